// Dense adjoint of the untruncated sweep, d = 3..9: d ln Z_l / d p_{q,P}.
//
// Z is linear in every qubit factor, so dZ/dw_q is the environment of that
// factor (Sec. 3.2.4: the contraction is differentiable in the local error
// probabilities, which the estimation of Eq. 10 back-propagates). For d <= 9
// the exact boundary state over one corner column has at most 2^(d+1)
// entries (one plaquette variable per row, absent plaquettes pinned to 0), so
// the states are kept dense on chip. One thread block owns one (syndrome,
// class) unit:
//   forward   L_{c+1} = T_c L_c for c = 0..d-1, T_c applied one qubit factor
//             at a time to states over d+2 bits and rescaled by a power of two
//             per column; L_1..L_{d-1} go to the block's global slice, and
//             ln Z_l = ln sum L_d + the accumulated exponents.
//   backward  for c = d-1..0: the transposed factors carry R_{c+1} back
//             through column c (G_d..G_0, all kept in shared memory) and G_0
//             gives R_c; then the factors are re-applied from L_c, and each
//             factor's environment is the contraction of the state before it
//             with G after it, bucketed by the factor's four plaquette
//             variables.
// <R_{c+1}|T_c|L_c> = sum_k env_k w_k of any one factor (Euler's identity for
// a linear function), so every ratio env / Z is scale-free.
//
// State layout before factor r (qubit (r, c)) of column c, bit positions of
// a (d+2)-bit index: bits 0..r hold beta_0..beta_r (corner column c+1), bits
// r+1..d hold alpha_{r+1}..alpha_d (corner column c), bit d+1 holds alpha_r.
// Factor r sums alpha_r out, brings beta_{r+1} in and moves alpha_{r+1} to
// bit d+1; it touches bits r, r+1 and d+1 only, so a thread owns the eight
// entries of one assignment of the other bits ("rest").
#include <math.h>
#include <stdint.h>

#include "mld_grad.h"
#include "mld_plan.h"

namespace mld {
namespace {

template <int D>
struct GradShape {
    static constexpr int N = D * D;
    static constexpr int HALF = 1 << (D + 1);       // states over one corner column
    static constexpr int SIZE = HALF << 1;          // states inside a column (one more bit)
    static constexpr int REST = SIZE >> 3;          // eight entries per thread and factor
    static constexpr int NT = REST >= 256 ? 256 : (REST >= 64 ? 64 : 32);
    static constexpr int NW = NT / 32;
    // shared memory (floats)
    static constexpr int off_w = 0;                          // 4N factor weights w_q[u + 2v]
    static constexpr int off_g = (4 * N + 3) & ~3;           // G_0..G_d, SIZE each
    static constexpr int off_f0 = off_g + (D + 1) * SIZE;     // forward state (ping)
    static constexpr int off_f1 = off_f0 + SIZE;              // forward state (pong)
    static constexpr int off_r = off_f1 + SIZE;               // HALF: L_{c+1} staging, R_{c+1}
    static constexpr int off_red = off_r + HALF;              // D x NW x 16 per-warp environment sums
    static constexpr int off_env = off_red + D * NW * 16;     // D x 16 environments of a column
    static constexpr int off_misc = off_env + D * 16;         // 32: per-warp reductions
    static constexpr int off_rep = off_misc + 32;             // N ints: representative x + 2z
    static constexpr int off_acc = (off_rep + N + 1) & ~1;    // 4N doubles: dL/dp of this block
    static constexpr int floats = off_acc + 8 * N;
    static constexpr int lfloats = (D - 1) * HALF;            // global: L_1..L_{d-1}
};

// Rows i whose plaquette (i, j) is a check (the others are pinned to 0).
template <int D>
__device__ __forceinline__ int present_rows(int j) {
    int m = 0;
#pragma unroll
    for (int i = 0; i <= D; ++i) m |= plaquette_is_check(D, i, j) ? 1 << i : 0;
    return m;
}

// Weights of factor (r, c) for every assignment k = a | a'<<1 | b<<2 | b'<<3
// of (alpha_r, alpha_{r+1}, beta_r, beta_{r+1}): w_q[u + 2v] with u (v) the
// XOR of the two X-type (Z-type) plaquettes around the qubit.
template <int D>
__device__ __forceinline__ void factor_weights(const float* w, int r, int c, float (&wr)[16]) {
    const float4 v = *reinterpret_cast<const float4*>(w + 4 * (r * D + c));
    const float W[4] = {v.x, v.y, v.z, v.w};
    const bool par = ((r + c) & 1) != 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int a = k & 1, ap = (k >> 1) & 1, b = (k >> 2) & 1, bp = (k >> 3) & 1;
        const int u0 = a ^ bp, v0 = ap ^ b;    // parity 0; parity 1 exchanges u and v
        wr[k] = par ? W[v0 + 2 * u0] : W[u0 + 2 * v0];
    }
}

__device__ __forceinline__ int rest_core(int rs, int r) {
    return (rs & ((1 << r) - 1)) | ((rs >> r) << (r + 2));
}

// Index of the corner-column state entry that feeds entry e of the state
// before factor 0 (bit 0 = beta_0 is free, bit d+1 = alpha_0).
template <int D>
__device__ __forceinline__ int left_index(int e) {
    constexpr int HALF = GradShape<D>::HALF;
    return (e & (HALF - 1) & ~1) | (e >> (D + 1));
}

// Sum of 16 per-lane values over the warp, scattered: lanes 2k and 2k+1
// return the total of slot k.
__device__ __forceinline__ float reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const bool hi = (lane & (2 * h)) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = hi ? v[i] : v[i + h];
            const float keep = hi ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * h);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int NW>
__device__ __forceinline__ float block_max_nonneg(float v, float* misc, int tid) {
    // non-negative floats (and NaN, which must win) order like their bit patterns
    unsigned u = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
    if ((tid & 31) == 0) misc[tid >> 5] = __uint_as_float(u);
    __syncthreads();
    u = __float_as_uint(misc[0]);
#pragma unroll
    for (int w = 1; w < NW; ++w) u = max(u, __float_as_uint(misc[w]));
    return __uint_as_float(u);
}

template <int NW>
__device__ __forceinline__ float block_sum(float v, float* misc, int tid) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) misc[tid >> 5] = v;
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += misc[w];
    return s;
}

// exact 2^-e for the exponent e of m (m = f 2^e, f in [0.5, 1))
__device__ __forceinline__ float inv_pow2_of(float m, int* e) {
    int ex = 0;
    frexpf(m, &ex);
    ex = ex < -126 ? -126 : (ex > 126 ? 126 : ex);
    *e = ex;
    return __int_as_float((127 - ex) << 23);
}

// Forward factor r: F_{r+1} from F_r (rows of one rest per thread).
template <int D>
__device__ __forceinline__ void factor_forward(const float* __restrict__ Fr, float* __restrict__ Fn,
                                               const float (&wr)[16], int r, int rs) {
    constexpr int PS = GradShape<D>::HALF;
    const int P0 = 1 << r, P1 = 2 << r, core = rest_core(rs, r);
    float x[8];   // x[b | a'<<1 | a<<2] = F_r[core + b P0 + a' P1 + a PS]
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = Fr[core + (k & 1) * P0 + ((k >> 1) & 1) * P1 + (k >> 2) * PS];
#pragma unroll
    for (int k = 0; k < 8; ++k) {   // k = b | b'<<1 | a'<<2 (output bits r, r+1, d+1)
        const int b = k & 1, bp = (k >> 1) & 1, ap = k >> 2;
        const int i0 = b | (ap << 1), wk = (ap << 1) | (b << 2) | (bp << 3);
        Fn[core + b * P0 + bp * P1 + ap * PS] = fmaf(x[i0], wr[wk], x[i0 | 4] * wr[wk | 1]);
    }
}

// Transposed factor r: G_r from G_{r+1}.
template <int D>
__device__ __forceinline__ void factor_backward(const float* __restrict__ Gn, float* __restrict__ Gr,
                                                const float (&wr)[16], int r, int rs) {
    constexpr int PS = GradShape<D>::HALF;
    const int P0 = 1 << r, P1 = 2 << r, core = rest_core(rs, r);
    float y[8];   // y[b | b'<<1 | a'<<2] = G_{r+1}[core + b P0 + b' P1 + a' PS]
#pragma unroll
    for (int k = 0; k < 8; ++k) y[k] = Gn[core + (k & 1) * P0 + ((k >> 1) & 1) * P1 + (k >> 2) * PS];
#pragma unroll
    for (int k = 0; k < 8; ++k) {   // k = b | a'<<1 | a<<2 (bits r, r+1, d+1 of G_r)
        const int b = k & 1, ap = (k >> 1) & 1, a = k >> 2;
        const int i0 = b | (ap << 2), wk = a | (ap << 1) | (b << 2);
        Gr[core + b * P0 + ap * P1 + a * PS] = fmaf(y[i0], wr[wk], y[i0 | 2] * wr[wk | 8]);
    }
}

// Environment of factor r (accumulated into e[k], k as in factor_weights)
// and, unless it is the column's last factor, the forward step.
template <int D>
__device__ __forceinline__ void factor_environment(const float* __restrict__ Fr, const float* __restrict__ Gn,
                                                   float* __restrict__ Fn, const float (&wr)[16], int r,
                                                   int rs, bool forward, float (&e)[16]) {
    constexpr int PS = GradShape<D>::HALF;
    const int P0 = 1 << r, P1 = 2 << r, core = rest_core(rs, r);
    float x[8], y[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int off = core + (k & 1) * P0 + ((k >> 1) & 1) * P1 + (k >> 2) * PS;
        x[k] = Fr[off];   // x[b | a'<<1 | a<<2]
        y[k] = Gn[off];   // y[b | b'<<1 | a'<<2]
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int a = k & 1, ap = (k >> 1) & 1, b = (k >> 2) & 1, bp = (k >> 3) & 1;
        e[k] = fmaf(x[b | (ap << 1) | (a << 2)], y[b | (bp << 1) | (ap << 2)], e[k]);
    }
    if (forward) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int b = k & 1, bp = (k >> 1) & 1, ap = k >> 2;
            const int i0 = b | (ap << 1), wk = (ap << 1) | (b << 2) | (bp << 3);
            Fn[core + b * P0 + bp * P1 + ap * PS] = fmaf(x[i0], wr[wk], x[i0 | 4] * wr[wk | 1]);
        }
    }
}

template <int D>
__global__ void __launch_bounds__(GradShape<D>::NT) grad_dense_kernel(GradDenseArgs g) {
    using S = GradShape<D>;
    constexpr int N = S::N, HALF = S::HALF, SIZE = S::SIZE, REST = S::REST, NT = S::NT, NW = S::NW;
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* wts = sm + S::off_w;
    float* G = sm + S::off_g;
    float* F0 = sm + S::off_f0;
    float* F1 = sm + S::off_f1;
    float* Rs = sm + S::off_r;
    float* red = sm + S::off_red;
    float* env = sm + S::off_env;
    float* misc = sm + S::off_misc;
    int* rep = reinterpret_cast<int*>(sm + S::off_rep);
    double* acc = reinterpret_cast<double*>(sm + S::off_acc);
    float* Lg = g.lws + (size_t)blockIdx.x * S::lfloats;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rs = tid;                    // this thread's rest (REST <= NT)
    const bool owns = rs < REST;

    for (int e = tid; e < 4 * N; e += NT) acc[e] = 0.0;

    for (int64_t unit = blockIdx.x; unit < 4 * g.B; unit += gridDim.x) {
        const int64_t b = unit >> 2;
        const int cls = (int)(unit & 3);
        const double up = g.dlogP ? g.dlogP[unit] : 0.0;
        if (up == 0.0 && !g.logP) continue;        // uniform over the block
        // representative E_{l,s} = f(s) X_L^{l_X} Z_L^{l_Z} (X_L on column 0,
        // Z_L on row 0) and the factor weights w_q[u + 2v] = p_q[E_q X^u Z^v]
        for (int q = tid; q < N; q += NT) {
            int x = 0, z = 0;
            const uint64_t* mk = g.dmask + (size_t)q * 2 * g.words;
            for (int w = 0; w < g.words; ++w) {
                const uint64_t sw = g.syn[b * g.words + w];
                x ^= __popcll(sw & mk[w]) & 1;
                z ^= __popcll(sw & mk[g.words + w]) & 1;
            }
            if ((cls & 1) && q % D == 0) x ^= 1;
            if ((cls & 2) && q < D) z ^= 1;
            const float4 p = *reinterpret_cast<const float4*>(g.noise + 4 * (size_t)q);
            const float row[4] = {p.x, p.y, p.z, p.w};   // I, X, Y, Z
#pragma unroll
            for (int uv = 0; uv < 4; ++uv) {
                const int xx = x ^ (uv & 1), zz = z ^ (uv >> 1);
                wts[4 * q + uv] = row[xx ? (zz ? 2 : 1) : (zz ? 3 : 0)];
            }
            rep[q] = x + 2 * z;
        }
        {
            const int pm0 = present_rows<D>(0);
            for (int e = tid; e < SIZE; e += NT) F0[e] = (left_index<D>(e) & ~pm0) == 0 ? 1.f : 0.f;
        }
        __syncthreads();

        // ---------------------------------------------------------------- forward
        float* Fa = F0;
        float* Fb = F1;
        int eL = 0;
        float total = 0.f;
        bool dead = false;
        for (int c = 0; c < D; ++c) {
            for (int r = 0; r < D; ++r) {
                float wr[16];
                factor_weights<D>(wts, r, c, wr);
                if (owns) factor_forward<D>(Fa, Fb, wr, r, rs);
                __syncthreads();
                float* t = Fa; Fa = Fb; Fb = t;
            }
            const int pmn = present_rows<D>(c + 1);
            float tmax = 0.f, tsum = 0.f;
            for (int bi = tid; bi < HALF; bi += NT) {
                const float v = (bi & ~pmn) == 0 ? Fa[bi] + Fa[bi | HALF] : 0.f;
                Rs[bi] = v;
                tmax = fmaxf(tmax, v);
                tsum += v;
            }
            if (c == D - 1) {
                total = block_sum<NW>(tsum, misc, tid);
                break;
            }
            const float m = block_max_nonneg<NW>(tmax, misc, tid);
            if (!(m > 0.f) || !(m < INFINITY)) { dead = true; break; }
            int ex = 0;
            const float s = inv_pow2_of(m, &ex);
            eL += ex;
            for (int e = tid; e < SIZE; e += NT) Fa[e] = Rs[left_index<D>(e)] * s;
            for (int bi = tid; bi < HALF; bi += NT) Lg[c * HALF + bi] = Rs[bi] * s;
            __syncthreads();
        }
        const double lz = (!dead && total > 0.f && total < INFINITY)
                              ? log((double)total) + (double)eL * 0.69314718055994530942
                              : (dead || total == 0.f ? -INFINITY : (double)NAN);
        if (g.logP && tid == 0) g.logP[unit] = lz;
        if (up == 0.0 || !(lz > -INFINITY) || !(lz < INFINITY)) {
            __syncthreads();
            continue;
        }

        // ---------------------------------------------------------------- backward
        for (int c = D - 1; c >= 0; --c) {
            {
                const int pmn = present_rows<D>(c + 1);
                float* GD = G + D * SIZE;
                for (int e = tid; e < SIZE; e += NT) {
                    const int bi = e & (HALF - 1);
                    GD[e] = c == D - 1 ? ((bi & ~pmn) == 0 ? 1.f : 0.f) : Rs[bi];
                }
                const int pm0 = present_rows<D>(0);
                for (int e = tid; e < SIZE; e += NT) {
                    const int li = left_index<D>(e);
                    F0[e] = c == 0 ? ((li & ~pm0) == 0 ? 1.f : 0.f) : Lg[(c - 1) * HALF + li];
                }
            }
            __syncthreads();
            for (int r = D - 1; r >= (c > 0 ? 0 : 1); --r) {
                float wr[16];
                factor_weights<D>(wts, r, c, wr);
                if (owns) factor_backward<D>(G + (r + 1) * SIZE, G + r * SIZE, wr, r, rs);
                __syncthreads();
            }
            if (c > 0) {
                // R_c = sum over beta_0 of G_0, rescaled
                const int pmc = present_rows<D>(c);
                float tmax = 0.f;
                for (int ai = tid; ai < HALF; ai += NT) {
                    const int e = (ai & ~1) | ((ai & 1) << (D + 1));
                    const float v = (ai & ~pmc) == 0 ? G[e] + G[e | 1] : 0.f;
                    Rs[ai] = v;
                    tmax = fmaxf(tmax, v);
                }
                const float m = block_max_nonneg<NW>(tmax, misc, tid);
                int ex = 0;
                const float s = (m > 0.f && m < INFINITY) ? inv_pow2_of(m, &ex) : 1.f;
                for (int ai = tid; ai < HALF; ai += NT) Rs[ai] *= s;
            }
            // re-apply the factors from L_c with each factor's environment
            float* Fa2 = F0;
            float* Fb2 = F1;
            for (int r = 0; r < D; ++r) {
                float wr[16], e[16];
                factor_weights<D>(wts, r, c, wr);
#pragma unroll
                for (int k = 0; k < 16; ++k) e[k] = 0.f;
                if (owns) factor_environment<D>(Fa2, G + (r + 1) * SIZE, Fb2, wr, r, rs, r < D - 1, e);
                const float tot = reduce_scatter16(e, lane);
                if ((lane & 1) == 0) red[(r * NW + warp) * 16 + (lane >> 1)] = tot;
                __syncthreads();
                float* t = Fa2; Fa2 = Fb2; Fb2 = t;
            }
            for (int t = tid; t < D * 16; t += NT) {
                float s = 0.f;
#pragma unroll
                for (int w = 0; w < NW; ++w) s += red[((t >> 4) * NW + w) * 16 + (t & 15)];
                env[t] = s;
            }
            __syncthreads();
            for (int t = tid; t < 4 * D; t += NT) {
                const int r = t >> 2, uv = t & 3;
                float w0[16];
                factor_weights<D>(wts, 0, c, w0);
                float zc = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k) zc = fmaf(env[k], w0[k], zc);
                const bool par = ((r + c) & 1) != 0;
                float eu = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int a = k & 1, ap = (k >> 1) & 1, bb = (k >> 2) & 1, bp = (k >> 3) & 1;
                    const int u = par ? (ap ^ bb) : (a ^ bp), v = par ? (a ^ bp) : (ap ^ bb);
                    if (u + 2 * v == uv) eu += env[r * 16 + k];
                }
                if (zc > 0.f) {
                    const int q = r * D + c, xx = (rep[q] & 1) ^ (uv & 1), zz = (rep[q] >> 1) ^ (uv >> 1);
                    acc[4 * q + (xx ? (zz ? 2 : 1) : (zz ? 3 : 0))] += up * (double)(eu / zc);
                }
            }
        }
        __syncthreads();
    }
    __syncthreads();
    for (int e = tid; e < 4 * N; e += NT)
        if (acc[e] != 0.0) atomicAdd(g.dnoise + e, acc[e]);
}

template <int D>
int64_t blocks_d(int sms, int64_t B) {
    using S = GradShape<D>;
    const size_t bytes = (size_t)S::floats * sizeof(float);
    if (cudaFuncSetAttribute(grad_dense_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grad_dense_kernel<D>, S::NT, bytes) != cudaSuccess ||
        per_sm < 1)
        return 0;
    int64_t nb = (int64_t)sms * per_sm;
    if (nb > 4 * B) nb = 4 * B;
    return nb < 1 ? 1 : nb;
}

template <int D>
bool launch_d(const GradDenseArgs& a, int64_t blocks, cudaStream_t s) {
    using S = GradShape<D>;
    const size_t bytes = (size_t)S::floats * sizeof(float);
    if (cudaFuncSetAttribute(grad_dense_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return false;
    grad_dense_kernel<D><<<(unsigned)blocks, S::NT, bytes, s>>>(a);
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace

bool grad_dense_supported(int d) { return d == 3 || d == 5 || d == 7 || d == 9; }

int64_t grad_dense_blocks(int d, int sms, int64_t B) {
    switch (d) {
        case 3: return blocks_d<3>(sms, B);
        case 5: return blocks_d<5>(sms, B);
        case 7: return blocks_d<7>(sms, B);
        case 9: return blocks_d<9>(sms, B);
    }
    return 0;
}

int64_t grad_dense_workspace_floats(int d) {
    switch (d) {
        case 3: return GradShape<3>::lfloats;
        case 5: return GradShape<5>::lfloats;
        case 7: return GradShape<7>::lfloats;
        case 9: return GradShape<9>::lfloats;
    }
    return 0;
}

bool launch_grad_dense(int d, const GradDenseArgs& a, int64_t blocks, cudaStream_t s) {
    switch (d) {
        case 3: return launch_d<3>(a, blocks, s);
        case 5: return launch_d<5>(a, blocks, s);
        case 7: return launch_d<7>(a, blocks, s);
        case 9: return launch_d<9>(a, blocks, s);
    }
    return false;
}

}  // namespace mld
