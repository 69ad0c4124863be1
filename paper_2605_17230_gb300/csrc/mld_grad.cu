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
    static constexpr int off_red = off_r + HALF;              // D x NW x 4 per-warp environment sums
    static constexpr int off_env = off_red + D * NW * 4;      // D x 4 environments of a column
    static constexpr int off_misc = off_env + D * 4;          // 32: per-warp reductions
    static constexpr int off_rep = off_misc + 32;             // N ints: representative x + 2z
    static constexpr int off_acc = (off_rep + N + 1) & ~1;    // 4N doubles: dL/dp of this block
    static constexpr int floats = off_acc + 8 * N;
    static constexpr int lfloats = (D - 1) * HALF;            // global: L_1..L_{d-1}
    // blocks per SM that shared memory allows (the register budget is held to it)
    static constexpr int MINB = (227 * 1024) / (floats * 4 + 1024) < 8 ? (227 * 1024) / (floats * 4 + 1024) : 8;
};

// Rows i whose plaquette (i, j) is a check (the others are pinned to 0).
template <int D>
__device__ __forceinline__ int present_rows(int j) {
    int m = 0;
#pragma unroll
    for (int i = 0; i <= D; ++i) m |= plaquette_is_check(D, i, j) ? 1 << i : 0;
    return m;
}

// Factor weights of qubit (r, c) are stored as Wp[u0 + 2 v0] with u0 =
// alpha_r ^ beta_{r+1} and v0 = alpha_{r+1} ^ beta_r: for parity (r + c) even
// these are the X and Z powers (u, v) of the factor p_q[E_q X^u Z^v]; for odd
// parity the two exchange roles, so Wp[j] = w_q[j with bits 0 and 1 swapped].
// Entry k = a | a'<<1 | b<<2 | b'<<3 of the factor then reads Wp[jk(k)].
__device__ __forceinline__ constexpr int jk(int k) {
    return ((k & 1) ^ ((k >> 3) & 1)) + 2 * (((k >> 1) & 1) ^ ((k >> 2) & 1));
}
template <int D>
__device__ __forceinline__ void factor_weights(const float* w, int r, int c, float (&Wp)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(w + 4 * (r * D + c));
    Wp[0] = v.x; Wp[1] = v.y; Wp[2] = v.z; Wp[3] = v.w;
}

__device__ __forceinline__ int rest_core(int rs, int r) {
    return (rs & ((1 << r) - 1)) | ((rs >> r) << (r + 2));
}

// Shared-memory position of entry e of the state before factor r (d >= 7).
// The 32 lanes of a warp own 32 consecutive rests, i.e. vary the five lowest
// index bits outside {r, r+1, d+1}; for r <= 4 two of those bits are bank
// bits, so a plain layout puts a warp on 8 or 16 banks. XORing bits 5 and 6
// into the bank bits with the masks below makes the lane -> bank map a
// bijection both for factor r-1 (which writes the state) and for factor r
// (which reads it); each mask pair was chosen so that, together with the
// bank bits left free by the two factors, it spans all five bank bits.
__device__ __forceinline__ int swz_mask5(int r) {
    return r == 0 ? 1 : r == 1 ? 5 : r == 2 ? 10 : r == 3 ? 20 : r == 4 ? 8 : 0;
}
__device__ __forceinline__ int swz_mask6(int r) {
    return r <= 1 ? 2 : r == 2 ? 4 : r == 3 ? 8 : r <= 5 ? 16 : 0;
}
template <int D>
__device__ __forceinline__ int phys(int e, int r) {
    if (D < 7) return e;
    return e ^ (((e >> 5) & 1) ? swz_mask5(r) : 0) ^ (((e >> 6) & 1) ? swz_mask6(r) : 0);
}

// Index of the corner-column state entry that feeds entry e of the state
// before factor 0 (bit 0 = beta_0 is free, bit d+1 = alpha_0).
template <int D>
__device__ __forceinline__ int left_index(int e) {
    constexpr int HALF = GradShape<D>::HALF;
    return (e & (HALF - 1) & ~1) | (e >> (D + 1));
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

// Shared-memory offsets of the eight entries of rest `core` in the layout of
// state index `lay`: o[k] holds the entry with bit r = k & 1, bit r+1 =
// (k >> 1) & 1 and bit d+1 = k >> 2. phys is linear over GF(2), so the
// offsets are one swizzled base XOR constants.
template <int D>
__device__ __forceinline__ void entry_offsets(int core, int r, int lay, int (&o)[8]) {
    constexpr int PS = GradShape<D>::HALF;
    const int base = phys<D>(core, lay);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = base ^ phys<D>((k & 1) * (1 << r) + ((k >> 1) & 1) * (2 << r) + (k >> 2) * PS, lay);
}

// Forward factor r: F_{r+1} from F_r (the eight entries of one rest).
//   F_{r+1}[b, b', a'] = sum_a F_r[b, a', a] w(a, a', b, b')
template <int D>
__device__ __forceinline__ void factor_forward(const float* __restrict__ Fr, float* __restrict__ Fn,
                                               const float (&Wp)[4], int r, int rs) {
    const int core = rest_core(rs, r);
    int oi[8], oo[8];
    entry_offsets<D>(core, r, r, oi);
    entry_offsets<D>(core, r, r + 1, oo);
    float x[8];   // x[b | a'<<1 | a<<2]
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = Fr[oi[k]];
#pragma unroll
    for (int k = 0; k < 8; ++k) {   // k = b | b'<<1 | a'<<2
        const int b = k & 1, bp = (k >> 1) & 1, ap = k >> 2;
        const int i0 = b | (ap << 1), wk = (ap << 1) | (b << 2) | (bp << 3);
        Fn[oo[k]] = fmaf(x[i0], Wp[jk(wk)], x[i0 | 4] * Wp[jk(wk | 1)]);
    }
}

// Transposed factor r: G_r from G_{r+1}.
//   G_r[b, a', a] = sum_b' G_{r+1}[b, b', a'] w(a, a', b, b')
template <int D>
__device__ __forceinline__ void factor_backward(const float* __restrict__ Gn, float* __restrict__ Gr,
                                                const float (&Wp)[4], int r, int rs) {
    const int core = rest_core(rs, r);
    int oi[8], oo[8];
    entry_offsets<D>(core, r, r + 1, oi);
    entry_offsets<D>(core, r, r, oo);
    float y[8];   // y[b | b'<<1 | a'<<2]
#pragma unroll
    for (int k = 0; k < 8; ++k) y[k] = Gn[oi[k]];
#pragma unroll
    for (int k = 0; k < 8; ++k) {   // k = b | a'<<1 | a<<2
        const int b = k & 1, ap = (k >> 1) & 1, a = k >> 2;
        const int i0 = b | (ap << 2), wk = a | (ap << 1) | (b << 2);
        Gr[oo[k]] = fmaf(y[i0], Wp[jk(wk)], y[i0 | 2] * Wp[jk(wk | 8)]);
    }
}

// Environment of factor r, accumulated per weight slot j (e[j] += sum of
// F_r x G_{r+1} over the entries k with jk(k) = j), and, unless r is the
// column's last factor, the forward step.
template <int D>
__device__ __forceinline__ void factor_environment(const float* __restrict__ Fr, const float* __restrict__ Gn,
                                                   float* __restrict__ Fn, const float (&Wp)[4], int r,
                                                   int rs, bool forward, float (&e)[4]) {
    const int core = rest_core(rs, r);
    int o0[8], o1[8];
    entry_offsets<D>(core, r, r, o0);
    entry_offsets<D>(core, r, r + 1, o1);
    float x[8], y[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x[k] = Fr[o0[k]];   // x[b | a'<<1 | a<<2]
        y[k] = Gn[o1[k]];   // y[b | b'<<1 | a'<<2]
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int a = k & 1, ap = (k >> 1) & 1, b = (k >> 2) & 1, bp = (k >> 3) & 1;
        e[jk(k)] = fmaf(x[b | (ap << 1) | (a << 2)], y[b | (bp << 1) | (ap << 2)], e[jk(k)]);
    }
    if (forward) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int b = k & 1, bp = (k >> 1) & 1, ap = k >> 2;
            const int i0 = b | (ap << 1), wk = (ap << 1) | (b << 2) | (bp << 3);
            Fn[o1[k]] = fmaf(x[i0], Wp[jk(wk)], x[i0 | 4] * Wp[jk(wk | 1)]);
        }
    }
}

// Sum of four per-lane values over the warp, scattered: lane l returns the
// total of slot (l >> 3) & 3.
__device__ __forceinline__ float reduce_scatter4(float (&v)[4], int lane) {
    {
        const bool hi = (lane & 16) != 0;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float send = hi ? v[i] : v[i + 2];
            const float keep = hi ? v[i + 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
    }
    const bool hi = (lane & 8) != 0;
    float t = (hi ? v[1] : v[0]) + __shfl_xor_sync(0xffffffffu, hi ? v[0] : v[1], 8);
    t += __shfl_xor_sync(0xffffffffu, t, 4);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    return t;
}

template <int D>
__global__ void __launch_bounds__(GradShape<D>::NT, GradShape<D>::MINB) grad_dense_kernel(GradDenseArgs g) {
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
        // Z_L on row 0) and the factor weights p_q[E_q X^u Z^v] (stored as Wp)
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
            const bool par = ((q / D + q % D) & 1) != 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int uv = par ? ((j & 1) << 1) | (j >> 1) : j;
                const int xx = x ^ (uv & 1), zz = z ^ (uv >> 1);
                wts[4 * q + j] = row[xx ? (zz ? 2 : 1) : (zz ? 3 : 0)];
            }
            rep[q] = x + 2 * z;
        }
        {
            const int pm0 = present_rows<D>(0);
            for (int e = tid; e < SIZE; e += NT) F0[phys<D>(e, 0)] = (left_index<D>(e) & ~pm0) == 0 ? 1.f : 0.f;
        }
        __syncthreads();

        // ---------------------------------------------------------------- forward
        float* Fa = F0;
        float* Fb = F1;
        int eL = 0;
        float total = 0.f;
        bool dead = false;
        for (int c = 0; c < D; ++c) {
#pragma unroll
            for (int r = 0; r < D; ++r) {
                float wr[4];
                factor_weights<D>(wts, r, c, wr);
                if (owns) factor_forward<D>(Fa, Fb, wr, r, rs);
                __syncthreads();
                float* t = Fa; Fa = Fb; Fb = t;
            }
            const int pmn = present_rows<D>(c + 1);
            float tmax = 0.f, tsum = 0.f;
            for (int bi = tid; bi < HALF; bi += NT) {
                const float v = (bi & ~pmn) == 0 ? Fa[phys<D>(bi, D)] + Fa[phys<D>(bi | HALF, D)] : 0.f;
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
            for (int e = tid; e < SIZE; e += NT) Fa[phys<D>(e, 0)] = Rs[left_index<D>(e)] * s;
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
                    GD[phys<D>(e, D)] = c == D - 1 ? ((bi & ~pmn) == 0 ? 1.f : 0.f) : Rs[bi];
                }
                const int pm0 = present_rows<D>(0);
                for (int e = tid; e < SIZE; e += NT) {
                    const int li = left_index<D>(e);
                    F0[phys<D>(e, 0)] = c == 0 ? ((li & ~pm0) == 0 ? 1.f : 0.f) : Lg[(c - 1) * HALF + li];
                }
            }
            __syncthreads();
#pragma unroll
            for (int r = D - 1; r >= 1; --r) {
                float wr[4];
                factor_weights<D>(wts, r, c, wr);
                if (owns) factor_backward<D>(G + (r + 1) * SIZE, G + r * SIZE, wr, r, rs);
                __syncthreads();
            }
            if (c > 0) {
                float wr[4];
                factor_weights<D>(wts, 0, c, wr);
                if (owns) factor_backward<D>(G + SIZE, G, wr, 0, rs);
                __syncthreads();
                // R_c = sum over beta_0 of G_0, rescaled
                const int pmc = present_rows<D>(c);
                float tmax = 0.f;
                for (int ai = tid; ai < HALF; ai += NT) {
                    const int e = (ai & ~1) | ((ai & 1) << (D + 1));
                    const float v = (ai & ~pmc) == 0 ? G[phys<D>(e, 0)] + G[phys<D>(e | 1, 0)] : 0.f;
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
#pragma unroll
            for (int r = 0; r < D; ++r) {
                float wr[4], e[4] = {0.f, 0.f, 0.f, 0.f};
                factor_weights<D>(wts, r, c, wr);
                if (owns) factor_environment<D>(Fa2, G + (r + 1) * SIZE, Fb2, wr, r, rs, r < D - 1, e);
                const float tot = reduce_scatter4(e, lane);
                if ((lane & 7) == 0) red[(r * NW + warp) * 4 + (lane >> 3)] = tot;
                __syncthreads();
                float* t = Fa2; Fa2 = Fb2; Fb2 = t;
            }
            for (int t = tid; t < D * 4; t += NT) {
                float s = 0.f;
#pragma unroll
                for (int w = 0; w < NW; ++w) s += red[((t >> 2) * NW + w) * 4 + (t & 3)];
                env[t] = s;
            }
            __syncthreads();
            // dZ/dp_{q,P} = env / <R|T|L>, with <R|T|L> = sum_j env_j Wp_j of factor 0
            for (int t = tid; t < 4 * D; t += NT) {
                const int r = t >> 2, uv = t & 3;
                float w0[4];
                factor_weights<D>(wts, 0, c, w0);
                float zc = 0.f;
#pragma unroll
                for (int j = 0; j < 4; ++j) zc = fmaf(env[j], w0[j], zc);
                const bool par = ((r + c) & 1) != 0;
                const float eu = env[4 * r + (par ? ((uv & 1) << 1) | (uv >> 1) : uv)];
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
