// Dense adjoint of the untruncated sweep, d = 3..13: d ln Z_l / d p_{q,P}.
// (Each block sums its units' gradients in a fixed order and a second
// kernel adds the blocks' sums in block order: reruns are bit-identical.)
//
// Z is linear in every qubit factor, so dZ/dw_q is the environment of that
// factor (Sec. 3.2.4: the contraction is differentiable in the local error
// probabilities, which the estimation of Eq. 10 back-propagates). The exact
// boundary state over one corner column has at most 2^(d+1) entries (one
// plaquette variable per row, absent plaquettes pinned to 0), so the states
// are kept dense: on chip for d <= 11; at d = 13 (128 KB per state inside a
// column) the states inside a column live in the block's global slice and
// only the two corner-column states R stay on chip. One thread block owns one
// (syndrome, class) unit:
//   forward   L_{c+1} = T_c L_c for c = 0..d-1, T_c applied qubit factor by
//             qubit factor to states over d+2 bits and rescaled by a power of
//             two per column; L_1..L_{d-1} go to the block's global slice, and
//             ln Z_l = ln sum L_d + the accumulated exponents.
//   backward  for c = d-1..0: the transposed factors carry R_{c+1} back
//             through column c (the states G_r kept in shared memory) and G_0
//             gives R_c; then the factors are re-applied from L_c, and each
//             factor's environment is the contraction of the state before it
//             with G after it, bucketed by the factor's weight slot.
// <R_{c+1}|T_c|L_c> = sum_j env_j w_j of any one factor (Euler's identity for
// a linear function), so every ratio env / Z is scale-free.
//
// State layout before factor r (qubit (r, c)) of column c, bit positions of
// a (d+2)-bit index: bits 0..r hold beta_0..beta_r (corner column c+1), bits
// r+1..d hold alpha_{r+1}..alpha_d (corner column c), bit d+1 holds alpha_r.
// Factor r sums alpha_r out, brings beta_{r+1} in and moves alpha_{r+1} to
// bit d+1, touching bits r, r+1 and d+1 only; factors r and r+1 together
// touch bits r, r+1, r+2 and d+1. So the factors are applied in pairs
// (r, r+1), r even, each thread holding in registers the sixteen entries of
// one assignment of the other bits (a "rest"); d odd leaves factor d-1 as a
// single step over eight entries per rest. Only the states before even
// factors (and after the last) are stored; the state between the two
// factors of a pair is recomputed in registers where it is needed.
#include <math.h>
#include <stdint.h>

#include "mld_dense_steps.cuh"
#include "mld_grad.h"
#include "mld_plan.h"

namespace mld {
namespace {

using namespace dense;

template <int D>
struct GradShape {
    static_assert(D % 2 == 1, "odd distances only");
    static constexpr int N = D * D;
    static constexpr int HALF = 1 << (D + 1);       // states over one corner column
    static constexpr int SIZE = HALF << 1;          // states inside a column (one more bit)
    static constexpr int REST1 = SIZE >> 3;         // rests of a single step (eight entries each)
    static constexpr int REST2 = SIZE >> 4;         // rests of a pair step (sixteen entries each)
    static constexpr int NT = REST2 >= 512 ? 512 : (REST2 >= 128 ? 128 : 32);
    // d >= 11: one block fills an SM's shared memory, so L_c is read from the
    // block's global slice, each step's environment sums are reduced at once,
    // and the representative's bits are recomputed where they are needed
    static constexpr bool BIG = D >= 11;
    // d >= 13: the G states (the states inside a column) are in the block's
    // global slice too; a thread takes several rests per step
    static constexpr bool HUGE = D >= 13;
    static constexpr int NW = NT / 32;
    static constexpr int NG = (D + 1) / 2;          // stored G states: r = 0, 2, .., d-1
    // shared memory (floats)
    static constexpr int off_w = 0;                          // 4N factor weights (slot order Wp)
    static constexpr int off_g = (4 * N + 3) & ~3;           // NG states of SIZE (on chip unless HUGE)
    static constexpr int off_l = off_g + (HUGE ? 0 : NG * SIZE);   // HALF: L_c for the environment pass
    static constexpr int off_ra = off_l + (BIG ? 0 : HALF);   // HALF: R_{c+1} (and staging)
    static constexpr int off_rb = off_ra + HALF;              // HALF: R_c being formed
    static constexpr int off_red = off_rb + HALF;             // per-warp environment sums:
    static constexpr int RED = BIG ? NW * 8 : D * NW * 4;     //   of one step (BIG) or of the column
    static constexpr int off_env = off_red + RED;             // D x 4 environments of a column
    static constexpr int off_misc = off_env + D * 4;          // 32: per-warp reductions
    static constexpr int off_rep = off_misc + 32;             // N ints: representative x + 2z
    static constexpr int floats = off_rep + (BIG ? 0 : N);
    static constexpr int lfloats = (D - 1) * HALF;            // global: L_1..L_{d-1}
    static constexpr int goff = lfloats + 8 * N;               // + the block's 4N double gradient sums
    static constexpr int slice = goff + (HUGE ? NG * SIZE : 0);   // + the G states (HUGE)
    static_assert(goff % 4 == 0 && slice % 4 == 0, "16-byte aligned slices");
    // blocks per SM that shared memory allows (the register budget is held to it)
    static constexpr int FIT0 = (227 * 1024) / (floats * 4 + 1024);
    static constexpr int FIT = FIT0 < 1 ? 1 : FIT0;   // one block of up to 227 KB always fits
    static constexpr int MINB = FIT < 16 ? FIT : 16;
    static_assert(floats * 4 <= 227 * 1024, "a block's shared memory is at most 227 KB");
};

// G state slot of the state before factor r (r even, or r = d).
template <int D>
__device__ __forceinline__ constexpr int gslot(int r) { return r == D ? (D + 1) / 2 : r / 2; }

// Shared-memory position of entry e of a stored state with layout index lay
// (the state before factor lay; d >= 7). The 32 lanes of a warp own 32
// consecutive rests, i.e. vary the five lowest index bits that the step
// leaves fixed; when the step touches bank bits (0..4), a plain layout puts
// the warp on 4 to 16 banks. XORing bits 5, 6 and 7 into the bank bits with
// these masks makes the lane -> bank map a bijection for both steps that
// access the state (the pair or single step that writes it and the one that
// reads it).
__device__ __forceinline__ constexpr int swz_mask(int lay, int bit) {
    return bit == 5 ? (lay == 0 ? 1 : lay == 2 ? 9 : lay == 4 ? 4 : 0)
         : bit == 6 ? (lay == 0 ? 2 : lay == 2 ? 18 : lay == 4 ? 8 : 0)
                    : (lay == 0 || lay == 2 ? 4 : lay == 4 || lay == 6 ? 16 : 0);
}
template <int D>
__device__ __forceinline__ int phys(int e, int lay) {
    if (D < 7) return e;
    return e ^ (((e >> 5) & 1) ? swz_mask(lay, 5) : 0) ^ (((e >> 6) & 1) ? swz_mask(lay, 6) : 0) ^
           (((e >> 7) & 1) ? swz_mask(lay, 7) : 0);
}

// ------------------------------------------------------------- single steps
// Entry k of a rest: bit r = k & 1, bit r+1 = (k >> 1) & 1, bit d+1 = k >> 2.
// phys is linear over GF(2), so the offsets are one swizzled base XOR
// constants.
template <int D>
__device__ __forceinline__ void single_offsets(int rs, int r, int lay, int (&o)[8]) {
    constexpr int PS = GradShape<D>::HALF;
    const int core = (rs & ((1 << r) - 1)) | ((rs >> r) << (r + 2));
    const int base = phys<D>(core, lay);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = base ^ phys<D>((k & 1) * (1 << r) + ((k >> 1) & 1) * (2 << r) + (k >> 2) * PS, lay);
}

// F_{r+1}[b, b', a'] = sum_a F_r[b, a', a] w(a, a', b, b')
template <int D>
__device__ __forceinline__ void single_forward(const float* __restrict__ Fr, float* __restrict__ Fn,
                                               const float (&Wp)[4], int r, int rs) {
    int oi[8], oo[8];
    single_offsets<D>(rs, r, r, oi);
    single_offsets<D>(rs, r, r + 1, oo);
    float x[8];   // x[b | a'<<1 | a<<2]
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = Fr[oi[k]];
#pragma unroll
    for (int k = 0; k < 8; ++k) {   // k = b | b'<<1 | a'<<2
        const int b = k & 1, bp = (k >> 1) & 1, ap = k >> 2, i0 = b | (ap << 1);
        Fn[oo[k]] = fmaf(x[i0], Wp[jw(0, ap, b, bp)], x[i0 | 4] * Wp[jw(1, ap, b, bp)]);
    }
}

// G_r[b, a', a] = sum_b' G_{r+1}[b, b', a'] w(a, a', b, b'). For the
// column's last factor, G_{r+1} = G_d is R_{c+1} for both values of the
// spare bit: read from the R buffer (HALF entries, plain layout).
template <int D, bool GR>
__device__ __forceinline__ void single_backward(const float* __restrict__ Gn, float* __restrict__ Gr,
                                                const float (&Wp)[4], int r, int rs) {
    constexpr int HALF = GradShape<D>::HALF;
    int oi[8], oo[8];
    single_offsets<D>(rs, r, r + 1, oi);
    single_offsets<D>(rs, r, r, oo);
    float y[8];   // y[b | b'<<1 | a'<<2]
#pragma unroll
    for (int k = 0; k < 8; ++k) y[k] = GR ? Gn[oi[k] & (HALF - 1)] : Gn[oi[k]];
#pragma unroll
    for (int k = 0; k < 8; ++k) {   // k = b | a'<<1 | a<<2
        const int b = k & 1, ap = (k >> 1) & 1, a = k >> 2, i0 = b | (ap << 2);
        Gr[oo[k]] = fmaf(y[i0], Wp[jw(a, ap, b, 0)], y[i0 | 2] * Wp[jw(a, ap, b, 1)]);
    }
}

// e[jw(a, a', b, b')] += F_r[b, a', a] G_{r+1}[b, b', a'] (G as in single_backward)
template <int D, bool GR>
__device__ __forceinline__ void single_environment(const float* __restrict__ Fr, const float* __restrict__ Gn,
                                                   int r, int rs, float (&e)[4]) {
    constexpr int HALF = GradShape<D>::HALF;
    int o0[8], o1[8];
    single_offsets<D>(rs, r, r, o0);
    single_offsets<D>(rs, r, r + 1, o1);
    float x[8], y[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x[k] = Fr[o0[k]];                                     // x[b | a'<<1 | a<<2]
        y[k] = GR ? Gn[o1[k] & (HALF - 1)] : Gn[o1[k]];       // y[b | b'<<1 | a'<<2]
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int a = k & 1, ap = (k >> 1) & 1, b = (k >> 2) & 1, bp = (k >> 3) & 1;
        e[jw(a, ap, b, bp)] = fmaf(x[b | (ap << 1) | (a << 2)], y[b | (bp << 1) | (ap << 2)], e[jw(a, ap, b, bp)]);
    }
}

// --------------------------------------------------------------- pair steps
// Entry g of a rest: bit r = g & 1, bit r+1 = (g >> 1) & 1, bit r+2 =
// (g >> 2) & 1, bit d+1 = g >> 3. Before factor r the four bits hold
// (beta_r, alpha_{r+1}, alpha_{r+2}, alpha_r); between the two factors
// (beta_r, beta_{r+1}, alpha_{r+2}, alpha_{r+1}); after factor r+1
// (beta_r, beta_{r+1}, beta_{r+2}, alpha_{r+2}).
template <int D>
__device__ __forceinline__ void pair_offsets(int rs, int r, int lay, int (&o)[16]) {
    constexpr int PS = GradShape<D>::HALF;
    const int core = (rs & ((1 << r) - 1)) | ((rs >> r) << (r + 3));
    const int base = phys<D>(core, lay);
#pragma unroll
    for (int g = 0; g < 16; ++g)
        o[g] = base ^ phys<D>((g & 1) * (1 << r) + ((g >> 1) & 1) * (2 << r) + ((g >> 2) & 1) * (4 << r) +
                                  (g >> 3) * PS, lay);
}

// Sum of 8 (4) per-lane values over the warp, scattered: lane l returns the
// total of slot (l >> 2) & 7 ((l >> 3) & 3).
__device__ __forceinline__ float reduce_scatter8(float (&v)[8], int lane) {
#pragma unroll
    for (int h = 4; h >= 1; h >>= 1) {
        const bool hi = (lane & (4 * h)) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = hi ? v[i] : v[i + h];
            const float keep = hi ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4 * h);
        }
    }
    float t = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 2);
    return t + __shfl_xor_sync(0xffffffffu, t, 1);
}
__device__ __forceinline__ float reduce_scatter4(float (&v)[4], int lane) {
#pragma unroll
    for (int h = 2; h >= 1; h >>= 1) {
        const bool hi = (lane & (8 * h)) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = hi ? v[i] : v[i + h];
            const float keep = hi ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8 * h);
        }
    }
    float t = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 4);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    return t + __shfl_xor_sync(0xffffffffu, t, 1);
}

template <int D>
__global__ void __launch_bounds__(GradShape<D>::NT, GradShape<D>::MINB) grad_dense_kernel(GradDenseArgs g) {
    using S = GradShape<D>;
    constexpr int N = S::N, HALF = S::HALF, SIZE = S::SIZE, NT = S::NT, NW = S::NW;
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* wts = sm + S::off_w;
    float* Lg = g.lws + (size_t)blockIdx.x * S::slice;
    float* G = S::HUGE ? Lg + S::goff : sm + S::off_g;   // G + gslot(r) * SIZE: the state before factor r
    float* Lb = sm + S::off_l;             // (d <= 9 only)
    float* Rcur = sm + S::off_ra;
    float* Rnxt = sm + S::off_rb;
    float* red = sm + S::off_red;
    float* env = sm + S::off_env;
    float* misc = sm + S::off_misc;
    int* rep = reinterpret_cast<int*>(sm + S::off_rep);   // (d <= 9 only)
    double* acc = reinterpret_cast<double*>(Lg + S::lfloats);   // this block's dL/dp, summed in unit order
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

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
            if constexpr (!S::BIG) rep[q] = x + 2 * z;
        }
        {
            const int pm0 = present_rows<D>(0);
            for (int e = tid; e < SIZE; e += NT) G[phys<D>(e, 0)] = (left_index<D>(e) & ~pm0) == 0 ? 1.f : 0.f;
        }
        __syncthreads();

        // ---------------------------------------------------------------- forward
        // the states ping-pong between G slots 0 and 1 (free until the backward pass)
        int eL = 0;
        float total = 0.f;
        bool dead = false;
        for (int c = 0; c < D; ++c) {
            float* Fa = G;
            float* Fb = G + SIZE;
#pragma unroll
            for (int r = 0; r + 1 < D; r += 2) {
                float W0[4], W1[4];
                factor_weights<D>(wts, r, c, W0);
                factor_weights<D>(wts, r + 1, c, W1);
                for_rests<S::REST2, NT>(tid, [&](int rs) {
                    int oi[16], oo[16];
                    pair_offsets<D>(rs, r, r, oi);
                    pair_offsets<D>(rs, r, r + 2, oo);
                    float X[16], Y[16], Z[16];
#pragma unroll
                    for (int m = 0; m < 16; ++m) X[m] = Fa[oi[m]];
                    pair_first(X, W0, Y);
                    pair_second(Y, W1, Z);
#pragma unroll
                    for (int m = 0; m < 16; ++m) Fb[oo[m]] = Z[m];
                });
                __syncthreads();
                float* t = Fa; Fa = Fb; Fb = t;
            }
            {
                float W[4];
                factor_weights<D>(wts, D - 1, c, W);
                for (int rs = tid; rs < S::REST1; rs += NT) single_forward<D>(Fa, Fb, W, D - 1, rs);
                __syncthreads();
                float* t = Fa; Fa = Fb; Fb = t;
            }
            const int pmn = present_rows<D>(c + 1);
            float tmax = 0.f, tsum = 0.f;
            for (int bi = tid; bi < HALF; bi += NT) {
                const float v = (bi & ~pmn) == 0 ? Fa[phys<D>(bi, D)] + Fa[phys<D>(bi | HALF, D)] : 0.f;
                Rcur[bi] = v;
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
            for (int e = tid; e < SIZE; e += NT) G[phys<D>(e, 0)] = Rcur[left_index<D>(e)] * s;
            for (int bi = tid; bi < HALF; bi += NT) Lg[c * HALF + bi] = Rcur[bi] * s;
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
        {
            const int pmd = present_rows<D>(D);
            for (int bi = tid; bi < HALF; bi += NT) Rcur[bi] = (bi & ~pmd) == 0 ? 1.f : 0.f;   // R_d
        }
        for (int c = D - 1; c >= 0; --c) {
            if constexpr (!S::BIG) {
                const int pm0 = present_rows<D>(0);
                for (int bi = tid; bi < HALF; bi += NT)
                    Lb[bi] = c == 0 ? ((bi & ~pm0) == 0 ? 1.f : 0.f) : Lg[(c - 1) * HALF + bi];
            }
            __syncthreads();
            {
                float W[4];
                factor_weights<D>(wts, D - 1, c, W);
                for (int rs = tid; rs < S::REST1; rs += NT)
                    single_backward<D, true>(Rcur, G + gslot<D>(D - 1) * SIZE, W, D - 1, rs);
                __syncthreads();
            }
#pragma unroll
            for (int r = D - 3; r >= 0; r -= 2) {
                if (r == 0 && c == 0) break;       // R_0 is not needed
                float W0[4], W1[4];
                factor_weights<D>(wts, r, c, W0);
                factor_weights<D>(wts, r + 1, c, W1);
                for_rests<S::REST2, NT>(tid, [&](int rs) {
                    int oi[16], oo[16];
                    pair_offsets<D>(rs, r, r + 2, oi);
                    pair_offsets<D>(rs, r, r, oo);
                    float Gz[16], Gy[16], Gx[16];
                    const float* Gn = G + gslot<D>(r + 2) * SIZE;
#pragma unroll
                    for (int m = 0; m < 16; ++m) Gz[m] = Gn[oi[m]];
                    pair_second_t(Gz, W1, Gy);
                    pair_first_t(Gy, W0, Gx);
                    float* Go = G + gslot<D>(r) * SIZE;
#pragma unroll
                    for (int m = 0; m < 16; ++m) Go[oo[m]] = Gx[m];
                });
                __syncthreads();
            }
            if (c > 0) {
                // R_c = sum over beta_0 of G_0, rescaled (R_{c+1} stays in Rcur for the pass below)
                const int pmc = present_rows<D>(c);
                float tmax = 0.f;
                for (int ai = tid; ai < HALF; ai += NT) {
                    const int e = (ai & ~1) | ((ai & 1) << (D + 1));
                    const float v = (ai & ~pmc) == 0 ? G[phys<D>(e, 0)] + G[phys<D>(e | 1, 0)] : 0.f;
                    Rnxt[ai] = v;
                    tmax = fmaxf(tmax, v);
                }
                const float m = block_max_nonneg<NW>(tmax, misc, tid);
                int ex = 0;
                const float s = (m > 0.f && m < INFINITY) ? inv_pow2_of(m, &ex) : 1.f;
                for (int ai = tid; ai < HALF; ai += NT) Rnxt[ai] *= s;
            }
            // re-apply the factors from L_c with each factor's environment; the
            // state after pair r goes to the slot of G_r, which pair r-2 (or
            // the extraction of R_c) has consumed; the first pair reads L_c
            // itself (beta_0 free, alpha_0 at bit d+1)
            const float* Fa = nullptr;
#pragma unroll
            for (int r = 0; r + 1 < D; r += 2) {
                float W0[4], W1[4];
                factor_weights<D>(wts, r, c, W0);
                factor_weights<D>(wts, r + 1, c, W1);
                float e[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // factor r, then factor r+1
                float* Fb = G + gslot<D>(r) * SIZE;
                for_rests<S::REST2, NT>(tid, [&](int rs) {
                    int o0[16], o2[16];
                    pair_offsets<D>(rs, r, r, o0);
                    pair_offsets<D>(rs, r, r + 2, o2);
                    const float* Gn = G + gslot<D>(r + 2) * SIZE;
                    float X[16], Gz[16], Y[16], Gy[16];
                    if (r == 0) {
                        const int core = rs << 3;      // rest bits above positions 0, 1, 2 (bit d+1 from g)
#pragma unroll
                        for (int m = 0; m < 16; ++m) {
                            const int lg = core | (m & 7) | ((m >> 3) << (D + 1));
                            const int li = left_index<D>(lg);
                            if constexpr (S::BIG)
                                X[m] = c == 0 ? ((li & ~present_rows<D>(0)) == 0 ? 1.f : 0.f) : Lg[(c - 1) * HALF + li];
                            else
                                X[m] = Lb[li];
                            Gz[m] = Gn[o2[m]];
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < 16; ++m) {
                            X[m] = Fa[o0[m]];
                            Gz[m] = Gn[o2[m]];
                        }
                    }
                    pair_first(X, W0, Y);
                    pair_second_t(Gz, W1, Gy);
#pragma unroll
                    for (int m = 0; m < 32; ++m) {
                        // factor r: sum over alpha_{r+2} of X (b_r, a_{r+1}, a_{r+2}, a_r) Gy (b_r, b_{r+1}, a_{r+2}, a_{r+1})
                        const int br = m & 1, ar1 = (m >> 1) & 1, ar2 = (m >> 2) & 1, ar = (m >> 3) & 1, br1 = m >> 4;
                        const int j = jw(ar, ar1, br, br1);
                        e[j] = fmaf(X[g4(br, ar1, ar2, ar)], Gy[g4(br, br1, ar2, ar1)], e[j]);
                    }
#pragma unroll
                    for (int m = 0; m < 32; ++m) {
                        // factor r+1: sum over beta_r of Y (b_r, b_{r+1}, a_{r+2}, a_{r+1}) Gz (b_r, b_{r+1}, b_{r+2}, a_{r+2})
                        const int br = m & 1, br1 = (m >> 1) & 1, ar2 = (m >> 2) & 1, ar1 = (m >> 3) & 1, br2 = m >> 4;
                        const int j = 4 + jw(ar1, ar2, br1, br2);
                        e[j] = fmaf(Y[g4(br, br1, ar2, ar1)], Gz[g4(br, br1, br2, ar2)], e[j]);
                    }
                    float Z[16];
                    pair_second(Y, W1, Z);
#pragma unroll
                    for (int m = 0; m < 16; ++m) Fb[o2[m]] = Z[m];
                });
                const float tot = reduce_scatter8(e, lane);
                if ((lane & 3) == 0) {
                    const int slot = lane >> 2;
                    if constexpr (S::BIG) red[warp * 8 + slot] = tot;
                    else red[((r + (slot >> 2)) * NW + warp) * 4 + (slot & 3)] = tot;
                }
                __syncthreads();
                if constexpr (S::BIG) {
                    if (tid < 8) {
                        float sum = 0.f;
                        for (int w = 0; w < NW; ++w) sum += red[w * 8 + tid];
                        env[(r + (tid >> 2)) * 4 + (tid & 3)] = sum;
                    }
                    __syncthreads();
                }
                Fa = Fb;
            }
            {
                float e[4] = {0.f, 0.f, 0.f, 0.f};
                for (int rs = tid; rs < S::REST1; rs += NT) single_environment<D, true>(Fa, Rcur, D - 1, rs, e);
                const float tot = reduce_scatter4(e, lane);
                if ((lane & 7) == 0) {
                    if constexpr (S::BIG) red[warp * 8 + (lane >> 3)] = tot;
                    else red[((D - 1) * NW + warp) * 4 + (lane >> 3)] = tot;
                }
                __syncthreads();
            }
            if constexpr (S::BIG) {
                if (tid < 4) {
                    float sum = 0.f;
                    for (int w = 0; w < NW; ++w) sum += red[w * 8 + tid];
                    env[(D - 1) * 4 + tid] = sum;
                }
            } else {
                for (int t = tid; t < D * 4; t += NT) {
                    float s = 0.f;
#pragma unroll
                    for (int w = 0; w < NW; ++w) s += red[((t >> 2) * NW + w) * 4 + (t & 3)];
                    env[t] = s;
                }
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
                    const int q = r * D + c;
                    int rx, rz;
                    if constexpr (S::BIG) {
                        rx = 0; rz = 0;
                        const uint64_t* mk = g.dmask + (size_t)q * 2 * g.words;
                        for (int w = 0; w < g.words; ++w) {
                            const uint64_t sw = g.syn[b * g.words + w];
                            rx ^= __popcll(sw & mk[w]) & 1;
                            rz ^= __popcll(sw & mk[g.words + w]) & 1;
                        }
                        if ((cls & 1) && c == 0) rx ^= 1;
                        if ((cls & 2) && r == 0) rz ^= 1;
                    } else {
                        rx = rep[q] & 1;
                        rz = rep[q] >> 1;
                    }
                    const int xx = rx ^ (uv & 1), zz = rz ^ (uv >> 1);
                    acc[4 * q + (xx ? (zz ? 2 : 1) : (zz ? 3 : 0))] += up * (double)(eu / zc);
                }
            }
            float* t = Rcur; Rcur = Rnxt; Rnxt = t;
        }
        __syncthreads();
    }
    // acc is the block's slot: grad_reduce_kernel adds the slots in block
    // order, so a rerun gives the same bits
}

// One block per gradient entry e: thread t sums the slots t, t + 256, ... in
// order, then a fixed-shape tree adds the 256 partial sums (deterministic).
__global__ void __launch_bounds__(256) grad_reduce_kernel(const float* __restrict__ ws, int64_t slice,
                                                          int64_t lfloats, int64_t blocks,
                                                          double* __restrict__ dnoise) {
    __shared__ double part[256];
    const int e = blockIdx.x, t = threadIdx.x;
    double s = 0.0;
    for (int64_t b = t; b < blocks; b += 256) s += reinterpret_cast<const double*>(ws + b * slice + lfloats)[e];
    part[t] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) part[t] += part[t + h];
        __syncthreads();
    }
    if (t == 0) dnoise[e] += part[0];
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
    if (cudaGetLastError() != cudaSuccess) return false;
    grad_reduce_kernel<<<4 * S::N, 256, 0, s>>>(a.lws, S::slice, S::lfloats, blocks, a.dnoise);
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace

bool grad_dense_supported(int d) { return d == 3 || d == 5 || d == 7 || d == 9 || d == 11 || d == 13; }

int64_t grad_dense_blocks(int d, int sms, int64_t B) {
    switch (d) {
        case 3: return blocks_d<3>(sms, B);
        case 5: return blocks_d<5>(sms, B);
        case 7: return blocks_d<7>(sms, B);
        case 9: return blocks_d<9>(sms, B);
        case 11: return blocks_d<11>(sms, B);
        case 13: return blocks_d<13>(sms, B);
    }
    return 0;
}

int64_t grad_dense_workspace_floats(int d) {
    switch (d) {
        case 3: return GradShape<3>::slice;
        case 5: return GradShape<5>::slice;
        case 7: return GradShape<7>::slice;
        case 9: return GradShape<9>::slice;
        case 11: return GradShape<11>::slice;
        case 13: return GradShape<13>::slice;
    }
    return 0;
}

bool launch_grad_dense(int d, const GradDenseArgs& a, int64_t blocks, cudaStream_t s) {
    switch (d) {
        case 3: return launch_d<3>(a, blocks, s);
        case 5: return launch_d<5>(a, blocks, s);
        case 7: return launch_d<7>(a, blocks, s);
        case 9: return launch_d<9>(a, blocks, s);
        case 11: return launch_d<11>(a, blocks, s);
        case 13: return launch_d<13>(a, blocks, s);
    }
    return false;
}

}  // namespace mld
