// Steps of the dense column transfer shared by the untruncated kernels that
// keep the boundary state dense (the adjoint and the d = 13 forward sweep).
//
// Within column c the state before factor r (qubit (r, c)) is indexed by d+2
// bits: bits 0..r hold beta_0..beta_r (corner column c+1), bits r+1..d hold
// alpha_{r+1}..alpha_d (corner column c) and bit d+1 holds alpha_r. Factor r
// sums alpha_r out, brings beta_{r+1} in and moves alpha_{r+1} to bit d+1;
// two consecutive factors (a pair) touch bits r, r+1, r+2 and d+1 only.
#pragma once

#include <math.h>
#include <stdint.h>

#include "mld_plan.h"

namespace mld {
namespace dense {

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
// The factor's entry (a, a', b, b') = (alpha_r, alpha_{r+1}, beta_r,
// beta_{r+1}) reads Wp[jw(a, a', b, b')].
__device__ __forceinline__ constexpr int jw(int a, int ap, int b, int bp) { return (a ^ bp) + 2 * (ap ^ b); }

template <int D>
__device__ __forceinline__ void factor_weights(const float* w, int r, int c, float (&Wp)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(w + 4 * (r * D + c));
    Wp[0] = v.x; Wp[1] = v.y; Wp[2] = v.z; Wp[3] = v.w;
}

// Index of the corner-column state entry that feeds entry e of the state
// before factor 0 (bit 0 = beta_0 is free, bit d+1 = alpha_0).
template <int D>
__device__ __forceinline__ int left_index(int e) {
    constexpr int HALF = 1 << (D + 1);
    return (e & (HALF - 1) & ~1) | (e >> (D + 1));
}

__device__ __forceinline__ constexpr int g4(int b0, int b1, int b2, int b3) { return b0 | (b1 << 1) | (b2 << 2) | (b3 << 3); }

// f(rs) for every rest rs of a pair step this thread owns: one (or none)
// while the block has a thread per rest, every NT-th one beyond that (d = 13).
template <int REST, int NT, typename F>
__device__ __forceinline__ void for_rests(int tid, F&& f) {
    if constexpr (REST <= NT) {
        if (tid < REST) f(tid);
    } else {
        for (int rs = tid; rs < REST; rs += NT) f(rs);
    }
}

// factor r on the sixteen entries: Y = state between the factors from X
__device__ __forceinline__ void pair_first(const float (&X)[16], const float (&W)[4], float (&Y)[16]) {
#pragma unroll
    for (int m = 0; m < 16; ++m) {   // m = (b_r, b_{r+1}, a_{r+2}, a_{r+1})
        const int br = m & 1, br1 = (m >> 1) & 1, ar2 = (m >> 2) & 1, ar1 = m >> 3;
        Y[m] = fmaf(X[g4(br, ar1, ar2, 0)], W[jw(0, ar1, br, br1)], X[g4(br, ar1, ar2, 1)] * W[jw(1, ar1, br, br1)]);
    }
}
// factor r+1: Z = state after the pair from Y
__device__ __forceinline__ void pair_second(const float (&Y)[16], const float (&W)[4], float (&Z)[16]) {
#pragma unroll
    for (int m = 0; m < 16; ++m) {   // m = (b_r, b_{r+1}, b_{r+2}, a_{r+2})
        const int br = m & 1, br1 = (m >> 1) & 1, br2 = (m >> 2) & 1, ar2 = m >> 3;
        Z[m] = fmaf(Y[g4(br, br1, ar2, 0)], W[jw(0, ar2, br1, br2)], Y[g4(br, br1, ar2, 1)] * W[jw(1, ar2, br1, br2)]);
    }
}
// transposed factor r+1: Gy (between the factors) from Gz (after the pair)
__device__ __forceinline__ void pair_second_t(const float (&Gz)[16], const float (&W)[4], float (&Gy)[16]) {
#pragma unroll
    for (int m = 0; m < 16; ++m) {   // m = (b_r, b_{r+1}, a_{r+2}, a_{r+1})
        const int br = m & 1, br1 = (m >> 1) & 1, ar2 = (m >> 2) & 1, ar1 = m >> 3;
        Gy[m] = fmaf(Gz[g4(br, br1, 0, ar2)], W[jw(ar1, ar2, br1, 0)], Gz[g4(br, br1, 1, ar2)] * W[jw(ar1, ar2, br1, 1)]);
    }
}
// transposed factor r: Gx (before the pair) from Gy
__device__ __forceinline__ void pair_first_t(const float (&Gy)[16], const float (&W)[4], float (&Gx)[16]) {
#pragma unroll
    for (int m = 0; m < 16; ++m) {   // m = (b_r, a_{r+1}, a_{r+2}, a_r)
        const int br = m & 1, ar1 = (m >> 1) & 1, ar2 = (m >> 2) & 1, ar = m >> 3;
        Gx[m] = fmaf(Gy[g4(br, 0, ar2, ar1)], W[jw(ar, ar1, br, 0)], Gy[g4(br, 1, ar2, ar1)] * W[jw(ar, ar1, br, 1)]);
    }
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

}  // namespace dense
}  // namespace mld
