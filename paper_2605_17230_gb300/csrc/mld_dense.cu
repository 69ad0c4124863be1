// Untruncated sweep with the boundary state kept dense, for the distances
// where the exact boundary MPS is larger than an SM's shared memory per warp
// (d = 13: bonds up to 64, 298 KB per unit) but the dense state of one unit
// fits one block (2^(d+2) floats inside a column: 128 KB at d = 13).
//
// At chi >= 2^floor(d/2) the boundary MPS of the column sweep (Eq. 7,
// Sec. 3.2.1) discards nothing: it is the exact boundary state over the
// plaquette variables of one corner column, written as a product of site
// tensors. This kernel keeps that state as the dense vector instead and
// applies the column's qubit factors to it one pair at a time, in place in
// shared memory (the steps and the bit layout of the dense adjoint; a rest's
// sixteen entries occupy the same positions before and after a pair step,
// so one buffer serves the whole column). One block owns one (syndrome, l_Z)
// unit; X_L is taken on column d-1, so the two classes
// l_X = 0, 1 share columns 0..d-2 and only the last column runs twice, from
// the corner state after column d-2. Power-of-two rescaling per column; the
// exponents are summed as integers and ln Z is formed in FP64.
#include <math.h>
#include <stdint.h>

#include <utility>

#include "mld_dense.h"
#include "mld_dense_steps.cuh"

namespace mld {
namespace {

using namespace dense;

template <int D>
struct DenseShape {
    static constexpr int N = D * D;
    static constexpr int HALF = 1 << (D + 1);      // a corner-column state
    static constexpr int SIZE = HALF << 1;         // a state inside a column
    static constexpr int REST1 = SIZE >> 3;        // rests of a single step (eight entries)
    static constexpr int REST2 = SIZE >> 4;        // rests of a pair step (sixteen entries)
    // d = 13: one block of 16 warps per SM (shared memory); d = 11: two
    // blocks of 8 warps, d = 9: four blocks of 4 warps (registers)
    static constexpr int NT = D >= 13 ? 512 : (D >= 11 ? 256 : 128);
    static constexpr int MINB = D >= 13 ? 1 : (D >= 11 ? 2 : 4);
    static constexpr int NW = NT / 32;
    // shared memory (floats)
    static constexpr int off_w = 0;                       // 4N factor weights (slot order Wp)
    static constexpr int off_s = (4 * N + 31) & ~31;      // SIZE: the state inside the column
    static constexpr int off_r = off_s + SIZE;             // HALF: the corner state after a column
    static constexpr int off_misc = off_r + HALF;          // 32: block reductions
    static constexpr int floats = off_misc + 32;
    static_assert(floats * 4 <= 227 * 1024, "one unit's state fits a block's shared memory");
    static_assert(REST2 >= NT, "every thread owns at least one rest of a pair step");
};

// Shared-memory position of entry e of a state inside a column: bits 5, 6
// and 7 XORed into the bank bits with masks 5, 9 and 18. The map is linear
// over GF(2) and the same for every step, so a step rewrites its entries in
// place. The 32 lanes of a warp (32 consecutive rests) hit 32 distinct banks
// in every pair and single step of d = 9, 11, 13 when no rest is skipped
// (checked exhaustively on the host); of the three-mask swizzles with that
// property, this one leaves the fewest same-bank pairs once the rests of
// absent plaquettes are skipped (measured at d = 13: 5.6% of the
// shared-memory wavefronts are conflicts, against 12.8% with masks 4, 9, 18).
// Two more masks (bits 8 and 9) removed nearly all of them but cost 13% more
// instructions and ran 8% slower: the kernel is issue-bound.
__host__ __device__ __forceinline__ constexpr int sphys(int e) {
    return e ^ (((e >> 5) & 1) ? 5 : 0) ^ (((e >> 6) & 1) ? 9 : 0) ^ (((e >> 7) & 1) ? 18 : 0);
}

// Position of entry m of a rest at `base`: base XOR the entry's swizzled bits.
// From step bit 8 on the entry bits lie above the swizzle's source bits and
// the base is zero at their positions, so the XOR is an addition of a
// compile-time constant (which the shared-memory load and store take as
// their immediate offset).
template <int OFF, bool ADD>
__device__ __forceinline__ int entry_at(int base) {
    if constexpr (ADD) return base + OFF;
    else return base ^ OFF;
}

// Factor weights of the D qubits of column c for class (lx, lz), stored in
// the slot order Wp[u0 + 2 v0] of the dense steps (u0 = alpha_r ^ beta_{r+1},
// v0 = alpha_{r+1} ^ beta_r; the two exchange roles at odd plaquette parity).
// Representative E = f(s) X_L^{lx} Z_L^{lz}: Z_L is Z on row 0, X_L is X on
// column d-1 (it differs from X on column 0 by X-type stabilisers).
template <int D>
__device__ __forceinline__ void qubit_weights(const DenseArgs& a, int64_t b, int q, int lx, int lz, float* wts) {
    int x = 0, z = 0;
    const uint64_t* mk = a.dmask + (size_t)q * 2 * a.words;
    for (int w = 0; w < a.words; ++w) {
        const uint64_t sw = a.syn[b * a.words + w];
        x ^= __popcll(sw & mk[w]) & 1;
        z ^= __popcll(sw & mk[a.words + w]) & 1;
    }
    if (lx && q % D == D - 1) x ^= 1;
    if (lz && q < D) z ^= 1;
    float row[4];
    if (a.noise_mode == MLD_NOISE_TABLE) {
        const float4 p = *reinterpret_cast<const float4*>(a.noise + 4 * (size_t)q);
        row[0] = p.x; row[1] = p.y; row[2] = p.z; row[3] = p.w;   // I, X, Y, Z
    } else {
        const float p = a.noise[b];
        row[0] = 1.f - p;
        row[1] = row[2] = row[3] = p * (1.f / 3.f);
    }
    const bool par = ((q / D + q % D) & 1) != 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int uv = par ? ((j & 1) << 1) | (j >> 1) : j;
        const int xx = x ^ (uv & 1), zz = z ^ (uv >> 1);
        wts[4 * q + j] = row[xx ? (zz ? 2 : 1) : (zz ? 3 : 0)];
    }
}

// Rest r_live of a step whose rest bits in `dead` are held at zero: r_live
// with a zero inserted at every set bit of `dead` (ascending).
__device__ __forceinline__ int expand_rest(int r_live, int dead) {
    for (int m = dead; m; m &= m - 1) {
        const int b = __ffs(m) - 1;
        r_live = ((r_live >> b) << (b + 1)) | (r_live & ((1 << b) - 1));
    }
    return r_live;
}

// Index bits of a pair step at factor r of column c that stay outside the
// step (rest bits) and carry an absent plaquette: a beta bit (0..r-1) of an
// absent plaquette of corner column c+1, whose entries the column's end
// discards, or an alpha bit (r+3..d) of an absent plaquette of corner column
// c, whose entries are zero until the factor that sums it out. Rests with
// such a bit set are skipped: the dead ones keep stale values nobody reads,
// the zero ones stay zero. Returned as rest bits (index bit i < r is rest bit
// i, index bit i > r+2 is rest bit i-3).
template <int D>
__host__ __device__ __forceinline__ int dead_pair_rest_bits(int r, int pa, int pb) {
    constexpr int FULL = (1 << (D + 1)) - 1;
    const int low = (1 << r) - 1;
    const int idx_hi = ~pa & FULL & ~((1 << (r + 3)) - 1);
    return (~pb & low) | ((idx_hi >> (r + 3)) << r);
}

// Pair step (R, R+1) of column c, in place on the live rests.
template <int D, int R, int M>
__device__ __forceinline__ constexpr int pair_off() {
    return sphys((M & 1) * (1 << R) + ((M >> 1) & 1) * (2 << R) + ((M >> 2) & 1) * (4 << R) +
                 (M >> 3) * DenseShape<D>::HALF);
}

template <int D, int R, int... Ms>
__device__ __forceinline__ void pair_step(float* S, const float* wts, int c, int tid, int pa, int pb,
                                          std::integer_sequence<int, Ms...>) {
    using Sh = DenseShape<D>;
    constexpr bool ADD = R >= 8;
    float W0[4], W1[4];
    factor_weights<D>(wts, R, c, W0);
    factor_weights<D>(wts, R + 1, c, W1);
    const int dead = dead_pair_rest_bits<D>(R, pa, pb);
    const int live = Sh::REST2 >> __popc(dead);
    for (int k = tid; k < live; k += Sh::NT) {
        const int rs = expand_rest(k, dead);
        const int base = sphys((rs & ((1 << R) - 1)) | ((rs >> R) << (R + 3)));
        float X[16] = {S[entry_at<pair_off<D, R, Ms>(), ADD>(base)]...};
        float Y[16], Z[16];
        pair_first(X, W0, Y);
        pair_second(Y, W1, Z);
        ((S[entry_at<pair_off<D, R, Ms>(), ADD>(base)] = Z[Ms]), ...);
    }
    __syncthreads();
}

template <int D, int... Is>
__device__ __forceinline__ void pair_steps(float* S, const float* wts, int c, int tid, int pa, int pb,
                                           std::integer_sequence<int, Is...>) {
    (pair_step<D, 2 * Is>(S, wts, c, tid, pa, pb, std::make_integer_sequence<int, 16>{}), ...);
}

// The single factor D-1 of column c, in place on the live rests.
template <int D, int K>
__device__ __forceinline__ constexpr int single_off() {
    constexpr int R = D - 1;
    return sphys((K & 1) * (1 << R) + ((K >> 1) & 1) * (2 << R) + (K >> 2) * DenseShape<D>::HALF);
}

template <int D, int... Ks>
__device__ __forceinline__ void single_step(float* S, const float* wts, int c, int tid, int pb,
                                            std::integer_sequence<int, Ks...>) {
    using Sh = DenseShape<D>;
    constexpr int R = D - 1;
    constexpr bool ADD = R >= 8;
    float W[4];
    factor_weights<D>(wts, R, c, W);
    // the rest bits are beta_0..beta_{d-2}; dead where the plaquette is absent
    const int dead = ~pb & ((1 << R) - 1);
    const int live = Sh::REST1 >> __popc(dead);
    for (int k = tid; k < live; k += Sh::NT) {
        const int base = sphys(expand_rest(k, dead));
        const float x[8] = {S[entry_at<single_off<D, Ks>(), ADD>(base)]...};   // x[b | a'<<1 | a<<2]
        float y[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {   // j = b | b'<<1 | a'<<2
            const int bb = j & 1, bp = (j >> 1) & 1, ap = j >> 2, i0 = bb | (ap << 1);
            y[j] = fmaf(x[i0], W[jw(0, ap, bb, bp)], x[i0 | 4] * W[jw(1, ap, bb, bp)]);
        }
        ((S[entry_at<single_off<D, Ks>(), ADD>(base)] = y[Ks]), ...);
    }
    __syncthreads();
}

// The D qubit factors of column c applied in place to the state S: pairs
// (r, r+1) for even r, then the single factor D-1, on the rests that hold
// live entries (every step's offsets are compile-time constants).
template <int D>
__device__ __forceinline__ void column_in_place(float* S, const float* wts, int c, int tid) {
    const int pa = present_rows<D>(c), pb = present_rows<D>(c + 1);
    pair_steps<D>(S, wts, c, tid, pa, pb, std::make_integer_sequence<int, (D - 1) / 2>{});
    single_step<D>(S, wts, c, tid, pb, std::make_integer_sequence<int, 8>{});
}

template <int D>
__global__ void __launch_bounds__(DenseShape<D>::NT, DenseShape<D>::MINB) dense_exact_kernel(DenseArgs a) {
    using Sh = DenseShape<D>;
    constexpr int N = Sh::N, HALF = Sh::HALF, SIZE = Sh::SIZE, NT = Sh::NT, NW = Sh::NW;
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* wts = sm + Sh::off_w;
    float* S = sm + Sh::off_s;
    float* R = sm + Sh::off_r;
    float* misc = sm + Sh::off_misc;
    const int tid = threadIdx.x;

    for (int64_t unit = blockIdx.x; unit < 2 * a.B; unit += gridDim.x) {
        const int64_t b = unit >> 1;
        const int lz = (int)(unit & 1);
        for (int q = tid; q < N; q += NT) qubit_weights<D>(a, b, q, 0, lz, wts);
        {
            const int pm0 = present_rows<D>(0);
            for (int e = tid; e < SIZE; e += NT) S[sphys(e)] = (left_index<D>(e) & ~pm0) == 0 ? 1.f : 0.f;
        }
        __syncthreads();
        int eL = 0;
        bool dead = false;
        // columns 0..d-2, shared by l_X = 0, 1; the corner state after column
        // d-2 stays in R
#pragma unroll 1
        for (int c = 0; c + 1 < D; ++c) {
            column_in_place<D>(S, wts, c, tid);
            const int pmn = present_rows<D>(c + 1);
            float tmax = 0.f;
            for (int bi = tid; bi < HALF; bi += NT) {
                const float v = (bi & ~pmn) == 0 ? S[sphys(bi)] + S[sphys(bi | HALF)] : 0.f;
                R[bi] = v;
                tmax = fmaxf(tmax, v);
            }
            const float m = block_max_nonneg<NW>(tmax, misc, tid);
            if (!(m > 0.f) || !(m < INFINITY)) {
                dead = true;
                if (!(m == 0.f) && tid == 0) atomicOr(a.status, 1 << MLD_ERR_NUMERIC);
                break;
            }
            int ex = 0;
            const float s = inv_pow2_of(m, &ex);
            eL += ex;
            if (c + 2 < D) {
                for (int e = tid; e < SIZE; e += NT) S[sphys(e)] = R[left_index<D>(e)] * s;
            } else {
                for (int bi = tid; bi < HALF; bi += NT) R[bi] *= s;
            }
            __syncthreads();
        }
        // the last column once per l_X from the corner state after column d-2
#pragma unroll 1
        for (int lx = 0; lx < 2; ++lx) {
            double lnz = -INFINITY;
            if (!dead) {
                if (lx == 1) {
                    for (int r = tid; r < D; r += NT) qubit_weights<D>(a, b, r * D + D - 1, 1, lz, wts);
                    __syncthreads();
                }
                for (int e = tid; e < SIZE; e += NT) S[sphys(e)] = R[left_index<D>(e)];
                __syncthreads();
                column_in_place<D>(S, wts, D - 1, tid);
                const int pmd = present_rows<D>(D);
                float tsum = 0.f;
                for (int bi = tid; bi < HALF; bi += NT)
                    tsum += (bi & ~pmd) == 0 ? S[sphys(bi)] + S[sphys(bi | HALF)] : 0.f;
                const float total = block_sum<NW>(tsum, misc, tid);
                if (!(total == total) || !(total < INFINITY)) {
                    if (tid == 0) atomicOr(a.status, 1 << MLD_ERR_NUMERIC);
                } else if (total > 0.f) {
                    lnz = log((double)total) + (double)eL * 0.69314718055994530942;
                }
            }
            if (tid == 0) a.logP[b * 4 + lx + 2 * lz] = lnz;
            __syncthreads();
        }
    }
}

template <int D>
int64_t blocks_d(int sms, int64_t B) {
    using Sh = DenseShape<D>;
    const size_t bytes = (size_t)Sh::floats * sizeof(float);
    if (cudaFuncSetAttribute(dense_exact_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_exact_kernel<D>, Sh::NT, bytes) !=
            cudaSuccess ||
        per_sm < 1)
        return 0;
    int64_t nb = (int64_t)sms * per_sm;
    if (nb > 2 * B) nb = 2 * B;
    return nb < 1 ? 1 : nb;
}

template <int D>
bool launch_d(const DenseArgs& a, int sms, cudaStream_t s) {
    const int64_t blocks = blocks_d<D>(sms, a.B);
    if (blocks < 1 || blocks > 0x7fffffff) return false;
    dense_exact_kernel<D><<<(unsigned)blocks, DenseShape<D>::NT, (size_t)DenseShape<D>::floats * sizeof(float), s>>>(a);
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace

bool dense_exact_supported(int d) { return d == 9 || d == 11 || d == 13; }

template <int D>
double flops_d() {
    // per (syndrome, l_Z): columns 0..d-2 once and column d-1 twice; 96 flops
    // per live rest of a pair step (two factors over sixteen entries, a fused
    // multiply-add and a multiply each) and 24 per live rest of the single step
    using Sh = DenseShape<D>;
    auto rows = [](int j) {
        int m = 0;
        for (int i = 0; i <= D; ++i) m |= plaquette_is_check(D, i, j) ? 1 << i : 0;
        return m;
    };
    double total = 0.0;
    for (int c = 0; c < D; ++c) {
        const int pa = rows(c), pb = rows(c + 1);
        double col = 0.0;
        for (int r = 0; r + 1 < D; r += 2)
            col += 96.0 * (Sh::REST2 >> __builtin_popcount(dead_pair_rest_bits<D>(r, pa, pb)));
        col += 24.0 * (Sh::REST1 >> __builtin_popcount(~pb & ((1 << (D - 1)) - 1)));
        total += (c == D - 1 ? 2.0 : 1.0) * col;
    }
    return 2.0 * total;
}

double dense_exact_flops_per_syndrome(int d) {
    switch (d) {
        case 9: return flops_d<9>();
        case 11: return flops_d<11>();
        case 13: return flops_d<13>();
    }
    return 0.0;
}

bool launch_dense_exact(int d, const DenseArgs& a, cudaStream_t s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    switch (d) {
        case 9: return launch_d<9>(a, sms, s);
        case 11: return launch_d<11>(a, sms, s);
        case 13: return launch_d<13>(a, sms, s);
    }
    return false;
}

}  // namespace mld
