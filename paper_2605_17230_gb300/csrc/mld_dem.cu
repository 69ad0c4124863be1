// Detector-picture MLD of a code-capacity error model (Sec. 3.2.2), d = 3..9.
//
// The model is a list of independent error mechanisms, each a Pauli on one
// qubit with its own probability. The detector picture sums over all error
// configurations and restricts them with parity constraints instead of
// enumerating a coset (the generator picture): Z_l(s) is the contraction of
// qubit tensors (the local contraction of the qubit's mechanism tensors
// diag(1 - p, p): the qubit's Pauli distribution), one parity tensor
// delta(XOR of incident bits = s_j) per detector, and two logical parity
// tensors.
//
// Layout on the grid: detectors are the plaquettes (i, j), qubit (r, c)
// touches the four around it. The sweep runs over qubit columns c and, within
// a column, rows r. Each detector's parity tensor is decomposed into a chain
// of two-input XORs along the sweep: the boundary state holds one partial
// parity per open detector, and a detector's delta is applied the moment its
// last qubit has been absorbed. The network is planar, so no passing tensors
// are needed. The logical parities (the x-bits on Z_L's support, row 0; the
// z-bits on X_L's support, column 0) are carried as two more state bits, so
// one sweep gives Z for all four observable values at once; the class l of
// E_{l,s} = f(s) X_L^{l_X} Z_L^{l_Z} reads the value obs(f(s)) xor (l_X, l_Z).
//
// State before qubit (r, c), bit positions of a (d+4)-bit index: 0..r-1 the
// finished partial parities g_0..g_{r-1} of corner column c+1 (all of column
// c's contributions in), r the partial parity g_r (from qubit (r-1, c)),
// r+1..d the parities f_{r+1}..f_d of corner column c (from column c-1),
// d+1 the parity f_r (which qubit (r, c) completes), d+2 and d+3 the two
// observables. Qubit (r, c) sums over its Pauli e: f_r ^ bit(e) must equal
// s(r, c) (the delta), f_{r+1} and g_r take bit(e), and g_{r+1} starts at
// bit(e); afterwards position r+1 holds g_{r+1} and d+1 holds f_{r+1}. With
// every detector complete after its last qubit, the contraction is exact
// (untruncated; the dense state is the boundary MPS at full bond dimension).
// Entries stay non-negative, so FP32 keeps relative accuracy; each column is
// rescaled by a power of two and ln Z accumulates the exponents in FP64.
#include <math.h>
#include <stdint.h>

#include <vector>

#include "mld_checks.h"
#include "mld_dem.h"

namespace mld {
namespace {

constexpr int kDemMaxD = 11;

struct DemParams {
    float P[kDemMaxD * kDemMaxD][4];                       // per qubit: Pr(E_q = e), e = x + 2z
    int16_t face_stab[(kDemMaxD + 1) * (kDemMaxD + 1)];    // [j (d+1) + i]: stabiliser of face (i, j), or -1
};

struct DemArgs {
    const uint64_t* dmask;     // [n][2][words]
    const uint64_t* syn;       // [B][words]
    double* logP;              // [B][4]
    uint8_t* argmax;           // [B] or nullptr
    int64_t B;
    int words;
};

template <int D>
struct DemShape {
    static constexpr int N = D * D;
    static constexpr int HALF = 1 << (D + 1);
    static constexpr int SIZE = 1 << (D + 4);
    static constexpr int SP = D + 1, OXP = D + 2, OZP = D + 3;   // spare and observable positions
    // d = 11: the 128 KB state fills a block's shared memory; one block of
    // 512 threads per SM
    static constexpr int NT = D >= 11 ? 512 : (D >= 9 ? 128 : (D >= 7 ? 64 : 32));
    static constexpr int NW = NT / 32;
    static constexpr int NF = (D + 1) * (D + 1);
    static constexpr int off_f = 0, off_sf = SIZE, off_misc = off_sf + ((NF + 3) & ~3);   // one state, updated in place
    static constexpr int PER = SIZE / NT;                           // entries per thread in a column transition
    static constexpr int floats = off_misc + 32;
    static constexpr int FIT = (227 * 1024) / (floats * 4 + 1024);
    // keep room for ~96 registers a thread at d = 9 (fewer spill there), ~84 below
    static constexpr int REGS = 65536 / (NT * (D >= 11 ? 128 : (D >= 9 ? 96 : 84)));
    static constexpr int MINB = FIT < REGS ? (FIT < 16 ? FIT : 16) : (REGS < 16 ? REGS : 16);
};

__host__ __device__ constexpr bool dem_face_present(int d, int i, int j) { return plaquette_is_check(d, i, j); }

// Bit that Pauli code e (x + 2z) contributes to face (i, j): X-type faces
// ((i + j) even) detect z, Z-type faces detect x; absent faces nothing.
__host__ __device__ constexpr int dem_face_bit(int d, int i, int j, int e) {
    return !dem_face_present(d, i, j) ? 0 : (((i + j) & 1) == 0 ? (e >> 1) & 1 : e & 1);
}

// Shared-memory position of entry e of the state (d >= 7). Every step
// updates its rests' entries in place, so one layout serves the whole sweep.
// The 32 lanes of a warp own 32 consecutive rests, i.e. vary the five lowest
// index bits the step leaves fixed; where a step touches bank bits (0..4),
// bits 5, 6 and 7 are XORed into the bank bits (masks 9, 18 and 28) so that
// the lane -> bank map is a bijection for every step pattern of the sweep:
// column 0's row 0 and its pairs of odd rows, the other columns' pairs of
// even rows and their last row.
template <int D>
__device__ __forceinline__ int dem_phys(int e) {
    if (D < 7) return e;
    return e ^ (((e >> 5) & 1) ? 9 : 0) ^ (((e >> 6) & 1) ? 18 : 0) ^ (((e >> 7) & 1) ? 28 : 0);
}

// Insert a zero bit at position p (positions must be inserted in ascending order).
__device__ __forceinline__ constexpr int insert_zero(int x, int p) { return (x & ((1 << p) - 1)) | ((x >> p) << (p + 1)); }
__device__ __forceinline__ constexpr int lbit(int l) { return l >= 0 ? 1 << l : 0; }

// Qubit (R, c) on entries held in registers. Local bit LA holds g_R, LB
// f_{R+1}, LS the spare f_R, LOX / LOZ the observables (-1 if the qubit does
// not feed them); other local bits pass through. Afterwards LA holds g_R,
// LB g_{R+1} and LS f_{R+1}. CR is a column of the same kind as c (face
// presence and types are compile-time); sr is the syndrome bit of face (R, c).
template <int D, int CR, int R, int NE, int LA, int LB, int LS, int LOX, int LOZ>
__device__ __forceinline__ void qubit_apply(const float (&in)[NE], float (&out)[NE], const float (&w)[4], int sr) {
    constexpr int MS = 1 << LS;
    constexpr int MASK = lbit(LA) | lbit(LB) | MS | lbit(LOX) | lbit(LOZ);
    // the delta on f_R: the input's spare bit must be sr ^ bit(e);
    // v1[li] / v0[li] is the entry (spare bit of li clear) whose spare bit is sr ^ 1 / sr
    float v0[NE], v1[NE];
#pragma unroll
    for (int li = 0; li < NE; ++li) {
        if (li & MS) continue;
        v0[li] = sr ? in[li | MS] : in[li];
        v1[li] = sr ? in[li] : in[li | MS];
    }
#pragma unroll
    for (int lo = 0; lo < NE; ++lo) {
        const int gr = (lo >> LA) & 1, gr1 = (lo >> LB) & 1, fr1 = (lo >> LS) & 1;
        const int ox = LOX >= 0 ? (lo >> (LOX >= 0 ? LOX : 0)) & 1 : 0;
        const int oz = LOZ >= 0 ? (lo >> (LOZ >= 0 ? LOZ : 0)) & 1 : 0;
        const int base = lo & ~MASK;
        float acc = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (dem_face_bit(D, R + 1, CR + 1, e) != gr1) continue;        // g_{R+1} starts at bit(e)
            const int src = base | ((gr ^ dem_face_bit(D, R, CR + 1, e)) << LA) |     // g_R
                            ((fr1 ^ dem_face_bit(D, R + 1, CR, e)) << LB) |            // f_{R+1}
                            (LOX >= 0 ? (ox ^ (e & 1)) << (LOX >= 0 ? LOX : 0) : 0) |
                            (LOZ >= 0 ? (oz ^ (e >> 1)) << (LOZ >= 0 ? LOZ : 0) : 0);
            acc = fmaf(w[e], dem_face_bit(D, R, CR, e) ? v1[src] : v0[src], acc);
        }
        out[lo] = acc;
    }
}

template <int KIND>
__device__ __forceinline__ constexpr int kind_column(int d) { return KIND == 0 ? 0 : KIND == 1 ? 2 : KIND == 2 ? 1 : d - 1; }

// Single qubit step R of a column of kind KIND (0 = column 0, 1 = interior
// even, 2 = interior odd, 3 = column d-1), in place: local bits 0 = position
// R, 1 = R+1, 2 = spare, then the observables the qubit feeds.
template <int D, int KIND, int R>
__device__ __forceinline__ void dem_single(float* __restrict__ F, const float (&w)[4], int sr, int tid) {
    using S = DemShape<D>;
    constexpr int CR = kind_column<KIND>(D);
    constexpr bool OX = R == 0, OZ = KIND == 0;
    constexpr int T = 3 + (OX ? 1 : 0) + (OZ ? 1 : 0), NE = 1 << T;
    constexpr int REST = S::SIZE >> T;
    constexpr int L3 = OX ? 3 : -1, L4 = OZ ? (OX ? 4 : 3) : -1;
    for (int rs = tid; rs < REST; rs += S::NT) {
        int core = insert_zero(insert_zero(insert_zero(rs, R), R + 1), S::SP);
        if (OX) core = insert_zero(core, S::OXP);
        if (OZ) core = insert_zero(core, S::OZP);
        const int base = dem_phys<D>(core);
        int o[NE];
        float in[NE], out[NE];
#pragma unroll
        for (int li = 0; li < NE; ++li) {
            const int off = ((li & 1) << R) | (((li >> 1) & 1) << (R + 1)) | (((li >> 2) & 1) << S::SP) |
                            (OX ? ((li >> 3) & 1) << S::OXP : 0) | (OZ ? ((li >> (OX ? 4 : 3)) & 1) << S::OZP : 0);
            o[li] = base ^ dem_phys<D>(off);
            in[li] = F[o[li]];
        }
        qubit_apply<D, CR, R, NE, 0, 1, 2, L3, L4>(in, out, w, sr);
#pragma unroll
        for (int lo = 0; lo < NE; ++lo) F[o[lo]] = out[lo];
    }
}

// Qubits R and R+1 of a column in one pass, in place: local bits 0 =
// position R, 1 = R+1, 2 = R+2, 3 = spare, 4 = the observable the rows feed
// (Z_L's x-parity on row 0 of columns 1..d-1; X_L's z-parity on every row of
// column 0, where the pairs start at row 1).
template <int D, int KIND, int R>
__device__ __forceinline__ void dem_pair(float* __restrict__ F, const float (&w0)[4], const float (&w1)[4], int s0,
                                         int s1, int tid) {
    using S = DemShape<D>;
    constexpr int CR = kind_column<KIND>(D);
    constexpr bool OZ = KIND == 0, OX = !OZ && R == 0;
    constexpr int POS4 = OZ ? S::OZP : S::OXP;
    constexpr int T = 4 + ((OX || OZ) ? 1 : 0), NE = 1 << T;
    constexpr int REST = S::SIZE >> T;
    for (int rs = tid; rs < REST; rs += S::NT) {
        int core = insert_zero(insert_zero(insert_zero(insert_zero(rs, R), R + 1), R + 2), S::SP);
        if (T == 5) core = insert_zero(core, POS4);
        const int base = dem_phys<D>(core);
        int o[NE];
        float in[NE], mid[NE], out[NE];
#pragma unroll
        for (int li = 0; li < NE; ++li) {
            const int off = ((li & 1) << R) | (((li >> 1) & 1) << (R + 1)) | (((li >> 2) & 1) << (R + 2)) |
                            (((li >> 3) & 1) << S::SP) | (T == 5 ? ((li >> 4) & 1) << POS4 : 0);
            o[li] = base ^ dem_phys<D>(off);
            in[li] = F[o[li]];
        }
        qubit_apply<D, CR, R, NE, 0, 1, 3, OX ? 4 : -1, OZ ? 4 : -1>(in, mid, w0, s0);
        qubit_apply<D, CR, R + 1, NE, 1, 2, 3, -1, OZ ? 4 : -1>(mid, out, w1, s1);
#pragma unroll
        for (int lo = 0; lo < NE; ++lo) F[o[lo]] = out[lo];
    }
}

template <int D>
__device__ __forceinline__ void qubit_weights(const DemParams& prm, int r, int c, float (&w)[4]) {
    const float* pq = prm.P[r * D + c];
    w[0] = pq[0]; w[1] = pq[1]; w[2] = pq[2]; w[3] = pq[3];
}

// Column 0: row 0 alone (it feeds both observables), then pairs of rows.
template <int D, int R>
__device__ __forceinline__ void dem_column0(float* F, const DemParams& prm, const int* sf, int tid) {
    if constexpr (R == 0) {
        float w[4];
        qubit_weights<D>(prm, 0, 0, w);
        dem_single<D, 0, 0>(F, w, sf[0], tid);
        __syncthreads();
        dem_column0<D, 1>(F, prm, sf, tid);
    } else if constexpr (R + 1 < D) {
        float w0[4], w1[4];
        qubit_weights<D>(prm, R, 0, w0);
        qubit_weights<D>(prm, R + 1, 0, w1);
        dem_pair<D, 0, R>(F, w0, w1, sf[R], sf[R + 1], tid);
        __syncthreads();
        dem_column0<D, R + 2>(F, prm, sf, tid);
    }
}

// Columns 1..d-1: pairs of rows, then the last row alone.
template <int D, int KIND, int R>
__device__ __forceinline__ void dem_column(float* F, const DemParams& prm, const int* sf, int c, int tid) {
    if constexpr (R + 1 < D) {
        float w0[4], w1[4];
        qubit_weights<D>(prm, R, c, w0);
        qubit_weights<D>(prm, R + 1, c, w1);
        dem_pair<D, KIND, R>(F, w0, w1, sf[c * (D + 1) + R], sf[c * (D + 1) + R + 1], tid);
        __syncthreads();
        dem_column<D, KIND, R + 2>(F, prm, sf, c, tid);
    } else if constexpr (R < D) {
        float w[4];
        qubit_weights<D>(prm, R, c, w);
        dem_single<D, KIND, R>(F, w, sf[c * (D + 1) + R], tid);
        __syncthreads();
    }
}

template <int NW>
__device__ __forceinline__ float dem_block_max(float v, float* misc, int tid) {
    unsigned u = __reduce_max_sync(0xffffffffu, __float_as_uint(v));   // v >= 0 (NaN wins)
    if ((tid & 31) == 0) misc[tid >> 5] = __uint_as_float(u);
    __syncthreads();
    u = __float_as_uint(misc[0]);
#pragma unroll
    for (int w = 1; w < NW; ++w) u = max(u, __float_as_uint(misc[w]));
    return __uint_as_float(u);
}

template <int D>
__global__ void __launch_bounds__(DemShape<D>::NT, DemShape<D>::MINB) dem_dense_kernel(DemArgs a, const __grid_constant__ DemParams prm) {
    using S = DemShape<D>;
    constexpr int N = S::N, HALF = S::HALF, SIZE = S::SIZE, NT = S::NT, NW = S::NW;
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    float* F = sm + S::off_f;
    int* sf = reinterpret_cast<int*>(sm + S::off_sf);     // syndrome bit of face (i, j) at j (d+1) + i
    float* misc = sm + S::off_misc;
    const int tid = threadIdx.x;

    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        const uint64_t* sw = a.syn + b * a.words;
        for (int f = tid; f < S::NF; f += NT) {
            const int k = prm.face_stab[f];
            sf[f] = k < 0 ? 0 : (int)((sw[k >> 6] >> (k & 63)) & 1);
        }
        // observables of the pure error f(s): x-parity on row 0, z-parity on column 0
        int ox_bit = 0, oz_bit = 0;
        for (int q = tid; q < N; q += NT) {
            if (q >= D && q % D != 0) continue;
            int x = 0, z = 0;
            const uint64_t* mk = a.dmask + (size_t)q * 2 * a.words;
            for (int w = 0; w < a.words; ++w) {
                x ^= __popcll(sw[w] & mk[w]) & 1;
                z ^= __popcll(sw[w] & mk[a.words + w]) & 1;
            }
            if (q < D) ox_bit ^= x;
            if (q % D == 0) oz_bit ^= z;
        }
        const int ox0 = __syncthreads_count(ox_bit) & 1;
        const int oz0 = __syncthreads_count(oz_bit) & 1;
        // column 0 starts with every parity 0
        for (int e = tid; e < SIZE; e += NT) F[e] = 0.f;
        __syncthreads();
        if (tid == 0) F[0] = 1.f;                     // entry 0 sits at position 0
        __syncthreads();

        int eL = 0;
        bool dead = false;
        for (int c = 0; c < D; ++c) {
            if (c == 0) dem_column0<D, 0>(F, prm, sf, tid);
            else if (c == D - 1) dem_column<D, 3, 0>(F, prm, sf, c, tid);
            else if (c & 1) dem_column<D, 2, 0>(F, prm, sf, c, tid);
            else dem_column<D, 1, 0>(F, prm, sf, c, tid);
            if (c == D - 1) break;
            // the delta of face (d, c), then corner column c+1 becomes the left column:
            // position 0 = new g_0 (parity 0), 1..d = f_1..f_d, spare = f_0. A gather,
            // so every thread loads its entries, the block max is the barrier, then
            // the rescaled entries are stored.
            const int sD = sf[c * (D + 1) + D];
            float v[S::PER];
            float tmax = 0.f;
#pragma unroll
            for (int k = 0; k < S::PER; ++k) {
                const int e = tid + k * NT;
                v[k] = 0.f;
                if (!(e & 1)) {
                    const int old = (e & (HALF - 1) & ~1) | ((e >> S::SP) & 1) | (sD << S::SP) | (e & (3 << S::OXP));
                    v[k] = F[dem_phys<D>(old)];
                }
                tmax = fmaxf(tmax, v[k]);
            }
            const float m = dem_block_max<NW>(tmax, misc, tid);
            if (!(m > 0.f) || !(m < INFINITY)) { dead = true; break; }
            int ex = 0;
            frexpf(m, &ex);
            ex = ex < -126 ? -126 : (ex > 126 ? 126 : ex);
            eL += ex;
            const float s = __int_as_float((127 - ex) << 23);
#pragma unroll
            for (int k = 0; k < S::PER; ++k) F[dem_phys<D>(tid + k * NT)] = v[k] * s;
            __syncthreads();
        }
        if (tid == 0) {
            double lz[4];
            if (dead) {
                for (int l = 0; l < 4; ++l) lz[l] = -INFINITY;
            } else {
                int g = 0;
                for (int i = 0; i <= D; ++i) g |= sf[D * (D + 1) + i] << i;        // corner column d
                const int base = g | (sf[(D - 1) * (D + 1) + D] << S::SP);         // delta of face (d, d-1)
                for (int l = 0; l < 4; ++l) {
                    const int ox = ox0 ^ (l & 1), oz = oz0 ^ (l >> 1);
                    const float z = F[dem_phys<D>(base | (ox << S::OXP) | (oz << S::OZP))];
                    lz[l] = z > 0.f ? log((double)z) + (double)eL * 0.69314718055994530942 : -INFINITY;
                }
            }
            int best = 0;
            for (int l = 0; l < 4; ++l) {
                a.logP[b * 4 + l] = lz[l];
                if (lz[l] > lz[best]) best = l;
            }
            if (a.argmax) a.argmax[b] = (uint8_t)best;
        }
        __syncthreads();
    }
}

template <int D>
mld_status launch_dem(const DemArgs& a, const DemParams& prm, cudaStream_t s) {
    using S = DemShape<D>;
    const size_t bytes = (size_t)S::floats * sizeof(float);
    if (cudaFuncSetAttribute(dem_dense_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return MLD_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dem_dense_kernel<D>, S::NT, bytes) != cudaSuccess ||
        per_sm < 1)
        return MLD_ERR_CUDA;
    int64_t blocks = (int64_t)sms * per_sm;
    if (blocks > a.B) blocks = a.B;
    dem_dense_kernel<D><<<(unsigned)blocks, S::NT, bytes, s>>>(a, prm);
    return cudaGetLastError() == cudaSuccess ? MLD_OK : MLD_ERR_CUDA;
}

}  // namespace
}  // namespace mld

extern "C" mld_status mld_decode_dem(const mld_code* Cc, const int32_t* mech_qubit, const int32_t* mech_pauli,
                                     const double* mech_p, int32_t n_mech, const uint64_t* syndromes, int64_t B,
                                     double* logP, uint8_t* argmax, void* stream) {
    using namespace mld;
    NvtxRange trace("mld_decode_dem");
    mld_code* C = const_cast<mld_code*>(Cc);
    if (!C || n_mech < 0 || B < 0) return MLD_ERR_INVALID_ARG;
    if (n_mech > 0 && (!mech_qubit || !mech_pauli || !mech_p)) return MLD_ERR_INVALID_ARG;
    if (C->d > kDemMaxD) return MLD_ERR_UNSUPPORTED;
    const int d = C->d, n = C->n;
    // each qubit's Pauli distribution: independent mechanisms compose by Pauli product
    std::vector<double> dist((size_t)n * 4, 0.0);
    for (int q = 0; q < n; ++q) dist[(size_t)q * 4] = 1.0;
    for (int32_t m = 0; m < n_mech; ++m) {
        const int q = mech_qubit[m], e = mech_pauli[m];
        const double p = mech_p[m];
        if (q < 0 || q >= n || e < 1 || e > 3 || !(p >= 0.0 && p <= 1.0)) return MLD_ERR_INVALID_ARG;
        double* r = &dist[(size_t)q * 4];
        const double o[4] = {r[0], r[1], r[2], r[3]};
        for (int k = 0; k < 4; ++k) r[k] = (1.0 - p) * o[k] + p * o[k ^ e];
    }
    if (B == 0) return MLD_OK;
    if (!syndromes || !logP) return MLD_ERR_INVALID_ARG;
    mld_status st = ensure_code_device(C);
    if (st != MLD_OK) return st;
    DemParams prm;
    for (int q = 0; q < kDemMaxD * kDemMaxD; ++q)
        for (int k = 0; k < 4; ++k) prm.P[q][k] = q < n ? (float)dist[(size_t)q * 4 + k] : 0.f;
    for (int f = 0; f < (kDemMaxD + 1) * (kDemMaxD + 1); ++f) prm.face_stab[f] = -1;
    int k = 0;
    for (int j = 0; j <= d; ++j)                 // stabiliser order: present plaquettes, column-major
        for (int i = 0; i <= d; ++i)
            if (plaquette_is_check(d, i, j)) prm.face_stab[j * (d + 1) + i] = (int16_t)k++;
    if (k != C->m) return MLD_ERR_CUDA;
    DemArgs a;
    a.dmask = C->d_dmask;
    a.syn = syndromes;
    a.logP = logP;
    a.argmax = argmax;
    a.B = B;
    a.words = C->words;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (d) {
        case 3: return launch_dem<3>(a, prm, s);
        case 5: return launch_dem<5>(a, prm, s);
        case 7: return launch_dem<7>(a, prm, s);
        case 9: return launch_dem<9>(a, prm, s);
        case 11: return launch_dem<11>(a, prm, s);
    }
    return MLD_ERR_UNSUPPORTED;
}
