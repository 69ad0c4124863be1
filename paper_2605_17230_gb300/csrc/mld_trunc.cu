// Rank-adaptive boundary-MPS sweep for truncating chi on sm_103a.
//
// Sec. 3.2.1: after each column's MPO is applied, the boundary MPS is brought
// to left-canonical form (QR, left to right) and compressed right to left by
// SVDs that keep the largest singular values, at most chi of them. Here the
// kept count at every cut is k = min(chi, #{sigma_j > cutoff * sigma_1}): the
// Schmidt spectra of these boundary states fall by seven orders of magnitude
// within the first ~20 values at p ~ 0.1 (kept bonds average 3..6 at d = 17
// and 25, p = 0.12), so a fixed bond of 32..128 would carry values below FP32
// resolution through every later product. Bonds are therefore runtime values
// per unit and every product, QR and Jacobi sweep runs on the actual shapes.
//
// Both factorisations are rank-revealing: Householder QR with column
// pivoting stops once every remaining column norm is at most cutoff times the
// largest one, so a QR of the left sweep keeps only the numerically
// significant rows of R (the carry, and with it the next site's row count,
// follows the numerical rank), and the SVD of a bond matrix T is taken from
// its pivoted triangle R by one-sided Jacobi on R^T (Drmac and Veselic's
// preconditioning: the rows of a pivoted R are nearly orthogonal, so few
// sweeps settle) over r' columns instead of all of T.
//
// One warp owns one (syndrome, l_Z) unit (both l_X classes: the X_L string
// sits on column d-1, columns 0..d-2 are swept once and the last column once
// per l_X from the state they leave); warps are persistent and take units
// from a device queue. The matrices are small (tens of rows), so a warp per
// unit keeps every step warp-synchronous and many units resident per SM.
// Each site step lays its buffers out from its actual shapes in the warp's
// shared-memory arena: the incoming carry at one end, the outgoing carry at
// the other (ends alternate from step to step, so a carry is never moved),
// the work buffers in between. A step whose buffers do not fit runs in the
// unit's global spill arena instead (L2-resident). The MPS and the column's
// Householder reflectors are stored compactly in the unit's global slice
// (written once and read back once per column). A unit whose shapes exceed
// the slice's capacities goes to an overflow list that the fixed-shape kernel
// (same truncation rule) decodes afterwards.
//
// Matrices are column-major (element (r, c) at c*ld + r) so that the column
// operations of Householder QR and one-sided Jacobi read consecutive
// addresses across a warp.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mld_internal.h"
#include "mld_trunc.h"

namespace mld {
namespace trunc {

constexpr int kWarpsPerBlock = 4;         // units per block
constexpr int kMaxSweeps = 40;
constexpr float kTol = 1.0e-5f;           // pair orthogonality threshold (as the fixed-shape kernel)
constexpr float kNoise = 1.0e-8f;         // rotations moving less than this of the block are skipped
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }

// Exact quotient e / d for 0 <= e < 2^20 and 1 <= d <= 2^10 by one multiply:
// (e + 1/2) / d lies at least 1/(2d) from an integer, far beyond the float
// rounding of the product.
struct FDiv {
    int d;
    float inv;
    __device__ explicit FDiv(int d_) : d(d_), inv(1.f / (float)d_) {}
    __device__ int q(int e) const { return __float2int_rz(((float)e + 0.5f) * inv); }
};

// Odd leading dimension: the columns of a matrix walked by one lane each then
// fall into distinct shared-memory banks.
__device__ __forceinline__ int odd(int k) { return k | 1; }

// Householder QR with column pivoting, in place, of a column-major K x N
// matrix (leading dimension ld). Step j swaps the column of largest remaining
// norm into place, forms its reflector (R on and above the diagonal, the tail
// below it with v_j[j] = 1 implied, tau[j]) and applies it to the later
// columns; piv[j] is the original index of the column now at j. It stops once
// every remaining column norm is at most thr_rel times the largest initial
// one (or after min(K, N, maxr) steps) and returns the step count r. The
// reflector is formed across the warp's lanes; the later columns are updated
// one per lane (their row loops run serially, with no cross-lane reduction).
// The reflector norm is taken of the column scaled by a power of two near its
// maximum (a column far below the matrix's largest entries would lose its
// squares to underflow).
__device__ __noinline__ int qrcp(float* M, int K, int ld, int N, float* tau, int* piv, float* nrm, float thr_rel,
                                 int maxr, unsigned long long* fl) {
    const int lane = threadIdx.x & 31;
    for (int c = lane; c < N; c += 32) {
        const float* col = M + c * ld;
        float s = 0.f;
#pragma unroll 2
        for (int r = 0; r < K; ++r) s = fmaf(col[r], col[r], s);
        nrm[c] = sqrtf(s);
        piv[c] = c;
    }
    __syncwarp();
    float thr = 0.f;
    for (int c = lane; c < N; c += 32) thr = fmaxf(thr, nrm[c]);
    thr = thr_rel * warp_max(thr);
    const int steps = imin(imin(K, N), maxr);
    int r = 0;
    for (int j = 0; j < steps; ++j) {
        float best = -1.f;
        int p = j;
        for (int c = j + lane; c < N; c += 32) {
            const float v = nrm[c];
            if (v > best) { best = v; p = c; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(kFull, best, o);
            const int oi = __shfl_xor_sync(kFull, p, o);
            if (ob > best || (ob == best && oi < p)) { best = ob; p = oi; }
        }
        if (!(best > thr && best > 0.f)) break;
        r = j + 1;
        float* vj = M + j * ld;
        if (p != j) {
            float* cp = M + p * ld;
            for (int rr = lane; rr < K; rr += 32) { const float t = vj[rr]; vj[rr] = cp[rr]; cp[rr] = t; }
            if (lane == 0) {
                const float tn = nrm[j]; nrm[j] = nrm[p]; nrm[p] = tn;
                const int ti = piv[j]; piv[j] = piv[p]; piv[p] = ti;
            }
            __syncwarp();
        }
        float mx = 0.f;
        for (int rr = j + 1 + lane; rr < K; rr += 32) mx = fmaxf(mx, fabsf(vj[rr]));
        mx = warp_max(mx);
        const float x0 = vj[j];
        int ex = 0;
        frexpf(fmaxf(mx, fabsf(x0)), &ex);
        ex = ex < -125 ? -125 : (ex > 126 ? 126 : ex);
        const float sc = pow2f(-ex), isc = pow2f(ex);
        float ss = 0.f;
        for (int rr = j + 1 + lane; rr < K; rr += 32) { const float x = vj[rr] * sc; ss = fmaf(x, x, ss); }
        ss = warp_sum(ss);
        float tj = 0.f, beta = x0, scal = 0.f;
        if (mx > 0.f) {
            const float x0s = x0 * sc;
            const float betas = -copysignf(sqrtf(fmaf(x0s, x0s, ss)), x0s);
            tj = (betas - x0s) / betas;
            scal = 1.f / (x0s - betas);
            beta = betas * isc;
        }
        __syncwarp();
        if (tj != 0.f)
            for (int rr = j + 1 + lane; rr < K; rr += 32) vj[rr] = (vj[rr] * sc) * scal;
        if (lane == 0) { vj[j] = beta; tau[j] = tj; }
        __syncwarp();
        // H_j on columns j+1 .. N-1 and their norms below row j: a group of G
        // lanes per column (G the largest power of two with (N-1-j) G <= 32),
        // the rows dealt round-robin over the group, the dot product and the
        // norm summed across it by shuffles
        const int rem = N - 1 - j;
        int G = 32;
        while (G > 1 && rem * G > 32) G >>= 1;
        const int groups = 32 / G, grp = lane / G, g = lane - grp * G;
        for (int base = j + 1; base < N; base += groups) {
            const int cc = base + grp;
            const bool act = cc < N;
            float* col = M + (act ? cc : j) * ld;
            float w = 0.f;
            if (act && tj != 0.f) {
                if (g == 0) w = col[j];
                for (int rr = j + 1 + g; rr < K; rr += G) w = fmaf(vj[rr], col[rr], w);
            }
            for (int o = G >> 1; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
            float s = 0.f;
            if (act) {
                if (tj != 0.f) {
                    w *= tj;
                    if (g == 0) col[j] -= w;
                }
                for (int rr = j + 1 + g; rr < K; rr += G) {
                    const float x = tj != 0.f ? fmaf(-vj[rr], w, col[rr]) : col[rr];
                    col[rr] = x;
                    s = fmaf(x, x, s);
                }
            }
            for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            if (act && g == 0) nrm[cc] = sqrtf(s);
        }
        __syncwarp();
        if (lane == 0) *fl += 3ULL * (K - j) + 6ULL * (K - j) * (N - 1 - j);
    }
    return r;
}

// Y <- Q Y for the columns of Y (column-major, leading dimension ldy), Q =
// H_0 ... H_{nr-1} with reflectors V (column-major, leading dimension ldv,
// v_j below row j) and tau. Columns n < split use set 0 (V0, tau0, nr0), the
// others set 1. A group of G lanes per column (G the largest power of two
// with ncols G <= 32), the rows dealt round-robin over the group and each
// reflector's dot product summed across it by shuffles.
__device__ __noinline__ void apply_q(const float* V0, const float* tau0, int nr0, const float* V1,
                                     const float* tau1, int nr1, int split, int ldv, int K, float* Y, int ldy,
                                     int ncols, unsigned long long* fl) {
    const int lane = threadIdx.x & 31;
    int G = 32;
    while (G > 1 && ncols * G > 32) G >>= 1;
    const int groups = 32 / G, grp = lane / G, g = lane - grp * G;
    const int nrmax = nr0 > nr1 ? nr0 : nr1;
    for (int base = 0; base < ncols; base += groups) {
        const int n = base + grp;
        const bool act = n < ncols;
        const bool s1 = n >= split;
        const float* Vs = s1 ? V1 : V0;
        const float* ts = s1 ? tau1 : tau0;
        const int nr = act ? (s1 ? nr1 : nr0) : 0;
        float* y = Y + (act ? n : 0) * ldy;
        // every lane runs nrmax steps so that the group shuffles stay uniform;
        // lane g owns the rows r = g (mod G) in every step, so no lane reads
        // another's writes (v_j[j] = 1 is implied)
        for (int j = nrmax - 1; j >= 0; --j) {
            const bool on = j < nr && ts[j] != 0.f;
            const float* v = Vs + j * ldv;
            const int r0 = j + ((g - j) & (G - 1));
            float w = 0.f;
            if (on)
                for (int r = r0; r < K; r += G) w = fmaf(r == j ? 1.f : v[r], y[r], w);
            for (int o = G >> 1; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
            if (on) {
                w *= ts[j];
                for (int r = r0; r < K; r += G) y[r] = fmaf(r == j ? -1.f : -v[r], w, y[r]);
            }
        }
    }
    if (lane == 0) {
        // sum_j 4 (K - j) over nr reflectors, per column
        const unsigned long long f0 = 2ULL * nr0 * (2 * K - nr0 + 1), f1 = 2ULL * nr1 * (2 * K - nr1 + 1);
        const int c0 = split < ncols ? split : ncols;
        *fl += f0 * c0 + f1 * (ncols - c0);
    }
    __syncwarp();
}

// One-sided Jacobi (Hestenes) on the n columns (length L, ld L) of X,
// accumulating the rotations into W (n x n, column-major, starts at I).
// Parallel tournament order: each round rotates n/2 disjoint pairs, one group
// of G lanes per pair (G a power of two). A pair is rotated when it is not
// orthogonal to kTol and the rotation moves more than kNoise of the block's
// Frobenius norm (below that it is FP32 rounding noise, which rotations
// regenerate). Rotation parameters: Rutishauser's formulas in FP32. Returns
// false when kMaxSweeps sweeps did not settle.
__device__ __forceinline__ bool jacobi(float* X, int L, int n, float* W, unsigned long long* fl) {
    const int lane = threadIdx.x & 31;
    float f2 = 0.f;
    for (int e = lane; e < L * n; e += 32) f2 = fmaf(X[e], X[e], f2);
    const float fro = sqrtf(warp_sum(f2));
    for (int e = lane; e < n * n; e += 32) W[e] = (e % (n + 1) == 0) ? 1.f : 0.f;
    __syncwarp();
    const int nvp = n + (n & 1), npairs = nvp >> 1;
    int G = 32;
    while (G > 1 && npairs * G > 32) G >>= 1;
    const int groups = 32 / G, grp = lane / G, g = lane - grp * G;
    int ev = 0, rt = 0;                        // pair evaluations and rotations by this group leader
    bool ok = n < 2;
    for (int sweep = 0; sweep < kMaxSweeps && !ok; ++sweep) {
        int rotated = 0;
        for (int round = 0; round < nvp - 1; ++round) {
            for (int base = 0; base < npairs; base += groups) {
                const int k = base + grp;
                int p = -1, q = -1;
                if (k < npairs) {
                    if (k == 0) { p = round; q = nvp - 1; }
                    else { p = (round + k) % (nvp - 1); q = (round - k + (nvp - 1)) % (nvp - 1); }
                    if (p >= n || q >= n) p = q = -1;
                }
                float al = 0.f, be = 0.f, ga = 0.f;
                if (p >= 0) {
                    const float* xp = X + p * L;
                    const float* xq = X + q * L;
                    for (int r = g; r < L; r += G) {
                        const float a = xp[r], b = xq[r];
                        al = fmaf(a, a, al); be = fmaf(b, b, be); ga = fmaf(a, b, ga);
                    }
                }
                for (int o = G >> 1; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(kFull, al, o);
                    be += __shfl_xor_sync(kFull, be, o);
                    ga += __shfl_xor_sync(kFull, ga, o);
                }
                if (p >= 0 && g == 0) ++ev;
                if (p >= 0 && ga != 0.f && fabsf(ga) > kTol * sqrtf(al) * sqrtf(be) &&
                    fabsf(ga) > kNoise * sqrtf(fmaxf(al, be)) * fro) {
                    const float zeta = (be - al) / (2.f * ga);
                    const float az = fabsf(zeta);
                    const float t = copysignf(1.f, zeta) / (az + (az < 1e18f ? sqrtf(fmaf(az, az, 1.f)) : az));
                    const float cs = 1.f / sqrtf(fmaf(t, t, 1.f)), sn = cs * t;
                    float* xp = X + p * L;
                    float* xq = X + q * L;
                    for (int r = g; r < L; r += G) {
                        const float a = xp[r], b = xq[r];
                        xp[r] = cs * a - sn * b;
                        xq[r] = sn * a + cs * b;
                    }
                    float* wp = W + p * n;
                    float* wq = W + q * n;
                    for (int r = g; r < n; r += G) {
                        const float a = wp[r], b = wq[r];
                        wp[r] = cs * a - sn * b;
                        wq[r] = sn * a + cs * b;
                    }
                    rotated = 1;
                    if (g == 0) ++rt;
                }
                __syncwarp();
            }
        }
        ok = !__any_sync(kFull, rotated);
    }
    // flops: 6L per evaluation, 6(L + n) per rotation, from the group leaders
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ev += __shfl_xor_sync(kFull, ev, o);
        rt += __shfl_xor_sync(kFull, rt, o);
    }
    if (lane == 0) *fl += 6ULL * L * ev + 6ULL * (L + n) * rt + 2ULL * L * n;
    __syncwarp();
    return ok;
}

// Per-unit state in shared memory beside the arena.
struct Small {
    float wcol[kMaxD * 4];
    uint64_t syn[kMaxSynWords];
    int Dold[kMaxD + 2], Dnew[kMaxD + 2], Dkeep[kMaxD + 2];
    int Kr[kMaxD + 2], R0[kMaxD + 2], R1[kMaxD + 2];   // left sweep: rows, kept rank of each beta block
    int Qoff[2 * kMaxD + 4];             // reflector store offset of each site's beta blocks (this column)
    int Moff[2][kMaxD + 2];              // site offsets in the two MPS buffers
    unsigned long long fl;               // executed flops of the current unit (lane 0 adds)
};

// Placement of one site step's buffers in an arena of `cap` floats: the
// incoming carry stays at its end (bottom or top), the work buffers follow
// it, the outgoing carry goes to the other end.
struct Placement {
    float* base;
    int cap;
    const float* in;
    float* work;
    bool out_top;
    int outsz;
};

// ---------------------------------------------------------------- the unit
struct Unit {
    const TruncArgs& a;
    Small& S;
    float* arena;         // on-chip arena (a.arena floats)
    float* mps0;          // global MPS buffers (0 and 1)
    float* mps1;
    float* qst;           // global reflector store
    float* spill;         // global spill arena (a.caps.spill floats)
    int64_t b;            // syndrome
    int lz;               // class l_Z of this unit
    int e2;               // accumulated power-of-two exponent
    bool zero, bad, ovf, timeout;
    // where the carry is: arena, start, size, at the top of the arena or not
    float* cbase;
    float* cptr;
    int csize;
    int cld;              // leading dimension (rows) of the carry
    bool ctop;

    __device__ int present(int i, int j) const { return plaquette_is_check(a.d, i, j) ? 2 : 1; }

    // Lay out a step with the current carry, an outgoing carry of at most
    // `out` floats and `work` floats of buffers; the spill arena when the
    // on-chip one is too small (the carry is copied there first).
    __device__ int capof(const float* base) const { return base == arena ? a.arena : (int)a.caps.spill; }
    __device__ bool place(int out, int work, Placement& P) {
        const int lane = threadIdx.x & 31;
        // the carry's footprint: from its start to its end of the arena
        const int foot = ctop ? capof(cbase) - (int)(cptr - cbase) : csize;
        int need = foot + out + work;
        float* base = cbase;
        int cap = capof(cbase);
        if (need > cap || (cbase != arena && csize + out + work <= a.arena)) {
            need = csize + out + work;
            if (need <= a.arena) { base = arena; cap = a.arena; }
            else if (need <= a.caps.spill) {
                base = spill;
                cap = (int)a.caps.spill;
                if (lane == 0) atomicAdd(a.bond_hist, 1ULL);   // bin 0: steps run in the spill arena
            } else { ovf = true; return false; }
            if (base != cbase) {
                for (int e = lane; e < csize; e += 32) base[e] = cptr[e];
            } else {                           // same arena, carry moved to its bottom
                // (only when it sits at the top with room to spare below it)
                for (int e = lane; e < csize; e += 32) {
                    const float v = cptr[e];
                    __syncwarp();
                    base[e] = v;
                }
            }
            __syncwarp();
            cbase = base;
            cptr = base;
            ctop = false;
        }
        P.base = base;
        P.cap = cap;
        P.in = cptr;
        if (!ctop) {
            P.work = base + csize;
            P.out_top = true;
        } else {
            P.work = base + out;
            P.out_top = false;
        }
        P.outsz = out;
        return true;
    }
    // the outgoing carry: at the top of the reserved region or at the bottom
    __device__ float* out_ptr(const Placement& P) const { return P.out_top ? P.base + P.cap - P.outsz : P.base; }
    __device__ void carry_is(const Placement& P, float* ptr, int size, int ld) {
        cbase = P.base;
        cptr = ptr;
        csize = size;
        cld = ld;
        ctop = P.out_top;
    }

    // factor weights of column c's qubits: wcol[r][u + 2v] = p_q[E_q xor X^u Z^v]
    __device__ void column_weights(int c, int lx) {
        const int d = a.d, lane = threadIdx.x & 31;
        for (int r = lane; r < d; r += 32) {
            const int q = r * d + c;
            const uint64_t* mk = a.dmask + (size_t)q * 2 * a.words;
            int x = 0, z = 0;
            for (int w = 0; w < a.words; ++w) {
                x ^= __popcll(S.syn[w] & mk[w]) & 1;
                z ^= __popcll(S.syn[w] & mk[a.words + w]) & 1;
            }
            if (lz && r == 0) z ^= 1;                 // Z_L on row 0
            if (lx && c == d - 1) x ^= 1;             // X_L on column d-1
            float row[4];
            if (a.noise_mode == MLD_NOISE_TABLE) {
                const float4 v = *reinterpret_cast<const float4*>(a.noise + 4 * (size_t)q);
                row[0] = v.x; row[1] = v.y; row[2] = v.z; row[3] = v.w;
            } else {
                const float p = a.noise[b];
                row[0] = 1.f - p; row[1] = row[2] = row[3] = p * (1.f / 3.f);
            }
            for (int uv = 0; uv < 4; ++uv) {
                const int xx = x ^ (uv & 1), zz = z ^ (uv >> 1);
                S.wcol[4 * r + uv] = row[(!xx && !zz) ? 0 : (xx && !zz) ? 1 : (xx && zz) ? 2 : 3];
            }
        }
    }

    // Column c: MPO apply + pivoted QR sweep left to right, then the SVD sweep
    // right to left, MPS buffer sb -> db.
    __device__ void sweep_column(int c, int lx, int sb, int db) {
        const int d = a.d, lane = threadIdx.x & 31;
        const float* src = sb ? mps1 : mps0;
        float* dst = db ? mps1 : mps0;
        column_weights(c, lx);
        // the carry before site 0 is [1], at the bottom of the on-chip arena
        cbase = arena;
        cptr = arena;
        csize = 1;
        cld = 1;
        ctop = false;
        if (lane == 0) arena[0] = 1.f;
        __syncwarp();
        // ------------------------------------------------------ left sweep
        // The carry's rows are (beta_{i-1}, j): block 0's r0 rows, then block
        // 1's; rsplit = r0 of the previous site (beta = 0 below it).
        int K = 1, rsplit = 1, qo = 0;
        for (int i = 0; i <= d; ++i) {
            if (K > a.caps.max_rows) { ovf = true; return; }
            const int pam = i == 0 ? 1 : present(i - 1, c);
            const int pa = present(i, c), pb = present(i, c + 1);
            const int Dl = S.Dold[i], Dr = S.Dold[i + 1];
            const int ncolA = pa * Dr;
            const int ncol = i < d ? ncolA : 1;
            const int rmax = imin(K, ncol);
            const int ldM = odd(K);
            const int ldo = pb * rmax;            // rows reserved in the outgoing carry
            // work: A | M (one beta block at a time) | tau, nrm, piv, ipiv (ncol each)
            const int sA = Dl * ncolA, sM = ldM * ncol;
            Placement P;
            if (!place(ldo * ncol, sA + sM + 4 * ncol, P)) return;
            const float* C = P.in;
            const int ldC = cld;
            float* A = P.work;
            float* M = A + sA;
            float* tau = M + sM;
            float* nrm = tau + ncol;
            int* piv = reinterpret_cast<int*>(nrm + ncol);
            int* ipiv = piv + ncol;
            float* Co = out_ptr(P);
            // stage the old site (Dl x ncolA, row-major as stored)
            const float* Ag = src + S.Moff[sb][i];
            for (int e = lane; e < sA; e += 32) A[e] = Ag[e];
            __syncwarp();
            const int par = (i - 1 + c) & 1;
            const float* wq = S.wcol + 4 * (i - 1);
            const FDiv dK(K), dDr(Dr);
            int rb[2] = {0, 0};
            int E = 0;                            // common exponent of the site's blocks
            bool any = false;
            for (int bp = 0; bp < pb; ++bp) {
                // M^{b'}[kappa][col] = sum_a w(a, a', beta(kappa), b') sum_l C[kappa][a Dl + l] A[l][col]
                // (qubit (i-1, c); at i = d alpha_d is summed into the single column)
                float mx = 0.f;
                for (int e = lane; e < K * ncol; e += 32) {
                    const int col = dK.q(e), kap = e - col * K;
                    const int beta = (i == 0 || kap < rsplit) ? 0 : 1;
                    float acc = 0.f;
                    const int apLo = i < d ? dDr.q(col) : 0, apHi = i < d ? apLo + 1 : pa;
                    for (int ap = apLo; ap < apHi; ++ap) {
                        const int cA = i < d ? col : ap;      // column of A (Dr = 1 at i = d)
                        for (int al = 0; al < pam; ++al) {
                            const float* crow = C + (al * Dl) * ldC + kap;
                            float x = 0.f;
#pragma unroll 2
                            for (int l = 0; l < Dl; ++l) x = fmaf(crow[l * ldC], A[l * ncolA + cA], x);
                            float w = 1.f;
                            if (i > 0) {
                                // parity 0: u = a ^ b', v = a' ^ beta; parity 1: u = a' ^ beta, v = a ^ b'
                                const int ab = ap ^ beta, ub = al ^ bp;
                                w = par == 0 ? wq[ub + 2 * ab] : wq[ab + 2 * ub];
                            }
                            acc = fmaf(w, x, acc);
                        }
                    }
                    M[col * ldM + kap] = acc;
                    mx = fmaxf(mx, fabsf(acc));
                }
                if (lane == 0) S.fl += 2ULL * K * ncolA * pam * (Dl + 1);
                mx = warp_max(mx);
                if (!(mx < INFINITY)) { bad = true; return; }
                if (mx == 0.f) continue;          // this block is zero: no rows
                // power-of-two scaling of the block (exact), exponent kept
                int ex;
                frexpf(mx, &ex);
                if (ex > 126 || ex < -125) { bad = true; return; }
                const float sc = pow2f(-ex);
                __syncwarp();
                for (int e = lane; e < sM; e += 32) M[e] *= sc;
                __syncwarp();
                // rank-revealing QR M^{b'} = Q [R; R22] P^T, R22 dropped
                const int r = qrcp(M, K, ldM, ncol, tau, piv, nrm, a.cutoff, rmax, &S.fl);
                rb[bp] = r;
                // reflectors (leading dimension K) and taus to the store
                const int qsz = K * r + r;
                if (qo + qsz > a.caps.q) { ovf = true; return; }
                float* Q = qst + qo;
                for (int j = 0; j < r; ++j)
                    for (int row = lane; row < K; row += 32) Q[j * K + row] = M[j * ldM + row];
                for (int j = lane; j < r; j += 32) Q[K * r + j] = tau[j];
                for (int j = lane; j < ncol; j += 32) ipiv[piv[j]] = j;
                __syncwarp();
                // the block's carry rows: R[j][position of col] (upper trapezoid),
                // on the site's common power-of-two scale
                int rel = 0;
                if (!any) E = ex;
                else if (ex > E) {                // rescale the rows already written
                    for (int col = 0; col < ncol; ++col)
                        for (int row = lane; row < rb[0]; row += 32)
                            Co[col * ldo + row] = ldexpf(Co[col * ldo + row], E - ex);
                    E = ex;
                } else rel = ex - E;
                any = true;
                const int row0 = bp == 0 ? 0 : rb[0];
                for (int col = 0; col < ncol; ++col) {
                    const int jp = ipiv[col];
                    for (int j = lane; j < r; j += 32)
                        Co[col * ldo + row0 + j] = j <= jp ? ldexpf(M[jp * ldM + j], rel) : 0.f;
                }
                if (lane == 0) S.Qoff[2 * i + bp] = qo;
                qo += qsz;
                __syncwarp();
            }
            if (!any) { zero = true; return; }
            e2 += E;
            if (lane == 0) { S.Kr[i] = K; S.R0[i] = rb[0]; S.R1[i] = rb[1]; }
            __syncwarp();
            carry_is(P, Co, ldo * ncol, ldo);
            K = rb[0] + rb[1];
            rsplit = rb[0];
        }
        // ----------------------------------------------------- right sweep
        int Sr = 1, mo = 0;
        for (int i = d; i >= 0; --i) {
            const int pb = present(i, c + 1);
            const int Ki = S.Kr[i], r0 = S.R0[i], r1 = S.R1[i];
            const int N = pb * Sr;
            const int mn = imin(Ki, N);
            const int ldT = odd(Ki);
            const int kcap = imin(mn, a.chi);
            // work: T (Ki x N) | X (N x mn) | W (mn x mn) | tau, nrm, piv (N) | sig, perm (mn)
            const int sT = ldT * N, sX = N * mn, sW = mn * mn;
            Placement P;
            if (!place(i == 0 ? 0 : ldT * kcap, sT + sX + sW + 3 * N + 2 * mn, P)) return;
            const float* G = P.in;
            const int ldG = cld;                  // rows (b', j): r0 + r1 of them
            float* T = P.work;
            float* X = T + sT;
            float* W = X + sX;
            float* tau = W + sW;
            float* nrm = tau + N;
            int* piv = reinterpret_cast<int*>(nrm + N);
            float* sig = reinterpret_cast<float*>(piv + N);
            int* perm = reinterpret_cast<int*>(sig + mn);
            // T^{b'} = Q^{b'} [G^{b'}; 0]: block b' of G is rows [b' r0, b' r0 + r_b')
            for (int n = 0; n < N; ++n) {
                const int bp = n >= Sr ? 1 : 0, s = n - bp * Sr;
                const int rr = bp ? r1 : r0, off = bp ? r0 : 0;
                for (int kap = lane; kap < Ki; kap += 32) T[n * ldT + kap] = kap < rr ? G[s * ldG + off + kap] : 0.f;
            }
            __syncwarp();
            {
                const float* Q0 = qst + S.Qoff[2 * i];
                const float* Q1 = qst + S.Qoff[2 * i + 1];
                apply_q(Q0, Q0 + Ki * r0, r0, Q1, Q1 + Ki * r1, r1, Sr, Ki, Ki, T, ldT, N, &S.fl);
                __syncwarp();
            }
            if (i == 0) {                         // Ki = 1: the orthogonality centre is the site
                if (mo + N > a.caps.mps) { ovf = true; return; }
                float* site = dst + mo;
                for (int e = lane; e < N; e += 32) site[e] = T[e * ldT];
                if (lane == 0) { S.Dnew[0] = 1; S.Moff[db][0] = mo; }
                __syncwarp();
                break;
            }
            // T P = Q_T [R; R22], R22 dropped; Jacobi on X = R^T (N x r')
            const int rp = qrcp(T, Ki, ldT, N, tau, piv, nrm, a.cutoff, mn, &S.fl);
            if (rp == 0) { zero = true; return; }
            for (int j = 0; j < rp; ++j)
                for (int n = lane; n < N; n += 32) X[j * N + n] = j <= n ? T[n * ldT + j] : 0.f;
            __syncwarp();
            if (!jacobi(X, N, rp, W, &S.fl)) timeout = true;
            // R = W Sigma U'^T: right vectors of T = P U', left = Q_T [W; 0];
            // keep k = min(chi, #{sigma > cutoff sigma_max}) largest
            float smax = 0.f;
            for (int j = lane; j < rp; j += 32) {
                float s2 = 0.f;
                for (int rr = 0; rr < N; ++rr) s2 = fmaf(X[j * N + rr], X[j * N + rr], s2);
                sig[j] = sqrtf(s2);
                smax = fmaxf(smax, sig[j]);
            }
            smax = warp_max(smax);
            __syncwarp();
            int kept = 0;
            for (int j = lane; j < rp; j += 32) kept += (sig[j] > a.cutoff * smax && sig[j] > 0.f);
            for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(kFull, kept, o);
            const int k = imin(kept, a.chi);
            if (k == 0) { zero = true; return; }
            if (k > a.caps.max_bond || mo + k * N > a.caps.mps) { ovf = true; return; }
            for (int j = lane; j < rp; j += 32) {
                const float sj = sig[j];
                int rank = 0;
                for (int m = 0; m < rp; ++m) rank += (sig[m] > sj) || (sig[m] == sj && m < j);
                if (rank < k) perm[rank] = j;
            }
            __syncwarp();
            float* site = dst + mo;
            for (int l = 0; l < k; ++l) {
                const float inv = 1.f / sig[perm[l]];
                for (int n = lane; n < N; n += 32) site[l * N + piv[n]] = X[perm[l] * N + n] * inv;
            }
            float* Gn = out_ptr(P);
            for (int l = 0; l < k; ++l) {
                const float sg = sig[perm[l]];
                for (int kap = lane; kap < Ki; kap += 32)
                    Gn[l * ldT + kap] = kap < rp ? W[perm[l] * rp + kap] * sg : 0.f;
            }
            if (lane == 0) {
                S.Dnew[i] = k;
                S.Moff[db][i] = mo;
                atomicAdd(a.bond_hist + (k < 64 ? k : 64), 1ULL);
            }
            __syncwarp();
            apply_q(T, tau, rp, T, tau, rp, k, ldT, Ki, Gn, ldT, k, &S.fl);
            __syncwarp();
            carry_is(P, Gn, ldT * kcap, ldT);
            mo += k * N;
            Sr = k;
        }
        for (int i = lane; i <= d; i += 32) S.Dold[i] = S.Dnew[i];
        if (lane == 0) S.Dold[d + 1] = 1;
        __syncwarp();
    }

    // Contraction of the MPS (buffer db) with all-ones vectors -> ln Z (FP64)
    __device__ double contract(int db) {
        const int d = a.d, lane = threadIdx.x & 31;
        float* v = arena;                 // bonds of at most 128 (the large capacities)
        float* vn = arena + 128;
        if (lane == 0) v[0] = 1.f;
        __syncwarp();
        for (int i = 0; i <= d; ++i) {
            const int Dl = S.Dold[i], Dr = S.Dold[i + 1];
            const int p = present(i, d);                            // corner column d
            const float* site = (db ? mps1 : mps0) + S.Moff[db][i];
            for (int s = lane; s < Dr; s += 32) {
                float acc = 0.f;
                for (int l = 0; l < Dl; ++l)
                    for (int bb = 0; bb < p; ++bb) acc = fmaf(v[l], site[l * p * Dr + bb * Dr + s], acc);
                vn[s] = acc;
            }
            __syncwarp();
            float* t = v; v = vn; vn = t;
        }
        const float z = v[0];
        __syncwarp();
        if (!(z == z)) bad = true;
        return z > 0.f ? log((double)z) + (double)e2 * 0.69314718055994530942 : -INFINITY;
    }

    __device__ void run(int64_t unit) {
        const int d = a.d, lane = threadIdx.x & 31;
        b = unit >> 1;
        lz = (int)(unit & 1);
        e2 = 0;
        zero = bad = ovf = timeout = false;
        for (int w = lane; w < a.words; w += 32) S.syn[w] = a.syn[b * a.words + w];
        // all-ones product state over corner column 0 (site i: 1 x p x 1 at 2i)
        for (int i = lane; i <= d; i += 32) {
            mps0[2 * i] = 1.f;
            mps0[2 * i + 1] = 1.f;
            S.Dold[i] = 1;
            S.Moff[0][i] = 2 * i;
        }
        if (lane == 0) { S.Dold[d + 1] = 1; S.fl = 0ULL; }
        __syncwarp();
        // passes: columns 0..d-2 (l_X = 0), then column d-1 once per l_X from
        // the state after column d-2 (kept in buffer sb, its bonds in Dkeep)
        double out[2] = {-INFINITY, -INFINITY};
        int sb = 0, e2p = 0;
        for (int pass = 0; pass < d + 1; ++pass) {
            const int c = pass < d - 1 ? pass : d - 1;
            const int lx = pass == d ? 1 : 0;
            if (pass == d - 1) {                  // keep the state for the second last-column pass
                e2p = e2;
                for (int i = lane; i <= d + 1; i += 32) S.Dkeep[i] = S.Dold[i];
                __syncwarp();
            } else if (pass == d) {
                e2 = e2p;
                zero = false;
                for (int i = lane; i <= d + 1; i += 32) S.Dold[i] = S.Dkeep[i];
                __syncwarp();
            }
            sweep_column(c, lx, sb, sb ^ 1);
            __syncwarp();
            if (bad || ovf) break;
            if (pass < d - 1) {
                if (zero) break;                  // every class of this unit vanishes
                sb ^= 1;
            } else if (!zero) {
                out[pass - (d - 1)] = contract(sb ^ 1);
            }
        }
        if (lane == 0) {
            if (ovf) {
                if (a.ovf_list) {
                    const int slot = atomicAdd(a.ovf_count, 1);
                    a.ovf_list[slot] = (int64_t)unit;
                } else {
                    atomicOr(a.status, 1 << MLD_ERR_UNSUPPORTED);
                }
            } else {
                a.logP[b * 4 + 2 * lz] = out[0];
                a.logP[b * 4 + 2 * lz + 1] = out[1];
            }
            if (bad) atomicOr(a.status, 1 << MLD_ERR_NUMERIC);
            if (timeout) atomicOr(a.status, 1 << MLD_ERR_TIMEOUT);
            atomicAdd(a.flops, (double)S.fl);
        }
        __syncwarp();
    }
};

// Shared memory of one unit: Small, then the arena (16-byte aligned).
__host__ __device__ constexpr size_t small_bytes() { return (sizeof(Small) + 15) & ~size_t(15); }
__host__ __device__ constexpr size_t unit_bytes(int arena) {
    return small_bytes() + (((size_t)arena * sizeof(float) + 15) & ~size_t(15));
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock, 4) trunc_kernel(TruncArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* mine = smem_raw + (size_t)warp * unit_bytes(a.arena);
    Small& S = *reinterpret_cast<Small*>(mine);
    float* arena = reinterpret_cast<float*>(mine + small_bytes());
    const int64_t slot = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    float* base = a.ws + slot * a.caps.slice();
    const unsigned long long units = a.in_list ? (unsigned long long)*a.in_count : 2ULL * (unsigned long long)a.B;
    for (;;) {
        unsigned long long idx = 0;
        if (lane == 0) idx = atomicAdd(a.next_unit, 1ULL);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= units) break;
        Unit u{a, S, arena, base, base + a.caps.mps, base + 2 * a.caps.mps,
               base + 2 * a.caps.mps + a.caps.q};
        u.run(a.in_list ? a.in_list[idx] : (int64_t)idx);
    }
}

}  // namespace trunc

int trunc_units_per_block() { return trunc::kWarpsPerBlock; }

size_t trunc_smem_bytes(int arena) { return trunc::kWarpsPerBlock * trunc::unit_bytes(arena); }

int trunc_blocks_per_sm(int arena) {
    const size_t smem = trunc_smem_bytes(arena);
    if (cudaFuncSetAttribute(trunc::trunc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trunc::trunc_kernel, 32 * trunc::kWarpsPerBlock, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

bool launch_trunc(const TruncArgs& a, int blocks, cudaStream_t s) {
    const size_t smem = trunc_smem_bytes(a.arena);
    if (cudaFuncSetAttribute(trunc::trunc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return false;
    trunc::trunc_kernel<<<blocks, 32 * trunc::kWarpsPerBlock, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace mld
