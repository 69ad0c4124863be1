// Boundary-MPS coset contraction on sm_103a (FP32 path) and the C-ABI.
//
// One warp owns one (syndrome, l_Z) unit -- both classes l_X = 0, 1, which
// share columns 0..d-2 (see decode_unit) -- and keeps its whole state in
// shared memory: the per-qubit weights, the boundary MPS, two carry buffers
// and the Householder store. A unit runs, for every qubit column c
// (Sec. 3.2.1, boundary MPS of the generator-picture network, Eq. 7):
//   left sweep   site i = 0..d: contract carry x old site x qubit factor into
//                one block per beta_i (the MPO.MPS product), rescale by a
//                power of two, Householder-QR the block if it is tall;
//   right sweep  site i = d..0: form the bond matrix T = Q [carry; 0] and
//                factor it: identity site, dense site, or (when chi is below
//                min(rows, cols)) a one-sided Jacobi SVD that keeps the chi
//                largest singular values.
// After the last column the MPS is contracted with all-ones vectors, giving
// Z_l(s) (Eq. 3) up to the accumulated power of two; ln Z is formed in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "mld_exact.h"
#include "mld_checks.h"
#include "mld_dem.h"
#include "mld_grad.h"
#include "mld_dense.h"
#include "mld_internal.h"
#include "mld_trunc.h"

extern "C" mld_status mld_code_build_host(int d, mld_code** out);

namespace mld {

constexpr int kMaxWarpsPerBlock = 8;
constexpr int kMaxJacobiSweeps = 40;
constexpr float kJacobiTol = 1.0e-5f;   // above the ~L*eps noise floor of FP32 dot products
constexpr float kJacobiNoise = 1.0e-8f; // rotations that move less than this (relative to the block) are skipped

struct DecodeArgs {
    const SiteStep* steps;
    float* gws;                // global workspace (nullptr: shared memory)
    const uint64_t* dmask;     // [n][2][words]
    const float* noise;
    const uint64_t* syn;
    double* logP;
    int* status;
    int64_t B;
    int d, n, words, noise_mode;
    int off_w, off_mps, off_buf0, off_buf1, off_q, off_svd, per_warp;
    int init_sizes[kMaxD + 1];
    float* qgws = nullptr;     // split mode: the kept tall blocks of each resident warp in global memory
    int64_t q_per_warp = 0;    // floats per warp of qgws
    float cutoff = 0.f;        // singular values <= cutoff * sigma_1 of a bond matrix are discarded
    const int64_t* ulist = nullptr;   // global mode: decode only these units (count at *ucount)
    const int* ucount = nullptr;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// sum over aligned groups of G lanes (G a power of two <= 32)
__device__ __forceinline__ float group_sum(float v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float pow2f(int e) {   // exact 2^e for -126 <= e <= 127
    return __int_as_float((e + 127) << 23);
}

__device__ __forceinline__ float group_max(float v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// weight of qubit factor at this step: w(a, a', b, b') = p_q[E_q xor X^u Z^v]
__device__ __forceinline__ float qweight(const float* wq, int parity, int a, int ap, int b, int bp) {
    int u, v;
    if (parity == 0) { u = a ^ bp; v = ap ^ b; }
    else { u = ap ^ b; v = a ^ bp; }
    return wq[u + 2 * v];
}

// ---------------------------------------------------------------- left sweep
__device__ __forceinline__ int qdiv(int x, int n, int l, bool p2) { return p2 ? (x >> l) : (x / n); }

// Left-sweep product of one site:
//   M^{b'}[k][(a', r')] = sum_a w(a, a', beta(k), b') X_a[k][(a', r')],
//   X_a[k][col] = sum_r C[k][a*Dl + r] A[r][col].
// The bond sum collapses for identity carries (st.cid: row k = (beta, j)
// with j = a*Dl + r picks one term) and for identity old sites (K_IDR:
// r = a'*Dr + r'; K_IDL: r = r' - a'*Dl when that lies in [0, Dl)); only a
// data site with a data carry is a real GEMM. At the last site alpha_d is
// summed (Dr = 1, ncol = 1).
__device__ void apply_site(const SiteStep& st, const float* __restrict__ C,
                           const float* __restrict__ A, float* __restrict__ M,
                           const float* __restrict__ wts, int lane, bool last) {
    const int K = st.K, pam = st.pam, pa = st.pa, pb = st.pb, Dl = st.Dl, Dr = st.Dr;
    const int ncolA = pa * Dr, ncol = st.ncol, kqp = st.kq_prev, par = st.parity;
    const bool p2 = st.pow2;
    const float* wq = st.qubit >= 0 ? wts + 4 * st.qubit : nullptr;
    float wr[16];                      // w(a, a', beta, b') for this qubit, index a | a'<<1 | beta<<2 | b'<<3
#pragma unroll
    for (int m = 0; m < 16; ++m)
        wr[m] = wq ? qweight(wq, par, m & 1, (m >> 1) & 1, (m >> 2) & 1, (m >> 3) & 1) : 1.f;
    const int ldc = pam * Dl;
    const int kind = st.okind;
    if (!st.cid && kind == K_DATA && !last && (ncolA & 3) == 0 && (Dr & 3) == 0) {
        // dense GEMM, four consecutive columns per lane (they share a')
        const int q4 = ncolA >> 2, lq4 = st.lncol - 2;
        for (int tI = lane; tI < K * q4; tI += 32) {
            const int k = qdiv(tI, q4, lq4, p2), col = (tI - k * q4) * 4, ap = qdiv(col, Dr, st.lDr, p2);
            float4 t0 = make_float4(0.f, 0.f, 0.f, 0.f), t1 = t0;
            const float* c0 = C + k * ldc;
            const float* c1 = c0 + Dl;
            for (int r = 0; r < Dl; ++r) {
                const float4 av = *reinterpret_cast<const float4*>(A + r * ncolA + col);
                const float x0 = c0[r];
                t0.x = fmaf(x0, av.x, t0.x); t0.y = fmaf(x0, av.y, t0.y);
                t0.z = fmaf(x0, av.z, t0.z); t0.w = fmaf(x0, av.w, t0.w);
                if (pam == 2) {
                    const float x1 = c1[r];
                    t1.x = fmaf(x1, av.x, t1.x); t1.y = fmaf(x1, av.y, t1.y);
                    t1.z = fmaf(x1, av.z, t1.z); t1.w = fmaf(x1, av.w, t1.w);
                }
            }
            const int beta = qdiv(k, kqp, st.lkqp, p2);
            for (int bp = 0; bp < pb; ++bp) {
                const float w0 = wr[(ap << 1) | (beta << 2) | (bp << 3)];
                const float w1 = pam == 2 ? wr[1 | (ap << 1) | (beta << 2) | (bp << 3)] : 0.f;
                float4 o;
                o.x = fmaf(w0, t0.x, w1 * t1.x); o.y = fmaf(w0, t0.y, w1 * t1.y);
                o.z = fmaf(w0, t0.z, w1 * t1.z); o.w = fmaf(w0, t0.w, w1 * t1.w);
                *reinterpret_cast<float4*>(M + (bp * K + k) * ncol + col) = o;
            }
        }
        return;
    }
    // general element loop (identity kinds, identity carries, odd shapes)
    const int nout = last ? K : K * ncolA;
    for (int e = lane; e < nout; e += 32) {
        int k, col;
        if (last) { k = e; col = 0; }
        else { k = qdiv(e, ncolA, st.lncol, p2); col = e - k * ncolA; }
        const int beta = qdiv(k, kqp, st.lkqp, p2);
        const int j = k - beta * kqp;              // identity carry: j = a*Dl + r
        const int ja = st.cid ? qdiv(j, Dl, st.lDl, p2) : 0;
        const int jr = j - ja * Dl;
        float acc[2] = {0.f, 0.f};                 // per b'
        const int apLo = last ? 0 : qdiv(col, Dr, st.lDr, p2);
        const int apHi = last ? pa : apLo + 1;
        for (int ap = apLo; ap < apHi; ++ap) {
            const int rp = last ? 0 : col - ap * Dr;
            float X[2] = {0.f, 0.f};
            if (st.cid) {
                float av;
                if (kind == K_DATA) av = A[jr * ncolA + ap * Dr + rp];
                else if (kind == K_IDR) av = (jr == ap * Dr + rp) ? 1.f : 0.f;
                else av = (rp == ap * Dl + jr) ? 1.f : 0.f;
                X[ja] = av;
            } else {
                for (int a = 0; a < pam; ++a) {
                    const float* crow = C + k * ldc + a * Dl;
                    float s = 0.f;
                    if (kind == K_DATA) {
                        for (int r = 0; r < Dl; ++r) s = fmaf(crow[r], A[r * ncolA + ap * Dr + rp], s);
                    } else if (kind == K_IDR) {
                        s = crow[ap * Dr + rp];
                    } else {
                        const int r = rp - ap * Dl;
                        s = (r >= 0 && r < Dl) ? crow[r] : 0.f;
                    }
                    X[a] = s;
                }
            }
            for (int bp = 0; bp < pb; ++bp)
                acc[bp] = fmaf(wr[(ap << 1) | (beta << 2) | (bp << 3)], X[0],
                               fmaf(wr[1 | (ap << 1) | (beta << 2) | (bp << 3)], X[1], acc[bp]));
        }
        for (int bp = 0; bp < pb; ++bp) M[(bp * K + k) * ncol + col] = acc[bp];
    }
}

// Rescale M (len floats) by 2^-e with e the exponent of max|M|; returns e.
// Sets *zero when M vanishes, *bad when it is not finite.
__device__ int renormalise(float* M, int len, int lane, bool* zero, bool* bad) {
    float mx = 0.f;
    for (int e = lane; e < len; e += 32) mx = fmaxf(mx, fabsf(M[e]));
    mx = warp_max(mx);
    if (!(mx < INFINITY)) { *bad = true; return 0; }    // inf or NaN
    if (mx == 0.f) { *zero = true; return 0; }
    int ex;
    frexpf(mx, &ex);
    if (ex > 126 || ex < -125) { *bad = true; return 0; }
    const float s = pow2f(-ex);
    __syncwarp();
    for (int e = lane; e < len; e += 32) M[e] *= s;
    return ex;
}

// Householder QR of the K x n block (row-major, ld = n), K > n, in place:
// R on and above the diagonal, reflector tails below, tau[j] beside. Run by
// a group of G lanes (g = lane index in the group). LAPACK sign convention.
__device__ void qr_block(float* M, float* tau, int K, int n, int g, int G) {
    for (int j = 0; j < n; ++j) {
        // the reflector from the column scaled by a power of two near its
        // maximum: a column far below the block's largest entries (common under
        // strongly biased noise) would otherwise lose its squares to underflow,
        // and the reciprocal of a tiny norm would overflow
        float mx = 0.f;
        for (int r = j + 1 + g; r < K; r += G) mx = fmaxf(mx, fabsf(M[r * n + j]));
        mx = group_max(mx, G);
        const float x0 = M[j * n + j];
        int ex = 0;
        frexpf(fmaxf(mx, fabsf(x0)), &ex);
        ex = ex < -125 ? -125 : (ex > 126 ? 126 : ex);
        const float sc = pow2f(-ex), isc = pow2f(ex);
        float ss = 0.f;
        for (int r = j + 1 + g; r < K; r += G) { const float x = M[r * n + j] * sc; ss = fmaf(x, x, ss); }
        ss = group_sum(ss, G);
        float tj = 0.f, beta = x0, scal = 0.f;
        if (mx > 0.f) {
            const float x0s = x0 * sc;
            const float betas = -copysignf(sqrtf(fmaf(x0s, x0s, ss)), x0s);
            tj = (betas - x0s) / betas;
            scal = 1.f / (x0s - betas);                // v_r = x_r / (x0 - beta) = (x_r sc) * scal
            beta = betas * isc;
        }
        __syncwarp();
        if (tj != 0.f)
            for (int r = j + 1 + g; r < K; r += G) M[r * n + j] = (M[r * n + j] * sc) * scal;
        if (g == 0) { M[j * n + j] = beta; tau[j] = tj; }
        __syncwarp();
        if (tj != 0.f) {
            for (int cc = j + 1 + g; cc < n; cc += G) {
                float w = M[j * n + cc];
                for (int r = j + 1; r < K; ++r) w = fmaf(M[r * n + j], M[r * n + cc], w);
                w *= tj;
                M[j * n + cc] -= w;
                for (int r = j + 1; r < K; ++r) M[r * n + cc] = fmaf(-M[r * n + j], w, M[r * n + cc]);
            }
        }
        __syncwarp();
    }
}

// Y (K x S, leading dim ldy) <- Q [Y0; 0] with Q = H_0 ... H_{n-1} from qr_block.
// The caller has written Y0 into rows 0..n-1 and zeros below. Lanes of a
// group of G split the columns.
__device__ void apply_q(const float* Mq, const float* tau, int K, int n, float* Y, int ldy, int S,
                        int g, int G) {
    for (int j = n - 1; j >= 0; --j) {
        const float tj = tau[j];
        if (tj != 0.f) {
            for (int s = g; s < S; s += G) {
                float w = Y[j * ldy + s];
                for (int r = j + 1; r < K; ++r) w = fmaf(Mq[r * n + j], Y[r * ldy + s], w);
                w *= tj;
                Y[j * ldy + s] -= w;
                for (int r = j + 1; r < K; ++r) Y[r * ldy + s] = fmaf(-Mq[r * n + j], w, Y[r * ldy + s]);
            }
        }
        __syncwarp();
    }
}

// One-sided Jacobi on the nv columns (length L, ld = ldx) of X, accumulating
// the rotations into acc (nv x nv, starts at I). Rotation parameters in
// FP32 (FP64 ones, at 1/64 of the FP32 rate on this GPU, cost 30% of the
// truncated sweep at d=9..11 and changed no result beyond 1e-5 in ln Z);
// cyclic round-robin order; bounded sweeps.
// A pair (p, q) is rotated when its columns are not orthogonal to kJacobiTol
// and the rotation moves a component that matters: the mass that would stay
// in the smaller column along the larger one, gamma / sqrt(max(alpha, beta)),
// exceeds kJacobiNoise of the block's Frobenius norm. Below that the pair is
// FP32 rounding noise, which rotations only regenerate (they would not
// settle); a fixed floor on the column norms instead left small but real
// overlaps unrotated, and their truncation cost up to 1e-4 in ln Z.
// Returns false if the sweep bound was hit.
__device__ bool jacobi(float* X, int L, int ldx, int nv, float* acc, int lane) {
    float fro2 = 0.f;
    for (int e = lane; e < L * nv; e += 32) {
        const float x = X[(e / nv) * ldx + (e % nv)];
        fro2 = fmaf(x, x, fro2);
    }
    const float fro = sqrtf(warp_sum(fro2));
    for (int e = lane; e < nv * nv; e += 32) acc[e] = (e / nv == e % nv) ? 1.f : 0.f;
    __syncwarp();
    const int nvp = nv + (nv & 1);
    const int npairs = nvp / 2;
    int G = 32;
    while (G > 1 && npairs * G > 32) G >>= 1;
    const int groups = 32 / G;
    const int grp = lane / G, g = lane % G;
    for (int sweep = 0; sweep < kMaxJacobiSweeps; ++sweep) {
        int rotated = 0;
        for (int round = 0; round < nvp - 1; ++round) {
            for (int base = 0; base < npairs; base += groups) {
                const int k = base + grp;
                int p = -1, q = -1;
                if (k < npairs) {
                    if (k == 0) { p = round; q = nvp - 1; }
                    else { p = (round + k) % (nvp - 1); q = (round - k + (nvp - 1)) % (nvp - 1); }
                    if (p >= nv || q >= nv) p = q = -1;
                }
                float al = 0.f, be = 0.f, ga = 0.f;
                if (p >= 0)
                    for (int r = g; r < L; r += G) {
                        const float xp = X[r * ldx + p], xq = X[r * ldx + q];
                        al = fmaf(xp, xp, al); be = fmaf(xq, xq, be); ga = fmaf(xp, xq, ga);
                    }
                al = group_sum(al, G); be = group_sum(be, G); ga = group_sum(ga, G);
                if (p >= 0 && ga != 0.f && fabsf(ga) > kJacobiTol * sqrtf(al) * sqrtf(be) &&
                    fabsf(ga) > kJacobiNoise * sqrtf(fmaxf(al, be)) * fro) {
                    // Rutishauser's rotation in FP32 (|zeta| large: t = 1/(2 zeta))
                    const float zeta = (be - al) / (2.f * ga);
                    const float az = fabsf(zeta);
                    const float t = copysignf(1.f, zeta) / (az + (az < 1e18f ? sqrtf(fmaf(az, az, 1.f)) : az));
                    const float cs = 1.f / sqrtf(fmaf(t, t, 1.f)), sn = cs * t;
                    for (int r = g; r < L; r += G) {
                        const float xp = X[r * ldx + p], xq = X[r * ldx + q];
                        X[r * ldx + p] = cs * xp - sn * xq;
                        X[r * ldx + q] = sn * xp + cs * xq;
                    }
                    for (int r = g; r < nv; r += G) {
                        const float xp = acc[r * nv + p], xq = acc[r * nv + q];
                        acc[r * nv + p] = cs * xp - sn * xq;
                        acc[r * nv + q] = sn * xp + cs * xq;
                    }
                    rotated = 1;
                }
                __syncwarp();
            }
        }
        if (!__any_sync(0xffffffffu, rotated)) return true;
    }
    return false;
}

// ------------------------------------------------------------------ kernel
// One (syndrome, class) unit on one warp (with pair, a (syndrome, l_Z) unit
// as below), with its state at ws (shared memory, or this warp's slice of the
// global workspace); returns ln Z.
//
// pair (optional): the unit is (syndrome, l_Z) = unit >> 1, unit & 1 and both
// classes l_X = 0, 1 are decoded, ln Z into pair[0] and pair[1]. X_L is then
// taken as X on column d-1 (it differs from X on column 0 by X-type
// stabilisers, so each coset is the same); the two representatives agree on
// columns 0..d-2, which are swept once, and the last column is swept once
// per class from the state they leave (the plan stores the last column's
// sites after its old ones). At truncated chi the approximation depends on
// the representative: this one is E_{l,s} with X_L on column d-1.
__device__ __forceinline__ double decode_unit(const DecodeArgs& a, float* ws, int64_t unit, int lane,
                                              double* pair = nullptr, float* qext = nullptr) {
    const int64_t b = pair ? unit >> 1 : unit >> 2;
    const int cls = pair ? (int)(unit & 1) << 1 : (int)(unit & 3);
    const int d = a.d, n = a.n;
    float* wts = ws + a.off_w;
    float* mps = ws + a.off_mps;
    float* qst = qext ? qext : ws + a.off_q;
    float* svd = ws + a.off_svd;
    float* bufA = ws + a.off_buf0;
    float* bufB = ws + a.off_buf1;

    // pure error f(s) = prod_{s_k=1} T_k (per-qubit parity of s & mask),
    // representative E_{l,s} = f * X_L^{l_X} * Z_L^{l_Z}, factor weights
    uint64_t sw[kMaxSynWords];
    for (int w = 0; w < a.words; ++w) sw[w] = a.syn[b * a.words + w];
    for (int q = lane; q < n; q += 32) {
        int x = 0, z = 0;
        const uint64_t* mk = a.dmask + (size_t)q * 2 * a.words;
        for (int w = 0; w < a.words; ++w) {
            x ^= __popcll(sw[w] & mk[w]) & 1;
            z ^= __popcll(sw[w] & mk[a.words + w]) & 1;
        }
        const int r = q / d, c = q - r * d;
        if ((cls & 1) && c == 0) x ^= 1;
        if ((cls & 2) && r == 0) z ^= 1;
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
            const int pidx = (!xx && !zz) ? 0 : (xx && !zz) ? 1 : (xx && zz) ? 2 : 3;
            wts[4 * q + uv] = row[pidx];
        }
    }
    (void)cls;
    // initial boundary MPS: all-ones product state over corner column 0
    {
        int o = 0;
        for (int i = 0; i <= d; ++i) {
            const int sz = a.init_sizes[i];
            if (lane < sz) mps[o + lane] = 1.f;
            o += (sz + 3) & ~3;
        }
    }
    __syncwarp();

    int e2 = 0;
    bool zero = false, bad = false, timeout = false;
    auto sweep_column = [&](int c) {
        const SiteStep* S = a.steps + (size_t)c * (d + 1);
        float* cin = bufA;
        float* cout = bufB;
        // ---- left sweep
        for (int i = 0; i <= d; ++i) {
            const SiteStep st = S[i];
            const int K = st.K, ncol = st.ncol, pb = st.pb;
            float* M = st.tall ? qst + st.offQ : cout;
            apply_site(st, cin, mps + st.offA, M, wts, lane, i == d);
            __syncwarp();
            e2 += renormalise(M, pb * K * ncol, lane, &zero, &bad);
            __syncwarp();
            if (zero || bad) break;
            if (st.tall && st.canon) {
                float* tau = qst + st.offQ + pb * K * ncol;
                if (pb == 2) {
                    const int hb = lane >> 4;
                    qr_block(M + hb * K * ncol, tau + hb * ncol, K, ncol, lane & 15, 16);
                } else {
                    qr_block(M, tau, K, ncol, lane, 32);
                }
                // R blocks -> carry rows b*kq .. (kq = ncol)
                for (int e = lane; e < pb * ncol * ncol; e += 32) {
                    const int bb = e / (ncol * ncol), rem = e - bb * ncol * ncol;
                    const int j = rem / ncol, cc = rem - j * ncol;
                    cout[e] = cc >= j ? M[bb * K * ncol + j * ncol + cc] : 0.f;
                }
                __syncwarp();
            }
            float* t = cin; cin = cout; cout = t;
        }
        if (zero || bad) return;
        // ---- right sweep; carry g (rows x S), T into t. A tall last block
        // kept as the site leaves an identity carry (st.gid).
        float* g = cin;
        float* t = cout;
        for (int i = d; i >= 0; --i) {
            const SiteStep st = S[i];
            const int rows = st.K, Sr = st.S, pb = st.pb, cols = pb * Sr, kq = st.kq;
            // T^b = Q^b [G^b; 0] (canonical column), M^b G^b (tall block kept
            // as the site) or G^b (wide block, Q = I). st.gid: the incoming
            // carry is the identity, G[row][s] = [row == s]. A binary-expansion
            // identity site (K_IDL) is not formed at all.
            const int gid = st.gid;
            if (st.nkind == K_IDL) {
                // nothing to form or store; the carry stays the identity
            } else if (st.tall && !st.canon) {
                const float* Mb = qst + st.offQ;
                const int nc = st.ncol;
                for (int e = lane; e < rows * cols; e += 32) {
                    const int r = e / cols, cc = e - r * cols, bb = cc / Sr, s = cc - bb * Sr;
                    const float* mrow = Mb + (bb * rows + r) * nc;
                    float acc = 0.f;
                    if (gid == 2) {                    // G^b = I_kq
                        acc = mrow[s];
                    } else if (gid) {                  // G = I: G^b selects columns b*kq ..
                        const int j = s - bb * kq;
                        acc = (j >= 0 && j < nc) ? mrow[j] : 0.f;
                    } else {
                        const float* gcol = g + (bb * kq) * Sr + s;
                        for (int j = 0; j < nc; ++j) acc = fmaf(mrow[j], gcol[j * Sr], acc);
                    }
                    t[e] = acc;
                }
                __syncwarp();
            } else if (st.tall) {
                for (int e = lane; e < rows * cols; e += 32) {
                    const int r = e / cols, cc = e - r * cols, bb = cc / Sr, s = cc - bb * Sr;
                    const int grow = bb * kq + r;
                    t[e] = r < kq ? (gid ? (grow == s ? 1.f : 0.f) : g[grow * Sr + s]) : 0.f;
                }
                __syncwarp();
                const float* Mq = qst + st.offQ;
                const float* tau = Mq + pb * rows * st.ncol;
                if (pb == 2) {
                    const int hb = lane >> 4;
                    apply_q(Mq + hb * rows * st.ncol, tau + hb * st.ncol, rows, st.ncol,
                            t + hb * Sr, cols, Sr, lane & 15, 16);
                } else {
                    apply_q(Mq, tau, rows, st.ncol, t, cols, Sr, lane, 32);
                }
            } else {
                for (int e = lane; e < rows * cols; e += 32) {
                    const int r = e / cols, cc = e - r * cols, bb = cc / Sr, s = cc - bb * Sr;
                    const int grow = bb * rows + r;
                    t[e] = gid ? (grow == s ? 1.f : 0.f) : g[grow * Sr + s];
                }
                __syncwarp();
            }
            float* site = mps + st.offN;
            const int Sl = st.Sl;
            if (st.rmode == R_IDENT) {
                float* tmp = g; g = t; t = tmp;        // site = identity (K_IDR), carry = T
            } else if (st.rmode == R_DENSE) {
                if (st.nkind == K_DATA)                // site = T, carry = identity (implicit)
                    for (int e = lane; e < rows * cols; e += 32) site[e] = t[e];
            } else {
                // truncated SVD of T keeping Sl singular values
                const int nv = rows < cols ? rows : cols;
                float* acc = svd;
                float* sig = svd + nv * nv;
                int* perm = reinterpret_cast<int*>(sig + nv);
                const bool tallT = rows >= cols;
                float* X;
                int L;
                if (tallT) { X = t; L = rows; }
                else {
                    X = g; L = cols;                   // X = T^T (cols x rows)
                    for (int e = lane; e < rows * cols; e += 32) {
                        const int r = e / cols, cc = e - r * cols;
                        X[cc * rows + r] = t[e];
                    }
                }
                __syncwarp();
                if (!jacobi(X, L, nv, nv, acc, lane)) timeout = true;
                for (int k = lane; k < nv; k += 32) {
                    float s2 = 0.f;
                    for (int r = 0; r < L; ++r) s2 = fmaf(X[r * nv + k], X[r * nv + k], s2);
                    sig[k] = sqrtf(s2);
                }
                __syncwarp();
                // the relative cutoff: values at or below cutoff * sigma_1 are
                // discarded (their site rows and carry columns written as zero)
                float smax = 0.f;
                for (int k = lane; k < nv; k += 32) smax = fmaxf(smax, sig[k]);
                const float sfloor = a.cutoff * warp_max(smax);
                for (int k = lane; k < nv; k += 32) {
                    int rank = 0;
                    const float sk = sig[k];
                    for (int j = 0; j < nv; ++j) rank += (sig[j] > sk) || (sig[j] == sk && j < k);
                    if (rank < Sl) perm[rank] = sk > sfloor ? k : -1;
                }
                __syncwarp();
                if (tallT) {
                    // T = X V^T: site = V[:, top]^T (Sl x cols), carry = X[:, top]
                    for (int e = lane; e < Sl * cols; e += 32) {
                        const int s = e / cols, cc = e - s * cols;
                        site[e] = perm[s] >= 0 ? acc[cc * nv + perm[s]] : 0.f;
                    }
                    for (int e = lane; e < rows * Sl; e += 32) {
                        const int r = e / Sl, s = e - r * Sl;
                        g[e] = perm[s] >= 0 ? X[r * nv + perm[s]] : 0.f;
                    }
                } else {
                    // T = U X^T: site = X[:, top]^T / sigma, carry = U[:, top] sigma
                    for (int e = lane; e < Sl * cols; e += 32) {
                        const int s = e / cols, cc = e - s * cols;
                        const float sg = perm[s] >= 0 ? sig[perm[s]] : 0.f;
                        site[e] = sg > 0.f ? X[cc * nv + perm[s]] / sg : 0.f;
                    }
                    for (int e = lane; e < rows * Sl; e += 32) {
                        const int r = e / Sl, s = e - r * Sl;
                        t[e] = perm[s] >= 0 ? acc[r * nv + perm[s]] * sig[perm[s]] : 0.f;
                    }
                    float* tmp = g; g = t; t = tmp;
                }
            }
            __syncwarp();
        }
    };
    const int cend = pair ? d - 1 : d;
    for (int c = 0; c < cend && !zero && !bad; ++c) {
        sweep_column(c);
    }
    auto contract = [&]() -> double {
    double logz;
    if (zero) {
        logz = -INFINITY;
    } else {
        // contract the final MPS with all-ones vectors
        const SiteStep* S = a.steps + (size_t)(d - 1) * (d + 1);
        float* v = bufA;
        float* vn = bufB;
        if (lane == 0) v[0] = 1.f;
        __syncwarp();
        for (int i = 0; i <= d; ++i) {
            const SiteStep st = S[i];
            const float* site = mps + st.offN;
            for (int s = lane; s < st.S; s += 32) {
                float acc = 0.f;
                if (st.nkind == K_IDR) {              // A[l][b][s] = [l == b*S + s]
                    for (int bb = 0; bb < st.pb; ++bb) acc += v[bb * st.S + s];
                } else if (st.nkind == K_IDL) {       // A[l][b][s] = [s == b*Sl + l]
                    acc = v[s % st.Sl];
                } else {
                    for (int sl = 0; sl < st.Sl; ++sl)
                        for (int bb = 0; bb < st.pb; ++bb) acc = fmaf(v[sl], site[(sl * st.pb + bb) * st.S + s], acc);
                }
                vn[s] = acc;
            }
            __syncwarp();
            float* tmp = v; v = vn; vn = tmp;
        }
        const float z = v[0];
        logz = z > 0.f ? log((double)z) + (double)e2 * 0.69314718055994530942 : -INFINITY;
        if (!(z == z)) bad = true;
    }
    return logz;
    };
    double logz = 0.0;
    if (!pair) {
        logz = contract();
    } else {
        // the last column once per l_X from the state after column d-2
        const int e2p = e2;
        const bool zerop = zero, badp = bad;
        for (int lx = 0; lx < 2; ++lx) {
            e2 = e2p;
            zero = zerop;
            bad = bad || badp;
            if (lx == 1) {
                // X on column d-1: w[u + 2v] = p[E xor X^u Z^v] becomes w[(u ^ 1) + 2v]
                if (lane < d) {
                    float* w = wts + 4 * (lane * d + d - 1);
                    const float w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3];
                    w[0] = w1; w[1] = w0; w[2] = w3; w[3] = w2;
                }
                __syncwarp();
            }
            if (!zero && !bad) sweep_column(d - 1);
            pair[lx] = contract();
            __syncwarp();
        }
    }
    if (lane == 0) {
        if (bad) atomicOr(a.status, 1 << MLD_ERR_NUMERIC);
        if (timeout) atomicOr(a.status, 1 << MLD_ERR_TIMEOUT);
    }
    return logz;
}

// Shared-memory mode: one unit per warp. Global-workspace mode (a.gws set,
// for states larger than a block's shared memory): a fixed set of resident
// warps, each with its own slice of the workspace, strides over the units.
// Split mode (a.qgws set): the same persistent warps keep everything but the
// kept tall blocks in shared memory, and those blocks (the largest part of
// the state, touched only by the QR and the Q application) in their slice
// of global memory, so that more units share an SM.
template <bool GLOBAL>
__global__ void __launch_bounds__(32 * kMaxWarpsPerBlock)
decode_fp32_kernel(DecodeArgs a) {
    extern __shared__ float4 smem4[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    // unit = (syndrome, l_Z); both l_X from one sweep of columns 0..d-2
    double lz[2];
    if (!GLOBAL && a.qgws) {
        const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
        float* ws = reinterpret_cast<float*>(smem4) + (size_t)warp * a.per_warp;
        float* qx = a.qgws + (size_t)gw * a.q_per_warp;
        for (int64_t unit = gw; unit < 2 * a.B; unit += nw) {
            decode_unit(a, ws, unit, lane, lz, qx);
            if (lane == 0) {
                a.logP[(unit >> 1) * 4 + 2 * (unit & 1)] = lz[0];
                a.logP[(unit >> 1) * 4 + 2 * (unit & 1) + 1] = lz[1];
            }
            __syncwarp();
        }
        return;
    }
    if constexpr (GLOBAL) {
        const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
        float* ws = a.gws + (size_t)gw * a.per_warp;
        const int64_t nunits = a.ulist ? (int64_t)*a.ucount : 2 * a.B;
        for (int64_t idx = gw; idx < nunits; idx += nw) {
            const int64_t unit = a.ulist ? a.ulist[idx] : idx;
            decode_unit(a, ws, unit, lane, lz);
            if (lane == 0) {
                a.logP[(unit >> 1) * 4 + 2 * (unit & 1)] = lz[0];
                a.logP[(unit >> 1) * 4 + 2 * (unit & 1) + 1] = lz[1];
            }
            __syncwarp();
        }
    } else {
        if (gw >= 2 * a.B) return;
        decode_unit(a, reinterpret_cast<float*>(smem4) + (size_t)warp * a.per_warp, gw, lane, lz);
        if (lane == 0) {
            a.logP[(gw >> 1) * 4 + 2 * (gw & 1)] = lz[0];
            a.logP[(gw >> 1) * 4 + 2 * (gw & 1) + 1] = lz[1];
        }
    }
}

__global__ void noise_check_kernel(const float* __restrict__ noise, int mode, int64_t count, int* status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        bool ok;
        if (mode == MLD_NOISE_TABLE) {
            const float4 v = reinterpret_cast<const float4*>(noise)[i];
            const float sum = (v.x + v.y) + (v.z + v.w);
            ok = v.x >= 0.f && v.y >= 0.f && v.z >= 0.f && v.w >= 0.f && fabsf(sum - 1.f) <= 1e-6f;   // NaN fails
        } else {
            const float p = noise[i];
            ok = p >= 0.f && p <= 1.f;
        }
        if (!ok) atomicOr(status, 1 << MLD_ERR_INVALID_ARG);
    }
}

bool launch_noise_check(const float* noise, int noise_mode, int64_t count, int* status, cudaStream_t s) {
    if (count <= 0) return true;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    noise_check_kernel<<<(unsigned)blocks, 256, 0, s>>>(noise, noise_mode, count, status);
    return cudaGetLastError() == cudaSuccess;
}

__global__ void argmax_kernel(const double* __restrict__ logP, uint8_t* __restrict__ am, int64_t B) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double* l = logP + 4 * b;
    int best = 0;
    for (int k = 1; k < 4; ++k)
        if (l[k] > l[best]) best = k;
    am[b] = (uint8_t)best;
}

}  // namespace mld

// =================================================================== C-ABI

namespace {

std::mutex g_plan_mutex;

// Device copies of the code tables, made on first use (the host-side
// construction needs no GPU).
mld_status ensure_device(mld_code* C) {
    if (C->d_dmask) return MLD_OK;
    const size_t mb = C->dmask.size() * sizeof(uint64_t);
    uint64_t* dm = nullptr;
    int* ds = nullptr;
    if (cudaMalloc(&dm, mb) != cudaSuccess) return MLD_ERR_NOMEM;
    if (cudaMalloc(&ds, sizeof(int)) != cudaSuccess) { cudaFree(dm); return MLD_ERR_NOMEM; }
    if (cudaMemcpy(dm, C->dmask.data(), mb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(ds, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(dm);
        cudaFree(ds);
        return MLD_ERR_CUDA;
    }
    C->d_status = ds;
    C->d_dmask = dm;
    return MLD_OK;
}

const mld_code::PlanDev* get_plan(mld_code* C, int chi, mld_status* st) {
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    if ((*st = ensure_device(C)) != MLD_OK) return nullptr;
    for (auto& p : C->plans)
        if (p.chi == chi) return &p;
    mld_code::PlanDev pd;
    pd.chi = chi;
    pd.plan = mld::make_plan(C->d, chi);
    pd.d_steps = nullptr;
    const size_t bytes = (size_t)pd.plan.nsteps * sizeof(mld::SiteStep);
    if (cudaMalloc(&pd.d_steps, bytes) != cudaSuccess) { *st = MLD_ERR_NOMEM; return nullptr; }
    if (cudaMemcpy(pd.d_steps, pd.plan.steps, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(pd.d_steps);
        *st = MLD_ERR_CUDA;
        return nullptr;
    }
    C->plans.push_back(pd);
    return &C->plans.back();
}

}  // namespace

namespace mld {
mld_status ensure_code_device(mld_code* C) {
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    return ensure_device(C);
}
}  // namespace mld

namespace {

// Grow a device buffer owned by the code object to at least `bytes`.
template <typename T>
mld_status grow(T** buf, size_t* have, size_t bytes) {
    if (bytes <= *have) return MLD_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    if (cudaMalloc(reinterpret_cast<void**>(buf), bytes) != cudaSuccess) return MLD_ERR_NOMEM;
    *have = bytes;
    return MLD_OK;
}

// Truncating chi: the rank-adaptive kernel (one warp per unit) over all units
// on every resident warp, with the smallest slice capacities that hold bonds
// of chi (bond 48, 64 or 128: 2.25, 4.5 or 17.8 MB per resident warp), or
// smaller ones if that workspace cannot be allocated or the code's cap is
// lower; the units it hands back go to a second pass of the same kernel with
// the bond-128 capacities on one block of warps per 4 SMs, and what that
// hands back (bonds above 128) to the fixed-shape kernel in global-workspace
// mode. (A unit handed back restarts from its first column on few warps, so
// the first pass's capacities decide how long that tail is: at d=25 with
// bond 48 the few units whose middle cuts keep up to 64 values took as long
// as the whole first pass, and at chi = 128 with bond 64 the tail cost 27%.) Later passes read their unit
// count on the device and exit at once when it is zero. Control block
// (bytes): [0] queue head of pass 1, [8] of pass 2, [16] overflow count of
// pass 1, [20] of pass 2, [24] executed flops (f64, accumulated), [32] bond
// histogram (65 x u64, accumulated).
constexpr size_t kTctlBytes = 1024;
constexpr int kTruncArena = 3072;        // on-chip work arena per unit (floats)

mld_status decode_truncated(mld_code* C, const mld::Plan& P, const mld::SiteStep* d_steps, const float* noise,
                            int noise_mode, const uint64_t* syn, int64_t B, int chi, double* logP,
                            cudaStream_t s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MLD_ERR_CUDA;
    const int64_t units = 2 * B;
    const int bps = mld::trunc_blocks_per_sm(kTruncArena);
    if (bps < 1) return MLD_ERR_CUDA;
    const int upb = mld::trunc_units_per_block();
    int64_t blocks1 = (int64_t)bps * sms;
    if (blocks1 > (units + upb - 1) / upb) blocks1 = (units + upb - 1) / upb;
    int64_t blocks2 = (sms + 3) / 4;
    const size_t ws2 = (size_t)blocks2 * upb * mld::kTruncLarge.slice();
    // first-pass capacities: the smallest that hold bonds of chi (at most the
    // cap set by mld_code_set_truncation_workspace); if that workspace cannot
    // be allocated, the next smaller ones
    const mld::TruncCaps order[3] = {mld::kTruncSmall, mld::kTruncMid, mld::kTruncLarge};
    const int cap_bond = C->trunc_first_bond > 0 ? C->trunc_first_bond : mld::kTruncLarge.max_bond;
    int ci = 0;
    while (ci < 2 && chi > order[ci].max_bond && order[ci + 1].max_bond <= cap_bond) ++ci;
    mld::TruncCaps caps1 = order[ci];
    mld_status st = grow(&C->d_tws, &C->tws_bytes,
                         std::max((size_t)blocks1 * upb * caps1.slice(), ws2) * sizeof(float));
    while (st == MLD_ERR_NOMEM && ci > 0) {
        (void)cudaGetLastError();                          // clear the failed allocation's error
        caps1 = order[--ci];
        st = grow(&C->d_tws, &C->tws_bytes,
                  std::max((size_t)blocks1 * upb * caps1.slice(), ws2) * sizeof(float));
    }
    if (st != MLD_OK) return st;
    const bool pass2 = chi > caps1.max_bond;   // otherwise only carry rows can overflow
    if (!C->d_tctl) {
        if (cudaMalloc(&C->d_tctl, kTctlBytes) != cudaSuccess) return MLD_ERR_NOMEM;
        if (cudaMemset(C->d_tctl, 0, kTctlBytes) != cudaSuccess) return MLD_ERR_CUDA;
    }
    if (2 * units > C->ovf_cap) {
        cudaFree(C->d_ovf);
        C->d_ovf = nullptr;
        C->ovf_cap = 0;
        if (cudaMalloc(&C->d_ovf, (size_t)2 * units * sizeof(int64_t)) != cudaSuccess) return MLD_ERR_NOMEM;
        C->ovf_cap = 2 * units;
    }
    char* ctl = static_cast<char*>(C->d_tctl);
    // queue heads and overflow counts start at zero (flops and histogram accumulate)
    if (cudaMemsetAsync(ctl, 0, 24, s) != cudaSuccess) return MLD_ERR_CUDA;
    mld::TruncArgs ta;
    ta.dmask = C->d_dmask;
    ta.noise = noise;
    ta.syn = syn;
    ta.logP = logP;
    ta.status = C->d_status;
    ta.B = B;
    ta.d = C->d;
    ta.n = C->n;
    ta.words = C->words;
    ta.noise_mode = noise_mode;
    ta.chi = chi;
    ta.cutoff = C->svd_cutoff;
    ta.arena = kTruncArena;
    ta.caps = caps1;
    ta.ws = C->d_tws;
    ta.next_unit = reinterpret_cast<unsigned long long*>(ctl);
    ta.in_list = nullptr;
    ta.in_count = nullptr;
    ta.ovf_list = C->d_ovf;
    ta.ovf_count = reinterpret_cast<int*>(ctl + 16);
    ta.flops = reinterpret_cast<double*>(ctl + 24);
    ta.bond_hist = reinterpret_cast<unsigned long long*>(ctl + 32);
    if (!mld::launch_trunc(ta, (int)blocks1, s)) return MLD_ERR_CUDA;
    const int64_t* last_list = C->d_ovf;
    const int* last_count = reinterpret_cast<const int*>(ctl + 16);
    if (pass2) {
        ta.caps = mld::kTruncLarge;
        ta.next_unit = reinterpret_cast<unsigned long long*>(ctl + 8);
        ta.in_list = C->d_ovf;
        ta.in_count = reinterpret_cast<const int*>(ctl + 16);
        ta.ovf_list = C->d_ovf + units;
        ta.ovf_count = reinterpret_cast<int*>(ctl + 20);
        if (!mld::launch_trunc(ta, (int)blocks2, s)) return MLD_ERR_CUDA;
        last_list = C->d_ovf + units;
        last_count = reinterpret_cast<const int*>(ctl + 20);
    }
    // the fixed-shape kernel over what is left (persistent warps, global
    // workspaces of at most 1 GiB in all)
    mld::DecodeArgs a;
    a.steps = d_steps;
    a.dmask = C->d_dmask;
    a.noise = noise;
    a.syn = syn;
    a.logP = logP;
    a.status = C->d_status;
    a.B = B;
    a.d = C->d;
    a.n = C->n;
    a.words = C->words;
    a.noise_mode = noise_mode;
    a.off_w = P.off_w;
    a.off_mps = P.off_mps;
    a.off_buf0 = P.off_buf0;
    a.off_buf1 = P.off_buf1;
    a.off_q = P.off_q;
    a.off_svd = P.off_svd;
    a.per_warp = P.floats_per_warp;
    for (int i = 0; i <= mld::kMaxD; ++i) a.init_sizes[i] = i <= C->d ? P.init_sizes[i] : 0;
    a.cutoff = C->svd_cutoff;
    a.ulist = last_list;
    a.ucount = last_count;
    const size_t pw = (size_t)P.floats_per_warp * sizeof(float);
    const int W = 4;
    int64_t nw = (int64_t)sms * 16;
    while (nw > W && (size_t)nw * pw > ((size_t)1 << 30)) nw /= 2;
    nw = (nw / W) * W;
    st = grow(&C->d_gws, &C->gws_bytes, (size_t)nw * pw);
    if (st != MLD_OK) return st;
    a.gws = C->d_gws;
    mld::decode_fp32_kernel<true><<<(unsigned)(nw / W), 32 * W, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? MLD_OK : MLD_ERR_CUDA;
}

}  // namespace

namespace mld {
// Whether an untruncated decode of this code runs the dense-state kernel:
// on request (mld_code_set_exact_kernel 2, d = 9, 11, 13), as mld_autotune
// chose for this chi, or by default at d = 11 and 13, where it is the faster
// exact kernel (measured: 2.61M against 2.07M syndromes/s for the split-TF32
// boundary-MPS kernel at d = 11; 556k against 140k at d = 13, where the
// exact boundary MPS needs 298 KB per unit and runs from global memory; at
// d = 9 the boundary-MPS kernel is faster, 19.2M against 10.8M).
bool uses_dense_exact(const mld_code* C, const Plan& P) {
    if (P.svd_sites != 0 || !dense_exact_supported(C->d) || C->exact_kernel == 1) return false;
    if (C->exact_kernel == 2) return true;
    for (const auto& kv : C->exact_tuned)
        if (kv.first == P.chi) return kv.second == 2;
    return C->d >= 11;
}

// Whether the untruncated or fixed-shape sweep of this code at this chi keeps
// its per-warp state in the global workspace (then mld_autotune's candidates
// are resident warps per SM).
bool state_in_global_workspace(const mld_code* C, int chi) {
    const Plan P = make_plan(C->d, chi);
    if (uses_dense_exact(C, P)) return false;
    const bool exact = P.svd_sites == 0 && exact_floats_per_warp(C->d) > 0;
    int dev = 0, max_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    const size_t pw = (size_t)(exact ? exact_floats_per_warp(C->d) : P.floats_per_warp) * sizeof(float);
    return pw > (size_t)max_optin;
}
}  // namespace mld

extern "C" {

const char* mld_status_string(mld_status s) {
    switch (s) {
        case MLD_OK: return "ok";
        case MLD_ERR_INVALID_ARG: return "invalid argument";
        case MLD_ERR_UNSUPPORTED: return "unsupported configuration";
        case MLD_ERR_CUDA: return "CUDA runtime error";
        case MLD_ERR_NOMEM: return "out of memory";
        case MLD_ERR_TIMEOUT: return "bounded device loop hit its limit";
        case MLD_ERR_NUMERIC: return "non-finite value on the device";
    }
    return "unknown status";
}

mld_status mld_code_create_rotated(int d, mld_code** out) {
    return mld_code_build_host(d, out);
}

void mld_code_destroy(mld_code* C) {
    if (!C) return;
    if (C->d_dmask) {
        for (auto& p : C->plans) cudaFree(p.d_steps);
        cudaFree(C->d_dmask);
        cudaFree(C->d_status);
        cudaFree(C->h_stage_dev);
        cudaFree(C->d_gws);
        cudaFree(C->d_gradws);
        cudaFree(C->d_tws);
        cudaFree(C->d_tctl);
        cudaFree(C->d_ovf);
        cudaFree(C->d_kw);
    }
    delete C;
}

mld_status mld_code_info(const mld_code* C, int* n, int* m, int* w) {
    if (!C) return MLD_ERR_INVALID_ARG;
    if (n) *n = C->n;
    if (m) *m = C->m;
    if (w) *w = C->words;
    return MLD_OK;
}

mld_status mld_code_layout(const mld_code* C, int32_t* type, int32_t* sup, uint8_t* lx, uint8_t* lz) {
    if (!C) return MLD_ERR_INVALID_ARG;
    for (int k = 0; k < C->m; ++k) {
        if (type) type[k] = C->stab_type[k];
        if (sup)
            for (int u = 0; u < 4; ++u) sup[4 * k + u] = C->stab_qubits[4 * k + u];
    }
    for (int q = 0; q < C->n; ++q) {
        if (lx) lx[q] = C->lx[q];
        if (lz) lz[q] = C->lz[q];
    }
    return MLD_OK;
}

int mld_decode_launches(void) { return 3; }

mld_status mld_code_set_exact_kernel(mld_code* C, int which) {
    if (!C || which < 0 || which > 2) return MLD_ERR_INVALID_ARG;
    if (which == 2 && !mld::dense_exact_supported(C->d)) return MLD_ERR_UNSUPPORTED;
    C->exact_kernel = which;
    return MLD_OK;
}

mld_status mld_decode_flops(const mld_code* C, int chi, int precision, double* out) {
    if (!C || chi < 1 || !out) return MLD_ERR_INVALID_ARG;
    if (precision != MLD_FP32 && precision != MLD_MIXED_BF16 && precision != MLD_MIXED_TF32)
        return MLD_ERR_INVALID_ARG;
    // every kernel sweeps columns 0..d-2 once per l_Z and the last column once
    // per class
    const mld::Plan P = mld::make_plan(C->d, chi);
    if (mld::uses_dense_exact(C, P)) {
        *out = mld::dense_exact_flops_per_syndrome(C->d);
        return MLD_OK;
    }
    *out = 2.0 * (P.flops_per_coset - P.flops_last_col) + 4.0 * P.flops_last_col;
    return MLD_OK;
}

mld_status mld_decode(const mld_code* Cc, const float* noise, int noise_mode, const uint64_t* syn,
                      int64_t B, int chi, int precision, double* logP, uint8_t* argmax, void* stream) {
    mld::NvtxRange trace("mld_decode");
    mld_code* C = const_cast<mld_code*>(Cc);
    if (!C || B < 0 || chi < 1) return MLD_ERR_INVALID_ARG;
    if (noise_mode != MLD_NOISE_TABLE && noise_mode != MLD_NOISE_DEPOL) return MLD_ERR_INVALID_ARG;
    if (precision != MLD_FP32 && precision != MLD_MIXED_BF16 && precision != MLD_MIXED_TF32)
        return MLD_ERR_INVALID_ARG;
    if (B == 0) return MLD_OK;
    if (!noise || !syn || !logP) return MLD_ERR_INVALID_ARG;
    if (noise_mode == MLD_NOISE_TABLE && (reinterpret_cast<uintptr_t>(noise) & 15)) return MLD_ERR_INVALID_ARG;
    mld_status st = MLD_OK;
    const mld_code::PlanDev* pd = get_plan(C, chi, &st);
    if (!pd) return st;
    const mld::Plan& P = pd->plan;
    mld::DecodeArgs a;
    a.steps = pd->d_steps;
    a.dmask = C->d_dmask;
    a.noise = noise;
    a.syn = syn;
    a.logP = logP;
    a.status = C->d_status;
    a.B = B;
    a.d = C->d;
    a.n = C->n;
    a.words = C->words;
    a.noise_mode = noise_mode;
    a.off_w = P.off_w;
    a.off_mps = P.off_mps;
    a.off_buf0 = P.off_buf0;
    a.off_buf1 = P.off_buf1;
    a.off_q = P.off_q;
    a.off_svd = P.off_svd;
    a.per_warp = P.floats_per_warp;
    a.cutoff = C->svd_cutoff;
    for (int i = 0; i <= mld::kMaxD; ++i) a.init_sizes[i] = i <= C->d ? P.init_sizes[i] : 0;
    int dev = 0, max_optin = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return MLD_ERR_CUDA;
    // untruncated chi (every kept dimension is min(rows, cols)): the
    // compile-time specialised kernel, when one exists for this d
    const bool exact = P.svd_sites == 0 && mld::exact_floats_per_warp(C->d) > 0;
    // the mixed-precision path exists for the untruncated specialised kernel
    // (TF32 tensor-core products); BF16 and truncating chi run FP32 only
    if (precision == MLD_MIXED_BF16 || (precision == MLD_MIXED_TF32 && !exact)) return MLD_ERR_UNSUPPORTED;
    // truncating chi: the rank-adaptive sweep, or the fixed-shape one when its
    // whole per-warp state fits 24 KB of shared memory (small chi and d, where
    // its compile-free static shapes beat the runtime ones), unless the
    // caller or mld_autotune chose
    int which = C->trunc_kernel;
    if (which == 0)
        for (const auto& kv : C->trunc_tuned)
            if (kv.first == chi) which = kv.second;
    if (which == 0) which = P.floats_per_warp <= 6144 ? 2 : 1;
    if (P.svd_sites != 0 && which == 1) {
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        if (!mld::launch_noise_check(noise, noise_mode, noise_mode == MLD_NOISE_TABLE ? C->n : B, C->d_status, s))
            return MLD_ERR_CUDA;
        const mld_status ts = decode_truncated(C, P, pd->d_steps, noise, noise_mode, syn, B, chi, logP, s);
        if (ts != MLD_OK) return ts;
        if (argmax) {
            mld::argmax_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(logP, argmax, B);
            if (cudaGetLastError() != cudaSuccess) return MLD_ERR_CUDA;
        }
        return MLD_OK;
    }
    if (mld::uses_dense_exact(C, P)) {
        // untruncated, dense boundary state (FP32 for either precision: no
        // product is MMA-shaped)
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        if (!mld::launch_noise_check(noise, noise_mode, noise_mode == MLD_NOISE_TABLE ? C->n : B, C->d_status, s))
            return MLD_ERR_CUDA;
        mld::DenseArgs da;
        da.dmask = C->d_dmask;
        da.noise = noise;
        da.syn = syn;
        da.logP = logP;
        da.status = C->d_status;
        da.B = B;
        da.words = C->words;
        da.noise_mode = noise_mode;
        if (!mld::launch_dense_exact(C->d, da, s)) return MLD_ERR_CUDA;
        if (argmax) {
            mld::argmax_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(logP, argmax, B);
            if (cudaGetLastError() != cudaSuccess) return MLD_ERR_CUDA;
        }
        return MLD_OK;
    }
    const size_t pw = (size_t)(exact ? mld::exact_floats_per_warp(C->d) : P.floats_per_warp) * sizeof(float);
    const int64_t units = 2 * B;                       // (syndrome, l_Z) pairs, both kernels
    int W = 1;
    float* gws = nullptr;
    int64_t gws_warps = 0;
    if (pw > (size_t)max_optin) {
        // state larger than a block's shared memory: persistent warps with
        // global-memory workspaces (R resident warps per SM: 16, or the
        // autotuned count; halved until the workspace is at most 8 GiB)
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MLD_ERR_CUDA;
        int R = 16;
        const int key = chi * 4 + precision;
        for (const auto& kv : C->tuned)
            if (kv.first == key && kv.second >= 1 && kv.second <= 64) R = kv.second;
        if (C->force_warps > 0) R = C->force_warps;
        W = R < 4 ? R : 4;
        int64_t nw = (int64_t)sms * R;
        while (nw > (int64_t)sms * W && (size_t)nw * pw > ((size_t)8 << 30)) nw /= 2;
        const int64_t need = ((units + W - 1) / W) * W;
        if (nw > need) nw = need;
        const size_t bytes = (size_t)nw * pw;
        if (bytes > C->gws_bytes) {
            cudaFree(C->d_gws);
            C->d_gws = nullptr;
            C->gws_bytes = 0;
            if (cudaMalloc(&C->d_gws, bytes) != cudaSuccess) return MLD_ERR_NOMEM;
            C->gws_bytes = bytes;
        }
        gws = C->d_gws;
        gws_warps = nw;
    } else {
        // warps per CTA: the autotuned shape if mld_autotune chose one, else
        // the most resident warps per SM (32 CTAs and 64 warps per SM at most,
        // 1 KB of shared memory reserved per CTA), fewest warps per CTA on ties
        int best = 0;
        for (int w = 1; w <= mld::kMaxWarpsPerBlock; ++w) {
            if (pw * w > (size_t)max_optin) break;
            int ctas = (int)((size_t)per_sm / (pw * w + 1024));
            ctas = ctas < 32 ? ctas : 32;
            int warps = ctas * w < 64 ? ctas * w : 64;
            if (warps > best) { best = warps; W = w; }
        }
        const int key = chi * 4 + precision;
        for (const auto& kv : C->tuned)
            if (kv.first == key && kv.second >= 1 && pw * kv.second <= (size_t)max_optin) W = kv.second;
        if (C->force_warps > 0 && pw * C->force_warps <= (size_t)max_optin) W = C->force_warps;
        // runtime-plan kernel: move the kept tall blocks to global memory when
        // that at least doubles the warps per SM (shared memory sets it)
        if (!exact && P.max_q > 0) {
            const size_t ps = (size_t)(P.off_q + ((P.max_svd + 3) & ~3)) * sizeof(float);
            int best_s = 0, Ws = 1;
            for (int w = 1; w <= mld::kMaxWarpsPerBlock; ++w) {
                if (ps * w > (size_t)max_optin) break;
                int ctas = (int)((size_t)per_sm / (ps * w + 1024));
                ctas = ctas < 32 ? ctas : 32;
                const int warps = ctas * w < 16 ? ctas * w : 16;   // registers: 16 warps of 8-warp CTAs
                if (warps > best_s) { best_s = warps; Ws = w; }
            }
            if (best_s >= 2 * best && C->force_warps == 0) {
                int sms = 0;
                if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                    return MLD_ERR_CUDA;
                int64_t nw = (int64_t)sms * (best_s / Ws) * Ws;
                const int64_t need = ((units + Ws - 1) / Ws) * Ws;
                if (nw > need) nw = need;
                const size_t qf = (size_t)((P.max_q + 3) & ~3);
                const size_t bytes = (size_t)nw * qf * sizeof(float);
                if (bytes > C->gws_bytes) {
                    cudaFree(C->d_gws);
                    C->d_gws = nullptr;
                    C->gws_bytes = 0;
                    if (cudaMalloc(&C->d_gws, bytes) != cudaSuccess) return MLD_ERR_NOMEM;
                    C->gws_bytes = bytes;
                }
                a.qgws = C->d_gws;
                a.q_per_warp = (int64_t)qf;
                a.off_svd = P.off_q;                   // shared-memory layout without the q area
                a.per_warp = P.off_q + ((P.max_svd + 3) & ~3);
                W = Ws;
                gws_warps = nw;
            }
        }
    }
    const size_t smem = gws ? 0 : (a.qgws ? (size_t)a.per_warp * sizeof(float) : pw) * W;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!mld::launch_noise_check(noise, noise_mode, noise_mode == MLD_NOISE_TABLE ? C->n : B, C->d_status, s))
        return MLD_ERR_CUDA;
    if (exact) {
        mld::ExactArgs ea;
        ea.dmask = C->d_dmask;
        ea.noise = noise;
        ea.syn = syn;
        ea.logP = logP;
        ea.status = C->d_status;
        ea.B = B;
        ea.noise_mode = noise_mode;
        ea.gws = gws;
        ea.gws_warps = gws_warps;
        if (!mld::launch_exact(C->d, ea, s, W, precision)) return MLD_ERR_CUDA;
        if (argmax) {
            mld::argmax_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(logP, argmax, B);
            if (cudaGetLastError() != cudaSuccess) return MLD_ERR_CUDA;
        }
        return MLD_OK;
    }
    auto kern = gws ? mld::decode_fp32_kernel<true> : mld::decode_fp32_kernel<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return MLD_ERR_CUDA;
    a.gws = gws;
    int64_t blocks = (units + W - 1) / W;
    if ((gws || a.qgws) && blocks > gws_warps / W) blocks = gws_warps / W;
    if (blocks > 0x7fffffff) return MLD_ERR_UNSUPPORTED;
    kern<<<(unsigned)blocks, 32 * W, smem, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return MLD_ERR_CUDA;
    if (argmax) {
        mld::argmax_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(logP, argmax, B);
        if (cudaGetLastError() != cudaSuccess) return MLD_ERR_CUDA;
    }
    return MLD_OK;
}

mld_status mld_decode_grad(const mld_code* Cc, const float* noise, const uint64_t* syn, int64_t B, int chi,
                           const double* dlogP, double* logP, double* dnoise, void* stream) {
    mld::NvtxRange trace("mld_decode_grad");
    mld_code* C = const_cast<mld_code*>(Cc);
    if (!C || B < 0 || chi < 1) return MLD_ERR_INVALID_ARG;
    if (B == 0) return MLD_OK;
    if (!noise || !syn || !dnoise || (reinterpret_cast<uintptr_t>(noise) & 15)) return MLD_ERR_INVALID_ARG;
    if (C->d > 13) return MLD_ERR_UNSUPPORTED;
    mld_status st = MLD_OK;
    const mld_code::PlanDev* pd = get_plan(C, chi, &st);
    if (!pd) return st;
    const mld::Plan& P = pd->plan;
    if (P.svd_sites != 0) return MLD_ERR_UNSUPPORTED;       // exact environments need untruncated chi
    const int d = C->d, n = C->n;
    if (!mld::launch_noise_check(noise, MLD_NOISE_TABLE, n, C->d_status, reinterpret_cast<cudaStream_t>(stream)))
        return MLD_ERR_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MLD_ERR_CUDA;
    if (!mld::grad_dense_supported(d)) return MLD_ERR_UNSUPPORTED;
    {
        // dense states (on chip, or in the block's global slice at d = 13): one
        // block per (syndrome, class) unit
        const int64_t blocks = mld::grad_dense_blocks(d, sms, B);
        if (blocks < 1) return MLD_ERR_CUDA;
        const size_t bytes = (size_t)blocks * mld::grad_dense_workspace_floats(d) * sizeof(float);
        if (bytes > C->gradws_bytes) {
            cudaFree(C->d_gradws);
            C->d_gradws = nullptr;
            C->gradws_bytes = 0;
            if (cudaMalloc(&C->d_gradws, bytes) != cudaSuccess) return MLD_ERR_NOMEM;
            C->gradws_bytes = bytes;
        }
        mld::GradDenseArgs ga;
        ga.dmask = C->d_dmask;
        ga.noise = noise;
        ga.syn = syn;
        ga.dlogP = dlogP;
        ga.logP = logP;
        ga.dnoise = dnoise;
        ga.lws = C->d_gradws;
        ga.B = B;
        ga.words = C->words;
        return mld::launch_grad_dense(d, ga, blocks, reinterpret_cast<cudaStream_t>(stream)) ? MLD_OK
                                                                                              : MLD_ERR_CUDA;
    }
}

mld_status mld_code_set_svd_cutoff(mld_code* C, double rel) {
    if (!C || !(rel >= 0.0) || !(rel < 1.0)) return MLD_ERR_INVALID_ARG;
    C->svd_cutoff = (float)rel;
    return MLD_OK;
}

mld_status mld_code_set_truncation_kernel(mld_code* C, int which) {
    if (!C || which < 0 || which > 2) return MLD_ERR_INVALID_ARG;
    C->trunc_kernel = which;
    return MLD_OK;
}

mld_status mld_code_set_truncation_workspace(mld_code* C, int max_bond) {
    if (!C || (max_bond != 0 && max_bond != mld::kTruncSmall.max_bond && max_bond != mld::kTruncMid.max_bond &&
               max_bond != mld::kTruncLarge.max_bond))
        return MLD_ERR_INVALID_ARG;
    C->trunc_first_bond = max_bond;
    return MLD_OK;
}

mld_status mld_decode_executed_flops(const mld_code* Cc, double* out) {
    mld_code* C = const_cast<mld_code*>(Cc);
    if (!C || !out) return MLD_ERR_INVALID_ARG;
    *out = 0.0;
    if (!C->d_tctl) return MLD_OK;
    char* ctl = static_cast<char*>(C->d_tctl);
    if (cudaMemcpy(out, ctl + 24, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return MLD_ERR_CUDA;
    if (cudaMemset(ctl + 24, 0, sizeof(double)) != cudaSuccess) return MLD_ERR_CUDA;
    return MLD_OK;
}

mld_status mld_decode_bond_histogram(const mld_code* Cc, int64_t* hist) {
    mld_code* C = const_cast<mld_code*>(Cc);
    if (!C || !hist) return MLD_ERR_INVALID_ARG;
    for (int k = 0; k <= 64; ++k) hist[k] = 0;
    if (!C->d_tctl) return MLD_OK;
    char* ctl = static_cast<char*>(C->d_tctl);
    if (cudaMemcpy(hist, ctl + 32, 65 * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess) return MLD_ERR_CUDA;
    if (cudaMemset(ctl + 32, 0, 65 * sizeof(int64_t)) != cudaSuccess) return MLD_ERR_CUDA;
    return MLD_OK;
}

mld_status mld_decode_status(const mld_code* C) {
    if (!C) return MLD_ERR_INVALID_ARG;
    if (!C->d_status) return MLD_OK;
    int h = 0;
    if (cudaMemcpy(&h, C->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MLD_ERR_CUDA;
    if (cudaMemset(C->d_status, 0, sizeof(int)) != cudaSuccess) return MLD_ERR_CUDA;
    if (h & (1 << MLD_ERR_INVALID_ARG)) return MLD_ERR_INVALID_ARG;
    if (h & (1 << MLD_ERR_NUMERIC)) return MLD_ERR_NUMERIC;
    if (h & (1 << MLD_ERR_TIMEOUT)) return MLD_ERR_TIMEOUT;
    return MLD_OK;
}

mld_status mld_decode_host(const mld_code* Cc, const float* noise, int noise_mode, const uint64_t* syn,
                           int64_t B, int chi, int precision, double* logP, uint8_t* argmax) {
    mld::NvtxRange trace("mld_decode_host");
    mld_code* C = const_cast<mld_code*>(Cc);
    if (!C || B < 0) return MLD_ERR_INVALID_ARG;
    if (B == 0) return MLD_OK;
    if (!noise || !syn || !logP) return MLD_ERR_INVALID_ARG;
    const size_t nb = noise_mode == MLD_NOISE_TABLE ? (size_t)C->n * 4 * sizeof(float) : (size_t)B * sizeof(float);
    const size_t sb = (size_t)B * C->words * sizeof(uint64_t);
    const size_t lb = (size_t)B * 4 * sizeof(double);
    const size_t ab = (size_t)B;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t need = al(nb) + al(sb) + al(lb) + al(ab);
    if (need > C->h_stage_bytes) {
        cudaFree(C->h_stage_dev);
        C->h_stage_dev = nullptr;
        C->h_stage_bytes = 0;
        if (cudaMalloc(&C->h_stage_dev, need) != cudaSuccess) return MLD_ERR_NOMEM;
        C->h_stage_bytes = need;
    }
    char* base = static_cast<char*>(C->h_stage_dev);
    float* dn = reinterpret_cast<float*>(base);
    uint64_t* ds = reinterpret_cast<uint64_t*>(base + al(nb));
    double* dl = reinterpret_cast<double*>(base + al(nb) + al(sb));
    uint8_t* da = reinterpret_cast<uint8_t*>(base + al(nb) + al(sb) + al(lb));
    cudaStream_t s = 0;
    if (cudaMemcpyAsync(dn, noise, nb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ds, syn, sb, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MLD_ERR_CUDA;
    mld_status st = mld_decode(C, dn, noise_mode, ds, B, chi, precision, dl, argmax ? da : nullptr, s);
    if (st != MLD_OK) return st;
    if (cudaMemcpyAsync(logP, dl, lb, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MLD_ERR_CUDA;
    if (argmax && cudaMemcpyAsync(argmax, da, ab, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MLD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MLD_ERR_CUDA;
    return mld_decode_status(C);
}

}  // extern "C"
