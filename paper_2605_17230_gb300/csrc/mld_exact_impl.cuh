#pragma once
// Kernel templates of the boundary-MPS sweep at untruncated bond dimension, specialised at compile
// time on the shape plan of distance d (sm_103a, FP32).
//
// When chi is at least the exact bond of every cut (2^floor(d/2) in this
// layout) no singular value is ever discarded (Sec. 3.2.1: the truncation
// keeps min(chi, #values)), every column is kept in the non-negative gauge
// (no QR, no SVD) and the shape of every step is a function of d alone. This
// kernel instantiates each site step of that plan as a template on its
// shapes (bond dimensions, block counts, site kinds), so index arithmetic is
// folded at compile time and identity sites cost no multiplications. The
// arithmetic is the same as the runtime-plan kernel's: MPO.MPS products per
// beta block, power-of-two renormalisation per site, bond-matrix products in
// the right sweep, contraction with all-ones vectors at the end.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "mld_exact.h"
#include "mld_internal.h"

namespace mld {
namespace exact {

constexpr int kExactChi = 1 << 20;

template <int D>
struct PlanOf {
    static constexpr Plan plan = make_plan(D, kExactChi);
};

template <int D>
struct LayoutOf {
    static constexpr ExactLayout lay = make_exact_layout(PlanOf<D>::plan);
    static_assert(exact_layout_valid(PlanOf<D>::plan, lay), "overlapping live intermediates");
};

// Columns c1 and c2 run the same code: every step has the same shapes,
// kinds, orientation, MPS offsets and arena offsets (only the qubits whose
// weights they read differ).
constexpr bool same_column(const Plan& P, const ExactLayout& L, int c1, int c2) {
    const int d = P.d;
    for (int i = 0; i <= d; ++i) {
        const SiteStep& a = P.steps[c1 * (d + 1) + i];
        const SiteStep& b = P.steps[c2 * (d + 1) + i];
        if (a.pam != b.pam || a.pa != b.pa || a.pb != b.pb || a.Dl != b.Dl || a.Dr != b.Dr || a.K != b.K ||
            a.ncol != b.ncol || a.kq != b.kq || a.kq_prev != b.kq_prev || a.tall != b.tall ||
            a.parity != b.parity || a.rmode != b.rmode || a.S != b.S || a.Sl != b.Sl || a.offA != b.offA ||
            a.offQ != b.offQ || a.offN != b.offN || a.canon != b.canon || a.cid != b.cid || a.okind != b.okind ||
            a.nkind != b.nkind || a.gid != b.gid)
            return false;
        const int k1 = c1 * (d + 1) + i, k2 = c2 * (d + 1) + i;
        if (L.cin[k1] != L.cin[k2] || L.mout[k1] != L.mout[k2] || L.gin[k1] != L.gin[k2] ||
            L.tout[k1] != L.tout[k2])
            return false;
    }
    return true;
}

// First column from which columns 0..d-2 repeat with period two (the bonds
// have reached the exact cut ranks and the orientation alternates): columns
// C0.. d-2 then run as a loop over one compiled pair. d - 1 when none repeat.
template <int D>
struct RepeatOf {
    static constexpr int find() {
        for (int c0 = 0; c0 + 2 <= D - 2; ++c0) {
            bool ok = true;
            for (int c = c0 + 2; c <= D - 2 && ok; ++c)
                ok = same_column(PlanOf<D>::plan, LayoutOf<D>::lay, c, c0 + ((c - c0) & 1));
            if (ok) return c0;
        }
        return D - 1;
    }
    static constexpr int c0 = find();
};

// Float index within a row of an M block of row length NC (the carry of the
// next left step, or a tall block kept for the right sweep). In the blocks a
// tensor-core step reads or writes (SW = 1) the row's float4 slots are
// XOR-permuted by the row index, so that the same column of eight consecutive
// rows falls in eight different bank groups (rows are multiples of 32 floats
// long) for the fragment loads; rows shorter than 8 floats, and every other
// block (whose reads are warp broadcasts), are stored as they are.
template <int NC, int SW>
__device__ __forceinline__ int swz(int row, int col) {
    if constexpr (SW && NC >= 8) {
        constexpr int Q = NC / 4 < 8 ? NC / 4 : 8;
        return col ^ ((row & (Q - 1)) << 2);
    } else {
        return col;
    }
}

// w(a, a', b, b') of the qubit factor, from its four weights p[E xor X^u Z^v]
// indexed u + 2v; the parity PAR selects which plaquette pair carries u.
template <int PAR>
__device__ __forceinline__ float wsel(const float4 w, int a, int ap, int b, int bp) {
    const int x1 = a ^ bp, x2 = ap ^ b;
    const int u = PAR ? x2 : x1, v = PAR ? x1 : x2;
    const int idx = u | (v << 1);
    return idx == 0 ? w.x : idx == 1 ? w.y : idx == 2 ? w.z : w.w;
}

// The eight weights w(a, a', beta, b') of a lane whose column fixes a',
// indexed a | b' << 1 | beta << 2.
template <int PAR>
__device__ __forceinline__ void weights8(const float4 w, int ap, float (&o)[8]) {
#pragma unroll
    for (int m = 0; m < 8; ++m) o[m] = wsel<PAR>(w, m & 1, ap, (m >> 2) & 1, (m >> 1) & 1);
}

// X_a[k][col] = sum_r C[k][a*DL + r] A[r][col] for the identity cases
// (identity carry and/or identity old site), where the sum has one term.
template <int DL, int DR, int PAM, int NCOLA, int KQP, int CID, int OKIND, int SW>
__device__ __forceinline__ void x_ident(const float* C, const float* A, int k, int ap, int rp, float X[2]) {
    constexpr int LDC = PAM * DL;
    X[0] = 0.f;
    X[1] = 0.f;
    if constexpr (CID) {
        const int j = k % KQP, ja = j / DL, jr = j % DL;
        float av;
        if constexpr (OKIND == K_DATA) av = A[jr * NCOLA + ap * DR + rp];
        else if constexpr (OKIND == K_IDR) av = (jr == ap * DR + rp) ? 1.f : 0.f;
        else av = (rp == ap * DL + jr) ? 1.f : 0.f;
        if (ja == 0) X[0] = av; else X[1] = av;
    } else {
#pragma unroll
        for (int a = 0; a < PAM; ++a) {
            const float* crow = C + k * LDC;
            if constexpr (OKIND == K_IDR) {
                X[a] = crow[swz<LDC, SW>(k, a * DL + ap * DR + rp)];
            } else {
                const int r = rp - ap * DL;
                X[a] = (r >= 0 && r < DL) ? crow[swz<LDC, SW>(k, a * DL + r)] : 0.f;
            }
        }
    }
}

__device__ __forceinline__ unsigned to_tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// D += A(16x8) B(8x8) on the tensor cores, TF32 operands, FP32 accumulate.
// Fragments (g = lane/4, t = lane%4): A rows g, g+8 x cols t, t+4; B rows
// t, t+4 x col g; D rows g, g+8 x cols 2t, 2t+1.
__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Split x into TF32 parts hi + lo (hi = x rounded to TF32, lo = the
// rounded remainder): products of the parts recover ~FP32 accuracy.
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

// The data-site product of the mixed-precision path: X_a = C_a A on the
// tensor cores, TF32 operands and FP32 accumulation, each operand split
// into TF32 hi + lo and the product taken as hi.hi + hi.lo + lo.hi (the
// lo.lo term is below FP32 rounding), then the FP32 qubit-factor epilogue
// M^{b'}[k][col] = sum_a w(a, a', beta, b') X_a[k][col].
// Per 16-row block kb and group of up to four 8-column tiles, the k-steps
// of 8 split one A fragment (both a) and the group's B fragments once and
// issue three MMAs per (tile, a).
template <int K, int PAM, int DL, int PA, int DR, int PB, int NCOL, int KQP, int PAR>
__device__ __forceinline__ float gemm_tf32(const float* __restrict__ C, const float* __restrict__ A,
                                           float* __restrict__ M, const float4 w, int lane) {
    constexpr int NCOLA = PA * DR;
    constexpr int LDC = PAM * DL;
    constexpr int KB = (K + 15) / 16;
    constexpr int NT = NCOLA / 8, KS = DL / 8;
    constexpr int NTG = NT < 4 ? NT : 4;
    constexpr int SW = 1;
    static_assert(DL % 8 == 0 && NCOLA % 8 == 0 && NT % NTG == 0, "tensor-core tile shape");
    const int g = lane >> 2, t = lane & 3;
    // the lane's weights for a' = 0 and a' = 1
    float wa[2][8];
    weights8<PAR>(w, 0, wa[0]);
    weights8<PAR>(w, 1, wa[1]);
    float mx = 0.f;
    // with one tile group, the split B fragments of the whole site stay in
    // registers across the row blocks
    constexpr bool BHOLD = NTG == NT && NT * KS <= 8;
    unsigned bhh[BHOLD ? KS : 1][BHOLD ? NT : 1][4];
    if constexpr (BHOLD) {
#pragma unroll
        for (int ks = 0; ks < KS; ++ks)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                split_tf32(A[(8 * ks + t) * NCOLA + nt * 8 + g], bhh[ks][nt][0], bhh[ks][nt][1]);
                split_tf32(A[(8 * ks + t + 4) * NCOLA + nt * 8 + g], bhh[ks][nt][2], bhh[ks][nt][3]);
            }
    }
#pragma unroll 1
    for (int kb = 0; kb < KB; ++kb) {
        const int r0 = kb * 16 + g, r1 = r0 + 8;
#pragma unroll
        for (int n0 = 0; n0 < NT; n0 += NTG) {
            float acc[NTG][2][4];
#pragma unroll
            for (int j = 0; j < NTG; ++j)
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[j][a][q] = 0.f;
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                unsigned ah[2][4], al[2][4];
#pragma unroll
                for (int a = 0; a < PAM; ++a) {
                    const float* c0 = C + r0 * LDC;
                    const float* c1 = C + r1 * LDC;
                    const int q0 = a * DL + 8 * ks + t;
                    split_tf32(r0 < K ? c0[swz<LDC, SW>(r0, q0)] : 0.f, ah[a][0], al[a][0]);
                    split_tf32(r1 < K ? c1[swz<LDC, SW>(r1, q0)] : 0.f, ah[a][1], al[a][1]);
                    split_tf32(r0 < K ? c0[swz<LDC, SW>(r0, q0 + 4)] : 0.f, ah[a][2], al[a][2]);
                    split_tf32(r1 < K ? c1[swz<LDC, SW>(r1, q0 + 4)] : 0.f, ah[a][3], al[a][3]);
                }
#pragma unroll
                for (int j = 0; j < NTG; ++j) {
                    const int nt = n0 + j;
                    unsigned bh0, bl0, bh1, bl1;
                    if constexpr (BHOLD) {
                        bh0 = bhh[ks][nt][0]; bl0 = bhh[ks][nt][1]; bh1 = bhh[ks][nt][2]; bl1 = bhh[ks][nt][3];
                    } else {
                        split_tf32(A[(8 * ks + t) * NCOLA + nt * 8 + g], bh0, bl0);
                        split_tf32(A[(8 * ks + t + 4) * NCOLA + nt * 8 + g], bh1, bl1);
                    }
#pragma unroll
                    for (int a = 0; a < PAM; ++a) {
                        mma_tf32(acc[j][a], al[a][0], al[a][1], al[a][2], al[a][3], bh0, bh1);
                        mma_tf32(acc[j][a], ah[a][0], ah[a][1], ah[a][2], ah[a][3], bl0, bl1);
                        mma_tf32(acc[j][a], ah[a][0], ah[a][1], ah[a][2], ah[a][3], bh0, bh1);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < NTG; ++j) {
                const int nt = n0 + j;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = kb * 16 + g + 8 * h;
                    if (k >= K) continue;
                    const bool beta = (k / KQP) != 0;
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int col = nt * 8 + 2 * t + e;
                        const int ap = col / DR;
                        const float x0 = acc[j][0][2 * h + e], x1 = PAM == 2 ? acc[j][1][2 * h + e] : 0.f;
#pragma unroll
                        for (int bp = 0; bp < PB; ++bp) {
                            const int m0 = (bp << 1) | (beta ? 4 : 0);
                            const float w0 = ap ? wa[1][m0] : wa[0][m0];
                            const float w1 = ap ? wa[1][m0 | 1] : wa[0][m0 | 1];
                            const float o = fmaf(w0, x0, w1 * x1);
                            M[(bp * K + k) * NCOL + swz<NCOL, SW>(bp * K + k, col)] = o;
                            mx = fmaxf(mx, fabsf(o));
                        }
                    }
                }
            }
        }
    }
    return mx;
}

// Four consecutive columns col..col+3 (one a', rp..rp+3) of X_a for the
// identity cases, as float4 (DR % 4 == 0; DL % 4 == 0 unless the carry is
// the identity).
template <int DL, int DR, int PAM, int NCOLA, int KQP, int CID, int OKIND, int SW>
__device__ __forceinline__ void x_ident4(const float* C, const float* A, int k, int ap, int rp, float4 X[2]) {
    constexpr int LDC = PAM * DL;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    X[0] = z;
    X[1] = z;
    if constexpr (CID) {
        const int j = k % KQP, ja = j / DL, jr = j % DL;
        float4 av;
        if constexpr (OKIND == K_DATA) {
            av = *reinterpret_cast<const float4*>(A + jr * NCOLA + ap * DR + rp);
        } else {
            const int hit = OKIND == K_IDR ? jr - (ap * DR + rp) : ap * DL + jr - rp;   // which of the four is 1
            av.x = hit == 0 ? 1.f : 0.f;
            av.y = hit == 1 ? 1.f : 0.f;
            av.z = hit == 2 ? 1.f : 0.f;
            av.w = hit == 3 ? 1.f : 0.f;
        }
        if (ja == 0) X[0] = av; else X[1] = av;
    } else {
#pragma unroll
        for (int a = 0; a < PAM; ++a) {
            const float* crow = C + k * LDC;
            if constexpr (OKIND == K_IDR) {
                X[a] = *reinterpret_cast<const float4*>(crow + swz<LDC, SW>(k, a * DL + ap * DR + rp));
            } else {
                const int r = rp - ap * DL;
                if (r >= 0 && r < DL) X[a] = *reinterpret_cast<const float4*>(crow + swz<LDC, SW>(k, a * DL + r));
            }
        }
    }
}

// Left-sweep site with four columns per lane (float4 loads and stores; the
// data-site product keeps four A columns in registers, so each broadcast C
// element feeds four FMAs). Lanes own column groups and every RG-th row; as
// in left_step the rows split at KQP into the two beta halves.
template <int K, int PAM, int DL, int PA, int DR, int PB, int NCOL, int KQP, int CID, int OKIND, int PAR, int SWC, int SWM>
__device__ __forceinline__ float left_cols4(const float* __restrict__ C, const float* __restrict__ A,
                                            float* __restrict__ M, const float4 w, int lane) {
    constexpr int NCOLA = PA * DR;
    constexpr int LDC = PAM * DL;
    constexpr int NCW = NCOLA / 4;                       // column groups
    constexpr int RG = NCW >= 32 ? 1 : 32 / NCW;
    constexpr int CPL = NCW >= 32 ? NCW / 32 : 1;
    constexpr int NK = (K + RG - 1) / RG;
    constexpr bool GEMM = !CID && OKIND == K_DATA;
    static_assert(NCOLA % 4 == 0 && DR % 4 == 0 && NCOL == NCOLA, "four-column groups");
    const int rg = lane / (32 / RG);
    const int cl = lane % (32 / RG);
    float mx = 0.f;
    if (K % RG != 0 && rg >= K) return mx;
#pragma unroll
    for (int cidx = 0; cidx < CPL; ++cidx) {
        const int col = 4 * (cl + 32 * cidx);
        const int ap = col / DR, rp = col % DR;
        float wp[8];
        weights8<PAR>(w, ap, wp);
        float4 acol[GEMM ? DL : 1];
        if constexpr (GEMM) {
#pragma unroll
            for (int r = 0; r < DL; ++r) acol[r] = *reinterpret_cast<const float4*>(A + r * NCOLA + col);
        }
        auto rows = [&](auto bt_tag, int j0, int j1) {
            constexpr int BT = decltype(bt_tag)::value;
            float wb[PB][2];
            const int beta_rt = BT >= 0 ? BT : (rg >= KQP ? 1 : 0);
#pragma unroll
            for (int bp = 0; bp < PB; ++bp) {
                wb[bp][0] = beta_rt ? wp[(bp << 1) | 4] : wp[bp << 1];
                wb[bp][1] = beta_rt ? wp[1 | (bp << 1) | 4] : wp[1 | (bp << 1)];
            }
            auto emit = [&](int k, const float4& x0, const float4& x1) {
#pragma unroll
                for (int bp = 0; bp < PB; ++bp) {
                    float4 o;
                    o.x = fmaf(wb[bp][0], x0.x, wb[bp][1] * x1.x);
                    o.y = fmaf(wb[bp][0], x0.y, wb[bp][1] * x1.y);
                    o.z = fmaf(wb[bp][0], x0.z, wb[bp][1] * x1.z);
                    o.w = fmaf(wb[bp][0], x0.w, wb[bp][1] * x1.w);
                    *reinterpret_cast<float4*>(M + (bp * K + k) * NCOL + swz<NCOL, SWM>(bp * K + k, col)) = o;
                    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(o.x), fabsf(o.y)), fmaxf(fabsf(o.z), fabsf(o.w))));
                }
            };
            if constexpr (GEMM) {
                constexpr int KUMAX = DL <= 8 ? 4 : DL <= 16 ? 2 : 1;
                constexpr int NH = (BT >= 0 && K != KQP) ? NK / 2 : NK;
                constexpr int KU = NH < KUMAX ? (NH < 1 ? 1 : NH) : KUMAX;
#pragma unroll 1
                for (int jj = j0; jj < j1; jj += KU) {
                    float4 x0[KU], x1[KU];
#pragma unroll
                    for (int u = 0; u < KU; ++u) {
                        x0[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                        x1[u] = x0[u];
                    }
#pragma unroll
                    for (int r = 0; r < DL; r += 4) {
#pragma unroll
                        for (int u = 0; u < KU; ++u) {
                            const int row = rg + (jj + u) * RG;
                            const float* c0 = C + row * LDC;
#pragma unroll
                            for (int a = 0; a < PAM; ++a) {
                                const float4 v = *reinterpret_cast<const float4*>(c0 + swz<LDC, SWC>(row, a * DL + r));
                                float4& x = a ? x1[u] : x0[u];
                                const float cv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    x.x = fmaf(cv[q], acol[r + q].x, x.x);
                                    x.y = fmaf(cv[q], acol[r + q].y, x.y);
                                    x.z = fmaf(cv[q], acol[r + q].z, x.z);
                                    x.w = fmaf(cv[q], acol[r + q].w, x.w);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < KU; ++u) emit(rg + (jj + u) * RG, x0[u], x1[u]);
                }
            } else {
#pragma unroll 2
                for (int jj = j0; jj < j1; ++jj) {
                    const int k = rg + jj * RG;
                    float4 X[2];
                    x_ident4<DL, DR, PAM, NCOLA, KQP, CID, OKIND, SWC>(C, A, k, ap, rp, X);
                    emit(k, X[0], X[1]);
                }
            }
        };
        if constexpr (K == KQP) {
            rows(std::integral_constant<int, 0>{}, 0, NK);
        } else if constexpr (KQP % RG == 0) {
            rows(std::integral_constant<int, 0>{}, 0, KQP / RG);
            rows(std::integral_constant<int, 1>{}, KQP / RG, NK);
        } else {
            static_assert(NK == 1, "a lane's rows straddle beta only when it has one row");
            rows(std::integral_constant<int, -1>{}, 0, NK);
        }
    }
    return mx;
}

// One left-sweep site: M^{b'}[k][col] = sum_a w(a, a', beta(k), b') X_a[k][col].
// Returns this lane's max |M|.
//
// Lanes own columns (col = cl + 32*cidx) and every RG-th row; the rows of a
// lane split at k = KQP into the beta = 0 and beta = 1 halves, so inside each
// half the factor weights are fixed registers.
template <int K, int PAM, int DL, int PA, int DR, int PB, int NCOL, int KQP, int CID, int OKIND, int LAST,
          int TEN, int PAR, int SWC, int SWM>
__device__ __forceinline__ float left_step(const float* __restrict__ C, const float* __restrict__ A,
                                        float* __restrict__ M, const float4 w, int lane) {
    constexpr int NCOLA = PA * DR;
    constexpr int LDC = PAM * DL;
    if constexpr (TEN) {
        static_assert(SWC && SWM, "a tensor-core step reads and writes swizzled blocks");
        return gemm_tf32<K, PAM, DL, PA, DR, PB, NCOL, KQP, PAR>(C, A, M, w, lane);
    }
    // four columns per lane where a step has at least 64 float4 outputs per
    // beta' block; for a data-site product only with the swizzled layout
    // (its four row groups read the same column of four rows)
    constexpr bool DATA_PRODUCT = !CID && OKIND == K_DATA;
    if constexpr (!LAST && DR % 4 == 0 && (CID || DL % 4 == 0) && K * NCOLA / 4 >= 64 &&
                  (!DATA_PRODUCT || (SWC && DL <= 32))) {
        return left_cols4<K, PAM, DL, PA, DR, PB, NCOL, KQP, CID, OKIND, PAR, SWC, SWM>(C, A, M, w, lane);
    }
    float mx = 0.f;
    if constexpr (LAST) {
        // alpha_d is summed (DR = 1, NCOL = 1): lanes over rows
        for (int k = lane; k < K; k += 32) {
            const int beta = k / KQP;
            float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
            for (int ap = 0; ap < PA; ++ap) {
                float X[2];
                if constexpr (!CID && OKIND == K_DATA) {
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        float s = 0.f;
                        if (a < PAM) {
                            const float* crow = C + k * LDC;
#pragma unroll
                            for (int r = 0; r < DL; ++r) s = fmaf(crow[swz<LDC, SWC>(k, a * DL + r)], A[r * NCOLA + ap], s);
                        }
                        X[a] = s;
                    }
                } else {
                    x_ident<DL, DR, PAM, NCOLA, KQP, CID, OKIND, SWC>(C, A, k, ap, 0, X);
                }
                acc0 = fmaf(wsel<PAR>(w, 0, ap, beta, 0), X[0], fmaf(wsel<PAR>(w, 1, ap, beta, 0), X[1], acc0));
                if (PB == 2)
                    acc1 = fmaf(wsel<PAR>(w, 0, ap, beta, 1), X[0], fmaf(wsel<PAR>(w, 1, ap, beta, 1), X[1], acc1));
            }
            M[k] = acc0;
            mx = fmaxf(mx, fabsf(acc0));
            if (PB == 2) {
                M[K + k] = acc1;
                mx = fmaxf(mx, fabsf(acc1));
            }
        }
        return mx;
    }
    static_assert((NCOLA & (NCOLA - 1)) == 0, "power-of-two columns");
    constexpr int RG = NCOLA >= 32 ? 1 : 32 / NCOLA;     // row groups across the warp
    constexpr int CPL = NCOLA >= 32 ? NCOLA / 32 : 1;    // columns per lane
    constexpr int NK = (K + RG - 1) / RG;                 // rows per lane
    constexpr bool GEMM = !CID && OKIND == K_DATA;
    const int rg = lane / (32 / RG);
    const int cl = lane % (32 / RG);
    if (K % RG != 0 && rg >= K) return 0.f;              // K < RG: lanes past the last row idle
#pragma unroll
    for (int cidx = 0; cidx < CPL; ++cidx) {
        const int col = cl + 32 * cidx;
        const int ap = col / DR, rp = col % DR;
        float wp[8];
        weights8<PAR>(w, ap, wp);
        float acol[GEMM ? DL : 1];
        if constexpr (GEMM) {
#pragma unroll
            for (int r = 0; r < DL; ++r) acol[r] = A[r * NCOLA + col];
        }
        // rows j0 <= j < j1 of this lane (k = rg + j*RG), all with beta = BT
        // (BT < 0: beta of the lane's single row, taken at run time)
        auto rows = [&](auto bt_tag, int j0, int j1) {
            constexpr int BT = decltype(bt_tag)::value;
            float wb[PB][2];
            const int beta_rt = BT >= 0 ? BT : (rg >= KQP ? 1 : 0);
#pragma unroll
            for (int bp = 0; bp < PB; ++bp) {
                wb[bp][0] = beta_rt ? wp[(bp << 1) | 4] : wp[bp << 1];
                wb[bp][1] = beta_rt ? wp[1 | (bp << 1) | 4] : wp[1 | (bp << 1)];
            }
            if constexpr (GEMM) {
                // KU rows per pass: 2*KU independent FMA chains
                constexpr int KUMAX = DL <= 16 ? 4 : DL <= 32 ? 2 : 1;
                constexpr int NH = (BT >= 0 && K != KQP) ? NK / 2 : NK;
                constexpr int KU = NH < KUMAX ? (NH < 1 ? 1 : NH) : KUMAX;
#pragma unroll 1
                for (int jj = j0; jj < j1; jj += KU) {
                    float x0[KU], x1[KU];
#pragma unroll
                    for (int u = 0; u < KU; ++u) {
                        x0[u] = 0.f;
                        x1[u] = 0.f;
                    }
                    if constexpr (DL % 4 == 0) {
#pragma unroll
                        for (int r = 0; r < DL; r += 4) {
#pragma unroll
                            for (int u = 0; u < KU; ++u) {
                                const int row = rg + (jj + u) * RG;
                                const float* c0 = C + row * LDC;
                                const float4 v0 = *reinterpret_cast<const float4*>(c0 + swz<LDC, SWC>(row, r));
                                x0[u] = fmaf(v0.x, acol[r], x0[u]);
                                x0[u] = fmaf(v0.y, acol[r + 1], x0[u]);
                                x0[u] = fmaf(v0.z, acol[r + 2], x0[u]);
                                x0[u] = fmaf(v0.w, acol[r + 3], x0[u]);
                                if (PAM == 2) {
                                    const float4 v1 = *reinterpret_cast<const float4*>(c0 + swz<LDC, SWC>(row, DL + r));
                                    x1[u] = fmaf(v1.x, acol[r], x1[u]);
                                    x1[u] = fmaf(v1.y, acol[r + 1], x1[u]);
                                    x1[u] = fmaf(v1.z, acol[r + 2], x1[u]);
                                    x1[u] = fmaf(v1.w, acol[r + 3], x1[u]);
                                }
                            }
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < DL; ++r) {
#pragma unroll
                            for (int u = 0; u < KU; ++u) {
                                const int row = rg + (jj + u) * RG;
                                const float* c0 = C + row * LDC;
                                x0[u] = fmaf(c0[swz<LDC, SWC>(row, r)], acol[r], x0[u]);
                                if (PAM == 2) x1[u] = fmaf(c0[swz<LDC, SWC>(row, DL + r)], acol[r], x1[u]);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < KU; ++u) {
                        const int k = rg + (jj + u) * RG;
#pragma unroll
                        for (int bp = 0; bp < PB; ++bp) {
                            const float o = fmaf(wb[bp][0], x0[u], wb[bp][1] * x1[u]);
                            M[(bp * K + k) * NCOL + swz<NCOL, SWM>(bp * K + k, col)] = o;
                            mx = fmaxf(mx, fabsf(o));
                        }
                    }
                }
            } else {
#pragma unroll 4
                for (int jj = j0; jj < j1; ++jj) {
                    const int k = rg + jj * RG;
                    float X[2];
                    x_ident<DL, DR, PAM, NCOLA, KQP, CID, OKIND, SWC>(C, A, k, ap, rp, X);
#pragma unroll
                    for (int bp = 0; bp < PB; ++bp) {
                        const float o = fmaf(wb[bp][0], X[0], wb[bp][1] * X[1]);
                        M[(bp * K + k) * NCOL + swz<NCOL, SWM>(bp * K + k, col)] = o;
                        mx = fmaxf(mx, fabsf(o));
                    }
                }
            }
        };
        if constexpr (K == KQP) {
            rows(std::integral_constant<int, 0>{}, 0, NK);
        } else if constexpr (KQP % RG == 0) {
            rows(std::integral_constant<int, 0>{}, 0, KQP / RG);
            rows(std::integral_constant<int, 1>{}, KQP / RG, NK);
        } else {
            static_assert(NK == 1, "a lane's rows straddle beta only when it has one row");
            rows(std::integral_constant<int, -1>{}, 0, NK);
        }
    }
    return mx;
}

// Element (r, cc) of T, cc = bb*S + s, for the steps without a product: a
// relabeling of the kept block M (TALL, GID 1 or 2), the identity pattern
// (GID, not TALL) or a relabeling of the carry G.
template <int ROWS, int S, int KQ, int NC, int TALL, int GID, int SW>
__device__ __forceinline__ float t_relabel(const float* __restrict__ Mq, const float* __restrict__ g, int r,
                                           int bb, int s) {
    if constexpr (TALL) {
        const int row = bb * ROWS + r;
        const float* mrow = Mq + row * NC;
        if constexpr (GID == 2) {
            return mrow[swz<NC, SW>(row, s)];
        } else {
            const int j = s - bb * KQ;
            return (j >= 0 && j < NC) ? mrow[swz<NC, SW>(row, j)] : 0.f;
        }
    } else {
        const int grow = bb * ROWS + r;
        if constexpr (GID) return (grow == s) ? 1.f : 0.f;
        else return g[grow * S + s];
    }
}

// One right-sweep site: T (ROWS x PB*S) from the kept block M (TALL) or the
// carry G, then IDENT (carry = T, written to t) or DENSE (site = T, written
// straight into the MPS buffer; carry = identity).
template <int ROWS, int S, int PB, int KQ, int NC, int TALL, int GID, int RMODE, int NKIND, int SW>
__device__ __forceinline__ void right_step(const float* __restrict__ Mq, const float* __restrict__ g,
                                        float* __restrict__ t, float* __restrict__ site, int lane) {
    constexpr int COLS = PB * S;
    float* dst = (RMODE == R_DENSE) ? site : t;
    if constexpr (NKIND == K_IDL) {
        return;                                   // identity site, identity carry: nothing to form
    } else if constexpr (TALL && GID == 0) {
        // T^{bb}[r][s] = sum_j M^{bb}[r][j] G[bb*KQ + j][s]: lanes own columns
        // cc (the G column in registers) and every RG-th row
        constexpr int RG = COLS >= 32 ? 1 : 32 / COLS;
        constexpr int CPL = COLS >= 32 ? COLS / 32 : 1;
        constexpr int NR = (ROWS + RG - 1) / RG;
        constexpr int KU = NR < 4 ? NR : 4;
        static_assert((COLS & (COLS - 1)) == 0 && NR % KU == 0, "power-of-two shapes");
        const int rg = lane / (32 / RG), cl = lane % (32 / RG);
        if (ROWS % RG != 0 && rg >= ROWS) return;
#pragma unroll
        for (int cidx = 0; cidx < CPL; ++cidx) {
            const int cc = cl + 32 * cidx, bb = cc / S, s = cc % S;
            float gcol[NC];
#pragma unroll
            for (int j = 0; j < NC; ++j) gcol[j] = g[(bb * KQ + j) * S + s];
#pragma unroll 1
            for (int j0 = 0; j0 < NR; j0 += KU) {
                float v[KU];
#pragma unroll
                for (int u = 0; u < KU; ++u) {
                    const int row = bb * ROWS + rg + (j0 + u) * RG;
                    const float* mrow = Mq + row * NC;
                    v[u] = 0.f;
                    if constexpr (NC % 4 == 0) {
#pragma unroll
                        for (int j = 0; j < NC; j += 4) {
                            const float4 m4 = *reinterpret_cast<const float4*>(mrow + swz<NC, SW>(row, j));
                            v[u] = fmaf(m4.x, gcol[j], v[u]);
                            v[u] = fmaf(m4.y, gcol[j + 1], v[u]);
                            v[u] = fmaf(m4.z, gcol[j + 2], v[u]);
                            v[u] = fmaf(m4.w, gcol[j + 3], v[u]);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < NC; ++j) v[u] = fmaf(mrow[swz<NC, SW>(row, j)], gcol[j], v[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < KU; ++u) dst[(rg + (j0 + u) * RG) * COLS + cc] = v[u];
            }
        }
    } else if constexpr (S % 4 == 0) {
        // four consecutive s of one (r, bb) per lane and pass
        constexpr int C4 = COLS / 4;
#pragma unroll 4
        for (int e4 = lane; e4 < ROWS * C4; e4 += 32) {
            const int r = e4 / C4, cc = 4 * (e4 % C4), bb = cc / S, s = cc % S;
            float4 v;
            if constexpr (!TALL && !GID) {
                v = *reinterpret_cast<const float4*>(g + (bb * ROWS + r) * S + s);
            } else if constexpr (TALL && GID == 1 && KQ % 4 == 0 && NC % 4 == 0) {
                const int j = s - bb * KQ;
                v = (j >= 0 && j < NC) ? *reinterpret_cast<const float4*>(Mq + (bb * ROWS + r) * NC +
                                                                          swz<NC, SW>(bb * ROWS + r, j))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                v.x = t_relabel<ROWS, S, KQ, NC, TALL, GID, SW>(Mq, g, r, bb, s);
                v.y = t_relabel<ROWS, S, KQ, NC, TALL, GID, SW>(Mq, g, r, bb, s + 1);
                v.z = t_relabel<ROWS, S, KQ, NC, TALL, GID, SW>(Mq, g, r, bb, s + 2);
                v.w = t_relabel<ROWS, S, KQ, NC, TALL, GID, SW>(Mq, g, r, bb, s + 3);
            }
            *reinterpret_cast<float4*>(dst + 4 * e4) = v;
        }
    } else {
#pragma unroll 4
        for (int e = lane; e < ROWS * COLS; e += 32) {
            const int r = e / COLS, cc = e % COLS, bb = cc / S, s = cc % S;
            dst[e] = t_relabel<ROWS, S, KQ, NC, TALL, GID, SW>(Mq, g, r, bb, s);
        }
    }
}

// Steps of at most this many outputs are inlined into the sweep; larger ones
// are calls shared by every site of the same shape. The calls of small steps
// cost more than their work (d=7: 1.55x, d=9: 1.2x once inlined); at d=13
// inlining raises register pressure past its 255 and halves the speed.
template <int D>
constexpr int kInlineOutputs = D <= 11 ? 1024 : 0;

template <int K, int PAM, int DL, int PA, int DR, int PB, int NCOL, int KQP, int CID, int OKIND, int LAST,
          int TEN, int PAR, int SWC, int SWM>
__device__ __noinline__ float left_step_call(const float* __restrict__ C, const float* __restrict__ A,
                                             float* __restrict__ M, const float4 w, int lane) {
    return left_step<K, PAM, DL, PA, DR, PB, NCOL, KQP, CID, OKIND, LAST, TEN, PAR, SWC, SWM>(C, A, M, w, lane);
}
template <int ROWS, int S, int PB, int KQ, int NC, int TALL, int GID, int RMODE, int NKIND, int SW>
__device__ __noinline__ void right_step_call(const float* __restrict__ Mq, const float* __restrict__ g,
                                             float* __restrict__ t, float* __restrict__ site, int lane) {
    right_step<ROWS, S, PB, KQ, NC, TALL, GID, RMODE, NKIND, SW>(Mq, g, t, site, lane);
}

template <int D, int PREC>
struct Ctx {
    float* wts;
    float* mps;
    float* arena;               // per-column intermediates at their layout offsets
    int lane;
    int e2;
    int pe;                     // exponent of the last block's max |M|, not yet folded
    int col;                    // qubit column being swept (the template column gives its shapes)
    bool zero, bad;
};

// Size of the data-site products that run on the tensor cores in the mixed
// kernel (smaller ones run in FP32: the split and the fragment traffic cost
// more than the tensor pipe saves there).
constexpr int kTensorMinK = 32, kTensorMinDL = 16, kTensorMinN = 32;

// Left step I of column C runs on the tensor cores.
template <int D, int PREC, int C, int I>
struct TensorStep {
    static constexpr SiteStep st = PlanOf<D>::plan.steps[C * (D + 1) + I];
    static constexpr bool value = PREC == MLD_MIXED_TF32 && I < D && !st.cid && st.okind == K_DATA &&
                                  st.K >= kTensorMinK && st.Dl >= kTensorMinDL && st.pa * st.Dr >= kTensorMinN;
};

// The M blocks of left step I are stored swizzled: it is a tensor-core step,
// or they are the carry of one (conflict-free fragment loads); every other
// block keeps the plain layout (its reads are warp broadcasts).
template <int D, int PREC, int C, int I>
struct SwizzledBlocks {
    static constexpr bool value = TensorStep<D, PREC, C, I>::value ||
                                  (I < D && !PlanOf<D>::plan.steps[C * (D + 1) + I].tall &&
                                   TensorStep<D, PREC, C, (I < D ? I + 1 : I)>::value);
};

template <int D, int PREC, int C, int I>
__device__ __forceinline__ void left_site(Ctx<D, PREC>& x) {
    constexpr SiteStep st = PlanOf<D>::plan.steps[C * (D + 1) + I];
    constexpr int ocin = LayoutOf<D>::lay.cin[C * (D + 1) + I];
    constexpr int omout = LayoutOf<D>::lay.mout[C * (D + 1) + I];
    if (x.zero || x.bad) return;
    const float* cin = x.arena + ocin;
    float* M = x.arena + omout;
    // power-of-two renormalisation, folded: the exponent of the previous
    // block's max |M| scales this site's factor (Z is linear in it), so no
    // block is rewritten and every block stays within one site's growth of 1
    const float sc = __int_as_float((127 - x.pe) << 23);
    x.e2 += x.pe;
    float4 w = I == 0 ? make_float4(1.f, 1.f, 1.f, 1.f)
                      : *reinterpret_cast<const float4*>(x.wts + 4 * ((I - 1) * D + x.col));
    w.x *= sc; w.y *= sc; w.z *= sc; w.w *= sc;
    constexpr int TEN = TensorStep<D, PREC, C, I>::value ? 1 : 0;
    constexpr int SWC = (I > 0 && SwizzledBlocks<D, PREC, C, (I > 0 ? I - 1 : 0)>::value) ? 1 : 0;
    constexpr int SWM = SwizzledBlocks<D, PREC, C, I>::value ? 1 : 0;
    constexpr bool SMALL = st.K * st.pa * st.Dr * st.pb <= kInlineOutputs<D>;
    float mx;
    if constexpr (SMALL)
        mx = left_step<st.K, st.pam, st.Dl, st.pa, st.Dr, st.pb, st.ncol, st.kq_prev, st.cid, st.okind,
                       (I == D), TEN, st.parity, SWC, SWM>(cin, x.mps + st.offA, M, w, x.lane);
    else
        mx = left_step_call<st.K, st.pam, st.Dl, st.pa, st.Dr, st.pb, st.ncol, st.kq_prev, st.cid, st.okind,
                            (I == D), TEN, st.parity, SWC, SWM>(cin, x.mps + st.offA, M, w, x.lane);
    // max |M| over the warp as the integer maximum of the bit patterns (the
    // order of non-negative floats); its biased exponent gives frexp's
    const unsigned mbits = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
    if (mbits >= 0x7f800000u) { x.bad = true; return; }
    if (mbits == 0u) { x.zero = true; return; }
    const int ex = (int)(mbits >> 23) - 126;           // mx = m 2^ex, m in [0.5, 1)
    if (ex > 126 || ex < -125) { x.bad = true; return; }
    x.pe = ex;
    __syncwarp();
}

template <int D, int PREC, int C, int IDX>
__device__ __forceinline__ void right_site(Ctx<D, PREC>& x) {
    constexpr int I = D - IDX;
    constexpr SiteStep st = PlanOf<D>::plan.steps[C * (D + 1) + I];
    constexpr int ogin = LayoutOf<D>::lay.gin[C * (D + 1) + I];
    constexpr int otout = LayoutOf<D>::lay.tout[C * (D + 1) + I];
    constexpr int omout = LayoutOf<D>::lay.mout[C * (D + 1) + I];
    if (x.zero || x.bad) return;
    if constexpr (st.K * st.pb * st.S <= kInlineOutputs<D>)
        right_step<st.K, st.S, st.pb, st.kq, st.ncol, st.tall, st.gid, st.rmode, st.nkind,
                   SwizzledBlocks<D, PREC, C, I>::value ? 1 : 0>(
            x.arena + omout, x.arena + ogin, x.arena + otout, x.mps + st.offN, x.lane);
    else
        right_step_call<st.K, st.S, st.pb, st.kq, st.ncol, st.tall, st.gid, st.rmode, st.nkind,
                        SwizzledBlocks<D, PREC, C, I>::value ? 1 : 0>(
            x.arena + omout, x.arena + ogin, x.arena + otout, x.mps + st.offN, x.lane);
    __syncwarp();
}

template <int D, int PREC, int C, int... Is>
__device__ __forceinline__ void column(Ctx<D, PREC>& x, std::integer_sequence<int, Is...>) {
    (left_site<D, PREC, C, Is>(x), ...);
    (right_site<D, PREC, C, Is>(x), ...);
}

template <int D, int PREC, int C>
__device__ __forceinline__ void column_at(Ctx<D, PREC>& x, int col) {
    x.col = col;
    column<D, PREC, C>(x, std::make_integer_sequence<int, D + 1>{});
}

template <int D, int PREC, int... Cs>
__device__ __forceinline__ void prefix_columns(Ctx<D, PREC>& x, std::integer_sequence<int, Cs...>) {
    (column_at<D, PREC, Cs>(x, Cs), ...);
}

// Columns 0..d-2: those before the repeating pattern one by one, the rest as
// a loop over the compiled pair (C0, C0 + 1). The loop keeps the kernel's
// code within the instruction cache; measured on GB300 it is 3-6% faster at
// d = 9 (FP32), 11 and 13, and 1.4% slower for the split-TF32 kernel at
// d = 9 (three of eight columns repeat there), which stays straight-line.
template <int D, int PREC>
__device__ __forceinline__ void all_columns(Ctx<D, PREC>& x) {
    constexpr int C0 = (D == 9 && PREC == MLD_MIXED_TF32) ? D - 1 : RepeatOf<D>::c0;
    if constexpr (C0 >= D - 1) {
        prefix_columns<D, PREC>(x, std::make_integer_sequence<int, D - 1>{});
    } else {
        prefix_columns<D, PREC>(x, std::make_integer_sequence<int, C0>{});
#pragma unroll 1
        for (int c = C0; c <= D - 2; c += 2) {
            column_at<D, PREC, C0>(x, c);
            if (c + 1 <= D - 2) column_at<D, PREC, C0 + 1>(x, c + 1);
        }
    }
}

// contract the final MPS (corner column d) with all-ones vectors
template <int D, int PREC, int I>
__device__ __forceinline__ void final_site(Ctx<D, PREC>& x) {
    constexpr SiteStep st = PlanOf<D>::plan.steps[(D - 1) * (D + 1) + I];
    const float* v = x.arena + ((I & 1) ? 64 : 0);
    float* vn = x.arena + ((I & 1) ? 0 : 64);
    const float* site = x.mps + st.offN;
    for (int s = x.lane; s < st.S; s += 32) {
        float acc = 0.f;
        if constexpr (st.nkind == K_IDR) {
#pragma unroll
            for (int bb = 0; bb < st.pb; ++bb) acc += v[bb * st.S + s];
        } else if constexpr (st.nkind == K_IDL) {
            acc = v[s % st.Sl];
        } else {
            for (int sl = 0; sl < st.Sl; ++sl)
#pragma unroll
                for (int bb = 0; bb < st.pb; ++bb) acc = fmaf(v[sl], site[(sl * st.pb + bb) * st.S + s], acc);
        }
        vn[s] = acc;
    }
    __syncwarp();
}

template <int D, int PREC, int... Is>
__device__ __forceinline__ void final_all(Ctx<D, PREC>& x, std::integer_sequence<int, Is...>) {
    (final_site<D, PREC, Is>(x), ...);
}

// initial boundary MPS: all-ones product state over corner column 0
template <int D, int I>
__host__ __device__ constexpr int init_offset() {
    int o = 0;
    for (int i = 0; i < I; ++i) o += (PlanOf<D>::plan.init_sizes[i] + 3) & ~3;
    return o;
}

template <int D, int I>
__host__ __device__ constexpr int init_size() { return PlanOf<D>::plan.init_sizes[I]; }

template <int D, int PREC, int... Is>
__device__ __forceinline__ void init_all(Ctx<D, PREC>& x, std::integer_sequence<int, Is...>) {
    ((x.lane < init_size<D, Is>() ? (void)(x.mps[init_offset<D, Is>() + x.lane] = 1.f) : (void)0), ...);
}

template <int D, int PREC>
__device__ __forceinline__ void decode_unit(const ExactArgs& a, float* ws, int64_t unit, int lane);

// A unit is (syndrome, l_Z): one warp sweeps the columns shared by the two
// classes l_X = 0, 1 once and the last column once per l_X (decode_unit).
// Shared-memory mode: one unit per warp. Global-workspace mode (a.gws set,
// for states larger than a block's shared memory): a fixed set of resident
// warps, each with its own slice of the workspace, strides over the units.
template <int D, int PREC, bool GLOBAL>
__global__ void __launch_bounds__(256) decode_exact_kernel(ExactArgs a) {
    constexpr int FPW = LayoutOf<D>::lay.floats_per_warp;
    extern __shared__ float4 smem4[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if constexpr (GLOBAL) {
        const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
        float* ws = a.gws + (size_t)gw * FPW;
        for (int64_t unit = gw; unit < 2 * a.B; unit += nw) {
            decode_unit<D, PREC>(a, ws, unit, lane);
            __syncwarp();
        }
    } else {
        if (gw >= 2 * a.B) return;
        decode_unit<D, PREC>(a, reinterpret_cast<float*>(smem4) + (size_t)warp * FPW, gw, lane);
    }
}

template <int D, int PREC>
__device__ __forceinline__ void decode_unit(const ExactArgs& a, float* ws, int64_t unit, int lane) {
    constexpr int OFF_W = LayoutOf<D>::lay.off_w, OFF_MPS = LayoutOf<D>::lay.off_mps;
    constexpr int OFF_ARENA = LayoutOf<D>::lay.off_arena;
    constexpr int n = D * D;
    const int64_t b = unit >> 1;
    const int lz = (int)(unit & 1);
    Ctx<D, PREC> x;
    x.wts = ws + OFF_W;
    x.mps = ws + OFF_MPS;
    x.arena = ws + OFF_ARENA;
    x.lane = lane;
    x.e2 = 0;
    x.pe = 0;
    x.zero = false;
    x.bad = false;

    // pure error f(s) = prod_{s_k=1} T_k, representative E_{l,s} =
    // f X_L^{l_X} Z_L^{l_Z}, and the four weights of every qubit factor.
    // Z_L is Z on row 0. X_L is taken as X on column d-1 rather than column
    // 0: the two differ by X-type stabilisers, so each coset (and Z_l) is
    // the same, and the classes l_X = 0, 1 then differ only in the last
    // column, which is swept once for each from the state after column d-2.
    constexpr int W = (n - 1 + 63) / 64;
    uint64_t sw[W];
#pragma unroll
    for (int u = 0; u < W; ++u) sw[u] = a.syn[b * W + u];
    for (int q = lane; q < n; q += 32) {
        int xb = 0, zb = 0;
        const uint64_t* mk = a.dmask + (size_t)q * 2 * W;
#pragma unroll
        for (int u = 0; u < W; ++u) {
            xb ^= __popcll(sw[u] & mk[u]) & 1;
            zb ^= __popcll(sw[u] & mk[W + u]) & 1;
        }
        const int r = q / D, c = q % D;
        (void)c;
        if (lz && r == 0) zb ^= 1;
        float row[4];
        if (a.noise_mode == MLD_NOISE_TABLE) {
            const float4 v = *reinterpret_cast<const float4*>(a.noise + 4 * (size_t)q);
            row[0] = v.x; row[1] = v.y; row[2] = v.z; row[3] = v.w;
        } else {
            const float p = a.noise[b];
            row[0] = 1.f - p; row[1] = row[2] = row[3] = p * (1.f / 3.f);
        }
#pragma unroll
        for (int uv = 0; uv < 4; ++uv) {
            const int xx = xb ^ (uv & 1), zz = zb ^ (uv >> 1);
            const int pidx = (!xx && !zz) ? 0 : (xx && !zz) ? 1 : (xx && zz) ? 2 : 3;
            x.wts[4 * q + uv] = row[pidx];
        }
    }
    init_all<D, PREC>(x, std::make_integer_sequence<int, D + 1>{});
    __syncwarp();
    all_columns<D, PREC>(x);
    // the last column once per l_X, each from the state after column d-2
    // (the last column writes its sites after the old ones, so they survive)
    const int e2 = x.e2, pe = x.pe;
    const bool zero = x.zero, bad = x.bad;
#pragma unroll 1
    for (int lx = 0; lx < 2; ++lx) {
        x.e2 = e2;
        x.pe = pe;
        x.zero = zero;
        x.bad = bad;
        if (lx == 1) {
            // X on column d-1: w[u + 2v] = p[E xor X^u Z^v] becomes w[(u ^ 1) + 2v]
            if (lane < D) {
                float4* w = reinterpret_cast<float4*>(x.wts + 4 * (lane * D + D - 1));
                const float4 v = *w;
                *w = make_float4(v.y, v.x, v.w, v.z);
            }
            __syncwarp();
        }
        column_at<D, PREC, D - 1>(x, D - 1);
        double logz = -INFINITY;
        if (!x.zero && !x.bad) {
            if (lane == 0) x.arena[0] = 1.f;
            __syncwarp();
            final_all<D, PREC>(x, std::make_integer_sequence<int, D + 1>{});
            const float z = x.arena[((D + 1) & 1) ? 64 : 0];
            if (!(z == z)) x.bad = true;
            else if (z > 0.f) logz = log((double)z) + (double)x.e2 * 0.69314718055994530942;
        }
        if (lane == 0) {
            a.logP[b * 4 + lx + 2 * lz] = logz;
            if (x.bad) atomicOr(a.status, 1 << MLD_ERR_NUMERIC);
        }
        __syncwarp();
    }
}

// States up to this many floats per warp run from shared memory; larger
// ones (d >= 13) from the global workspace.
constexpr int kSharedFloatsMax = (227 * 1024) / 4;

template <int D, int PREC>
bool launch_dp(const ExactArgs& a, cudaStream_t s, int warps_per_block) {
    constexpr int FPW = LayoutOf<D>::lay.floats_per_warp;
    constexpr bool GLOBAL = FPW > kSharedFloatsMax;
    if (GLOBAL != (a.gws != nullptr)) return false;
    const size_t smem = GLOBAL ? 0 : (size_t)FPW * sizeof(float) * warps_per_block;
    if (cudaFuncSetAttribute(decode_exact_kernel<D, PREC, GLOBAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return false;
    const int64_t units = 2 * a.B;                      // (syndrome, l_Z)
    int64_t blocks = (units + warps_per_block - 1) / warps_per_block;
    if (GLOBAL && blocks > a.gws_warps / warps_per_block) blocks = a.gws_warps / warps_per_block;
    decode_exact_kernel<D, PREC, GLOBAL><<<(unsigned)blocks, 32 * warps_per_block, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess;
}

// Distances with data-site products of the tensor-core size; at the others
// a mixed-precision request runs the FP32 kernel.
template <int D>
constexpr bool kTensorPays = D == 9 || D == 11;

template <int D>
bool launch_d(const ExactArgs& a, cudaStream_t s, int warps_per_block, int precision) {
    if constexpr (kTensorPays<D>) {
        if (precision == MLD_MIXED_TF32) return launch_dp<D, MLD_MIXED_TF32>(a, s, warps_per_block);
    } else {
        if (precision == MLD_MIXED_TF32) return launch_dp<D, MLD_FP32>(a, s, warps_per_block);
    }
    if (precision == MLD_FP32) return launch_dp<D, MLD_FP32>(a, s, warps_per_block);
    return false;
}

}  // namespace exact
}  // namespace mld
