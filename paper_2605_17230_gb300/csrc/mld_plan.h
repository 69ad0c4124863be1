// Shape plan of the boundary-MPS sweep (host and device, usable in
// constant expressions so that kernels can specialise on it).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define MLD_HD __host__ __device__
#else
#define MLD_HD
#endif

namespace mld {

constexpr int kMaxD = 25;
constexpr int kMaxN = kMaxD * kMaxD;
constexpr int kMaxSynWords = (kMaxN - 1 + 63) / 64;
constexpr int kMaxSteps = kMaxD * (kMaxD + 1);

// Kind of a boundary-MPS site tensor A[l][p][r]. Identity kinds are exact
// relabelings of the bond: they are not stored and never multiplied.
enum SiteKind : int16_t {
    K_DATA = 0,    // dense tensor stored in the MPS buffer
    K_IDR = 1,     // A[l][p][r] = [l == p*Dr + r]   (Dl = pa*Dr)
    K_IDL = 2      // A[l][p][r] = [r == p*Dl + l]   (Dr = pa*Dl)
};

// Right-sweep factorisation of the bond matrix T (rows x cols) of one site.
enum RMode : int16_t {
    R_IDENT = 0,   // cols <= rows, cols <= chi: site = identity, carry = T
    R_DENSE = 1,   // rows < cols, rows <= chi: site = T, carry = identity
    R_SVD = 2      // chi < min(rows, cols): truncated SVD keeps chi values
};

// One site i (plaquette row i, 0..d) of one column transfer c.
//
// Left sweep (apply the column MPO and bring the result to left-canonical
// form): the carry C[kappa][a*Dl + r] (K rows; a = alpha_{i-1}; r = old bond
// left of site i) is contracted with the old site A[r][a'*Dr + r'] and the
// qubit factor of qubit (i-1, c), w(alpha_{i-1}, alpha_i, beta_{i-1}, beta_i),
// giving for each beta_i = b' one block M^{b'}[kappa][a'*Dr + r'] (K x ncol).
// A tall block (K > ncol) is QR-factored; otherwise Q = I and R = M.
// The new carry stacks the R^{b'} blocks: row kappa' = b'*kq + j.
//
// Gauge. A column with no truncating bond (every right-sweep factorisation
// keeps min(rows, cols)) needs no canonical form: its tall blocks are kept
// as they are (site = M, carry = identity), so every tensor of the column
// stays entrywise non-negative and FP32 keeps relative accuracy in every
// coset. Only columns that truncate (canon = 1) are QR-canonicalised, since
// the SVD truncation is optimal only against a left-isometric left part.
struct SiteStep {
    int16_t pam = 0, pa = 0, pb = 0;   // dims of alpha_{i-1} (1 at i = 0), alpha_i, beta_i
    int16_t Dl = 0, Dr = 0;            // old MPS bonds left and right of site i
    int16_t K = 0;                     // rows of the M blocks (= rows of the incoming carry)
    int16_t ncol = 0;                  // columns of an M block: pa*Dr, or 1 at i = d (alpha_d summed)
    int16_t kq = 0;                    // min(K, ncol)
    int16_t kq_prev = 0;               // kq of site i-1 (beta_{i-1} = kappa / kq_prev); 1 at i = 0
    int16_t tall = 0;                  // K > ncol
    int16_t parity = 0;                // (i-1 + c) & 1: orientation of the qubit factor
    int16_t qubit = 0;                 // (i-1)*d + c, or -1 at i = 0
    int16_t rmode = 0;                 // right-sweep factorisation (RMode)
    int16_t S = 0;                     // new bond right of site i
    int16_t Sl = 0;                    // new bond left of site i
    int32_t offA = 0;                  // old site A in the MPS buffer (floats)
    int32_t offQ = 0;                  // tall: blocks at offQ + b*K*ncol, tau at offQ + pb*K*ncol + b*ncol
    int32_t offN = 0;                  // new site (Sl x pb x S) in the MPS buffer
    int16_t canon = 0;                 // column is QR-canonicalised (it has an R_SVD site)
    int16_t cid = 0;                   // incoming carry is an identity (skip the GEMM)
    int16_t okind = 0;                 // kind of the old site A (SiteKind)
    int16_t nkind = 0;                 // kind of the new site written by the right sweep
    int16_t gid = 0;                   // right sweep: incoming carry G is I (1) or I per beta block (2)
    int16_t pow2 = 0;                  // every dimension of this step is a power of two
    int8_t lK = 0, lncol = 0, lkq = 0, lkqp = 0, lDl = 0, lDr = 0, lS = 0, lSl = 0;   // log2 of the dims
};

struct Plan {
    int d = 0, chi = 0;
    int steps_per_col = 0;            // d + 1
    int nsteps = 0;                   // d * (d + 1)
    SiteStep steps[kMaxSteps] = {};   // column-major: steps[c*(d+1) + i]
    // per-warp shared-memory layout (floats, 4-aligned)
    int off_w = 0, off_mps = 0, off_buf0 = 0, off_buf1 = 0, off_q = 0, off_svd = 0;
    int floats_per_warp = 0;
    int max_buf = 0, max_mps = 0, max_q = 0, max_svd = 0;
    int svd_sites = 0;                // number of sites that truncate
    double flops_per_coset = 0.0;     // counted flops of this schedule
    double flops_last_col = 0.0;      // of which the last column (d-1)
    int init_sizes[kMaxD + 1] = {};   // initial product-state site sizes
};

MLD_HD constexpr bool plaquette_is_check(int d, int i, int j) {
    const bool in_rows = i >= 1 && i <= d - 1, in_cols = j >= 1 && j <= d - 1;
    if (in_rows && in_cols) return true;                                // interior
    if ((i == 0 || i == d) && in_cols) return ((i + j) & 1) == 0;       // X-type, top/bottom
    if ((j == 0 || j == d) && in_rows) return ((i + j) & 1) == 1;       // Z-type, left/right
    return false;
}

constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int align4(int x) { return (x + 3) & ~3; }
constexpr int8_t log2_or_zero(int x, int& ok) {
    int l = 0;
    while ((1 << l) < x) ++l;
    if ((1 << l) != x) { ok = 0; return 0; }
    return static_cast<int8_t>(l);
}

// Shapes of every step of the sweep for (d, chi); see SiteStep.
constexpr Plan make_plan(int d, int chi) {
    Plan P{};
    P.d = d;
    P.chi = chi;
    P.steps_per_col = d + 1;
    P.nsteps = d * (d + 1);
    int D[kMaxD + 2] = {};              // D[i]: old bond left of site i; D[d+1] = 1
    for (int i = 0; i < kMaxD + 2; ++i) D[i] = 1;
    int max_buf = 4, max_mps = 0, max_q = 0, max_svd = 0;
    double flops = 0.0;
    // initial product state over corner column 0
    {
        int tot = 0;
        for (int i = 0; i <= d; ++i) {
            P.init_sizes[i] = plaquette_is_check(d, i, 0) ? 2 : 1;
            tot += align4(P.init_sizes[i]);
        }
        max_mps = tot;
    }
    int offA[kMaxD + 1] = {};
    {
        int o = 0;
        for (int i = 0; i <= d; ++i) { offA[i] = o; o += align4(P.init_sizes[i]); }
    }
    double flops_prefix = 0.0;
    for (int c = 0; c < d; ++c) {
        if (c == d - 1) flops_prefix = flops;
        SiteStep* S = &P.steps[c * (d + 1)];
        int pa[kMaxD + 1] = {}, pb[kMaxD + 1] = {};
        for (int i = 0; i <= d; ++i) {
            pa[i] = plaquette_is_check(d, i, c) ? 2 : 1;
            pb[i] = plaquette_is_check(d, i, c + 1) ? 2 : 1;
        }
        // ---- left sweep: apply the column MPO, QR the tall blocks
        int K = 1, kq_prev = 1, qoff = 0;
        for (int i = 0; i <= d; ++i) {
            SiteStep& st = S[i];
            st = SiteStep{};
            st.pam = static_cast<int16_t>(i == 0 ? 1 : pa[i - 1]);
            st.pa = static_cast<int16_t>(pa[i]);
            st.pb = static_cast<int16_t>(pb[i]);
            st.Dl = static_cast<int16_t>(D[i]);
            st.Dr = static_cast<int16_t>(D[i + 1]);
            st.K = static_cast<int16_t>(K);
            const int ncolA = pa[i] * D[i + 1];
            const int ncol = i < d ? ncolA : 1;
            st.ncol = static_cast<int16_t>(ncol);
            const int kq = cmin(K, ncol);
            st.kq = static_cast<int16_t>(kq);
            st.kq_prev = static_cast<int16_t>(kq_prev);
            st.tall = static_cast<int16_t>(K > ncol);
            st.parity = static_cast<int16_t>(((i - 1 + c) & 1));
            st.qubit = static_cast<int16_t>(i == 0 ? -1 : (i - 1) * d + c);
            st.offA = offA[i];
            st.offQ = 0;
            const int pam = st.pam, Dl = D[i], pbi = pb[i];
            max_buf = cmax(max_buf, align4(K * pam * Dl));            // incoming carry
            if (st.tall) {
                st.offQ = qoff;
                qoff += align4(pbi * K * ncol + pbi * ncol);
                max_buf = cmax(max_buf, align4(pbi * kq * ncol));     // R blocks
            } else {
                max_buf = cmax(max_buf, align4(pbi * K * ncol));      // M blocks = carry
            }
            K = pbi * kq;
            kq_prev = kq;
        }
        max_q = cmax(max_q, qoff);
        // ---- right sweep: bond matrices T (rows x pb*S), truncate to chi
        int Sr = 1;
        int newD[kMaxD + 2] = {};
        for (int i = 0; i < kMaxD + 2; ++i) newD[i] = 1;
        for (int i = d; i >= 0; --i) {
            SiteStep& st = S[i];
            const int rows = st.K, cols = st.pb * Sr;
            const int keep = cmin(chi, cmin(rows, cols));
            int mode = R_DENSE;
            if (rows == 1) mode = R_DENSE;
            else if (keep < cmin(rows, cols)) mode = R_SVD;
            else if (cols <= rows) mode = R_IDENT;
            else mode = R_DENSE;
            st.rmode = static_cast<int16_t>(mode);
            st.S = static_cast<int16_t>(Sr);
            st.Sl = static_cast<int16_t>(keep);
            max_buf = cmax(max_buf, align4(rows * cols));                // T (or T^T)
            if (mode == R_DENSE) max_buf = cmax(max_buf, align4(rows * rows));   // identity carry
            if (mode == R_SVD) max_buf = cmax(max_buf, align4(rows * keep));     // U*S carry
            if (mode == R_SVD) {
                const int nv = cmin(rows, cols);
                max_svd = cmax(max_svd, align4(nv * nv + 2 * nv));
                ++P.svd_sites;
            }
            newD[i] = keep;
            Sr = keep;
        }
        // gauge of the column, identity carries and the counted flops
        int canon = 0;
        for (int i = 0; i <= d; ++i) canon |= S[i].rmode == R_SVD;
        for (int i = 0; i <= d; ++i) {
            SiteStep& st = S[i];
            st.canon = static_cast<int16_t>(canon);
            st.cid = static_cast<int16_t>(i == 0 || (!canon && S[i - 1].tall));
            const int K = st.K, ncolA = st.pa * st.Dr, pbi = st.pb;
            // (the apply's kind of old site is known only after the previous
            // column; counted below, once okind is set)
            (void)ncolA;
            if (st.tall) {
                const int n = st.ncol;
                if (canon) {
                    for (int j = 0; j < n; ++j)                                   // Householder QR
                        flops += pbi * (2.0 * (K - j) + 4.0 * (K - j) * (n - 1 - j));
                    for (int j = 0; j < n; ++j) flops += pbi * 4.0 * (K - j) * st.S;   // Q [G; 0]
                } else {
                    flops += pbi * 2.0 * K * n * st.S;                            // M G
                }
            }
        }
        // kinds of the new sites (right sweep): IDENT writes an identity
        // relabeling (K_IDR); a DENSE step whose incoming carry is the
        // identity and whose left block was wide (Q = I) writes the
        // binary-expansion identity (K_IDL); everything else is data.
        {
            // gid = 1: the carry is the identity matrix (after a DENSE step);
            // gid = 2: the stacked identity left by a kept tall last block,
            // one identity per beta block (G^b = I_kq, kq = S = 1 at i = d)
            int gid = (S[d].tall && !canon) ? 2 : 0;
            for (int i = d; i >= 0; --i) {
                SiteStep& st = S[i];
                st.gid = static_cast<int16_t>(gid);
                if (st.rmode == R_IDENT) {
                    st.nkind = K_IDR;
                    gid = 0;
                } else if (st.rmode == R_DENSE) {
                    st.nkind = (gid && !st.tall) ? K_IDL : K_DATA;
                    gid = 1;
                } else {
                    st.nkind = K_DATA;
                    gid = 0;
                }
            }
        }
        // old-site kinds of this column come from the previous column
        for (int i = 0; i <= d; ++i) S[i].okind = static_cast<int16_t>(c == 0 ? K_DATA : P.steps[(c - 1) * (d + 1) + i].nkind);
        // apply flops: a data site against a data carry is a GEMM
        // (2 K pam Dl ncolA) plus the factor (2 pb K ncolA pam); identity
        // carries or identity sites leave the factor products only
        for (int i = 0; i <= d; ++i) {
            const SiteStep& st = S[i];
            const double ncolA = st.pa * st.Dr;
            if (!st.cid && st.okind == K_DATA) flops += 2.0 * st.K * st.pam * st.Dl * ncolA;
            flops += 2.0 * st.pb * st.K * ncolA * (st.cid ? 1 : st.pam);
        }
        // new MPS layout: only data sites are stored (overwrites the old
        // layout once the left sweep is done). The last column's sites go
        // after the old ones, so that its old sites survive the column and
        // the column can be swept again from them (a kernel may sweep it once
        // per representative of X_L, which differ only in that column).
        int old_tot = 0;
        for (int i = 0; i <= d; ++i)
            if (S[i].okind == K_DATA) old_tot += align4(S[i].Dl * S[i].pa * S[i].Dr);
        int o = c == d - 1 ? old_tot : 0;
        for (int i = 0; i <= d; ++i) {
            S[i].offN = o;
            if (S[i].nkind == K_DATA) o += align4(S[i].Sl * S[i].pb * S[i].S);
        }
        max_mps = cmax(max_mps, cmax(o, old_tot));
        for (int i = 0; i <= d; ++i) offA[i] = S[i].offN;
        for (int i = 0; i <= d; ++i) {
            SiteStep& st = S[i];
            int ok = 1;
            st.lK = log2_or_zero(st.K, ok);
            st.lncol = log2_or_zero(st.ncol, ok);
            st.lkq = log2_or_zero(st.kq, ok);
            st.lkqp = log2_or_zero(st.kq_prev, ok);
            st.lDl = log2_or_zero(st.Dl, ok);
            st.lDr = log2_or_zero(st.Dr, ok);
            st.lS = log2_or_zero(st.S, ok);
            st.lSl = log2_or_zero(st.Sl, ok);
            st.pow2 = static_cast<int16_t>(ok);
        }
        for (int i = 0; i < kMaxD + 2; ++i) D[i] = newD[i];
        D[d + 1] = 1;
    }
    P.max_buf = max_buf;
    P.max_mps = max_mps;
    P.max_q = max_q;
    P.max_svd = max_svd;
    P.off_w = 0;
    P.off_mps = align4(4 * d * d);
    P.off_buf0 = P.off_mps + align4(max_mps);
    P.off_buf1 = P.off_buf0 + align4(max_buf);
    P.off_q = P.off_buf1 + align4(max_buf);
    P.off_svd = P.off_q + align4(max_q);
    P.floats_per_warp = P.off_svd + align4(max_svd);
    P.flops_per_coset = flops;
    P.flops_last_col = flops - flops_prefix;
    return P;
}

// Shared-memory layout of the untruncated sweep (a plan without truncating
// columns). Every intermediate of a column -- the carry a left step passes to
// the next, a tall block kept until the right sweep reaches its site, the
// bond matrix T a right step passes to the one above -- lives in one per-warp
// arena only between the step that writes it and the last step that reads it
// (left step i at time i, right step i at time 2d+1-i). Offsets are assigned
// from both ends of an arena sized to the largest total of simultaneously
// live objects: each object goes to the end opposite the most recently
// written object it overlaps in time, so a growing carry chain alternates
// ends instead of fragmenting.
struct ExactLayout {
    int cin[kMaxSteps] = {};    // left step: incoming carry (when cid == 0)
    int mout[kMaxSteps] = {};   // left step: its M blocks (the next carry, or the kept tall block)
    int gin[kMaxSteps] = {};    // right step: incoming carry G (when gid == 0)
    int tout[kMaxSteps] = {};   // right step: T (R_IDENT)
    int arena = 0;              // floats of the arena
    int off_w = 0, off_mps = 0, off_arena = 0, floats_per_warp = 0;
    int ok = 0;                 // the plan truncates nowhere, so the layout applies
};

constexpr int kMaxColObj = 2 * (kMaxD + 1);

// The intermediates of column c: [start, end] step times and sizes; idm[i] /
// idt[i] index the output of left step i / the T of right step i (-1: none).
struct ColumnObjects {
    int n = 0;
    int st[kMaxColObj] = {}, en[kMaxColObj] = {}, sz[kMaxColObj] = {};
    int idm[kMaxD + 1] = {}, idt[kMaxD + 1] = {};
};

constexpr ColumnObjects column_objects(const Plan& P, int c) {
    ColumnObjects O{};
    const int d = P.d;
    const SiteStep* S = &P.steps[c * (d + 1)];
    for (int i = 0; i <= d; ++i) {
        O.st[O.n] = i;
        O.en[O.n] = S[i].tall ? 2 * d + 1 - i : i + 1;
        O.sz[O.n] = align4(S[i].pb * S[i].K * S[i].ncol);
        O.idm[i] = O.n++;
    }
    for (int i = d; i >= 0; --i) {
        O.idt[i] = -1;
        if (S[i].rmode == R_IDENT) {
            O.st[O.n] = 2 * d + 1 - i;
            O.en[O.n] = O.st[O.n] + 1;
            O.sz[O.n] = align4(S[i].K * S[i].pb * S[i].S);
            O.idt[i] = O.n++;
        }
    }
    return O;
}

constexpr ExactLayout make_exact_layout(const Plan& P) {
    ExactLayout L{};
    if (P.svd_sites != 0) return L;
    L.ok = 1;
    const int d = P.d;
    // the arena's lower bound: the largest total of live objects at one time
    int cap = 128;                                  // the final contraction's two vectors: [0, 64), [64, 128)
    for (int c = 0; c < d; ++c) {
        const ColumnObjects O = column_objects(P, c);
        for (int t = 0; t <= 2 * d + 2; ++t) {
            int live = 0;
            for (int a = 0; a < O.n; ++a)
                if (O.st[a] <= t && t <= O.en[a]) live += O.sz[a];
            cap = cmax(cap, live);
        }
    }
    int hw = cap;
    for (int c = 0; c < d; ++c) {
        const ColumnObjects O = column_objects(P, c);
        int off[kMaxColObj] = {}, top[kMaxColObj] = {};
        for (int a = 0; a < O.n; ++a) {
            // the end opposite the most recently written live object
            int recent = -1;
            for (int b = 0; b < a; ++b)
                if (O.st[a] <= O.en[b] && O.st[b] <= O.en[a] && (recent < 0 || O.st[b] >= O.st[recent]))
                    recent = b;
            const bool want_top = recent >= 0 && !top[recent];
            int o = 0;
            bool placed = false;
            if (want_top) {                         // highest free offset below the cap
                o = cap - O.sz[a];
                bool moved = true;
                while (moved && o >= 0) {
                    moved = false;
                    for (int b = 0; b < a; ++b) {
                        const bool live = O.st[a] <= O.en[b] && O.st[b] <= O.en[a];
                        if (live && o < off[b] + O.sz[b] && off[b] < o + O.sz[a]) {
                            o = off[b] - O.sz[a];
                            moved = true;
                        }
                    }
                }
                placed = o >= 0;
            }
            if (!placed) {                          // lowest free offset
                o = 0;
                bool moved = true;
                while (moved) {
                    moved = false;
                    for (int b = 0; b < a; ++b) {
                        const bool live = O.st[a] <= O.en[b] && O.st[b] <= O.en[a];
                        if (live && o < off[b] + O.sz[b] && off[b] < o + O.sz[a]) {
                            o = off[b] + O.sz[b];
                            moved = true;
                        }
                    }
                }
            }
            off[a] = o;
            top[a] = placed ? 1 : 0;
            hw = cmax(hw, o + O.sz[a]);
        }
        for (int i = 0; i <= d; ++i) {
            const int k = c * (d + 1) + i;
            L.mout[k] = off[O.idm[i]];
            L.cin[k] = i > 0 ? off[O.idm[i - 1]] : 0;
            L.tout[k] = O.idt[i] >= 0 ? off[O.idt[i]] : 0;
            L.gin[k] = i == d ? off[O.idm[d]] : (O.idt[i + 1] >= 0 ? off[O.idt[i + 1]] : 0);
        }
    }
    L.arena = hw;
    L.off_w = 0;
    L.off_mps = align4(4 * d * d);
    L.off_arena = L.off_mps + align4(P.max_mps);
    L.floats_per_warp = L.off_arena + align4(hw);
    return L;
}

// Compile-time check of a layout: objects live at the same time never share
// a float, and every object lies inside the arena.
constexpr bool exact_layout_valid(const Plan& P, const ExactLayout& L) {
    if (!L.ok) return false;
    const int d = P.d;
    for (int c = 0; c < d; ++c) {
        const ColumnObjects O = column_objects(P, c);
        int off[kMaxColObj] = {};
        for (int i = 0; i <= d; ++i) {
            off[O.idm[i]] = L.mout[c * (d + 1) + i];
            if (O.idt[i] >= 0) off[O.idt[i]] = L.tout[c * (d + 1) + i];
        }
        for (int a = 0; a < O.n; ++a) {
            if (off[a] < 0 || off[a] + O.sz[a] > L.arena || (off[a] & 3)) return false;
            for (int b = 0; b < a; ++b) {
                const bool live = O.st[a] <= O.en[b] && O.st[b] <= O.en[a];
                const bool mem = off[a] < off[b] + O.sz[b] && off[b] < off[a] + O.sz[a];
                if (live && mem) return false;
            }
        }
        for (int i = 1; i <= d; ++i)               // a left step reads what the one before it wrote
            if (L.cin[c * (d + 1) + i] != L.mout[c * (d + 1) + i - 1]) return false;
    }
    return L.arena >= 128;
}

}  // namespace mld
