// Host runtime: rotated-code construction, destabiliser table and the
// per-column shape plan of the boundary-MPS sweep.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "mld_internal.h"

namespace {

bool is_check(int d, int i, int j) {
    const bool in_rows = i >= 1 && i <= d - 1, in_cols = j >= 1 && j <= d - 1;
    if (in_rows && in_cols) return true;                                // interior
    if ((i == 0 || i == d) && in_cols) return ((i + j) & 1) == 0;       // X-type, top/bottom
    if ((j == 0 || j == d) && in_rows) return ((i + j) & 1) == 1;       // Z-type, left/right
    return false;
}

// Solve A x = e_k over GF(2) for every unit right-hand side of a set of
// constraint rows (each row a bitset over n unknowns). Rows are reduced by
// Gauss-Jordan elimination on [A | I]; columns are scanned from the last
// unknown to the first. Returns one solution per row (free unknowns = 0).
bool gf2_right_inverse(int n, const std::vector<std::vector<uint64_t>>& rows_in,
                       std::vector<std::vector<uint8_t>>* sol) {
    const int R = static_cast<int>(rows_in.size());
    const int wn = (n + 63) / 64, wr = (R + 63) / 64, W = wn + wr;
    std::vector<std::vector<uint64_t>> a(R, std::vector<uint64_t>(W, 0));
    for (int r = 0; r < R; ++r) {
        for (int w = 0; w < wn; ++w) a[r][w] = rows_in[r][w];
        a[r][wn + r / 64] |= 1ULL << (r % 64);
    }
    auto bit = [&](int r, int c) { return (a[r][c / 64] >> (c % 64)) & 1ULL; };
    std::vector<int> pivot_of_row(R, -1);
    int rank = 0;
    for (int c = n - 1; c >= 0 && rank < R; --c) {
        int p = -1;
        for (int r = rank; r < R; ++r)
            if (bit(r, c)) { p = r; break; }
        if (p < 0) continue;
        std::swap(a[p], a[rank]);
        for (int r = 0; r < R; ++r)
            if (r != rank && bit(r, c))
                for (int w = 0; w < W; ++w) a[r][w] ^= a[rank][w];
        pivot_of_row[rank] = c;
        ++rank;
    }
    if (rank != R) return false;
    sol->assign(R, std::vector<uint8_t>(n, 0));
    for (int k = 0; k < R; ++k)
        for (int r = 0; r < R; ++r)
            if (bit(r, 64 * wn + k)) (*sol)[k][pivot_of_row[r]] = 1;
    return true;
}

}  // namespace

namespace mld {

static int align4(int x) { return (x + 3) & ~3; }

// Shapes of every step of the sweep for (d, chi); see SiteStep.
Plan make_plan(int d, int chi) {
    Plan P;
    P.d = d;
    P.chi = chi;
    P.steps_per_col = d + 1;
    P.steps.resize(static_cast<size_t>(d) * (d + 1));
    std::vector<int> D(d + 2, 1);       // D[i]: old bond left of site i; D[d+1] = 1
    int max_buf = 4, max_mps = 0, max_q = 0, max_svd = 0;
    double flops = 0.0;
    // initial product state over corner column 0
    {
        int tot = 0;
        for (int i = 0; i <= d; ++i) {
            P.init_sizes[i] = is_check(d, i, 0) ? 2 : 1;
            tot += align4(P.init_sizes[i]);
        }
        max_mps = tot;
    }
    std::vector<int> offA(d + 1, 0);
    {
        int o = 0;
        for (int i = 0; i <= d; ++i) { offA[i] = o; o += align4(P.init_sizes[i]); }
    }
    for (int c = 0; c < d; ++c) {
        SiteStep* S = &P.steps[static_cast<size_t>(c) * (d + 1)];
        std::vector<int> pa(d + 1), pb(d + 1);
        for (int i = 0; i <= d; ++i) {
            pa[i] = is_check(d, i, c) ? 2 : 1;
            pb[i] = is_check(d, i, c + 1) ? 2 : 1;
        }
        // ---- left sweep: apply the column MPO, QR the tall blocks
        int K = 1, kq_prev = 1, qoff = 0;
        for (int i = 0; i <= d; ++i) {
            SiteStep& st = S[i];
            std::memset(&st, 0, sizeof(st));
            st.pam = static_cast<int16_t>(i == 0 ? 1 : pa[i - 1]);
            st.pa = static_cast<int16_t>(pa[i]);
            st.pb = static_cast<int16_t>(pb[i]);
            st.Dl = static_cast<int16_t>(D[i]);
            st.Dr = static_cast<int16_t>(D[i + 1]);
            st.K = static_cast<int16_t>(K);
            const int ncolA = pa[i] * D[i + 1];
            const int ncol = i < d ? ncolA : 1;
            st.ncol = static_cast<int16_t>(ncol);
            const int kq = std::min(K, ncol);
            st.kq = static_cast<int16_t>(kq);
            st.kq_prev = static_cast<int16_t>(kq_prev);
            st.tall = static_cast<int16_t>(K > ncol);
            st.parity = static_cast<int16_t>(((i - 1 + c) & 1));
            st.qubit = static_cast<int16_t>(i == 0 ? -1 : (i - 1) * d + c);
            st.offA = offA[i];
            st.offQ = 0;
            const int pam = st.pam, Dl = D[i], pbi = pb[i];
            max_buf = std::max(max_buf, align4(K * pam * Dl));            // incoming carry
            if (st.tall) {
                st.offQ = qoff;
                qoff += align4(pbi * K * ncol + pbi * ncol);
                max_buf = std::max(max_buf, align4(pbi * kq * ncol));     // R blocks
            } else {
                max_buf = std::max(max_buf, align4(pbi * K * ncol));      // M blocks = carry
            }
            K = pbi * kq;
            kq_prev = kq;
        }
        max_q = std::max(max_q, qoff);
        // ---- right sweep: bond matrices T (rows x pb*S), truncate to chi
        int Sr = 1;
        std::vector<int> newD(d + 2, 1);
        for (int i = d; i >= 0; --i) {
            SiteStep& st = S[i];
            const int rows = st.K, cols = st.pb * Sr;
            const int keep = std::min(chi, std::min(rows, cols));
            int mode;
            if (rows == 1) mode = R_DENSE;
            else if (keep < std::min(rows, cols)) mode = R_SVD;
            else if (cols <= rows) mode = R_IDENT;
            else mode = R_DENSE;
            st.rmode = static_cast<int16_t>(mode);
            st.S = static_cast<int16_t>(Sr);
            st.Sl = static_cast<int16_t>(keep);
            max_buf = std::max(max_buf, align4(rows * cols));                // T (or T^T)
            if (mode == R_DENSE) max_buf = std::max(max_buf, align4(rows * rows));   // identity carry
            if (mode == R_SVD) max_buf = std::max(max_buf, align4(rows * keep));     // U*S carry
            if (mode == R_SVD) {
                const int nv = std::min(rows, cols);
                max_svd = std::max(max_svd, align4(nv * nv + 2 * nv));
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
            if (st.cid) {
                flops += 1.0 * pbi * K * ncolA;                                  // A x w
            } else {
                flops += 2.0 * K * st.pam * st.Dl * ncolA;                       // C x A
                flops += 2.0 * pbi * K * ncolA * st.pam;                         // x w
            }
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
        // new MPS layout (overwrites the old one once the left sweep is done)
        int o = 0, old_tot = 0;
        for (int i = 0; i <= d; ++i) old_tot += align4(S[i].Dl * S[i].pa * S[i].Dr);
        for (int i = 0; i <= d; ++i) {
            S[i].offN = o;
            o += align4(S[i].Sl * S[i].pb * S[i].S);
        }
        max_mps = std::max(max_mps, std::max(o, old_tot));
        for (int i = 0; i <= d; ++i) offA[i] = S[i].offN;
        D = newD;
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
    return P;
}

}  // namespace mld

// ---------------------------------------------------------------- code ----

extern "C" mld_status mld_code_build_host(int d, mld_code** out);

mld_status mld_code_build_host(int d, mld_code** out) {
    if (!out) return MLD_ERR_INVALID_ARG;
    *out = nullptr;
    if (d < 3 || d > mld::kMaxD || (d % 2) == 0) return MLD_ERR_INVALID_ARG;
    mld_code* C = new (std::nothrow) mld_code();
    if (!C) return MLD_ERR_NOMEM;
    C->d = d;
    C->n = d * d;
    for (int j = 0; j <= d; ++j)
        for (int i = 0; i <= d; ++i) {
            if (!is_check(d, i, j)) continue;
            C->stab_type.push_back(((i + j) & 1) ? 1 : 0);
            int qs[4] = {-1, -1, -1, -1}, t = 0;
            const int rr[4] = {i - 1, i - 1, i, i}, cc[4] = {j - 1, j, j - 1, j};
            for (int u = 0; u < 4; ++u)
                if (rr[u] >= 0 && rr[u] < d && cc[u] >= 0 && cc[u] < d) qs[t++] = rr[u] * d + cc[u];
            for (int u = 0; u < 4; ++u) C->stab_qubits.push_back(qs[u]);
        }
    C->m = static_cast<int>(C->stab_type.size());
    C->words = (C->m + 63) / 64;
    C->lx.assign(C->n, 0);
    C->lz.assign(C->n, 0);
    for (int r = 0; r < d; ++r) C->lx[r * d] = 1;     // X_L: column 0
    for (int c = 0; c < d; ++c) C->lz[c] = 1;         // Z_L: row 0
    // Destabilisers split into a pure-Z part (for X-type checks: rows are the
    // X-type checks plus X_L, unknowns the z-bits) and a pure-X part (Z-type
    // checks plus Z_L, unknowns the x-bits).
    C->dmask.assign(static_cast<size_t>(C->n) * 2 * C->words, 0);
    const int wn = (C->n + 63) / 64;
    for (int part = 0; part < 2; ++part) {            // part 0: X-type checks -> z-bits
        std::vector<int> ids;
        std::vector<std::vector<uint64_t>> rows;
        for (int k = 0; k < C->m; ++k) {
            if (C->stab_type[k] != part) continue;
            std::vector<uint64_t> row(wn, 0);
            for (int u = 0; u < 4; ++u) {
                int q = C->stab_qubits[4 * k + u];
                if (q >= 0) row[q / 64] |= 1ULL << (q % 64);
            }
            rows.push_back(row);
            ids.push_back(k);
        }
        std::vector<uint64_t> lrow(wn, 0);
        const std::vector<uint8_t>& L = part == 0 ? C->lx : C->lz;   // commute with X_L / Z_L
        for (int q = 0; q < C->n; ++q)
            if (L[q]) lrow[q / 64] |= 1ULL << (q % 64);
        rows.push_back(lrow);
        std::vector<std::vector<uint8_t>> sol;
        if (!gf2_right_inverse(C->n, rows, &sol)) { delete C; return MLD_ERR_UNSUPPORTED; }
        const int which = part == 0 ? 1 : 0;          // X-type checks get z-bits
        for (size_t t = 0; t < ids.size(); ++t) {
            const int k = ids[t];
            for (int q = 0; q < C->n; ++q)
                if (sol[t][q])
                    C->dmask[(static_cast<size_t>(q) * 2 + which) * C->words + k / 64] |= 1ULL << (k % 64);
        }
    }
    *out = C;
    return MLD_OK;
}

// E_{l,s} = f(s) * X_L^{l_X} * Z_L^{l_Z} for l = I, X, Z, Y (host).
extern "C" mld_status mld_code_representatives(const mld_code* C, const uint64_t* syn, int64_t B,
                                               uint8_t* reps) {
    if (!C || B < 0 || (B > 0 && (!syn || !reps))) return MLD_ERR_INVALID_ARG;
    const int n = C->n, d = C->d, W = C->words;
    for (int64_t b = 0; b < B; ++b) {
        const uint64_t* s = syn + b * W;
        for (int q = 0; q < n; ++q) {
            int x = 0, z = 0;
            const uint64_t* mk = C->dmask.data() + static_cast<size_t>(q) * 2 * W;
            for (int w = 0; w < W; ++w) {
                x ^= __builtin_popcountll(s[w] & mk[w]) & 1;
                z ^= __builtin_popcountll(s[w] & mk[W + w]) & 1;
            }
            for (int l = 0; l < 4; ++l) {
                const int xx = x ^ ((l & 1) && (q % d) == 0);
                const int zz = z ^ ((l & 2) && (q / d) == 0);
                reps[(static_cast<size_t>(b) * 4 + l) * n + q] = static_cast<uint8_t>(xx | (zz << 1));
            }
        }
    }
    return MLD_OK;
}
