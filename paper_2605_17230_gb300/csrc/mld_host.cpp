// Host runtime: rotated-code construction, destabiliser table and the
// per-column shape plan of the boundary-MPS sweep.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "mld_internal.h"

namespace {

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
            if (!mld::plaquette_is_check(d, i, j)) continue;
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
