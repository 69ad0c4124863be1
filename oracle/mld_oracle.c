/*
 * FP64 CPU oracle for maximum-likelihood decoding (MLD) of the rotated
 * surface code under independent Pauli noise.
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled and called by the test
 * suite, by the package's smoke check and by the CPU-baseline leg of the
 * benchmark. The decoder library never links it and shares no code with it:
 * the code construction, the destabiliser solve and the contraction below are
 * written independently of the CUDA path.
 *
 * What it computes (arxiv 2605.17230):
 *  - Coset partition function Z_l(s) = sum over errors E with syndrome s and
 *    logical class l of Pr(E)  (Eq. 3, "coset_prob", Sec. 2.3), with
 *    Pr(E) = prod_q p^{(q)}_{E_q} for independent Pauli noise (Sec. 3.1.1).
 *  - The MLD decision argmax_l Z_l(s)  (Eq. 4, "mld_formal").
 *  - Z_l(s) is evaluated in the generator picture (Eq. 7, Sec. 3.2.1): a sum
 *    over binary stabiliser variables alpha_k of Pr(E_{l,s} * prod S_k^alpha_k),
 *    done EXACTLY by eliminating the variables one corner column at a time
 *    (dense transfer over the 2^(d+1) assignments of a column, one qubit
 *    factor at a time). No truncation, no approximation.
 *  - Independent checks of that contraction: brute force over all 4^n Paulis
 *    (orc_bruteforce_table, n <= 13) and plain enumeration of the 2^(n-1)
 *    stabiliser-group elements (orc_group_logz, n <= 25).
 *  - Derivatives d ln Z / d p_{q,P}: Z is linear in every qubit's probability
 *    vector, so dZ/dp_{q,P} is Z with qubit q's vector replaced by the
 *    indicator of P (orc_coset_dlogz). This is the quantity the differentiable
 *    estimation of Sec. 3.2.4 (Eq. 10) back-propagates.
 *
 * Conventions (restated from the paper's definitions; the paper's figure of
 * the lattice is not available, so this layout is the reading adopted):
 *  - data qubit (r,c), 0<=r,c<d, index r*d+c; plaquette (i,j), 0<=i,j<=d,
 *    touches qubits (i-1,j-1),(i-1,j),(i,j-1),(i,j) inside the patch;
 *    X-type iff i+j even. Interior plaquettes present; on rows 0 and d only
 *    X-type, on columns 0 and d only Z-type ones (d^2-1 checks, Sec. 2.1).
 *  - stabiliser index = column-major order of present plaquettes.
 *  - Z_L = Z on row 0, X_L = X on column 0; class = l_X + 2 l_Z with
 *    l_X = <E,Z_L>, l_Z = <E,X_L>  (order I, X, Z, Y).
 *  - Pauli code x + 2z; noise rows (p_I, p_X, p_Y, p_Z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 25
#define ORC_MAXN (ORC_MAXD * ORC_MAXD)
#define ORC_DENSE_MAXD 21

typedef struct {
    int d, n, m;                       /* qubits, stabilisers (= n-1) */
    int built;
    int pi[ORC_MAXN], pj[ORC_MAXN];    /* plaquette position of stabiliser k */
    int type[ORC_MAXN];                /* 0 = X-type, 1 = Z-type */
    int nsup[ORC_MAXN];
    int sup[ORC_MAXN][4];
    int sid[ORC_MAXD + 1][ORC_MAXD + 1];   /* stabiliser id at (i,j), -1 if absent */
    uint8_t *tx, *tz;                  /* destabilisers: [m][n] x-bits and z-bits */
} ocode;

static ocode g_codes[ORC_MAXD + 1];

static int plaquette_present(int d, int i, int j) {
    if (i >= 1 && i <= d - 1 && j >= 1 && j <= d - 1) return 1;
    if ((i == 0 || i == d) && j >= 1 && j <= d - 1 && ((i + j) % 2 == 0)) return 1;
    if ((j == 0 || j == d) && i >= 1 && i <= d - 1 && ((i + j) % 2 == 1)) return 1;
    return 0;
}

/* p^{(q)} index (paper order I, X, Y, Z) of the Pauli with bits (x, z). */
static int paper_index(int x, int z) {
    if (!x && !z) return 0;
    if (x && !z) return 1;
    if (x && z) return 2;
    return 3;
}

/* ---- GF(2) solve for destabilisers -------------------------------------
 * T_k must satisfy <T_k, S_j> = [j == k] for every generator S_j and
 * <T_k, X_L> = <T_k, Z_L> = 0, so that f(s) = prod_{s_k=1} T_k has syndrome
 * s and trivial logical class. Unknown: the 2n bits (x_0..x_{n-1},
 * z_0..z_{n-1}). Equation for an X-type S_j: sum of z over its support; for
 * a Z-type one: sum of x; for X_L: sum of z on column 0; for Z_L: sum of x on
 * row 0. Gauss-Jordan elimination with the row operations tracked in an
 * augmented identity block gives all m right-hand sides at once. */
static int build_destabilisers(ocode* C) {
    const int n = C->n, m = C->m, rows = m + 2, cols = 2 * n;
    const int W = (cols + rows + 63) / 64;
    uint64_t* A = (uint64_t*)calloc((size_t)rows * W, sizeof(uint64_t));
    int* pivcol = (int*)malloc(sizeof(int) * rows);
    if (!A || !pivcol) { free(A); free(pivcol); return -1; }
#define SETB(r, c) (A[(size_t)(r) * W + (c) / 64] |= (1ULL << ((c) % 64)))
#define GETB(r, c) ((A[(size_t)(r) * W + (c) / 64] >> ((c) % 64)) & 1ULL)
    for (int k = 0; k < m; ++k)
        for (int t = 0; t < C->nsup[k]; ++t) {
            int q = C->sup[k][t];
            SETB(k, C->type[k] == 0 ? n + q : q);
        }
    for (int r = 0; r < C->d; ++r) SETB(m, n + r * C->d);      /* X_L: z-bits on column 0 */
    for (int c = 0; c < C->d; ++c) SETB(m + 1, c);              /* Z_L: x-bits on row 0 */
    for (int r = 0; r < rows; ++r) SETB(r, cols + r);           /* augmented identity */
    int rank = 0;
    for (int col = 0; col < cols && rank < rows; ++col) {
        int piv = -1;
        for (int r = rank; r < rows; ++r) if (GETB(r, col)) { piv = r; break; }
        if (piv < 0) continue;
        if (piv != rank)
            for (int w = 0; w < W; ++w) {
                uint64_t t = A[(size_t)piv * W + w];
                A[(size_t)piv * W + w] = A[(size_t)rank * W + w];
                A[(size_t)rank * W + w] = t;
            }
        for (int r = 0; r < rows; ++r)
            if (r != rank && GETB(r, col))
                for (int w = 0; w < W; ++w) A[(size_t)r * W + w] ^= A[(size_t)rank * W + w];
        pivcol[rank++] = col;
    }
    if (rank != rows) { free(A); free(pivcol); return -2; }
    /* Row r of the reduced system reads  x[pivcol[r]] = (P e_k)[r]  with the
     * free unknowns set to 0; (P e_k)[r] is augmented column k of row r. */
    for (int k = 0; k < m; ++k) {
        uint8_t* tx = C->tx + (size_t)k * n;
        uint8_t* tz = C->tz + (size_t)k * n;
        memset(tx, 0, n);
        memset(tz, 0, n);
        for (int r = 0; r < rows; ++r)
            if (GETB(r, cols + k)) {
                int c = pivcol[r];
                if (c < n) tx[c] = 1; else tz[c - n] = 1;
            }
    }
#undef SETB
#undef GETB
    free(A);
    free(pivcol);
    return 0;
}

static const ocode* get_code(int d) {
    if (d < 3 || d > ORC_MAXD || (d % 2) == 0) return NULL;
    ocode* C = &g_codes[d];
    if (C->built) return C;
    C->d = d;
    C->n = d * d;
    int k = 0;
    for (int i = 0; i <= d; ++i)
        for (int j = 0; j <= d; ++j) C->sid[i][j] = -1;
    for (int j = 0; j <= d; ++j)
        for (int i = 0; i <= d; ++i) {
            if (!plaquette_present(d, i, j)) continue;
            C->pi[k] = i;
            C->pj[k] = j;
            C->type[k] = ((i + j) % 2 == 0) ? 0 : 1;
            C->nsup[k] = 0;
            const int rr[4] = {i - 1, i - 1, i, i}, cc[4] = {j - 1, j, j - 1, j};
            for (int t = 0; t < 4; ++t)
                if (rr[t] >= 0 && rr[t] < d && cc[t] >= 0 && cc[t] < d)
                    C->sup[k][C->nsup[k]++] = rr[t] * d + cc[t];
            C->sid[i][j] = k;
            ++k;
        }
    C->m = k;
    C->tx = (uint8_t*)malloc((size_t)C->m * C->n);
    C->tz = (uint8_t*)malloc((size_t)C->m * C->n);
    if (!C->tx || !C->tz || build_destabilisers(C) != 0) return NULL;
    C->built = 1;
    return C;
}

/* ---- representatives ------------------------------------------------------ */

static int syn_bit(const uint64_t* s, int k) { return (int)((s[k / 64] >> (k % 64)) & 1ULL); }

/* E_{l,s} = f(s) * X_L^{l_X} * Z_L^{l_Z}; f(s) = product of T_k over s_k = 1. */
static void representative(const ocode* C, const uint64_t* syn, int l, uint8_t* E) {
    const int n = C->n, d = C->d;
    uint8_t x[ORC_MAXN], z[ORC_MAXN];
    memset(x, 0, n);
    memset(z, 0, n);
    for (int k = 0; k < C->m; ++k)
        if (syn_bit(syn, k)) {
            const uint8_t* tx = C->tx + (size_t)k * n;
            const uint8_t* tz = C->tz + (size_t)k * n;
            for (int q = 0; q < n; ++q) { x[q] ^= tx[q]; z[q] ^= tz[q]; }
        }
    if (l & 1) for (int r = 0; r < d; ++r) x[r * d] ^= 1;     /* X_L on column 0 */
    if (l & 2) for (int c = 0; c < d; ++c) z[c] ^= 1;         /* Z_L on row 0 */
    for (int q = 0; q < n; ++q) E[q] = (uint8_t)(x[q] | (z[q] << 1));
}

/* ---- exact contraction of the generator-picture sum (Eq. 7) -------------
 * Variables alpha live on present plaquettes. Corner column j holds the
 * plaquettes (i, j), i = 0..d; qubit column c touches corner columns c and
 * c+1 only. psi(a) over corner column c (bit i = variable of plaquette (i,c),
 * 0 for absent plaquettes) is the sum over all variables left of column c of
 * the product of the qubit factors of columns < c. One column step:
 *    psi'(b) = sum_a psi(a) prod_r w_{(r,c)}(a_r, a_{r+1}, b_r, b_{r+1}),
 * where w_q(..) = p^{(q)}[E_q xor X^u Z^v], u (v) the xor of the variables of
 * the X-type (Z-type) plaquettes touching q. The product is multiplied in one
 * qubit at a time and each a_r summed out as soon as its last factor is in
 * (a variable-elimination order); the working array has d+2 bits: bits 0..r
 * hold b_0..b_r, bit d+1 holds a_r, bits r+1..d hold a_{r+1}..a_d. */

typedef struct { double v[16]; } qtab;   /* weight per (a_r, a_r1, b_r, b_r1) */

static void qubit_table(const ocode* C, const double* pq, int Eq, int r, int c, qtab* t) {
    /* corners of qubit (r,c): (r,c)->a_r, (r+1,c)->a_r1, (r,c+1)->b_r, (r+1,c+1)->b_r1 */
    const int ci[4] = {r, r + 1, r, r + 1}, cj[4] = {c, c, c + 1, c + 1};
    for (int m = 0; m < 16; ++m) {
        int val[4] = {m & 1, (m >> 1) & 1, (m >> 2) & 1, (m >> 3) & 1};
        int u = 0, v = 0;
        for (int t = 0; t < 4; ++t) {
            int k = C->sid[ci[t]][cj[t]];
            if (k < 0) continue;                       /* absent: variable fixed at 0 */
            if (C->type[k] == 0) u ^= val[t]; else v ^= val[t];
        }
        int x = (Eq & 1) ^ u, z = ((Eq >> 1) & 1) ^ v;
        t->v[m] = pq[paper_index(x, z)];
    }
}

static void zero_absent(const ocode* C, int col, double* psi) {
    const int d = C->d;
    size_t size = (size_t)1 << (d + 1);
    uint64_t absent = 0;
    for (int i = 0; i <= d; ++i) if (C->sid[i][col] < 0) absent |= 1ULL << i;
    for (size_t a = 0; a < size; ++a) if (a & absent) psi[a] = 0.0;
}

/* ln Z of the coset {E * S : S in stabiliser group}; noise rows [n][4].
 * work must hold 2 * 2^(d+2) doubles. */
static double coset_logz_dense(const ocode* C, const double* noise, const uint8_t* E,
                               double* work, const double* override_row, int override_q) {
    const int d = C->d;
    const size_t size = (size_t)1 << (d + 2), half = (size_t)1 << (d + 1);
    const size_t spare = half;
    double* A = work;
    double* B = work + size;
    long long scale2 = 0;
    /* column 0: all assignments of the present plaquettes weigh 1 */
    for (size_t a = 0; a < half; ++a) A[a] = 1.0;
    zero_absent(C, 0, A);
    for (int c = 0; c < d; ++c) {
        /* prepare layout: bit 0 = b_0 (free), bit d+1 = a_0, bits 1..d = a_1..a_d */
        for (size_t idx = 0; idx < size; ++idx) {
            size_t a0 = (idx >> (d + 1)) & 1;
            B[idx] = A[(idx & ~(size_t)1 & (half - 1)) | a0];
        }
        { double* t = A; A = B; B = t; }
        for (int r = 0; r < d; ++r) {
            const int q = r * d + c;
            qtab tab;
            qubit_table(C, (q == override_q) ? override_row : noise + 4 * q, E[q], r, c, &tab);
            const size_t bit1 = (size_t)1 << (r + 1);
            for (size_t idx = 0; idx < size; ++idx) {
                int br = (int)((idx >> r) & 1), br1 = (int)((idx >> (r + 1)) & 1);
                int ar1 = (int)((idx >> (d + 1)) & 1);
                size_t base = (idx & ~bit1 & ~spare) | ((size_t)ar1 << (r + 1));
                double s = 0.0;
                for (int a = 0; a < 2; ++a) {
                    size_t old = base | ((size_t)a << (d + 1));
                    s += A[old] * tab.v[a | (ar1 << 1) | (br << 2) | (br1 << 3)];
                }
                B[idx] = s;
            }
            { double* t = A; A = B; B = t; }
        }
        /* sum the last a_d (bit d+1) out; result over corner column c+1 */
        for (size_t b = 0; b < half; ++b) B[b] = A[b] + A[b | spare];
        { double* t = A; A = B; B = t; }
        zero_absent(C, c + 1, A);
        double mx = 0.0;
        for (size_t b = 0; b < half; ++b) if (fabs(A[b]) > mx) mx = fabs(A[b]);
        if (mx == 0.0) return -INFINITY;
        int e;
        frexp(mx, &e);
        for (size_t b = 0; b < half; ++b) A[b] = ldexp(A[b], -e);
        scale2 += e;
    }
    double z = 0.0;
    for (size_t b = 0; b < half; ++b) z += A[b];
    if (z <= 0.0) return -INFINITY;
    return log(z) + (double)scale2 * log(2.0);
}

static void depol_row(double p, double* row) {
    row[0] = 1.0 - p;
    row[1] = row[2] = row[3] = p / 3.0;
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ============================ exported API ================================ */

int orc_code_info(int d, int* n, int* m, int* syn_words) {
    const ocode* C = get_code(d);
    if (!C) return -1;
    *n = C->n;
    *m = C->m;
    *syn_words = (C->m + 63) / 64;
    return 0;
}

/* type[m]; support[m][4] padded with -1; lx[n] = X_L support; lz[n] = Z_L support */
int orc_layout(int d, int32_t* type, int32_t* support, uint8_t* lx, uint8_t* lz) {
    const ocode* C = get_code(d);
    if (!C) return -1;
    for (int k = 0; k < C->m; ++k) {
        type[k] = C->type[k];
        for (int t = 0; t < 4; ++t) support[4 * k + t] = t < C->nsup[k] ? C->sup[k][t] : -1;
    }
    for (int q = 0; q < C->n; ++q) {
        lx[q] = (uint8_t)((q % d) == 0);
        lz[q] = (uint8_t)((q / d) == 0);
    }
    return 0;
}

/* destabilisers as Pauli codes [m][n] */
int orc_destabilisers(int d, uint8_t* T) {
    const ocode* C = get_code(d);
    if (!C) return -1;
    for (size_t i = 0; i < (size_t)C->m * C->n; ++i) T[i] = (uint8_t)(C->tx[i] | (C->tz[i] << 1));
    return 0;
}

/* syndrome bits (uint8 [B][m]) and class (uint8 [B]) of Pauli errors E [B][n] */
int orc_syndrome_class(int d, const uint8_t* E, int64_t B, uint8_t* bits, uint8_t* cls) {
    const ocode* C = get_code(d);
    if (!C) return -1;
    const int n = C->n;
    for (int64_t b = 0; b < B; ++b) {
        const uint8_t* e = E + (size_t)b * n;
        for (int k = 0; k < C->m; ++k) {
            int s = 0;
            for (int t = 0; t < C->nsup[k]; ++t) {
                int q = C->sup[k][t];
                s ^= C->type[k] == 0 ? ((e[q] >> 1) & 1) : (e[q] & 1);
            }
            bits[(size_t)b * C->m + k] = (uint8_t)s;
        }
        int lx = 0, lz = 0;
        for (int c = 0; c < d; ++c) lx ^= e[c] & 1;           /* <E, Z_L> */
        for (int r = 0; r < d; ++r) lz ^= (e[r * d] >> 1) & 1; /* <E, X_L> */
        cls[b] = (uint8_t)(lx + 2 * lz);
    }
    return 0;
}

/* representatives E_{l,s} for all 4 classes: reps [B][4][n] */
int orc_representatives(int d, const uint64_t* syn, int64_t B, uint8_t* reps) {
    const ocode* C = get_code(d);
    if (!C) return -1;
    const int w = (C->m + 63) / 64;
    for (int64_t b = 0; b < B; ++b)
        for (int l = 0; l < 4; ++l)
            representative(C, syn + (size_t)b * w, l, reps + ((size_t)b * 4 + l) * C->n);
    return 0;
}

/* ln Z of the coset of each representative. noise_stride = 0 (shared [n][4])
 * or 4n (one table per representative). */
int orc_coset_logz(int d, const double* noise, int64_t noise_stride, const uint8_t* reps,
                   int64_t B, double* logz, int nthreads) {
    const ocode* C = get_code(d);
    if (!C || d > ORC_DENSE_MAXD) return -1;
    set_threads(nthreads);
    const size_t wsz = (size_t)2 << (d + 2);
    int err = 0;
#pragma omp parallel
    {
        double* work = (double*)malloc(wsz * sizeof(double));
        if (!work) {
#pragma omp atomic write
            err = -3;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t b = 0; b < B; ++b) {
            if (!work) continue;
            logz[b] = coset_logz_dense(C, noise + b * noise_stride, reps + (size_t)b * C->n,
                                       work, NULL, -1);
        }
        free(work);
    }
    return err;
}

/* Decode syndromes: logP[B][4] = ln Z_l(s_b), argmax[B] (ties -> lowest class;
 * -inf entries never win unless all are -inf, then class 0).
 * noise_mode 0: table [n][4] shared; 1: depolarizing p[B]; 2: tables [B][n][4]. */
int orc_decode(int d, const double* noise, int noise_mode, const uint64_t* syn, int64_t B,
               double* logP, uint8_t* argmax, int nthreads) {
    const ocode* C = get_code(d);
    if (!C || d > ORC_DENSE_MAXD) return -1;
    set_threads(nthreads);
    const int n = C->n, w = (C->m + 63) / 64;
    const size_t wsz = (size_t)2 << (d + 2);
    int err = 0;
#pragma omp parallel
    {
        double* work = (double*)malloc(wsz * sizeof(double));
        double* tab = (double*)malloc(sizeof(double) * 4 * n);
        uint8_t E[ORC_MAXN];
        if (!work || !tab) {
#pragma omp atomic write
            err = -3;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t b = 0; b < B; ++b) {
            if (!work || !tab) continue;
            const double* nz;
            if (noise_mode == 0) nz = noise;
            else if (noise_mode == 1) { for (int q = 0; q < n; ++q) depol_row(noise[b], tab + 4 * q); nz = tab; }
            else nz = noise + (size_t)b * 4 * n;
            int best = 0;
            for (int l = 0; l < 4; ++l) {
                representative(C, syn + (size_t)b * w, l, E);
                logP[b * 4 + l] = coset_logz_dense(C, nz, E, work, NULL, -1);
                if (l > 0 && logP[b * 4 + l] > logP[b * 4 + best]) best = l;
            }
            if (argmax) argmax[b] = (uint8_t)best;
        }
        free(work);
        free(tab);
    }
    return err;
}

/* d ln Z / d p_{q,P} (all four entries of every row treated as independent)
 * for the coset of each representative: out [B][n][4]. Z is multilinear in
 * the rows, so dZ/dp_{q,P} is the contraction with row q set to e_P. */
int orc_coset_dlogz(int d, const double* noise, int64_t noise_stride, const uint8_t* reps,
                    int64_t B, double* logz, double* out, int nthreads) {
    const ocode* C = get_code(d);
    if (!C || d > ORC_DENSE_MAXD) return -1;
    set_threads(nthreads);
    const int n = C->n;
    const size_t wsz = (size_t)2 << (d + 2);
    const int64_t jobs = B * (int64_t)(4 * n + 1);
    int err = 0;
#pragma omp parallel
    {
        double* work = (double*)malloc(wsz * sizeof(double));
        if (!work) {
#pragma omp atomic write
            err = -3;
        }
#pragma omp for schedule(dynamic, 8)
        for (int64_t j = 0; j < jobs; ++j) {
            if (!work) continue;
            int64_t b = j / (4 * n + 1);
            int k = (int)(j % (4 * n + 1));
            const double* nz = noise + b * noise_stride;
            const uint8_t* E = reps + (size_t)b * n;
            if (k == 4 * n) {
                logz[b] = coset_logz_dense(C, nz, E, work, NULL, -1);
            } else {
                double row[4] = {0, 0, 0, 0};
                row[k % 4] = 1.0;
                double lzq = coset_logz_dense(C, nz, E, work, row, k / 4);
                out[(size_t)b * 4 * n + k] = lzq;   /* ln dZ; divided below */
            }
        }
        free(work);
    }
    if (err) return err;
    for (int64_t b = 0; b < B; ++b)
        for (int k = 0; k < 4 * n; ++k) {
            double v = out[(size_t)b * 4 * n + k];
            out[(size_t)b * 4 * n + k] = isinf(v) && v < 0 ? 0.0 : exp(v - logz[b]);
        }
    return 0;
}

/* Brute force over all 4^n Paulis (n <= 13): Z[s][l] for every syndrome
 * index s (bit k = stabiliser k) and class l. Eq. 3 summed literally. */
int orc_bruteforce_table(int d, const double* noise, double* Z) {
    const ocode* C = get_code(d);
    if (!C || C->n > 13) return -1;
    const int n = C->n, m = C->m;
    const uint64_t total = 1ULL << (2 * n);
    memset(Z, 0, sizeof(double) * ((size_t)4 << m));
    uint8_t e[ORC_MAXN];
    for (uint64_t t = 0; t < total; ++t) {
        double pr = 1.0;
        for (int q = 0; q < n; ++q) {
            e[q] = (uint8_t)((t >> (2 * q)) & 3);
            pr *= noise[4 * q + paper_index(e[q] & 1, e[q] >> 1)];
        }
        uint64_t s = 0;
        for (int k = 0; k < m; ++k) {
            int b = 0;
            for (int u = 0; u < C->nsup[k]; ++u) {
                int q = C->sup[k][u];
                b ^= C->type[k] == 0 ? (e[q] >> 1) : (e[q] & 1);
            }
            s |= (uint64_t)b << k;
        }
        int lx = 0, lz = 0;
        for (int c = 0; c < d; ++c) lx ^= e[c] & 1;
        for (int r = 0; r < d; ++r) lz ^= e[r * d] >> 1;
        Z[s * 4 + (uint64_t)(lx + 2 * lz)] += pr;
    }
    return 0;
}

/* Plain enumeration of the stabiliser group (n <= 25): ln of
 * sum_alpha Pr(E * prod_k S_k^alpha_k), the first line of Eq. 7 summed term by
 * term (Gray-code order, each term's product recomputed from scratch). */
int orc_group_logz(int d, const double* noise, const uint8_t* rep, double* logz, int nthreads) {
    const ocode* C = get_code(d);
    if (!C || C->n > 25) return -1;
    set_threads(nthreads);
    const int n = C->n, m = C->m;
    uint32_t sx[ORC_MAXN], sz[ORC_MAXN];
    for (int k = 0; k < m; ++k) {
        sx[k] = sz[k] = 0;
        for (int t = 0; t < C->nsup[k]; ++t) {
            if (C->type[k] == 0) sx[k] |= 1u << C->sup[k][t];
            else sz[k] |= 1u << C->sup[k][t];
        }
    }
    uint32_t ex = 0, ez = 0;
    for (int q = 0; q < n; ++q) { ex |= (uint32_t)(rep[q] & 1) << q; ez |= (uint32_t)((rep[q] >> 1) & 1) << q; }
    const uint64_t total = 1ULL << m;
    const int chunks = 256;
    double sum = 0.0;
#pragma omp parallel for reduction(+ : sum) schedule(dynamic, 1)
    for (int ch = 0; ch < chunks; ++ch) {
        uint64_t lo = total * (uint64_t)ch / chunks, hi = total * (uint64_t)(ch + 1) / chunks;
        if (lo >= hi) continue;
        uint64_t g = lo ^ (lo >> 1);
        uint32_t px = ex, pz = ez;
        for (int k = 0; k < m; ++k) if ((g >> k) & 1) { px ^= sx[k]; pz ^= sz[k]; }
        double part = 0.0;
        for (uint64_t t = lo; t < hi; ++t) {
            double pr = 1.0;
            for (int q = 0; q < n; ++q)
                pr *= noise[4 * q + paper_index((px >> q) & 1, (pz >> q) & 1)];
            part += pr;
            /* Gray step t -> t+1 flips bit ctz(t+1) */
            uint64_t nx = t + 1;
            if (nx < hi) {
                int k = __builtin_ctzll(nx);
                px ^= sx[k];
                pz ^= sz[k];
            }
        }
        sum += part;
    }
    *logz = sum > 0.0 ? log(sum) : -INFINITY;
    return 0;
}
