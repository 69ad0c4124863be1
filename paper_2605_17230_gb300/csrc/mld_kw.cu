// Kac-Ward planar solver for independent X/Z noise (Sec. 3.1.3).
//
// Under independent noise Pr(E) = prod_q Px_q(x_q) Pz_q(z_q), so the coset
// sums factorise: Z_(lX,lZ)(s) = ZX_lX(s) ZZ_lZ(s). Each part is a random-bond
// Ising model: spins on the plaquettes of one type, a coupling per qubit, two
// ghost spins for the qubits on the boundary that meets one plaquette of the
// type. With Px(e) = (1 + t (-1)^e) / 2, t = 1 - 2p, the high-temperature
// expansion gives ZX = 2^(nP - n) ES, where ES sums prod t_e s_e
// (s_e = (-1)^(representative bit)) over the even subgraphs of the graph in
// which the ghosts are tied by a path whose last edge has weight +1 (sector 0)
// or -1 (sector 1, the coset of E times the logical). Kac and Ward's formula
// for a straight-line planar drawing gives ES^2 = det(I - Lambda), Lambda over
// directed edges, Lambda[e -> f] = t_f exp(i theta / 2) with theta the turn
// from e to f (no backtracking). ES is a probability up to a positive factor,
// so ln ZX = (nP - n) ln 2 + ln|det| / 2.
//
// Device algorithm. With the directed edges ordered by the x coordinate of
// their midpoint, I - Lambda is banded (bandwidth about 3d) apart from the tie
// path's middle edge, which is ordered last as a two-row, two-column border,
// and the sector edge's two columns are the last two of the band. One warp
// eliminates one matrix with partial pivoting, streaming: only the rows and
// columns of the current band window are in shared memory (rows enter as the
// elimination reaches them; a row leaves when it has been the pivot). The
// border columns and a second copy of the two sector columns (their sector-1
// values) are carried beside the window, so both sectors share every step
// but the last: a 4 x 4 determinant per sector (the two remaining band rows,
// the two border rows). ln|det| accumulates the pivots' squared moduli as a
// mantissa and a power-of-two exponent. Complex FP32 or FP64.
//
// Floating point: ES sums signed terms. For a class far less likely than the
// leading one they cancel, and its ln Z then carries an error of order
// eps * cond(I - Lambda) relative to the leading class's Z; the leading class
// and the decision keep full accuracy (measured figures in the tests).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "mld_checks.h"
#include "mld_dem.h"
#include "mld_internal.h"
#include "mld_kw.h"

namespace mld {

// ---------------------------------------------------------------------------
// Host: the spin graph, its drawing and the ordered matrix
// ---------------------------------------------------------------------------

namespace {

struct KwEdge {
    int u, v, src;   // src: qubit, -1 weight 1, -2 sector
};

}  // namespace

std::vector<int> kw_zmap(int d) {
    std::vector<int> m((size_t)d * d);
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) m[(size_t)r * d + c] = (d - 1 - c) * d + r;
    return m;
}

bool build_kw_graph(int d, KwGraph* g) {
    if (d < 3 || (d & 1) == 0) return false;
    std::vector<double> px, py;
    std::vector<int> vid((size_t)(d + 1) * (d + 1), -1);
    auto add_vertex = [&](double x, double y) {
        px.push_back(x);
        py.push_back(y);
        return (int)px.size() - 1;
    };
    // X-type plaquette (i, j) at (j, -i)
    for (int i = 0; i <= d; ++i)
        for (int j = 0; j <= d; ++j)
            if (plaquette_is_check(d, i, j) && ((i + j) & 1) == 0) vid[(size_t)i * (d + 1) + j] = add_vertex(j, -i);
    const int n_plaq = (int)px.size();
    const double far = 3.0 * d, ymid = -0.5 * d;
    const int gl = add_vertex(-far, ymid), gr = add_vertex(d - 1 + far, ymid);
    const int ca = add_vertex(-far, -d - far), cb = add_vertex(d - 1 + far, -d - far);
    std::vector<KwEdge> E;
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            int ends[4], ne = 0;
            for (int di = 0; di < 2; ++di)
                for (int dj = 0; dj < 2; ++dj) {
                    const int v = vid[(size_t)(r + di) * (d + 1) + (c + dj)];
                    if (v >= 0) ends[ne++] = v;
                }
            const int q = r * d + c;
            if (ne == 2) {
                E.push_back({ends[0], ends[1], q});
                continue;
            }
            if (ne != 1 || (c != 0 && c != d - 1)) return false;
            const int u = ends[0], gh = c == 0 ? gl : gr;
            bool twice = false;
            for (const KwEdge& e : E) twice |= (e.u == u && e.v == gh);
            if (!twice) {
                E.push_back({u, gh, q});
            } else {
                // the plaquette's second qubit on this boundary: a bend point
                // between the plaquette and the ghost keeps the edges distinct
                const int bend = add_vertex(px[u] + (c == 0 ? -0.5 : 0.5), py[u] - 0.3);
                E.push_back({u, bend, q});
                E.push_back({bend, gh, -1});
            }
        }
    const int e_la = (int)E.size();
    E.push_back({gl, ca, -1});
    const int e_ab = (int)E.size();
    E.push_back({ca, cb, -1});
    const int e_br = (int)E.size();
    E.push_back({cb, gr, -2});
    const int m = (int)E.size();
    (void)e_la;
    // order: every edge but the border by midpoint x (then top to bottom),
    // the sector edge last of the band, the border edge after it
    std::vector<int> order;
    for (int e = 0; e < m; ++e)
        if (e != e_ab && e != e_br) order.push_back(e);
    auto mx = [&](int e) { return px[E[e].u] + px[E[e].v]; };
    auto my = [&](int e) { return py[E[e].u] + py[E[e].v]; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (mx(a) != mx(b)) return mx(a) < mx(b);
        return my(a) > my(b);
    });
    order.push_back(e_br);
    order.push_back(e_ab);
    const int N = 2 * m, Nb = N - 2;
    std::vector<int> pos_of(N);          // directed edge (2e: u->v, 2e+1: v->u) -> row
    for (int k = 0; k < m; ++k) {
        pos_of[2 * order[k]] = 2 * k;
        pos_of[2 * order[k] + 1] = 2 * k + 1;
    }
    std::vector<int> tail(N), head(N);
    for (int e = 0; e < m; ++e) {
        tail[2 * e] = E[e].u;
        head[2 * e] = E[e].v;
        tail[2 * e + 1] = E[e].v;
        head[2 * e + 1] = E[e].u;
    }
    std::vector<std::vector<int>> leaving(px.size());
    for (int k = 0; k < N; ++k) leaving[tail[k]].push_back(k);
    auto angle = [&](int k) { return atan2(py[head[k]] - py[tail[k]], px[head[k]] - px[tail[k]]); };
    // rows in elimination order
    std::vector<int> dir_at(N);
    for (int k = 0; k < N; ++k) dir_at[pos_of[k]] = k;
    g->d = d;
    g->N = N;
    g->Nb = Nb;
    g->n_plaq = n_plaq;
    g->row_start.assign(1, 0);
    g->col.clear();
    g->src.clear();
    g->ph_re.clear();
    g->ph_im.clear();
    g->ext0.assign(Nb, 0);
    int bl = 0, bu = 0;
    for (int i = 0; i < N; ++i) {
        const int k = dir_at[i];
        int ext = i;
        for (int f : leaving[head[k]]) {
            if (head[f] == tail[k]) continue;
            double th = angle(f) - angle(k);
            while (th > M_PI) th -= 2.0 * M_PI;
            while (th <= -M_PI) th += 2.0 * M_PI;
            const int j = pos_of[f];
            g->col.push_back(j);
            g->src.push_back(E[f >> 1].src);
            g->ph_re.push_back(cos(0.5 * th));
            g->ph_im.push_back(sin(0.5 * th));
            if (i < Nb && j < Nb) {
                bl = std::max(bl, i - j);
                bu = std::max(bu, j - i);
                ext = std::max(ext, j);
            }
        }
        if (i < Nb) g->ext0[i] = ext;
        g->row_start.push_back((int)g->col.size());
    }
    g->bl = bl;
    g->bu = bu;
    // the sector edge must be the band's last pair
    if (pos_of[2 * e_br] != Nb - 2 || pos_of[2 * e_br + 1] != Nb - 1) return false;
    return true;
}

}  // namespace mld

// ---------------------------------------------------------------------------
// Device: streaming banded elimination, one warp per syndrome
// ---------------------------------------------------------------------------

namespace mld {
namespace {

template <typename T>
struct Cplx;
template <>
struct Cplx<float> {
    using type = float2;
};
template <>
struct Cplx<double> {
    using type = double2;
};

constexpr int kKwMaxColsPerLane = 5;   // (bl + bu) / 32 rounded up; 5 covers d <= 25

struct KwArgs {
    // the graph (device copies)
    const int* row_start;
    const int* col;
    const int* src;
    const double2* ph;
    const int* ext0;
    const int* zmap;
    int N, Nb, bl, bu;
    int WR, WC, RS;     // window rows (bl + 1), window band columns (bl + bu + 1), row stride (WC + 4)
    int n, words;
    double cst;         // (n_plaq - n) ln 2
    size_t warp_bytes;  // shared memory per warp
    // the decode
    const uint64_t* dmask;
    const float* px;
    const float* pz;    // NULL: bit-flip noise
    const uint64_t* syn;
    int64_t B;
    double* logP;
    uint8_t* argmax;
    int* status;
};

// Per-warp shared memory: the window rows (WR band slots, then the two border
// rows; each RS entries: WC band columns by column index mod WC, the two
// border columns, the two sector-1 columns), the multipliers and active-row
// list of a step, the weights of the current part, the row map (logical row
// mod WR -> slot) and each slot's last nonzero band column.
struct KwLayout {
    size_t a, mult, wt, map, ext, act, total;
};

__host__ __device__ inline size_t kw_align(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline KwLayout kw_layout(int WR, int RS, int n, size_t cbytes) {
    KwLayout L;
    L.a = 0;
    L.mult = kw_align(L.a + (size_t)(WR + 2) * RS * cbytes);
    L.wt = kw_align(L.mult + (size_t)(WR + 2) * cbytes);
    L.map = kw_align(L.wt + (size_t)n * (cbytes / 2));
    L.ext = kw_align(L.map + (size_t)WR * 4);
    L.act = kw_align(L.ext + (size_t)(WR + 2) * 4);
    L.total = kw_align(L.act + (size_t)(WR + 2) * 4);
    return L;
}

template <typename T, typename C>
__device__ __forceinline__ C kw_entry(const KwArgs& a, const T* wt, int e, bool sector1) {
    const int s = a.src[e];
    const T w = s >= 0 ? wt[s] : (s == -1 ? T(1) : (sector1 ? T(-1) : T(1)));
    const double2 p = a.ph[e];
    C v;
    v.x = -w * (T)p.x;
    v.y = -w * (T)p.y;
    return v;
}

// Writes band row i (its diagonal and successors) into a zeroed slot.
template <typename T, typename C>
__device__ __forceinline__ void kw_load_row(const KwArgs& a, const T* wt, C* R, int i, int lane) {
    const int e0 = a.row_start[i], e1 = a.row_start[i + 1];
    for (int e = e0 + lane; e < e1; e += 32) {
        const int j = a.col[e];
        if (j < a.Nb) {
            R[j % a.WC] = kw_entry<T, C>(a, wt, e, false);
            if (j >= a.Nb - 2) R[a.WC + 2 + (j - (a.Nb - 2))] = kw_entry<T, C>(a, wt, e, true);
        } else {
            R[a.WC + (j - a.Nb)] = kw_entry<T, C>(a, wt, e, false);
        }
    }
    if (lane == 0) {
        R[i % a.WC].x = T(1);
        if (i >= a.Nb - 2) R[a.WC + 2 + (i - (a.Nb - 2))].x = T(1);
    }
}

// ln Z of one part for both sectors (returned on every lane). Weights wt[q]
// = (-1)^bit * (1 - 2p) for the part's qubits (turned-lattice index).
template <typename T>
__device__ void kw_part(const KwArgs& a, unsigned char* base, double out[2]) {
    using C = typename Cplx<T>::type;
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const KwLayout L = kw_layout(a.WR, a.RS, a.n, sizeof(C));
    C* A = reinterpret_cast<C*>(base + L.a);
    C* mult = reinterpret_cast<C*>(base + L.mult);
    const T* wt = reinterpret_cast<const T*>(base + L.wt);
    int* map = reinterpret_cast<int*>(base + L.map);
    int* ext = reinterpret_cast<int*>(base + L.ext);
    int* act = reinterpret_cast<int*>(base + L.act);
    const int WR = a.WR, WC = a.WC, RS = a.RS, Nb = a.Nb;

    // initial window: band rows 0..WR-1, columns 0..WC-1, the border rows
    for (int i = lane; i < (WR + 2) * RS; i += 32) A[i] = C{T(0), T(0)};
    for (int r = lane; r < WR; r += 32) map[r] = r;
    __syncwarp();
    const int rows0 = WR < Nb ? WR : Nb;
    for (int i = 0; i < rows0; ++i) {
        kw_load_row<T, C>(a, wt, A + (size_t)i * RS, i, lane);
        if (lane == 0) ext[i] = a.ext0[i];
    }
    for (int t = 0; t < 2; ++t) {
        const int i = Nb + t;
        C* R = A + (size_t)(WR + t) * RS;
        for (int e = a.row_start[i] + lane; e < a.row_start[i + 1]; e += 32) {
            const int j = a.col[e];
            if (j >= Nb) R[WC + (j - Nb)] = kw_entry<T, C>(a, wt, e, false);
            else {
                if (j < WC) R[j] = kw_entry<T, C>(a, wt, e, false);
                if (j >= Nb - 2) R[WC + 2 + (j - (Nb - 2))] = kw_entry<T, C>(a, wt, e, true);
            }
        }
        if (lane == 0) R[WC + t].x += T(1);
    }
    __syncwarp();

    T mant = T(1);
    int expo = 0;
    bool dead = false;
    int colk = 0;
    for (int k = 0; k < Nb - 2; ++k, colk = (colk + 1 == WC) ? 0 : colk + 1) {
        const int kend = (k + a.bl < Nb - 1) ? k + a.bl : Nb - 1;
        // pivot: the largest |entry| of column k among the band rows k..kend
        T best = T(-1);
        int bi = k;
        for (int r = k + lane; r <= kend; r += 32) {
            const C v = A[(size_t)map[r % WR] * RS + colk];
            const T m2 = v.x * v.x + v.y * v.y;
            if (m2 > best) {
                best = m2;
                bi = r;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const T ob = __shfl_xor_sync(FULL, best, o);
            const int oi = __shfl_xor_sync(FULL, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (!(best > T(0))) {
            dead = true;
            break;
        }
        if (lane == 0 && bi != k) {
            const int t0 = map[k % WR];
            map[k % WR] = map[bi % WR];
            map[bi % WR] = t0;
        }
        __syncwarp();
        const int ps = map[k % WR];
        C* P = A + (size_t)ps * RS;
        const C u = P[colk];
        const T inv2 = T(1) / best;
        const C inv = C{u.x * inv2, -u.y * inv2};
        if (lane == 0) {
            int e;
            mant *= best;
            mant = sizeof(T) == 4 ? (T)frexpf((float)mant, &e) : (T)frexp((double)mant, &e);
            expo += e;
        }
        // multipliers of the rows below (band rows k+1..kend, then the border rows)
        const int cnt1 = kend - k, ncand = cnt1 + 2;
        int nact = 0;
        for (int base_i = 0; base_i < ncand; base_i += 32) {
            const int idx = base_i + lane;
            const bool valid = idx < ncand;
            const int s = !valid ? 0 : (idx < cnt1 ? map[(k + 1 + idx) % WR] : WR + (idx - cnt1));
            C v = C{T(0), T(0)};
            if (valid) v = A[(size_t)s * RS + colk];
            const bool nz = valid && (v.x != T(0) || v.y != T(0));
            const unsigned bal = __ballot_sync(FULL, nz);
            if (nz) {
                const int slot = nact + __popc(bal & ((1u << lane) - 1u));
                act[slot] = s;
                mult[slot] = C{v.x * inv.x - v.y * inv.y, v.x * inv.y + v.y * inv.x};
                A[(size_t)s * RS + colk] = C{T(0), T(0)};
            }
            nact += __popc(bal);
        }
        const int extp = ext[ps];
        __syncwarp();
        // the pivot row's columns k+1..extp (lane-strided) and its four extra columns
        C U[kKwMaxColsPerLane];
        int pc[kKwMaxColsPerLane];
#pragma unroll
        for (int t = 0; t < kKwMaxColsPerLane; ++t) {
            const int c = k + 1 + lane + 32 * t;
            int p = colk + 1 + lane + 32 * t;
            if (p >= WC) p -= WC;
            pc[t] = c <= extp ? p : -1;
            U[t] = c <= extp ? P[p] : C{T(0), T(0)};
        }
        const C Ux = lane < 4 ? P[WC + lane] : C{T(0), T(0)};
        for (int q = 0; q < nact; ++q) {
            const int s = act[q];
            const C m = mult[q];
            C* R = A + (size_t)s * RS;
#pragma unroll
            for (int t = 0; t < kKwMaxColsPerLane; ++t) {
                if (pc[t] >= 0) {
                    C r = R[pc[t]];
                    r.x -= m.x * U[t].x - m.y * U[t].y;
                    r.y -= m.x * U[t].y + m.y * U[t].x;
                    R[pc[t]] = r;
                }
            }
            if (lane < 4) {
                C r = R[WC + lane];
                r.x -= m.x * Ux.x - m.y * Ux.y;
                r.y -= m.x * Ux.y + m.y * Ux.x;
                R[WC + lane] = r;
            }
            if (lane == 0 && s < WR && ext[s] < extp) ext[s] = extp;
        }
        __syncwarp();
        // the pivot row leaves; row k + WR takes its slot; column k + WC enters
        const int rin = k + WR;
        if (rin < Nb) {
            for (int i = lane; i < RS; i += 32) P[i] = C{T(0), T(0)};
            __syncwarp();
            kw_load_row<T, C>(a, wt, P, rin, lane);
            if (lane == 0) ext[ps] = a.ext0[rin];
        }
        const int jn = k + WC;
        if (jn < Nb && lane < 2) {
            const int i = Nb + lane;
            for (int e = a.row_start[i]; e < a.row_start[i + 1]; ++e)
                if (a.col[e] == jn) A[(size_t)(WR + lane) * RS + colk] = kw_entry<T, C>(a, wt, e, false);
        }
        __syncwarp();
    }

    // the last two band rows and the border rows against the sector columns
    // (regular: sector 0; the carried copies: sector 1) and the border columns
    // ln prod |u_kk|^2 (the mantissa and exponent live on lane 0)
    const double lm = __shfl_sync(FULL, log((double)mant) + (double)expo * 0.69314718055994530942, 0);
    double res = -INFINITY;
    if (!dead && lane < 2) {
        const int rows[4] = {map[(Nb - 2) % WR], map[(Nb - 1) % WR], WR, WR + 1};
        const int cols[4] = {lane == 0 ? (Nb - 2) % WC : WC + 2, lane == 0 ? (Nb - 1) % WC : WC + 3, WC, WC + 1};
        double fr[4][4], fi[4][4];
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
                const C v = A[(size_t)rows[r] * RS + cols[c]];
                fr[r][c] = (double)v.x;
                fi[r][c] = (double)v.y;
            }
        double lg = 0.0;
        for (int c = 0; c < 4 && lg > -INFINITY; ++c) {
            int p = c;
            double bm = -1.0;
            for (int r = c; r < 4; ++r) {
                const double m2 = fr[r][c] * fr[r][c] + fi[r][c] * fi[r][c];
                if (m2 > bm) {
                    bm = m2;
                    p = r;
                }
            }
            if (!(bm > 0.0)) {
                lg = -INFINITY;
                break;
            }
            for (int x = 0; x < 4; ++x) {
                const double tr = fr[c][x], ti = fi[c][x];
                fr[c][x] = fr[p][x];
                fi[c][x] = fi[p][x];
                fr[p][x] = tr;
                fi[p][x] = ti;
            }
            lg += 0.5 * log(bm);
            const double ir = fr[c][c] / bm, ii = -fi[c][c] / bm;
            for (int r = c + 1; r < 4; ++r) {
                const double mr = fr[r][c] * ir - fi[r][c] * ii, mi = fr[r][c] * ii + fi[r][c] * ir;
                for (int x = c; x < 4; ++x) {
                    fr[r][x] -= mr * fr[c][x] - mi * fi[c][x];
                    fi[r][x] -= mr * fi[c][x] + mi * fr[c][x];
                }
            }
        }
        // ln|det| = ln prod |u_kk| + ln|det F| = lm / 2 + lg
        res = a.cst + 0.5 * (0.5 * lm + lg);
    }
    out[0] = __shfl_sync(FULL, res, 0);
    out[1] = __shfl_sync(FULL, res, 1);
    if (dead && lane == 0) atomicOr(a.status, 1 << MLD_ERR_NUMERIC);
}

}  // namespace
}  // namespace mld

namespace mld {
namespace {

// One warp per syndrome, persistent over the batch: the representative's
// bits from the destabiliser masks, the X part, the Z part (or the bit-flip
// rule), then the four classes and the argmax.
template <typename T>
__global__ void __launch_bounds__(32) kw_decode_kernel(KwArgs a) {
    extern __shared__ __align__(16) unsigned char kw_smem[];
    using C = typename Cplx<T>::type;
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    unsigned char* base = kw_smem;
    const KwLayout L = kw_layout(a.WR, a.RS, a.n, sizeof(C));
    T* wt = reinterpret_cast<T*>(base + L.wt);
    const int n = a.n;
    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        const uint64_t* sb = a.syn + b * a.words;
        bool bad = false, zany = false;
        for (int q = lane; q < n; q += 32) {
            const uint64_t* mk = a.dmask + (size_t)q * 2 * a.words;
            int x = 0;
            for (int w = 0; w < a.words; ++w) x ^= __popcll(sb[w] & mk[w]) & 1;
            const float p = a.px[q];
            bad |= !(p > 0.f && p < 1.f);
            wt[q] = (x ? T(-1) : T(1)) * (T(1) - T(2) * (T)p);
            if (!a.pz) {
                int z = 0;
                for (int w = 0; w < a.words; ++w) z ^= __popcll(sb[w] & mk[a.words + w]) & 1;
                zany |= z != 0;
            }
        }
        __syncwarp();
        double lx[2], lz[2];
        kw_part<T>(a, base, lx);
        if (a.pz) {
            __syncwarp();
            for (int qt = lane; qt < n; qt += 32) {
                const int q = a.zmap[qt];
                const uint64_t* mk = a.dmask + (size_t)q * 2 * a.words;
                int z = 0;
                for (int w = 0; w < a.words; ++w) z ^= __popcll(sb[w] & mk[a.words + w]) & 1;
                const float p = a.pz[q];
                bad |= !(p > 0.f && p < 1.f);
                wt[qt] = (z ? T(-1) : T(1)) * (T(1) - T(2) * (T)p);
            }
            __syncwarp();
            kw_part<T>(a, base, lz);
        } else {
            // no Z errors: only the coset holding the identity's z-part has
            // weight, and only if the representative has no z-bits
            zany = __any_sync(FULL, zany);
            lz[0] = zany ? -INFINITY : 0.0;
            lz[1] = -INFINITY;
        }
        bad = __any_sync(FULL, bad);
        if (lane == 0) {
            if (bad) atomicOr(a.status, 1 << MLD_ERR_INVALID_ARG);
            int best = 0;
            double v[4];
            for (int l = 0; l < 4; ++l) {
                v[l] = lx[l & 1] + lz[l >> 1];
                if (v[l] > v[best]) best = l;
                a.logP[b * 4 + l] = v[l];
            }
            if (a.argmax) a.argmax[b] = (uint8_t)best;
        }
        __syncwarp();
    }
}

std::mutex g_kw_mutex;

// The code's Kac-Ward tables on the device, built on first use.
mld_status ensure_kw(mld_code* C) {
    std::lock_guard<std::mutex> lock(g_kw_mutex);
    if (C->d_kw) return MLD_OK;
    KwGraph g;
    if (!build_kw_graph(C->d, &g)) return MLD_ERR_UNSUPPORTED;
    if ((g.bl + g.bu + 31) / 32 > kKwMaxColsPerLane) return MLD_ERR_UNSUPPORTED;
    const int nnz = (int)g.col.size();
    const std::vector<int> zmap = kw_zmap(C->d);
    std::vector<int> ints;
    ints.insert(ints.end(), g.row_start.begin(), g.row_start.end());
    ints.insert(ints.end(), g.col.begin(), g.col.end());
    ints.insert(ints.end(), g.src.begin(), g.src.end());
    ints.insert(ints.end(), g.ext0.begin(), g.ext0.end());
    ints.insert(ints.end(), zmap.begin(), zmap.end());
    const size_t ph_off = kw_align(ints.size() * sizeof(int));
    std::vector<double> ph((size_t)2 * nnz);
    for (int e = 0; e < nnz; ++e) {
        ph[2 * (size_t)e] = g.ph_re[e];
        ph[2 * (size_t)e + 1] = g.ph_im[e];
    }
    const size_t bytes = ph_off + ph.size() * sizeof(double);
    void* blob = nullptr;
    if (cudaMalloc(&blob, bytes) != cudaSuccess) return MLD_ERR_NOMEM;
    if (cudaMemcpy(blob, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy((char*)blob + ph_off, ph.data(), ph.size() * sizeof(double), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cudaFree(blob);
        return MLD_ERR_CUDA;
    }
    C->kw_N = g.N;
    C->kw_Nb = g.Nb;
    C->kw_bl = g.bl;
    C->kw_bu = g.bu;
    C->kw_nplaq = g.n_plaq;
    C->kw_nnz = nnz;
    C->kw_ph_off = ph_off;
    C->d_kw = blob;
    return MLD_OK;
}

template <typename T>
mld_status launch_kw(KwArgs a, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    const KwLayout L = kw_layout(a.WR, a.RS, a.n, sizeof(C));
    a.warp_bytes = L.total;
    int dev = 0, sms = 0, smem_max = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return MLD_ERR_CUDA;
    if (L.total > (size_t)smem_max) return MLD_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(kw_decode_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total) !=
        cudaSuccess)
        return MLD_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kw_decode_kernel<T>, 32, L.total) != cudaSuccess ||
        per_sm < 1)
        return MLD_ERR_UNSUPPORTED;
    int64_t blocks = (int64_t)sms * per_sm;
    if (blocks > a.B) blocks = a.B;
    kw_decode_kernel<T><<<(unsigned)blocks, 32, L.total, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? MLD_OK : MLD_ERR_CUDA;
}

}  // namespace
}  // namespace mld

extern "C" mld_status mld_decode_xz(const mld_code* Cc, const float* px, const float* pz, const uint64_t* syndromes,
                                    int64_t B, int precision, double* logP, uint8_t* argmax, void* stream) {
    using namespace mld;
    NvtxRange trace("mld_decode_xz");
    mld_code* C = const_cast<mld_code*>(Cc);
    if (!C || B < 0 || (precision != MLD_FP32 && precision != MLD_FP64)) return MLD_ERR_INVALID_ARG;
    if (B == 0) return MLD_OK;
    if (!px || !syndromes || !logP) return MLD_ERR_INVALID_ARG;
    mld_status st = ensure_code_device(C);
    if (st != MLD_OK) return st;
    st = ensure_kw(C);
    if (st != MLD_OK) return st;
    KwArgs a;
    const int* ib = reinterpret_cast<const int*>(C->d_kw);
    const int N = C->kw_N, Nb = C->kw_Nb, nnz = C->kw_nnz;
    a.row_start = ib;
    a.col = ib + (N + 1);
    a.src = a.col + nnz;
    a.ext0 = a.src + nnz;
    a.zmap = a.ext0 + Nb;
    a.ph = reinterpret_cast<const double2*>(reinterpret_cast<const char*>(C->d_kw) + C->kw_ph_off);
    a.N = N;
    a.Nb = Nb;
    a.bl = C->kw_bl;
    a.bu = C->kw_bu;
    a.WR = a.bl + 1;
    a.WC = a.bl + a.bu + 1;
    a.RS = a.WC + 4;
    a.n = C->n;
    a.words = C->words;
    a.cst = (double)(C->kw_nplaq - C->n) * 0.69314718055994530942;
    a.warp_bytes = 0;
    a.dmask = C->d_dmask;
    a.px = px;
    a.pz = pz;
    a.syn = syndromes;
    a.B = B;
    a.logP = logP;
    a.argmax = argmax;
    a.status = C->d_status;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return precision == MLD_FP64 ? launch_kw<double>(a, s) : launch_kw<float>(a, s);
}
