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
// (d <= 13) or one block of four warps (d >= 15, with look-ahead: while warps
// 1-3 apply step k to columns k+2.., warp 0 applies it to column k+1, places
// the entering row and takes step k+1's pivot and multipliers) eliminates
// one matrix with partial pivoting, streaming: only the rows and
// columns of the current band window are in shared memory (rows enter as the
// elimination reaches them; a row leaves when it has been the pivot). The
// border columns and a second copy of the two sector columns (their sector-1
// values) are carried beside the window, so both sectors share every step
// but the last: a 4 x 4 determinant per sector (the two remaining band rows,
// the two border rows). ln|det| accumulates the pivots' squared moduli as a
// mantissa and a power-of-two exponent. Complex FP32 or FP64.
//
// Floating point: ES sums signed terms, so the elimination loses accuracy
// with the conditioning of I - Lambda: a class far less likely than the
// leading one can carry an error of order eps * cond relative to the leading
// class's Z, and at low error rates (large |t|, an ill-conditioned matrix)
// even the leading class can: measured against FP64 over 4,096 syndromes,
// complex FP32 keeps the leading ln Z within 1.1e-3 at p = 0.10 up to d = 25,
// but reaches 0.097 (p = 0.05) and 0.29 (p = 0.02) at d = 25 on rare
// syndromes, and one decision of 4,096 differed at d = 17, p = 0.02. FP64 is
// the accurate mode.
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
constexpr int kKwRowSlots = 32;        // successors per row, padded (at most d + 1 at a ghost)
constexpr int kKwMaxChunks = 3;        // (bl + 2) / 32 rounded up: candidate rows of one step

struct KwArgs {
    // the graph (device copies): row i's successors at [i * 32, i * 32 + 32),
    // column -1 for padding
    const int* ecol;
    const int* esrc;
    const double2* eph;
    const int* ext0;
    const int* zmap;
    int N, Nb, bl, bu;
    int WR, WC, RS;     // window rows (bl + 1), window band columns (bl + bu + 1), row stride (WC + 4)
    int n, words;
    double cst;         // (n_plaq - n) ln 2
    // the decode
    const uint64_t* dmask;
    const float* px;
    const float* pz;    // NULL: bit-flip noise
    const uint64_t* syn;
    int64_t B;
    double* logP;
    uint8_t* argmax;
    int* status;
    double* flops;      // executed-flop counter (one atomic add per part)
};

// Warps per syndrome window of the look-ahead block kernel.
constexpr int kKwWarps = 4;

// Shared memory of the one-warp kernel: the window rows (WR band slots, then
// the two border rows; each RS entries: WC band columns by column index mod
// WC, the two border columns, the two sector-1 columns), the weights of the
// current part, the row map (logical row mod WR -> slot) and each slot's last
// nonzero band column.
struct KwLayout {
    size_t a, wt, map, ext, total;
};

__host__ __device__ inline size_t kw_align(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline KwLayout kw_layout(int WR, int RS, int n, size_t cbytes) {
    KwLayout L;
    L.a = 0;
    L.wt = kw_align(L.a + (size_t)(WR + 2) * RS * cbytes);
    L.map = kw_align(L.wt + (size_t)n * (cbytes / 2));
    L.ext = kw_align(L.map + (size_t)WR * 4);
    L.total = kw_align(L.ext + (size_t)(WR + 2) * 4);
    return L;
}

// This lane's successor of row i: its column (-1 if none) and its values in
// sector 0 and, for the sector columns, sector 1.
template <typename T, typename C>
__device__ __forceinline__ int kw_fetch(const KwArgs& a, const T* wt, int i, int lane, C& v, C& v1) {
    const int j = a.ecol[i * kKwRowSlots + lane];
    if (j >= 0) {
        const int s = a.esrc[i * kKwRowSlots + lane];
        const double2 p = a.eph[i * kKwRowSlots + lane];
        const T w = s >= 0 ? wt[s] : T(1);      // -1 and the sector edge in sector 0: weight 1
        v = C{-w * (T)p.x, -w * (T)p.y};
        v1 = s == -2 ? C{(T)p.x, (T)p.y} : v;   // the sector edge in sector 1: weight -1
    }
    return j;
}

// Writes band row i, fetched by kw_fetch on every lane, into a zeroed slot.
template <typename T, typename C>
__device__ __forceinline__ void kw_place_row(const KwArgs& a, C* R, int i, int j, const C& v, const C& v1,
                                             int lane) {
    if (j >= 0) {
        if (j < a.Nb) {
            R[j % a.WC] = v;
            if (j >= a.Nb - 2) R[a.WC + 2 + (j - (a.Nb - 2))] = v1;
        } else {
            R[a.WC + (j - a.Nb)] = v;
        }
    }
    if (lane == 0) {
        R[i % a.WC].x = T(1);
        if (i >= a.Nb - 2) R[a.WC + 2 + (i - (a.Nb - 2))].x = T(1);
    }
}

template <typename C, typename T>
__device__ __forceinline__ void kw_axpy(C& r, const C& m, const C& u) {
    r.x -= m.x * u.x - m.y * u.y;
    r.y -= m.x * u.y + m.y * u.x;
}

// ln Z of one part for both sectors (returned on every lane). Weights wt[q]
// = (-1)^bit * (1 - 2p) for the part's qubits (turned-lattice index).
template <typename T, int NT, int RU>
__device__ __forceinline__ void kw_part_warp(const KwArgs& a, unsigned char* base, double out[2]) {
    using C = typename Cplx<T>::type;
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const KwLayout L = kw_layout(a.WR, a.RS, a.n, sizeof(C));
    C* A = reinterpret_cast<C*>(base + L.a);
    const T* wt = reinterpret_cast<const T*>(base + L.wt);
    int* map = reinterpret_cast<int*>(base + L.map);
    int* ext = reinterpret_cast<int*>(base + L.ext);
    const int WR = a.WR, WC = a.WC, RS = a.RS, Nb = a.Nb;
    const C zero = C{T(0), T(0)};

    // initial window: band rows 0..WR-1 (columns 0..WC-1), the border rows
    for (int i = lane; i < (WR + 2) * RS; i += 32) A[i] = zero;
    for (int r = lane; r < WR; r += 32) map[r] = r;
    __syncwarp();
    const int rows0 = WR < Nb ? WR : Nb;
    for (int i = 0; i < rows0; ++i) {
        C v, v1;
        const int j = kw_fetch<T, C>(a, wt, i, lane, v, v1);
        kw_place_row<T, C>(a, A + (size_t)i * RS, i, j, v, v1, lane);
        if (lane == 0) ext[i] = a.ext0[i];
    }
    // border rows: entries in the first WC band columns, the border and the
    // sector-1 columns now; later band columns when they enter the window
    // (each lane keeps its entry of both rows)
    int bj[2];
    C bv[2];
    for (int t = 0; t < 2; ++t) {
        C v1;
        bj[t] = kw_fetch<T, C>(a, wt, Nb + t, lane, bv[t], v1);
        C* R = A + (size_t)(WR + t) * RS;
        const int j = bj[t];
        if (j >= Nb) R[WC + (j - Nb)] = bv[t];
        else if (j >= 0) {
            if (j < WC) R[j] = bv[t];
            if (j >= Nb - 2) R[WC + 2 + (j - (Nb - 2))] = v1;
        }
        if (lane == 0) R[WC + t].x += T(1);
    }
    __syncwarp();

    long long rows_done = 0, cols_done = 0;   // multipliers and updated row-columns (lane 0)
    T mant = T(1);
    int expo = 0;
    bool dead = false;
    int colk = 0, kmod = 0;    // k mod WC, k mod WR
    for (int k = 0; k < Nb - 2; ++k) {
        const int kend = (k + a.bl < Nb - 1) ? k + a.bl : Nb - 1;
        // the row entering at the end of this step: fetched now, placed later
        const int rin = k + WR;
        C nv = zero, nv1 = zero;
        int nj = -1, next = 0;
        if (rin < Nb) {
            nj = kw_fetch<T, C>(a, wt, rin, lane, nv, nv1);
            next = a.ext0[rin];
        }
        // pivot: the largest |entry| of column k among the band rows k..kend
        T best = T(-1);
        int boff = 0;
        for (int off = lane; off <= kend - k; off += 32) {
            int mp = kmod + off;
            if (mp >= WR) mp -= WR;
            const C v = A[(size_t)map[mp] * RS + colk];
            const T m2 = v.x * v.x + v.y * v.y;
            if (m2 > best) {
                best = m2;
                boff = off;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const T ob = __shfl_xor_sync(FULL, best, o);
            const int oo = __shfl_xor_sync(FULL, boff, o);
            if (ob > best || (ob == best && oo < boff)) {
                best = ob;
                boff = oo;
            }
        }
        if (!(best > T(0))) {
            dead = true;
            break;
        }
        if (lane == 0 && boff != 0) {
            int mp = kmod + boff;
            if (mp >= WR) mp -= WR;
            const int t0 = map[kmod];
            map[kmod] = map[mp];
            map[mp] = t0;
        }
        __syncwarp();
        const int ps = map[kmod];
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
        const int extp = ext[ps];
        // multipliers of the rows below (band rows k+1..kend, then the two
        // border rows): candidate idx = 32 c + lane holds its slot and
        // multiplier in registers; the ballot marks the nonzero ones
        const int cnt1 = kend - k, ncand = cnt1 + 2;
        int sl[kKwMaxChunks];
        C mv[kKwMaxChunks];
        unsigned msk[kKwMaxChunks];
#pragma unroll
        for (int c = 0; c < kKwMaxChunks; ++c) {
            const int idx = 32 * c + lane;
            int s = 0;
            C v = zero;
            if (idx < cnt1) {
                int mp = kmod + 1 + idx;
                if (mp >= WR) mp -= WR;
                s = map[mp];
            } else if (idx < ncand) {
                s = WR + (idx - cnt1);
            }
            if (idx < ncand) v = A[(size_t)s * RS + colk];
            const bool nz = v.x != T(0) || v.y != T(0);
            msk[c] = __ballot_sync(FULL, nz);
            sl[c] = s;
            mv[c] = C{v.x * inv.x - v.y * inv.y, v.x * inv.y + v.y * inv.x};
            if (nz) {
                A[(size_t)s * RS + colk] = zero;
                if (s < WR && ext[s] < extp) ext[s] = extp;
            }
        }
        if (lane == 0) {
            int na = 0;
#pragma unroll
            for (int c = 0; c < kKwMaxChunks; ++c) na += __popc(msk[c]);
            rows_done += na;
            cols_done += (long long)na * (extp - k + 4);
        }
        // the pivot row's columns k+1..extp (lane-strided) and its four extra columns
        C U[NT];
        int pc[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int c = k + 1 + lane + 32 * t;
            int p = colk + 1 + lane + 32 * t;
            if (p >= WC) p -= WC;
            pc[t] = c <= extp ? p : -1;
            U[t] = c <= extp ? P[p] : zero;
        }
        const C Ux = lane < 4 ? P[WC + lane] : zero;
        // rank-one update, RU rows at a time: all loads, then the updates
#pragma unroll
        for (int c = 0; c < kKwMaxChunks; ++c) {
            unsigned mask = msk[c];
            while (mask) {
                int s[RU];
                C m[RU];
                bool ok[RU];
#pragma unroll
                for (int j = 0; j < RU; ++j) {
                    ok[j] = mask != 0u;
                    const int src = ok[j] ? __ffs(mask) - 1 : 0;
                    mask &= mask - 1u;
                    s[j] = __shfl_sync(FULL, sl[c], src);
                    m[j].x = __shfl_sync(FULL, mv[c].x, src);
                    m[j].y = __shfl_sync(FULL, mv[c].y, src);
                }
                C r[RU][NT], rx[RU];
#pragma unroll
                for (int j = 0; j < RU; ++j) {
#pragma unroll
                    for (int t = 0; t < NT; ++t)
                        if (ok[j] && pc[t] >= 0) r[j][t] = A[(size_t)s[j] * RS + pc[t]];
                    if (ok[j] && lane < 4) rx[j] = A[(size_t)s[j] * RS + WC + lane];
                }
#pragma unroll
                for (int j = 0; j < RU; ++j) {
#pragma unroll
                    for (int t = 0; t < NT; ++t)
                        if (ok[j] && pc[t] >= 0) {
                            kw_axpy<C, T>(r[j][t], m[j], U[t]);
                            A[(size_t)s[j] * RS + pc[t]] = r[j][t];
                        }
                    if (ok[j] && lane < 4) {
                        kw_axpy<C, T>(rx[j], m[j], Ux);
                        A[(size_t)s[j] * RS + WC + lane] = rx[j];
                    }
                }
            }
        }
        __syncwarp();
        // the pivot row leaves; row k + WR takes its slot; column k + WC
        // enters (its position is colk)
        if (rin < Nb) {
            for (int i = lane; i < RS; i += 32) P[i] = zero;
            __syncwarp();
            kw_place_row<T, C>(a, P, rin, nj, nv, nv1, lane);
            if (lane == 0) ext[ps] = next;
        }
        const int jn = k + WC;
#pragma unroll
        for (int t = 0; t < 2; ++t)
            if (bj[t] == jn && jn < Nb) A[(size_t)(WR + t) * RS + colk] = bv[t];
        __syncwarp();
        colk = colk + 1 == WC ? 0 : colk + 1;
        kmod = kmod + 1 == WR ? 0 : kmod + 1;
    }

    // ln prod |u_kk|^2 (the mantissa and exponent live on lane 0)
    const double lm = __shfl_sync(FULL, log((double)mant) + (double)expo * 0.69314718055994530942, 0);
    // the last two band rows and the border rows against the sector columns
    // (regular: sector 0; the carried copies: sector 1) and the border columns
    double res = -INFINITY;
    if (!dead && lane < 2) {
        int m0 = kmod, m1 = kmod + 1 == WR ? 0 : kmod + 1;   // k = Nb - 2 here
        const int rows[4] = {map[m0], map[m1], WR, WR + 1};
        const int cols[4] = {lane == 0 ? colk : WC + 2, lane == 0 ? (colk + 1 == WC ? 0 : colk + 1) : WC + 3, WC,
                             WC + 1};
        double fr[4][4], fi[4][4];
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
                const C v = A[(size_t)rows[r] * RS + cols[c]];
                fr[r][c] = (double)v.x;
                fi[r][c] = (double)v.y;
            }
        double lg = 0.0;
        for (int c = 0; c < 4; ++c) {
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
    // per active row a complex multiplier (6 flops), per updated column a
    // complex multiply-subtract (8 flops)
    if (lane == 0 && a.flops) atomicAdd(a.flops, 6.0 * (double)rows_done + 8.0 * (double)cols_done);
    if (dead && lane == 0) atomicOr(a.status, 1 << MLD_ERR_NUMERIC);
}

// One warp per syndrome (d <= 13), persistent over the batch: the
// representative's bits from the destabiliser masks, the X part, the Z part
// (or the bit-flip rule), then the four classes and the argmax.
template <typename T, int NT>
__global__ void __launch_bounds__(32) kw_decode_warp_kernel(KwArgs a) {
    constexpr int RU = sizeof(T) == 4 ? 4 : 2;   // rows per update group
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
        kw_part_warp<T, NT, RU>(a, base, lx);
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
            kw_part_warp<T, NT, RU>(a, base, lz);
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

// ln|det| of the 4 x 4 complex matrix A[rows[r] * RS + cols[c]], in FP64
// with partial pivoting (-inf if it is singular).
template <typename C>
__device__ __forceinline__ double kw_logdet4(const C* A, int RS, const int rows[4], const int cols[4]) {
    double fr[4][4], fi[4][4];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            const C v = A[(size_t)rows[r] * RS + cols[c]];
            fr[r][c] = (double)v.x;
            fi[r][c] = (double)v.y;
        }
    double lg = 0.0;
    for (int c = 0; c < 4; ++c) {
        int p = c;
        double bm = -1.0;
        for (int r = c; r < 4; ++r) {
            const double m2 = fr[r][c] * fr[r][c] + fi[r][c] * fi[r][c];
            if (m2 > bm) {
                bm = m2;
                p = r;
            }
        }
        if (!(bm > 0.0)) return -INFINITY;
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
    return lg;
}

// Shared memory of the look-ahead block kernel: WR + 1 band slots (one spare
// takes each step's entering row) and the two border rows, each RS entries;
// the active-row lists, multipliers and control words of two consecutive
// steps; the weights; the row map; each slot's last nonzero band column.
struct KwLayoutLA {
    size_t a, mult, wt, map, ext, act, ctl, total;
};

__host__ __device__ inline KwLayoutLA kw_layout_la(int WR, int RS, int n, size_t cbytes) {
    KwLayoutLA L;
    L.a = 0;
    L.mult = kw_align(L.a + (size_t)(WR + 3) * RS * cbytes);
    L.wt = kw_align(L.mult + (size_t)2 * (WR + 2) * cbytes);
    L.map = kw_align(L.wt + (size_t)n * (cbytes / 2));
    L.ext = kw_align(L.map + (size_t)WR * 4);
    L.act = kw_align(L.ext + (size_t)(WR + 3) * 4);
    L.ctl = kw_align(L.act + (size_t)2 * (WR + 2) * 4);
    L.total = kw_align(L.ctl + 64);
    return L;
}

// Warp 0's part of a step, for step j (column j at position colj, logical
// row j at map position kmodj): the pivot among rows j..j+bl, the row
// exchange, the pivot's squared modulus into the mantissa, the multipliers
// of the rows below (band rows, then the border rows at slots BR, BR+1) into
// the lists of buffer b, column j of those rows zeroed, their extents grown.
// Lane l holds the rows at offsets l, l + 32, l + 64 from j (slot and column
// j entry) from the pivot search to the multipliers; the exchange swaps two
// of them between lanes.
template <typename T, typename C>
__device__ __forceinline__ void kw_la_pivot(const KwArgs& a, C* A, C* mult, int* map, int* ext, int* act, int* ctl,
                                            int j, int colj, int kmodj, int b, int lane, T& mant, int& expo,
                                            long long& rows_done, long long& cols_done) {
    const unsigned FULL = 0xffffffffu;
    const int WR = a.WR, RS = a.RS, Nb = a.Nb, BR = a.WR + 1;
    const C zero = C{T(0), T(0)};
    const int kend = (j + a.bl < Nb - 1) ? j + a.bl : Nb - 1;
    const int span = kend - j;                       // offsets 0..span
    int sl[kKwMaxChunks];
    C vv[kKwMaxChunks];
    T best = T(-1);
    int boff = 0;
#pragma unroll
    for (int c = 0; c < kKwMaxChunks; ++c) {
        const int off = lane + 32 * c;
        sl[c] = 0;
        vv[c] = zero;
        if (off <= span) {
            int mp = kmodj + off;
            if (mp >= WR) mp -= WR;
            sl[c] = map[mp];
            vv[c] = A[(size_t)sl[c] * RS + colj];
            const T m2 = vv[c].x * vv[c].x + vv[c].y * vv[c].y;
            if (m2 > best) {
                best = m2;
                boff = off;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const T ob = __shfl_xor_sync(FULL, best, o);
        const int oo = __shfl_xor_sync(FULL, boff, o);
        if (ob > best || (ob == best && oo < boff)) {
            best = ob;
            boff = oo;
        }
    }
    if (!(best > T(0))) {
        if (lane == 0) ctl[b * 4 + 3] = 1;
        return;
    }
    if (boff != 0) {
        // exchange offsets 0 and boff in the map and in the lanes' registers
        const int lb = boff & 31, cb = boff >> 5;
        const int s_b = __shfl_sync(FULL, cb == 0 ? sl[0] : (cb == 1 ? sl[1] : sl[2]), lb);
        const C v_b = cb == 0 ? vv[0] : (cb == 1 ? vv[1] : vv[2]);
        const T vbx = __shfl_sync(FULL, v_b.x, lb), vby = __shfl_sync(FULL, v_b.y, lb);
        const int s_0 = __shfl_sync(FULL, sl[0], 0);
        const T v0x = __shfl_sync(FULL, vv[0].x, 0), v0y = __shfl_sync(FULL, vv[0].y, 0);
        if (lane == 0) {
            int mp = kmodj + boff;
            if (mp >= WR) mp -= WR;
            map[kmodj] = s_b;
            map[mp] = s_0;
            sl[0] = s_b;
            vv[0] = C{vbx, vby};
        }
        if (lane == lb) {
#pragma unroll
            for (int c = 0; c < kKwMaxChunks; ++c)
                if (c == cb) {
                    sl[c] = s_0;
                    vv[c] = C{v0x, v0y};
                }
        }
    }
    const int ps = __shfl_sync(FULL, sl[0], 0);
    const C u = C{__shfl_sync(FULL, vv[0].x, 0), __shfl_sync(FULL, vv[0].y, 0)};
    const T inv2 = T(1) / best;
    const C inv = C{u.x * inv2, -u.y * inv2};
    if (lane == 0) {
        int e;
        mant *= best;
        mant = sizeof(T) == 4 ? (T)frexpf((float)mant, &e) : (T)frexp((double)mant, &e);
        expo += e;
    }
    const int extp = ext[ps];
    int* actb = act + b * (WR + 2);
    C* multb = mult + b * (WR + 2);
    int nact = 0;
    // band rows: offsets 1..span, from the registers
#pragma unroll
    for (int c = 0; c < kKwMaxChunks; ++c) {
        const int off = lane + 32 * c;
        const bool nz = off >= 1 && off <= span && (vv[c].x != T(0) || vv[c].y != T(0));
        const unsigned bal = __ballot_sync(FULL, nz);
        if (nz) {
            const int q = nact + __popc(bal & ((1u << lane) - 1u));
            const int s = sl[c];
            actb[q] = s;
            multb[q] = C{vv[c].x * inv.x - vv[c].y * inv.y, vv[c].x * inv.y + vv[c].y * inv.x};
            A[(size_t)s * RS + colj] = zero;
            if (ext[s] < extp) ext[s] = extp;
        }
        nact += __popc(bal);
    }
    // the border rows
    {
        C v = zero;
        if (lane < 2) v = A[(size_t)(BR + lane) * RS + colj];
        const bool nz = lane < 2 && (v.x != T(0) || v.y != T(0));
        const unsigned bal = __ballot_sync(FULL, nz);
        if (nz) {
            const int q = nact + __popc(bal & ((1u << lane) - 1u));
            actb[q] = BR + lane;
            multb[q] = C{v.x * inv.x - v.y * inv.y, v.x * inv.y + v.y * inv.x};
            A[(size_t)(BR + lane) * RS + colj] = zero;
        }
        nact += __popc(bal);
    }
    if (lane == 0) {
        ctl[b * 4 + 0] = ps;
        ctl[b * 4 + 1] = extp;
        ctl[b * 4 + 2] = nact;
        ctl[b * 4 + 3] = 0;
        rows_done += nact;
        cols_done += (long long)nact * (extp - j + 4);
    }
    __syncwarp();
}

// ln Z of one part for both sectors, W warps per syndrome with look-ahead:
// in step k warp 0 applies step k's update to column k+1, places the
// entering row in the spare slot and takes step k+1's pivot and multipliers,
// while warps 1..W-1 apply step k's update to columns k+2.. and the extra
// columns. One block barrier per step; step k's lists are in buffer k & 1.
template <typename T, int NT, int W>
__device__ __forceinline__ void kw_part_la(const KwArgs& a, unsigned char* base, double out[2]) {
    using C = typename Cplx<T>::type;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const KwLayoutLA L = kw_layout_la(a.WR, a.RS, a.n, sizeof(C));
    C* A = reinterpret_cast<C*>(base + L.a);
    C* mult = reinterpret_cast<C*>(base + L.mult);
    const T* wt = reinterpret_cast<const T*>(base + L.wt);
    int* map = reinterpret_cast<int*>(base + L.map);
    int* ext = reinterpret_cast<int*>(base + L.ext);
    int* act = reinterpret_cast<int*>(base + L.act);
    int* ctl = reinterpret_cast<int*>(base + L.ctl);          // per buffer: pivot slot, its last column, active rows, dead
    double* res2 = reinterpret_cast<double*>(base + L.ctl + 32);
    const int WR = a.WR, WC = a.WC, RS = a.RS, Nb = a.Nb, BR = a.WR + 1;
    const C zero = C{T(0), T(0)};

    for (int i = tid; i < (WR + 3) * RS; i += 32 * W) A[i] = zero;
    for (int r = tid; r < WR; r += 32 * W) map[r] = r;
    __syncthreads();
    const int rows0 = WR < Nb ? WR : Nb;
    for (int i = warp; i < rows0; i += W) {
        C v, v1;
        const int j = kw_fetch<T, C>(a, wt, i, lane, v, v1);
        kw_place_row<T, C>(a, A + (size_t)i * RS, i, j, v, v1, lane);
        if (lane == 0) ext[i] = a.ext0[i];
    }
    // border rows (warp 0 keeps each lane's entry of both)
    int bj[2] = {-1, -1};
    C bv[2] = {zero, zero};
    if (warp == 0) {
        for (int t = 0; t < 2; ++t) {
            C v1;
            bj[t] = kw_fetch<T, C>(a, wt, Nb + t, lane, bv[t], v1);
            C* R = A + (size_t)(BR + t) * RS;
            const int j = bj[t];
            if (j >= Nb) R[WC + (j - Nb)] = bv[t];
            else if (j >= 0) {
                if (j < WC) R[j] = bv[t];
                if (j >= Nb - 2) R[WC + 2 + (j - (Nb - 2))] = v1;
            }
            if (lane == 0) R[WC + t].x += T(1);
        }
    }
    __syncthreads();

    T mant = T(1);
    int expo = 0;
    long long rows_done = 0, cols_done = 0;
    int spare = WR;                         // the free band slot (warp 0)
    // warp 0 reads the table entries of the row entering at step k during
    // step k-1 (column, weight source, phase, extent), off its critical path
    int fj = -1, fs = 0, fext = 0;
    double2 fph = make_double2(0.0, 0.0);
    auto prefetch = [&](int i) {
        if (i < Nb) {
            fj = a.ecol[i * kKwRowSlots + lane];
            fs = a.esrc[i * kKwRowSlots + lane];
            fph = a.eph[i * kKwRowSlots + lane];
            fext = a.ext0[i];
        }
    };
    if (warp == 0) prefetch(WR);
    if (warp == 0)
        kw_la_pivot<T, C>(a, A, mult, map, ext, act, ctl, 0, 0, 0, 0, lane, mant, expo, rows_done, cols_done);
    __syncthreads();
    bool dead = false;
    int colk = 0, kmod = 0;    // k mod WC, k mod WR
    for (int k = 0; k < Nb - 2; ++k) {
        const int b = k & 1;
        if (ctl[b * 4 + 3]) {
            dead = true;
            break;
        }
        const int ps = ctl[b * 4 + 0], extp = ctl[b * 4 + 1], nact = ctl[b * 4 + 2];
        const int* actb = act + b * (WR + 2);
        const C* multb = mult + b * (WR + 2);
        const C* P = A + (size_t)ps * RS;
        const int colk1 = colk + 1 == WC ? 0 : colk + 1;
        const int kmod1 = kmod + 1 == WR ? 0 : kmod + 1;
        if (warp == 0) {
            // step k's update of column k+1
            const C u1 = k + 1 <= extp ? P[colk1] : zero;
            for (int q = lane; q < nact; q += 32) {
                C* R = A + (size_t)actb[q] * RS;
                C r = R[colk1];
                kw_axpy<C, T>(r, multb[q], u1);
                R[colk1] = r;
            }
            // row k + WR enters in the spare slot (its map position is
            // k's); the pivot's slot becomes the spare
            const int rin = k + WR;
            if (rin < Nb) {
                const int j = fj, ext_in = fext;
                const T w = fs >= 0 ? wt[fs] : T(1);
                const C v = C{-w * (T)fph.x, -w * (T)fph.y};
                const C v1 = fs == -2 ? C{(T)fph.x, (T)fph.y} : v;
                prefetch(rin + 1);
                C* R = A + (size_t)spare * RS;
                for (int i = lane; i < RS; i += 32) R[i] = zero;
                __syncwarp();
                kw_place_row<T, C>(a, R, rin, j, v, v1, lane);
                if (lane == 0) {
                    ext[spare] = ext_in;
                    map[kmod] = spare;
                }
                spare = ps;
            }
            // the border rows' entries of the entering column k + WC
            const int jn = k + WC;
#pragma unroll
            for (int t = 0; t < 2; ++t)
                if (bj[t] == jn && jn < Nb) A[(size_t)(BR + t) * RS + colk] = bv[t];
            __syncwarp();
            if (k + 1 < Nb - 2)
                kw_la_pivot<T, C>(a, A, mult, map, ext, act, ctl, k + 1, colk1, kmod1, b ^ 1, lane, mant, expo,
                                  rows_done, cols_done);
        } else {
            // step k's update of columns k+2..extp and the four extra columns
            C U[NT];
            int pc[NT];
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int c = k + 1 + lane + 32 * t;
                int p = colk + 1 + lane + 32 * t;
                if (p >= WC) p -= WC;
                pc[t] = (c >= k + 2 && c <= extp) ? p : -1;
                U[t] = pc[t] >= 0 ? P[p] : zero;
            }
            const C Ux = lane < 4 ? P[WC + lane] : zero;
            for (int q = warp - 1; q < nact; q += W - 1) {
                C* R = A + (size_t)actb[q] * RS;
                const C m = multb[q];
                C r[NT], rx;
#pragma unroll
                for (int t = 0; t < NT; ++t)
                    if (pc[t] >= 0) r[t] = R[pc[t]];
                if (lane < 4) rx = R[WC + lane];
#pragma unroll
                for (int t = 0; t < NT; ++t)
                    if (pc[t] >= 0) {
                        kw_axpy<C, T>(r[t], m, U[t]);
                        R[pc[t]] = r[t];
                    }
                if (lane < 4) {
                    kw_axpy<C, T>(rx, m, Ux);
                    R[WC + lane] = rx;
                }
            }
        }
        __syncthreads();
        colk = colk1;
        kmod = kmod1;
    }

    if (warp == 0) {
        const double lm = __shfl_sync(FULL, log((double)mant) + (double)expo * 0.69314718055994530942, 0);
        double res = -INFINITY;
        if (!dead && lane < 2) {
            const int m0 = kmod, m1 = kmod + 1 == WR ? 0 : kmod + 1;   // k = Nb - 2 here
            const int rows[4] = {map[m0], map[m1], BR, BR + 1};
            const int cols[4] = {lane == 0 ? colk : WC + 2, lane == 0 ? (colk + 1 == WC ? 0 : colk + 1) : WC + 3,
                                 WC, WC + 1};
            res = a.cst + 0.5 * (0.5 * lm + kw_logdet4<C>(A, RS, rows, cols));
        }
        if (lane < 2) res2[lane] = res;
        if (dead && lane == 0) atomicOr(a.status, 1 << MLD_ERR_NUMERIC);
        if (lane == 0 && a.flops) atomicAdd(a.flops, 6.0 * (double)rows_done + 8.0 * (double)cols_done);
    }
    __syncthreads();
    out[0] = res2[0];
    out[1] = res2[1];
    __syncthreads();
}

// One block of W warps per syndrome with the look-ahead schedule (d >= 15),
// persistent over the batch; the same steps as kw_decode_warp_kernel.
template <typename T, int NT>
__global__ void __launch_bounds__(32 * kKwWarps) kw_decode_la_kernel(KwArgs a) {
    constexpr int W = kKwWarps;
    extern __shared__ __align__(16) unsigned char kw_smem[];
    using C = typename Cplx<T>::type;
    const int tid = threadIdx.x;
    unsigned char* base = kw_smem;
    const KwLayoutLA L = kw_layout_la(a.WR, a.RS, a.n, sizeof(C));
    T* wt = reinterpret_cast<T*>(base + L.wt);
    const int n = a.n;
    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        const uint64_t* sb = a.syn + b * a.words;
        int bad = 0, zany = 0;
        for (int q = tid; q < n; q += 32 * W) {
            const uint64_t* mk = a.dmask + (size_t)q * 2 * a.words;
            int x = 0;
            for (int w = 0; w < a.words; ++w) x ^= __popcll(sb[w] & mk[w]) & 1;
            const float p = a.px[q];
            bad |= !(p > 0.f && p < 1.f);
            wt[q] = (x ? T(-1) : T(1)) * (T(1) - T(2) * (T)p);
            if (!a.pz) {
                int z = 0;
                for (int w = 0; w < a.words; ++w) z ^= __popcll(sb[w] & mk[a.words + w]) & 1;
                zany |= z;
            }
        }
        zany = __syncthreads_or(zany);
        double lx[2], lz[2];
        kw_part_la<T, NT, W>(a, base, lx);
        if (a.pz) {
            for (int qt = tid; qt < n; qt += 32 * W) {
                const int q = a.zmap[qt];
                const uint64_t* mk = a.dmask + (size_t)q * 2 * a.words;
                int z = 0;
                for (int w = 0; w < a.words; ++w) z ^= __popcll(sb[w] & mk[a.words + w]) & 1;
                const float p = a.pz[q];
                bad |= !(p > 0.f && p < 1.f);
                wt[qt] = (z ? T(-1) : T(1)) * (T(1) - T(2) * (T)p);
            }
            __syncthreads();
            kw_part_la<T, NT, W>(a, base, lz);
        } else {
            lz[0] = zany ? -INFINITY : 0.0;
            lz[1] = -INFINITY;
        }
        bad = __syncthreads_or(bad);
        if (tid == 0) {
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
    }
}

std::mutex g_kw_mutex;

// The code's Kac-Ward tables on the device, built on first use.
mld_status ensure_kw(mld_code* C) {
    std::lock_guard<std::mutex> lock(g_kw_mutex);
    if (C->d_kw) return MLD_OK;
    KwGraph g;
    if (!build_kw_graph(C->d, &g)) return MLD_ERR_UNSUPPORTED;
    if ((g.bl + g.bu + 31) / 32 > kKwMaxColsPerLane || (g.bl + 2 + 31) / 32 > kKwMaxChunks)
        return MLD_ERR_UNSUPPORTED;
    const int N = g.N, S = kKwRowSlots;
    const std::vector<int> zmap = kw_zmap(C->d);
    // row i's successors padded to S slots: columns (-1 pad), weight sources,
    // then each band row's last column and the quarter-turn map; the phases
    // as double pairs after them
    std::vector<int> ints((size_t)2 * N * S, 0);
    std::vector<double> ph((size_t)2 * N * S, 0.0);
    for (int i = 0; i < N; ++i) {
        const int e0 = g.row_start[i], e1 = g.row_start[i + 1];
        if (e1 - e0 > S) return MLD_ERR_UNSUPPORTED;
        for (int t = 0; t < S; ++t) {
            const int e = e0 + t;
            ints[(size_t)i * S + t] = e < e1 ? g.col[e] : -1;
            ints[(size_t)N * S + (size_t)i * S + t] = e < e1 ? g.src[e] : 0;
            ph[2 * ((size_t)i * S + t)] = e < e1 ? g.ph_re[e] : 0.0;
            ph[2 * ((size_t)i * S + t) + 1] = e < e1 ? g.ph_im[e] : 0.0;
        }
    }
    ints.insert(ints.end(), g.ext0.begin(), g.ext0.end());
    ints.insert(ints.end(), zmap.begin(), zmap.end());
    const size_t ph_off = kw_align(ints.size() * sizeof(int));
    const int nnz = N * S;
    const size_t cnt_off = kw_align(ph_off + ph.size() * sizeof(double));
    const size_t bytes = cnt_off + 16;
    void* blob = nullptr;
    if (cudaMalloc(&blob, bytes) != cudaSuccess) return MLD_ERR_NOMEM;
    if (cudaMemcpy(blob, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy((char*)blob + ph_off, ph.data(), ph.size() * sizeof(double), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cudaFree(blob);
        return MLD_ERR_CUDA;
    }
    if (cudaMemset((char*)blob + cnt_off, 0, 16) != cudaSuccess) {
        cudaFree(blob);
        return MLD_ERR_CUDA;
    }
    C->kw_cnt_off = cnt_off;
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

template <typename K>
mld_status launch_kw_kernel(K kernel, int threads, size_t bytes, const KwArgs& a, cudaStream_t s) {
    int dev = 0, sms = 0, smem_max = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return MLD_ERR_CUDA;
    if (bytes > (size_t)smem_max) return MLD_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return MLD_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, bytes) != cudaSuccess ||
        per_sm < 1)
        return MLD_ERR_UNSUPPORTED;
    int64_t blocks = (int64_t)sms * per_sm;
    if (blocks > a.B) blocks = a.B;
    kernel<<<(unsigned)blocks, threads, bytes, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? MLD_OK : MLD_ERR_CUDA;
}

// One warp per syndrome while the window is small (up to 3 pivot-row columns
// per lane, d <= 13: measured faster there, 1.77 M against 1.15 M syndromes/s
// for four warps at d = 9); the look-ahead block of kKwWarps warps per
// syndrome above (d = 17: 277 k against 148 k for one warp; d = 25: 69 k
// against 26 k).
template <typename T, int NT>
mld_status launch_kw_nt(const KwArgs& a, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    if constexpr (NT <= 3)
        return launch_kw_kernel(kw_decode_warp_kernel<T, NT>, 32, kw_layout(a.WR, a.RS, a.n, sizeof(C)).total, a, s);
    else
        return launch_kw_kernel(kw_decode_la_kernel<T, NT>, 32 * kKwWarps,
                                kw_layout_la(a.WR, a.RS, a.n, sizeof(C)).total, a, s);
}

// Columns of the pivot row per lane: (bl + bu) / 32 rounded up (2 at d <= 9,
// 3 at d <= 13, 4 at d <= 17, 5 up to d = 25).
template <typename T>
mld_status launch_kw(const KwArgs& a, cudaStream_t s) {
    switch ((a.bl + a.bu + 31) / 32) {
        case 1:
        case 2: return launch_kw_nt<T, 2>(a, s);
        case 3: return launch_kw_nt<T, 3>(a, s);
        case 4: return launch_kw_nt<T, 4>(a, s);
        case 5: return launch_kw_nt<T, 5>(a, s);
    }
    return MLD_ERR_UNSUPPORTED;
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
    const int N = C->kw_N, Nb = C->kw_Nb, S = kKwRowSlots;
    a.ecol = ib;
    a.esrc = ib + (size_t)N * S;
    a.ext0 = ib + (size_t)2 * N * S;
    a.zmap = a.ext0 + Nb;
    a.eph = reinterpret_cast<const double2*>(reinterpret_cast<const char*>(C->d_kw) + C->kw_ph_off);
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
    a.dmask = C->d_dmask;
    a.px = px;
    a.pz = pz;
    a.syn = syndromes;
    a.B = B;
    a.logP = logP;
    a.argmax = argmax;
    a.status = C->d_status;
    a.flops = reinterpret_cast<double*>(reinterpret_cast<char*>(C->d_kw) + C->kw_cnt_off);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return precision == MLD_FP64 ? launch_kw<double>(a, s) : launch_kw<float>(a, s);
}

extern "C" mld_status mld_decode_xz_executed_flops(const mld_code* Cc, double* out) {
    mld_code* C = const_cast<mld_code*>(Cc);
    if (!C || !out) return MLD_ERR_INVALID_ARG;
    *out = 0.0;
    if (!C->d_kw) return MLD_OK;
    char* cnt = static_cast<char*>(C->d_kw) + C->kw_cnt_off;
    if (cudaMemcpy(out, cnt, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return MLD_ERR_CUDA;
    if (cudaMemset(cnt, 0, sizeof(double)) != cudaSuccess) return MLD_ERR_CUDA;
    return MLD_OK;
}
