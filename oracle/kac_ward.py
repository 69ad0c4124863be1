"""Kac-Ward evaluation of the coset partition functions under independent X/Z
noise (Sec. 3.1.3 of arxiv 2605.17230), in FP64 with numpy.

TEST INFRASTRUCTURE ONLY (imported by ``tests/`` and the benchmark's CPU leg).
It shares no code with the decoder package. It is a second, independent exact
method beside the variable elimination of ``mld_oracle.c``: the two agree on
every class where both are exact, which pins both.

What is computed. Under independent noise a Pauli's probability factorises,
Pr(E) = prod_q Px_q(x_q) Pz_q(z_q), so Z_(lX,lZ)(s) = ZX_lX(s) * ZZ_lZ(s):
the X part is a sum over the X-type stabiliser group acting on the x-bits of a
representative, the Z part the same with Z-type stabilisers and z-bits. Take
the X part. Write Px(e) = (1 + t (-1)^e) / 2 with t = 1 - 2 p, and give each
X-type plaquette a spin sigma = (-1)^alpha (alpha = whether its stabiliser is
applied). Qubit q then contributes (1 + t_q s_q sigma_u sigma_v) / 2 with
s_q = (-1)^(x_q) and u, v its two X-type plaquettes; a qubit on column 0 or
d-1 has one such plaquette and couples it to a ghost spin L or R. The ghosts
are tied by an extra edge of weight +1 (sector 0: sigma_L = sigma_R) or -1
(sector 1: sigma_L = -sigma_R, which is the coset of E X_L, X_L being X on a
column). Summing every spin (ghosts included) and expanding the products
(high-temperature expansion) gives

    ZX_sector = 2^(nP - n) * ES,   ES = sum over even subgraphs of prod t_e s_e,

with nP the number of X-type plaquettes and n the number of qubits (the
factor 1/4 removes the two ghost sums; a degree-two vertex inserted into an
edge with an extra weight-1 edge changes neither side). For a graph drawn in
the plane with straight edges, Kac and Ward's formula gives
ES^2 = det(I - Lambda), with Lambda over directed edges:
Lambda[e -> f] = t_f exp(i theta/2) when f leaves the vertex e enters,
f is not e reversed, and theta is the turning angle from e to f (Sec. 3.1.3).
ES > 0 (it is a probability up to a positive factor), so
ln ZX = (nP - n) ln 2 + ln|det(I - Lambda)| / 2.

The Z part is the same construction on the Z-type plaquettes: qubits on rows
0 and d-1 have one Z-type plaquette and couple it to ghosts T and B (top,
bottom); sector 1 is the coset of E Z_L (Z on a row).

Embedding (a reading: the paper gives none): plaquette (i, j) at the point
(x, y) = (j, -i), qubit (r, c) at (c + 1/2, -(r + 1/2)). Every ghost edge is
drawn through the point of its qubit (a degree-two vertex there), so that two
qubits joining the same plaquette to the same ghost are distinct segments; the
ghosts lie far outside the patch and the tie edge runs around it through two
corner points. The determinant is numpy's slogdet (LU with partial pivoting).

Floating point: ES is a sum of signed terms. For the class of larger weight
the terms mostly agree in sign; for a class far less likely than the other
one they cancel, and ln|det| then carries an absolute error of order
eps * cond relative to the leading class. With eps = 2^-53 this is invisible
for the sizes and rates the tests use, but it is a property of the method, not
of this code.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

from . import code_info, representatives


def _present(d: int, i: int, j: int) -> bool:
    """Plaquette (i, j), 0 <= i, j <= d, exists: every interior one; on rows 0
    and d only those with i + j even (X-type); on columns 0 and d only those
    with i + j odd (Z-type). Same layout as the exact oracle's."""
    row_in = 1 <= i <= d - 1
    col_in = 1 <= j <= d - 1
    if row_in and col_in:
        return True
    if i in (0, d) and col_in:
        return (i + j) % 2 == 0
    if j in (0, d) and row_in:
        return (i + j) % 2 == 1
    return False


def planar_graph(d: int, part: str):
    """The spin graph of one part ('x' or 'z') with its straight-line embedding.

    Returns (pos, edges, n_plaq): pos a list of points, edges a list of
    (u, v, qubit) with qubit = -1 for a segment of weight 1 and -2 for the
    ghost tie (weight +1 or -1 by sector)."""
    parity = 0 if part == "x" else 1
    pos, vid = [], {}

    def vertex(key, xy):
        if key not in vid:
            vid[key] = len(pos)
            pos.append(xy)
        return vid[key]

    for i in range(d + 1):
        for j in range(d + 1):
            if _present(d, i, j) and (i + j) % 2 == parity:
                vertex(("p", i, j), (float(j), -float(i)))
    n_plaq = len(pos)
    far = 4.0 * d
    mid = (d - 1) / 2.0
    if part == "x":       # ghosts left and right, tie around the bottom
        g0 = vertex("g0", (-far, -mid))
        g1 = vertex("g1", (d - 1 + far, -mid))
        c0 = vertex("c0", (-far, -d - far))
        c1 = vertex("c1", (d - 1 + far, -d - far))
    else:                 # ghosts top and bottom, tie around the right
        g0 = vertex("g0", (mid, far))
        g1 = vertex("g1", (mid, -(d - 1) - far))
        c0 = vertex("c0", (d + far, far))
        c1 = vertex("c1", (d + far, -(d - 1) - far))
    edges = []
    for r in range(d):
        for c in range(d):
            q = r * d + c
            ends = [vid[("p", i, j)] for (i, j) in ((r, c), (r, c + 1), (r + 1, c), (r + 1, c + 1))
                    if ("p", i, j) in vid]
            if len(ends) == 2:
                edges.append((ends[0], ends[1], q))
                continue
            assert len(ends) == 1
            if part == "x":
                ghost = g0 if c == 0 else g1
                assert c in (0, d - 1)
            else:
                ghost = g0 if r == 0 else g1
                assert r in (0, d - 1)
            mid_q = vertex(("q", r, c), (c + 0.5, -(r + 0.5)))
            edges.append((ends[0], mid_q, q))
            edges.append((mid_q, ghost, -1))
    edges.append((g0, c0, -1))
    edges.append((c0, c1, -1))
    edges.append((c1, g1, -2))
    return pos, edges, n_plaq


def kac_ward_matrix(pos, edges, t):
    """I - Lambda over directed edges (2e: u -> v, 2e + 1: v -> u) for edge
    weights t[e]."""
    m = len(edges)
    heads, tails = [], []
    for (u, v, _) in edges:
        tails += [u, v]
        heads += [v, u]
    leaving = {}
    for k in range(2 * m):
        leaving.setdefault(tails[k], []).append(k)

    def direction(k):
        a, b = pos[tails[k]], pos[heads[k]]
        return math.atan2(b[1] - a[1], b[0] - a[0])

    M = np.eye(2 * m, dtype=np.complex128)
    for k in range(2 * m):
        for f in leaving[heads[k]]:
            if heads[f] == tails[k]:
                continue            # no backtracking
            theta = direction(f) - direction(k)
            theta = (theta + math.pi) % (2.0 * math.pi) - math.pi
            M[k, f] -= t[f // 2] * cmath.exp(0.5j * theta)
    return M


def part_logz(d: int, part: str, p, bits, sector: int) -> float:
    """ln of one part's coset sum: p [n] the flip probabilities of that part,
    bits [n] the representative's x-bits (part 'x') or z-bits (part 'z')."""
    pos, edges, n_plaq = planar_graph(d, part)
    n = d * d
    t = np.empty(len(edges))
    for e, (_, _, q) in enumerate(edges):
        if q >= 0:
            t[e] = (1.0 - 2.0 * p[q]) * (-1.0 if bits[q] else 1.0)
        elif q == -1:
            t[e] = 1.0
        else:
            t[e] = -1.0 if sector else 1.0
    _, logabs = np.linalg.slogdet(kac_ward_matrix(pos, edges, t))
    return (n_plaq - n) * math.log(2.0) + 0.5 * logabs


def decode_xz(d: int, px, pz, syn):
    """ln Z_l(s) for l = I, X, Z, Y ([B][4], class l_X + 2 l_Z) under
    independent X/Z noise with per-qubit flip probabilities px, pz, and the
    argmax. pz = None is bit-flip noise: classes with l_Z = 1 get -inf and a
    syndrome with a nonzero X-type part (impossible without Z errors) gets -inf
    for every class."""
    n, _, _ = code_info(d)
    px = np.asarray(px, dtype=np.float64).reshape(n)
    reps = representatives(d, syn)[:, 0, :]
    out = np.empty((reps.shape[0], 4))
    for b, rep in enumerate(reps):
        xb, zb = rep & 1, rep >> 1
        zx = [part_logz(d, "x", px, xb, s) for s in (0, 1)]
        if pz is None:
            # only E with z-bits equal to a stabiliser (or Z_L times one) have
            # weight; the representative has no z-bits iff the X-type
            # syndrome part is zero, and then l_Z = 0 holds the identity
            zz = [0.0, -math.inf] if not zb.any() else [-math.inf, -math.inf]
        else:
            pzv = np.asarray(pz, dtype=np.float64).reshape(n)
            zz = [part_logz(d, "z", pzv, zb, s) for s in (0, 1)]
        for lz in (0, 1):
            for lx in (0, 1):
                out[b, lx + 2 * lz] = zx[lx] + zz[lz]
    return out, np.argmax(out, axis=1).astype(np.uint8)


def xz_table(px, pz) -> np.ndarray:
    """The Pauli table [n][4] (I, X, Y, Z) of independent X/Z noise."""
    px = np.asarray(px, dtype=np.float64)
    pz = np.zeros_like(px) if pz is None else np.asarray(pz, dtype=np.float64)
    return np.stack([(1 - px) * (1 - pz), px * (1 - pz), px * pz, (1 - px) * pz], axis=1)
