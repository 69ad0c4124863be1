"""Boundary-MPS contraction (Sec. 3.2.1 of arxiv 2605.17230) in FP64, numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows the paper's steps for the generator-picture network (Eq. 7) swept
column by column:
  * the boundary MPS starts as the first column of the network: one binary
    site per plaquette of corner column 0 (absent plaquettes have a single
    value, 0), all entries 1;
  * for each later column: (i) contract every tensor of that column's MPO
    into the matching MPS site, which multiplies the bond by the MPO bond
    (q = 4 here: the pair (alpha_i, beta_i) of variables shared by the qubit
    factors on both sides of a site); (ii) compress back to at most ``chi``
    by successive SVD truncations that keep the largest singular values;
  * after the last column, contracting the MPS with all-ones vectors gives Z.

Reading of step (ii), which the paper leaves open: the applied MPS is first
brought to left-canonical form by a left-to-right QR sweep (no truncation),
then a right-to-left sweep takes the SVD of every bond matrix and keeps
min(chi, number of singular values) of them, absorbing U*S into the left
neighbour. Each finished column is rescaled by a power of two (exact) and
the exponent is kept in the log.

The MPO of qubit column c: site i (plaquette row i) carries alpha_i (corner
column c, input) and beta_i (corner column c+1, output). The factor of
qubit (i-1, c), which depends on (alpha_{i-1}, alpha_i, beta_{i-1}, beta_i),
sits on site i; the right bond of site i copies (alpha_i, beta_i).

No truncation happens when chi is at least the exact bond; the result then
equals the dense contraction of ``mld_oracle.c`` (pinned in the tests). For a
smaller chi the value is the algorithm's approximation; it is pinned by a
dense restatement of the same rule (the tests apply each column's transfer to
the full 2^(d+1) state and then take, cut by cut from the last bond to the
first, the optimal rank-chi truncation of that vector, which is what a
right-to-left SVD sweep of a left-canonical MPS computes), at d = 5 and 7.
"""
from __future__ import annotations

import math

import numpy as np

from . import code_info, layout, representatives


def _present_map(d):
    """present[i][j] for plaquette (i, j) and its type (0 X, 1 Z)."""
    typ = np.full((d + 1, d + 1), -1, dtype=np.int64)
    for j in range(d + 1):
        for i in range(d + 1):
            ok = (1 <= i <= d - 1 and 1 <= j <= d - 1) or \
                 (i in (0, d) and 1 <= j <= d - 1 and (i + j) % 2 == 0) or \
                 (j in (0, d) and 1 <= i <= d - 1 and (i + j) % 2 == 1)
            if ok:
                typ[i, j] = (i + j) % 2
    return typ


def _paper_index(x, z):
    return {(0, 0): 0, (1, 0): 1, (1, 1): 2, (0, 1): 3}[(x, z)]


def _qubit_factor(typ, noise_q, e, r, c):
    """w[a_r, a_r1, b_r, b_r1] = p_q[E_q xor X^u Z^v] for qubit (r, c)."""
    w = np.zeros((2, 2, 2, 2))
    corners = [(r, c), (r + 1, c), (r, c + 1), (r + 1, c + 1)]
    for idx in np.ndindex(2, 2, 2, 2):
        u = v = 0
        for val, (i, j) in zip(idx, corners):
            t = typ[i, j]
            if t == 0:
                u ^= val
            elif t == 1:
                v ^= val
        w[idx] = noise_q[_paper_index((e & 1) ^ u, ((e >> 1) & 1) ^ v)]
    return w


def column_mpo(d, typ, noise, E, c):
    """MPO of qubit column c as a list of tensors M_i[ml, a_i, b_i, mr]."""
    dims_a = [2 if typ[i, c] >= 0 else 1 for i in range(d + 1)]
    dims_b = [2 if typ[i, c + 1] >= 0 else 1 for i in range(d + 1)]
    mpo = []
    for i in range(d + 1):
        da, db = dims_a[i], dims_b[i]
        ml = 1 if i == 0 else dims_a[i - 1] * dims_b[i - 1]
        mr = 1 if i == d else da * db
        M = np.zeros((ml, da, db, mr))
        for a in range(da):
            for b in range(db):
                if i == 0:
                    wval = np.ones((1,))
                else:
                    q = (i - 1) * d + c
                    w = _qubit_factor(typ, noise[q], int(E[q]), i - 1, c)
                    wval = np.array([w[pa, a, pb, b] for pa in range(dims_a[i - 1])
                                     for pb in range(dims_b[i - 1])])
                for m in range(ml):
                    if i == d:
                        M[m, a, b, 0] = wval[m]
                    else:
                        M[m, a, b, a * db + b] = wval[m]
        mpo.append(M)
    return mpo


def apply_mpo(mps, mpo):
    """(i): B_i[(l,ml), b, (r,mr)] = sum_a A_i[l, a, r] M_i[ml, a, b, mr]."""
    out = []
    for A, M in zip(mps, mpo):
        B = np.einsum("lar,mabn->lmbrn", A, M)
        l, m, b, r, n = B.shape
        out.append(B.reshape(l * m, b, r * n))
    return out


def compress(mps, chi):
    """(ii): left-to-right QR, then right-to-left SVD keeping min(chi, #sv)."""
    mps = [t.copy() for t in mps]
    L = len(mps)
    for i in range(L - 1):
        l, p, r = mps[i].shape
        Q, R = np.linalg.qr(mps[i].reshape(l * p, r))
        mps[i] = Q.reshape(l, p, Q.shape[1])
        mps[i + 1] = np.einsum("ab,bpr->apr", R, mps[i + 1])
    for i in range(L - 1, 0, -1):
        l, p, r = mps[i].shape
        U, S, Vh = np.linalg.svd(mps[i].reshape(l, p * r), full_matrices=False)
        k = min(chi, S.shape[0])
        mps[i] = Vh[:k].reshape(k, p, r)
        mps[i - 1] = np.einsum("lpa,ab->lpb", mps[i - 1], U[:, :k] * S[:k])
    return mps


def coset_logz_mps(d, noise, E, chi):
    """ln Z of the coset of E by the boundary-MPS sweep at bond dimension chi."""
    typ = _present_map(d)
    mps = [np.ones((1, 2 if typ[i, 0] >= 0 else 1, 1)) for i in range(d + 1)]
    log2 = 0
    for c in range(d):
        mps = compress(apply_mpo(mps, column_mpo(d, typ, noise, E, c)), chi)
        mx = max(np.abs(t).max() for t in mps)
        if mx == 0.0:
            return -math.inf
        e = math.frexp(mx)[1]
        mps[0] = np.ldexp(mps[0], -e)
        log2 += e
    v = np.ones((1,))
    for t in mps:
        v = np.einsum("l,lpr->r", v, t)
    z = float(v[0])
    return math.log(z) + log2 * math.log(2.0) if z > 0 else -math.inf


def decode_mps(d, noise, syn, chi, xl_column=0):
    """ln Z_l(s) for l = I, X, Z, Y ([B][4]) by the boundary-MPS sweep.

    The coset of E_{l,s} = f(s) X_L^{l_X} Z_L^{l_Z} does not depend on which X
    string is taken as X_L (X on any column: they differ by X-type
    stabilisers), but at truncated chi the sweep's approximation does (Sec.
    3.2.1 contracts one fixed representative). xl_column picks the column of
    the X string used for l_X = 1 (the GPU kernels take column d-1)."""
    n, _, _ = code_info(d)
    noise = np.asarray(noise, dtype=np.float64)
    reps = representatives(d, syn).copy()
    if xl_column != 0:
        # move the X string of the l_X = 1 classes from column 0 to xl_column
        # (Pauli code x + 2z: X flips bit 0)
        move = np.zeros(n, np.uint8)
        move[0::d] ^= 1
        move[xl_column::d] ^= 1
        reps[:, 1] ^= move
        reps[:, 3] ^= move
    B = reps.shape[0]
    out = np.zeros((B, 4))
    for b in range(B):
        nz = noise if noise.ndim == 2 else (
            np.stack([1 - noise[b], noise[b] / 3, noise[b] / 3, noise[b] / 3]) * np.ones((n, 1))
            if noise.ndim == 1 else noise[b])
        for l in range(4):
            out[b, l] = coset_logz_mps(d, nz, reps[b, l], chi)
    return out


__all__ = ["column_mpo", "apply_mpo", "compress", "coset_logz_mps", "decode_mps", "layout"]
