"""Pins of the Kac-Ward oracle (Sec. 3.1.3) against facts it does not compute
itself: the exact variable elimination of the generator picture (Eq. 7),
brute force over all Paulis at d = 3, normalisation over all syndromes, and the
even-subgraph sum written term by term on a small graph."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import kac_ward as kw


def _all_syndromes(d):
    m = d * d - 1
    bits = ((np.arange(1 << m)[:, None] >> np.arange(m)[None, :]) & 1).astype(np.uint8)
    return synth.pack_bits(bits)


@pytest.mark.parametrize("d", [3, 5, 7, 9])
def test_equals_variable_elimination_independent_xz(d):
    """Both parts and both sectors against the exact contraction, on sampled
    syndromes of per-qubit random rates (no class far below the other at these
    rates, so FP64 cancellation stays far below the tolerance)."""
    n = d * d
    rng = np.random.default_rng(100 + d)
    px, pz = rng.uniform(0.03, 0.3, n), rng.uniform(0.03, 0.3, n)
    tab = kw.xz_table(px, pz)
    syn = synth.syndromes_of(d, synth.sample_errors(d, tab, 6, seed=d))
    ref, am_ref = oracle.decode(d, tab, syn)
    lp, am = kw.decode_xz(d, px, pz, syn)
    np.testing.assert_allclose(lp, ref, rtol=0, atol=1e-9)
    np.testing.assert_array_equal(am, am_ref)


@pytest.mark.parametrize("d", [3, 5, 7])
def test_bitflip_equals_variable_elimination(d):
    """pz = None: the l_Z = 1 classes and impossible syndromes are -inf exactly
    where the exact contraction gives zero."""
    n = d * d
    rng = np.random.default_rng(7 + d)
    px = rng.uniform(0.02, 0.25, n)
    tab = kw.xz_table(px, None)
    syn = synth.syndromes_of(d, synth.sample_errors(d, tab, 6, seed=3 * d))
    # add a syndrome with an X-type bit set: impossible under bit-flip noise
    t, _, _, _ = oracle.layout(d)
    bits = np.zeros((1, n - 1), np.uint8)
    bits[0, int(np.nonzero(t == 0)[0][0])] = 1
    syn = np.concatenate([syn, synth.pack_bits(bits)])
    ref, _ = oracle.decode(d, tab, syn)
    lp, _ = kw.decode_xz(d, px, None, syn)
    np.testing.assert_array_equal(np.isfinite(lp), np.isfinite(ref))
    fin = np.isfinite(ref)
    np.testing.assert_allclose(lp[fin], ref[fin], rtol=0, atol=1e-10)
    assert not np.isfinite(lp[-1]).any()


def test_bruteforce_and_normalisation_d3():
    """Every syndrome of d = 3: equal to brute force over all 4^9 Paulis, and
    the probabilities of all (syndrome, class) pairs sum to one."""
    d, n = 3, 9
    rng = np.random.default_rng(5)
    px, pz = rng.uniform(0.05, 0.4, n), rng.uniform(0.05, 0.4, n)
    tab = kw.xz_table(px, pz)
    Z = oracle.bruteforce_table(d, tab)
    lp, _ = kw.decode_xz(d, px, pz, _all_syndromes(d))
    np.testing.assert_allclose(lp, np.log(Z), rtol=0, atol=1e-12)
    assert abs(np.exp(lp).sum() - 1.0) < 1e-12


def test_kac_ward_determinant_is_the_even_subgraph_sum():
    """det(I - Lambda) = ES^2 on the d = 3 spin graphs, with ES summed over all
    edge subsets of even degree (every vertex, ghosts and bend points
    included), for both parts and both tie signs."""
    d = 3
    rng = np.random.default_rng(9)
    for part in ("x", "z"):
        pos, edges, _ = kw.planar_graph(d, part)
        m = len(edges)
        for tie in (1.0, -1.0):
            t = np.array([rng.uniform(-0.9, 0.9) if q >= 0 else (1.0 if q == -1 else tie)
                          for (_, _, q) in edges])
            masks = np.arange(1 << m, dtype=np.int64)
            bits = (masks[:, None] >> np.arange(m)[None, :]) & 1
            odd = np.zeros((1 << m, len(pos)), np.int64)
            for e, (u, v, _) in enumerate(edges):
                odd[:, u] ^= bits[:, e]
                odd[:, v] ^= bits[:, e]
            weight = np.prod(np.where(bits == 1, t[None, :], 1.0), axis=1)
            es = float(weight[~odd.any(axis=1)].sum())
            det = np.linalg.det(kw.kac_ward_matrix(pos, edges, t))
            assert abs(det.imag) < 1e-9 * max(1.0, abs(det.real))
            assert abs(det.real - es * es) < 1e-9 * max(1.0, es * es)


def test_graph_is_planar_straight_line():
    """No two edges of the embedding cross or overlap (shared end points
    aside): the precondition of the Kac-Ward formula."""
    def cross(a, b, c, d):
        def orient(p, q, r):
            v = (q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0])
            return 0 if abs(v) < 1e-12 else (1 if v > 0 else -1)
        o1, o2, o3, o4 = orient(a, b, c), orient(a, b, d), orient(c, d, a), orient(c, d, b)
        return o1 * o2 < 0 and o3 * o4 < 0
    for d in (3, 5, 7):
        for part in ("x", "z"):
            pos, edges, _ = kw.planar_graph(d, part)
            for (e1, e2) in itertools.combinations(edges, 2):
                if len({e1[0], e1[1], e2[0], e2[1]}) < 4:
                    # a shared end: the two segments must leave it at different angles
                    s = ({e1[0], e1[1]} & {e2[0], e2[1]}).pop()
                    o1 = e1[1] if e1[0] == s else e1[0]
                    o2 = e2[1] if e2[0] == s else e2[0]
                    a1 = math.atan2(pos[o1][1] - pos[s][1], pos[o1][0] - pos[s][0])
                    a2 = math.atan2(pos[o2][1] - pos[s][1], pos[o2][0] - pos[s][0])
                    assert abs(a1 - a2) > 1e-9
                    continue
                assert not cross(pos[e1[0]], pos[e1[1]], pos[e2[0]], pos[e2[1]])
