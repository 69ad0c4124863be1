"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: brute force
over all Paulis, the stabiliser-group sum written term by term, closed forms,
symmetries of the code, the bit-flip random-bond Ising form (Eq. 6), and
the multilinearity of Z in the noise rows.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import oracle.mps as omps
import synth


def _all_syndromes(d):
    m = d * d - 1
    bits = ((np.arange(1 << m)[:, None] >> np.arange(m)[None, :]) & 1).astype(np.uint8)
    return synth.pack_bits(bits)


def _random_noise(n, seed, lo=0.01, hi=0.3):
    rng = np.random.default_rng(seed)
    t = rng.uniform(lo, hi, size=(n, 4))
    t[:, 0] = rng.uniform(0.5, 0.9, size=n)
    return t / t.sum(axis=1, keepdims=True)


# --- brute force: Eq. 3 summed over all 4^n Paulis --------------------------

@pytest.mark.parametrize("noise_kind", ["depolarizing", "random"])
def test_dense_equals_bruteforce_d3_all_syndromes(noise_kind):
    d, n = 3, 9
    noise = synth.depolarizing(n, 0.1) if noise_kind == "depolarizing" else _random_noise(n, 5)
    Z = oracle.bruteforce_table(d, noise)
    logP, am = oracle.decode(d, noise, _all_syndromes(d))
    np.testing.assert_allclose(logP, np.log(Z), rtol=0, atol=1e-12)
    # the decision is unique unless two cosets tie (exact under symmetric noise);
    # at a tie the pick must be one of the maxima
    lz = np.log(Z)
    top = np.sort(lz, axis=1)
    clear = top[:, -1] - top[:, -2] > 1e-9
    np.testing.assert_array_equal(am[clear], np.argmax(Z, axis=1)[clear])
    assert np.all(lz[np.arange(len(am)), am] >= top[:, -1] - 1e-9)


def test_normalisation_sum_over_syndromes_and_classes_d3():
    d, n = 3, 9
    noise = _random_noise(n, 11)
    logP, _ = oracle.decode(d, noise, _all_syndromes(d))
    assert abs(np.exp(logP).sum() - 1.0) < 1e-12
    assert abs(oracle.bruteforce_table(d, noise).sum() - 1.0) < 1e-12


# --- the stabiliser-group sum of Eq. 7, term by term ------------------------

def test_dense_equals_group_enumeration_d5():
    d, n = 5, 25
    noise = _random_noise(n, 3, 0.02, 0.2)
    E = synth.sample_errors(d, noise, 3, seed=21)
    reps = oracle.representatives(d, synth.syndromes_of(d, E))
    dense = oracle.coset_logz(d, noise, reps.reshape(-1, n))
    for k, rep in enumerate(reps.reshape(-1, n)):
        g = oracle.group_logz(d, noise, rep)
        assert abs(g - dense[k]) < 1e-11 * max(1.0, abs(g))


# --- closed forms -----------------------------------------------------------

@pytest.mark.parametrize("d", [3, 5, 7])
def test_fully_depolarized_closed_form(d):
    """p_I = p_X = p_Y = p_Z = 1/4: every coset holds 2^(n-1) Paulis of
    weight 4^-n, so ln Z = -(n+1) ln 2 for every syndrome and class."""
    n = d * d
    noise = np.full((n, 4), 0.25)
    E = synth.sample_errors(d, noise, 8, seed=2)
    logP, _ = oracle.decode(d, noise, synth.syndromes_of(d, E))
    np.testing.assert_allclose(logP, -(n + 1) * math.log(2.0), rtol=0, atol=1e-12)


def test_zero_noise_limit():
    """p = 0: only the identity has weight; Z_I(0) = 1, all other Z vanish."""
    d, n = 5, 25
    noise = synth.depolarizing(n, 0.0)
    syn = np.zeros((1, synth.syn_words(d)), np.uint64)
    logP, am = oracle.decode(d, noise, syn)
    assert logP[0, 0] == 0.0 and np.all(np.isneginf(logP[0, 1:])) and am[0] == 0


def test_small_p_limit_minimum_weight_d3():
    """p -> 0: ln Z_l(s) = ln N_min + w_min ln(p/3) + (n-w_min) ln(1-p) + O(p),
    with (w_min, N_min) the minimum weight and its multiplicity in the coset,
    found by enumerating all 4^n Paulis."""
    d, n = 3, 9
    codes = ((np.arange(4 ** n)[:, None] >> (2 * np.arange(n))[None, :]) & 3).astype(np.uint8)
    bits, cls = oracle.syndrome_class(d, codes)
    sidx = oracle.syndrome_index(bits).astype(np.int64)
    w = (codes != 0).sum(axis=1)
    key = sidx * 4 + cls
    wmin = np.full(4 << (n - 1), 99)
    np.minimum.at(wmin, key, w)
    nmin = np.zeros(4 << (n - 1), np.int64)
    np.add.at(nmin, key, (w == wmin[key]).astype(np.int64))
    p = 1e-7
    logP, am = oracle.decode(d, synth.depolarizing(n, p), _all_syndromes(d))
    expect = np.log(nmin) + wmin * math.log(p / 3) + (n - wmin) * math.log(1 - p)
    np.testing.assert_allclose(logP.reshape(-1), expect, rtol=0, atol=1e-4)
    # the decision is the coset of minimum weight whenever that is unique
    W = wmin.reshape(-1, 4)
    uniq = (W == W.min(axis=1, keepdims=True)).sum(axis=1) == 1
    np.testing.assert_array_equal(am[uniq], W.argmin(axis=1)[uniq])


def test_low_weight_errors_decode_to_their_class_d5():
    """Every error of weight <= (d-1)/2 is corrected by MLD at small p."""
    d, n = 5, 25
    errs = []
    for qs in itertools.chain(itertools.combinations(range(n), 1), itertools.combinations(range(n), 2)):
        for ps in itertools.product((1, 2, 3), repeat=len(qs)):
            e = np.zeros(n, np.uint8)
            e[list(qs)] = ps
            errs.append(e)
    E = np.array(errs)
    _, am = oracle.decode(d, synth.depolarizing(n, 1e-3), synth.syndromes_of(d, E))
    np.testing.assert_array_equal(am, synth.true_class(d, E))


# --- destabilisers, representatives and gauge invariance --------------------

@pytest.mark.parametrize("d", [3, 5, 9, 13])
def test_destabilisers_and_representatives(d):
    n, m, _ = oracle.code_info(d)
    T = oracle.destabilisers(d)
    bits = ((synth.syndromes_of(d, T)[:, :, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1))
    bits = bits.reshape(m, -1)[:, :m].astype(np.uint8)
    np.testing.assert_array_equal(bits, np.eye(m, dtype=np.uint8))
    assert not synth.true_class(d, T).any()
    E = synth.sample_errors(d, synth.depolarizing(n, 0.15), 64, seed=d)
    syn = synth.syndromes_of(d, E)
    reps = oracle.representatives(d, syn)
    for l in range(4):
        np.testing.assert_array_equal(synth.syndromes_of(d, reps[:, l]), syn)
        assert (synth.true_class(d, reps[:, l]) == l).all()


def _stabiliser_product(d, alpha):
    E = np.zeros(d * d, np.uint8)
    for a, (t, qs) in zip(alpha, synth.stabilizers(d)):
        if a:
            E[qs] ^= 1 if t == 0 else 2
    return E


@pytest.mark.parametrize("d", [5, 7])
def test_gauge_invariance_and_true_coset(d):
    """Z depends only on the coset: E and E*S give the same value, and the
    representative built from (syndrome, class) of E lies in E's coset."""
    n = d * d
    noise = _random_noise(n, d, 0.01, 0.15)
    rng = np.random.default_rng(d)
    E = synth.sample_errors(d, noise, 6, seed=99)
    ES = np.array([e ^ _stabiliser_product(d, rng.integers(0, 2, n - 1)) for e in E])
    z1 = oracle.coset_logz(d, noise, E)
    z2 = oracle.coset_logz(d, noise, ES)
    np.testing.assert_allclose(z1, z2, rtol=0, atol=1e-11)
    reps = oracle.representatives(d, synth.syndromes_of(d, E))
    cls = synth.true_class(d, E)
    z3 = oracle.coset_logz(d, noise, reps[np.arange(len(E)), cls])
    np.testing.assert_allclose(z1, z3, rtol=0, atol=1e-11)


# --- symmetries of the patch -------------------------------------------------

def _swap_xz_codes(E):
    return ((E & 1) << 1) | ((E >> 1) & 1)


def _rotate(d, E, noise, quarter):
    """Map qubit (r,c) to (c, d-1-r) (quarter turn, with X<->Z) or to
    (d-1-r, d-1-c) (half turn); both map the stabiliser group onto itself."""
    E2 = np.zeros_like(E)
    N2 = np.zeros_like(noise)
    for r in range(d):
        for c in range(d):
            q = r * d + c
            q2 = (c * d + (d - 1 - r)) if quarter else ((d - 1 - r) * d + (d - 1 - c))
            E2[..., q2] = _swap_xz_codes(E[..., q]) if quarter else E[..., q]
            N2[q2] = noise[q][[0, 3, 2, 1]] if quarter else noise[q]
    return E2, N2


@pytest.mark.parametrize("quarter", [True, False])
def test_rotation_symmetry(quarter):
    d, n = 7, 49
    noise = _random_noise(n, 17, 0.01, 0.12)
    E = synth.sample_errors(d, noise, 6, seed=5)
    E2, N2 = _rotate(d, E, noise, quarter)
    np.testing.assert_allclose(oracle.coset_logz(d, noise, E), oracle.coset_logz(d, N2, E2),
                               rtol=0, atol=1e-11)


# --- independent X/Z noise and the bit-flip RBIM (Eq. 6) --------------------

def test_independent_xz_noise_factorises():
    """P(X^u Z^v) = q_x(u) q_z(v) makes Z_l = Z^x_{l_X} Z^z_{l_Z}, hence
    ln Z_I + ln Z_Y = ln Z_X + ln Z_Z."""
    d, n = 7, 49
    rng = np.random.default_rng(4)
    qx = rng.uniform(0.02, 0.2, n)
    qz = rng.uniform(0.02, 0.2, n)
    noise = np.stack([(1 - qx) * (1 - qz), qx * (1 - qz), qx * qz, (1 - qx) * qz], axis=1)
    E = synth.sample_errors(d, noise, 16, seed=8)
    lp, _ = oracle.decode(d, noise, synth.syndromes_of(d, E))
    np.testing.assert_allclose(lp[:, 0] + lp[:, 3], lp[:, 1] + lp[:, 2], rtol=0, atol=1e-10)


@pytest.mark.parametrize("d", [3, 5])
def test_bitflip_random_bond_ising(d):
    """Bit-flip noise: Z of the coset of E equals (p(1-p))^{n/2} times the RBIM
    partition function sum_sigma prod_q exp(K eta_q prod_{f ni q} sigma_f) over
    spins on the X-type plaquettes, K = ln((1-p)/p)/2, eta_q = (-1)^{x_q}
    (Eq. 6); cosets that need a Z component have Z = 0."""
    n = d * d
    p = 0.08
    noise = np.zeros((n, 4))
    noise[:, 0], noise[:, 1] = 1 - p, p
    xplaq = [qs for t, qs in synth.stabilizers(d) if t == 0]
    E = synth.sample_errors(d, noise, 4, seed=13)
    K = 0.5 * math.log((1 - p) / p)
    for e in E:
        eta = np.where(e & 1, -1.0, 1.0)
        total = 0.0
        for spins in itertools.product((1, -1), repeat=len(xplaq)):
            prod = np.ones(n)
            for s, qs in zip(spins, xplaq):
                prod[qs] *= s
            total += math.exp(K * float((eta * prod).sum()))
        expect = 0.5 * n * math.log(p * (1 - p)) + math.log(total)
        got = oracle.coset_logz(d, noise, e[None])[0]
        assert abs(got - expect) < 1e-10
        zl = e.copy()
        zl[:d] ^= 2                      # times Z_L (row 0): needs a Z component
        assert np.isneginf(oracle.coset_logz(d, noise, zl[None])[0])


# --- derivatives --------------------------------------------------------------

@pytest.mark.parametrize("d", [3, 5])
def test_derivatives_finite_differences_and_euler(d):
    """dZ/dp_{q,P} against central differences, and the Euler identity
    sum_P p_{q,P} d ln Z/d p_{q,P} = 1 (Z is linear in each row)."""
    n = d * d
    noise = _random_noise(n, 31 + d, 0.02, 0.2)
    E = synth.sample_errors(d, noise, 2, seed=3)
    lz, g = oracle.coset_dlogz(d, noise, E)
    np.testing.assert_allclose((g * noise[None]).sum(axis=2), 1.0, rtol=0, atol=1e-11)
    h = 1e-6
    rng = np.random.default_rng(d)
    for q in rng.choice(n, 4, replace=False):
        for P in range(4):
            up = noise.copy(); up[q, P] += h
            dn = noise.copy(); dn[q, P] -= h
            fd = (oracle.coset_logz(d, up, E) - oracle.coset_logz(d, dn, E)) / (2 * h)
            np.testing.assert_allclose(g[:, q, P], fd, rtol=1e-6, atol=1e-8)


# --- the FP64 boundary-MPS mode at exact bond dimension ----------------------

@pytest.mark.parametrize("d,chi", [(3, 2), (5, 4), (7, 8), (9, 16)])
def test_mps_mode_exact_at_full_bond(d, chi):
    """With chi >= 2^floor(d/2) no singular value is discarded and the
    boundary-MPS sweep equals the exact contraction."""
    n = d * d
    noise = synth.depolarizing(n, 0.15)
    syn = synth.syndromes_of(d, synth.sample_errors(d, noise, 2, seed=1))
    ref, _ = oracle.decode(d, noise, syn)
    np.testing.assert_allclose(omps.decode_mps(d, noise, syn, chi), ref, rtol=0, atol=1e-9)


@pytest.mark.parametrize("col", [2, 4])
def test_mps_mode_x_string_column(col):
    """X on any column is an X_L (they differ by X-type stabilisers): at the
    exact bond the sweep gives the same Z_l for the representative with the X
    string on another column; below it the value depends on the
    representative (the truncation of a different network)."""
    d, n = 5, 25
    noise = synth.biased(n, 0.12, 5.0)
    syn = synth.syndromes_of(d, synth.sample_errors(d, noise, 3, seed=2))
    ref, _ = oracle.decode(d, noise, syn)
    np.testing.assert_allclose(omps.decode_mps(d, noise, syn, 4, xl_column=col), ref, rtol=0, atol=1e-9)
    a = omps.decode_mps(d, noise, syn, 2, xl_column=0)
    b = omps.decode_mps(d, noise, syn, 2, xl_column=col)
    np.testing.assert_array_equal(a[:, [0, 2]], b[:, [0, 2]])   # l_X = 0: the same network
    assert np.abs(a - b).max() > 0


def test_mps_mode_truncation_converges():
    """Below the exact bond the error shrinks as chi grows (Sec. 3.2.1)."""
    d, n = 9, 81
    noise = synth.depolarizing(n, 0.15)
    syn = synth.syndromes_of(d, synth.sample_errors(d, noise, 2, seed=3))
    ref, _ = oracle.decode(d, noise, syn)
    errs = [np.abs(omps.decode_mps(d, noise, syn, chi) - ref).max() for chi in (2, 4, 8, 16)]
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < 1e-9


# --- stored expected values (written by tests/golden/make_golden.py) ----------

def _golden(name):
    import os
    rows = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden", name))
            if not l.startswith("#")]
    return rows


def test_golden_d3_bruteforce_table():
    rows = _golden("d3_p010_bruteforce.txt")
    ref = np.array([[float(v) for v in r[1:5]] for r in rows])
    logP, _ = oracle.decode(3, synth.depolarizing(9, 0.10), _all_syndromes(3))
    np.testing.assert_allclose(logP, ref, rtol=0, atol=1e-12)


def test_golden_d5_group_enumeration():
    rows = _golden("d5_group_enum.txt")
    syn = np.array([[int(r[0])] for r in rows], dtype=np.uint64)
    ref = np.array([[float(v) for v in r[1:5]] for r in rows])
    logP, _ = oracle.decode(5, synth.depolarizing(25, 0.12), syn)
    np.testing.assert_allclose(logP, ref, rtol=0, atol=1e-11)


# ---------------------------------------------------------------- detector error models (Sec. 3.2.2)

def test_dem_qubit_table_closed_forms():
    """Closed forms of composing independent mechanisms on one qubit."""
    d, n = 3, 9
    # one X mechanism: (1 - p, p, 0, 0)
    t = oracle.dem_qubit_table(d, [4], [1], [0.2])
    np.testing.assert_allclose(t[4], [0.8, 0.2, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(t[0], [1.0, 0.0, 0.0, 0.0], atol=0)
    # independent X and Z (code capacity with independent flips): product form
    px, pz = 0.11, 0.07
    t = oracle.dem_qubit_table(d, [2, 2], [1, 2], [px, pz])
    np.testing.assert_allclose(t[2], [(1 - px) * (1 - pz), px * (1 - pz), px * pz, (1 - px) * pz], atol=1e-15)
    # two X mechanisms: odd number fires
    t = oracle.dem_qubit_table(d, [1, 1], [1, 1], [0.1, 0.3])
    np.testing.assert_allclose(t[1], [0.9 * 0.7 + 0.1 * 0.3, 0.1 * 0.7 + 0.9 * 0.3, 0, 0], atol=1e-15)
    # X, Y, Z mechanisms: enumerate the eight on/off patterns by hand
    ps = (0.05, 0.02, 0.08)
    t = oracle.dem_qubit_table(d, [7, 7, 7], [1, 3, 2], ps)
    want = np.zeros(4)
    for bx in (0, 1):
        for by in (0, 1):
            for bz in (0, 1):
                w = (ps[0] if bx else 1 - ps[0]) * (ps[1] if by else 1 - ps[1]) * (ps[2] if bz else 1 - ps[2])
                x = bx ^ by
                z = bz ^ by
                want[{(0, 0): 0, (1, 0): 1, (1, 1): 2, (0, 1): 3}[(x, z)]] += w
    np.testing.assert_allclose(t[7], want, atol=1e-15)
    assert abs(t.sum(axis=1) - 1).max() < 1e-15
    with pytest.raises(ValueError):
        oracle.dem_qubit_table(d, [n], [1], [0.1])
    with pytest.raises(ValueError):
        oracle.dem_qubit_table(d, [0], [0], [0.1])


def test_dem_definition_equals_generator_picture():
    """Summing over mechanism configurations (the detector picture's sum)
    equals the generator picture's coset sums with the composed per-qubit
    table, for every syndrome and class: by brute force over all 4^n Paulis
    and by the dense variable-elimination contraction."""
    d = 3
    rng = np.random.default_rng(5)
    q = np.repeat(np.arange(9), 2)
    pauli = rng.integers(1, 4, q.size)
    p = rng.uniform(0.01, 0.3, q.size)
    Zd = oracle.dem_bruteforce_table(d, q, pauli, p)
    tab = oracle.dem_qubit_table(d, q, pauli, p)
    Zg = oracle.bruteforce_table(d, tab)
    assert abs(Zd.sum() - 1.0) < 1e-12
    np.testing.assert_allclose(Zd, Zg, rtol=1e-12, atol=1e-300)
    m = 8
    bits = ((np.arange(1 << m)[:, None] >> np.arange(m)) & 1).astype(np.uint8)
    syn = np.array([synth.pack_bits(b[None])[0] for b in bits])
    lp, _ = oracle.decode(d, tab, syn)
    np.testing.assert_allclose(lp, np.log(Zd), rtol=0, atol=1e-11)


def test_mechanism_sampler_matches_composed_table():
    """The seeded mechanism sampler's per-qubit Pauli frequencies agree with
    the oracle's composition of the same mechanisms (within 5 sigma)."""
    d, B = 3, 200000
    q, c, p = synth.mechanism_model(d, seed=11, median=0.08)
    E = synth.sample_mechanisms(d, q, c, p, B, seed=12)
    tab = oracle.dem_qubit_table(d, q, c, p)
    code_to_row = np.array([0, 1, 3, 2])
    for qq in range(d * d):
        f = np.bincount(code_to_row[E[:, qq]], minlength=4) / B
        sig = np.sqrt(tab[qq] * (1 - tab[qq]) / B)
        assert (np.abs(f - tab[qq]) <= 5 * sig + 1e-12).all(), (qq, f, tab[qq])


# --- the boundary-MPS mode at truncated chi, against dense cut truncations ---

def _dense_column_transfer(d, psi, noise, E, c):
    """psi'(beta) = sum_alpha psi(alpha) prod_r w_r(alpha_r, alpha_r+1, beta_r, beta_r+1)
    over corner columns c (alpha) and c+1 (beta), every position binary (an
    absent plaquette's variable is pinned to 0 by zero entries). The qubit
    factor of (r, c) is p_q[E_q xor X^u Z^v], u (v) the XOR of the variables of
    its X-type (Z-type) corner plaquettes (Eq. 7, generator picture). Written
    here from the layout of synth, not from the oracle."""
    L = d + 1
    idx = np.arange(1 << L)
    bits = (idx[:, None] >> (L - 1 - np.arange(L))[None, :]) & 1      # position 0 = most significant
    a = bits[None, :, :]                                               # alpha [1, S, L]
    b = bits[:, None, :]                                               # beta  [S, 1, L]
    code_of = np.array([[0, 3], [1, 2]])                              # noise column of (x, z)
    T = np.ones((1 << L, 1 << L))
    for r in range(d):
        q = r * d + c
        u = np.zeros_like(T, dtype=np.int64)
        v = np.zeros_like(T, dtype=np.int64)
        for (i, j), var in (((r, c), a[..., r]), ((r + 1, c), a[..., r + 1]),
                            ((r, c + 1), b[..., r]), ((r + 1, c + 1), b[..., r + 1])):
            if not synth._present(d, i, j):
                continue
            if (i + j) % 2 == 0:
                u = u ^ var
            else:
                v = v ^ var
        x = (int(E[q]) & 1) ^ u
        z = ((int(E[q]) >> 1) & 1) ^ v
        T *= noise[q][code_of[x, z]]
    pres_b = np.array([synth._present(d, i, c + 1) for i in range(L)])
    keep = np.all(bits[:, ~pres_b] == 0, axis=1)                      # beta of absent positions = 0
    return (T @ psi) * keep


def _dense_truncated_logz(d, noise, E, chi, gaps):
    """ln Z of the boundary-MPS rule computed on the dense state: after each
    column, cut by cut from the last bond to the first, the best rank-chi
    approximation (Eckart-Young, numpy SVD) of the full 2^(d+1) vector
    matricised at that cut. The right-to-left SVD sweep of a left-canonical
    MPS performs exactly this sequence of projections."""
    L = d + 1
    idx = np.arange(1 << L)
    bits = (idx[:, None] >> (L - 1 - np.arange(L))[None, :]) & 1
    pres = np.array([synth._present(d, i, 0) for i in range(L)])
    psi = np.all(bits[:, ~pres] == 0, axis=1).astype(np.float64)
    log_scale = 0.0
    for c in range(d):
        psi = _dense_column_transfer(d, psi, noise, E, c)
        for k in range(L - 2, -1, -1):                                # cut between positions k, k+1
            M = psi.reshape(1 << (k + 1), 1 << (L - 1 - k))
            U, S, Vh = np.linalg.svd(M, full_matrices=False)
            if chi < len(S) and S[chi] > 1e-12 * S[0]:
                gaps.append((S[chi - 1] - S[chi]) / S[chi - 1])
            kk = min(chi, len(S))
            psi = ((U[:, :kk] * S[:kk]) @ Vh[:kk]).reshape(-1)
        m = np.abs(psi).max()
        psi = psi / m
        log_scale += math.log(m)
    return math.log(psi.sum()) + log_scale


def _posterior(x):
    return np.exp(x - np.logaddexp.reduce(x, axis=1, keepdims=True))


def _mps_and_dense(d, chi, seed):
    n = d * d
    noise = synth.lognormal_biased(n, seed=seed, median=0.15)
    syn = synth.syndromes_of(d, synth.sample_errors(d, noise, 2, seed=41))
    reps = oracle.representatives(d, syn)
    gaps = []
    ref = np.array([[_dense_truncated_logz(d, noise, reps[b, l], chi, gaps) for l in range(4)]
                    for b in range(len(syn))])
    got = np.array([[omps.coset_logz_mps(d, noise, reps[b, l], chi) for l in range(4)]
                    for b in range(len(syn))])
    return ref, got, gaps


@pytest.mark.parametrize("d,chi", [(5, 2), (5, 3), (7, 4), (7, 6)])
def test_mps_mode_truncation_equals_dense_cut_truncations(d, chi):
    """At truncated chi the boundary-MPS mode (left QR sweep, then right-to-left
    SVD keeping min(chi, #values), Sec. 3.2.1) equals, column by column, the
    dense transfer followed by the optimal rank-chi truncation of the dense
    state at every cut from the last to the first. Per-qubit noise keeps the
    singular values at each cut apart (relative gap at the cut above 1e-3),
    so the truncation is unique; rates near 0.15 make the discarded weight
    matter. Both sides round in FP64 relative to the largest coset, so the
    bar is 1e-10 on the leading coset's ln Z and on the posterior Pr(l|s)."""
    ref, got, gaps = _mps_and_dense(d, chi, 40 + d)
    assert gaps and min(gaps) > 1e-3                          # no tie at any cut
    lead = np.argmax(ref, axis=1)
    rows = np.arange(len(ref))
    assert np.abs(got[rows, lead] - ref[rows, lead]).max() < 1e-10
    assert np.abs(_posterior(got) - _posterior(ref)).max() < 1e-10


def test_dense_cut_pin_detects_a_missing_canonical_sweep(monkeypatch):
    """The pin above has the power to catch a plausible mistake: truncating the
    applied MPS by right-to-left SVDs without first bringing it to
    left-canonical form (a sub-optimal truncation that still converges in
    chi) moves the leading ln Z and the posterior far beyond the pin's 1e-10
    (by 1e-3 to 1e-1 on these cases)."""

    def compress_without_qr(mps, chi_):
        mps = [t.copy() for t in mps]
        for i in range(len(mps) - 1, 0, -1):
            l, p, r = mps[i].shape
            U, S, Vh = np.linalg.svd(mps[i].reshape(l, p * r), full_matrices=False)
            k = min(chi_, S.shape[0])
            mps[i] = Vh[:k].reshape(k, p, r)
            mps[i - 1] = np.einsum("lpa,ab->lpb", mps[i - 1], U[:, :k] * S[:k])
        return mps

    monkeypatch.setattr(omps, "compress", compress_without_qr)
    for d, chi in [(5, 2), (7, 4)]:
        ref, got, _ = _mps_and_dense(d, chi, 40 + d)
        lead = np.argmax(ref, axis=1)
        rows = np.arange(len(ref))
        assert max(np.abs(got[rows, lead] - ref[rows, lead]).max(),
                   np.abs(_posterior(got) - _posterior(ref)).max()) > 1e-4
