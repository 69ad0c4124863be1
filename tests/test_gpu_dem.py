"""Detector-picture decode of code-capacity error-mechanism models
(mld_decode_dem, Sec. 3.2.2) against the oracle: the configuration-sum
definition (brute force, d = 3) and the generator picture with the composed
per-qubit table (any d), element by element; against the generator-picture
CUDA path at the bench size; and the degenerate inputs."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_17230_gb300 as m
    m.load()
    return m


def _model(d, seed, lo=0.005, hi=0.15):
    """0..3 mechanisms per qubit, random Pauli types (repeats allowed)."""
    rng = np.random.default_rng(seed)
    q, c, p = [], [], []
    for qq in range(d * d):
        for _ in range(rng.integers(0, 4)):
            q.append(qq)
            c.append(rng.integers(1, 4))
            p.append(rng.uniform(lo, hi))
    return np.array(q, np.int32), np.array(c, np.int32), np.array(p, np.float64)


def _compare(lp, ref, atol=2e-5):
    # FP32 sums over d^2 qubit steps: rounding stays near 1e-5 at d = 9 (the
    # decoding tolerance on ln P is 1e-3)
    fin = np.isfinite(ref)
    assert (np.isfinite(lp) == fin).all()
    np.testing.assert_allclose(lp[fin], ref[fin], rtol=0, atol=atol)


@pytest.mark.parametrize("d,B", [(3, 256), (5, 301), (7, 257), (9, 65), (11, 40)])
def test_dem_vs_generator_oracle(mld, d, B):
    q, c, p = _model(d, seed=d)
    tab = oracle.dem_qubit_table(d, q, c, p)
    E = synth.sample_errors(d, tab, B, seed=100 + d)
    syn = synth.syndromes_of(d, E)
    code = mld.Code(d)
    lp, am = code.decode_dem(q, c, p, torch.tensor(syn.view(np.int64), device="cuda"))
    torch.cuda.synchronize()
    ref, ram = oracle.decode(d, tab, syn)
    lp = lp.cpu().numpy()
    _compare(lp, ref)
    srt = np.sort(ref, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 1e-4
    assert np.array_equal(am.cpu().numpy()[clear], ram[clear])


def test_dem_vs_configuration_sum_d3(mld):
    """Every syndrome of d = 3 against the sum over all 2^18 mechanism
    configurations (the definition), including classes of probability 0."""
    d = 3
    rng = np.random.default_rng(7)
    q = np.repeat(np.arange(9), 2).astype(np.int32)
    c = rng.integers(1, 4, q.size).astype(np.int32)
    p = rng.uniform(0.01, 0.3, q.size)
    Z = oracle.dem_bruteforce_table(d, q, c, p)
    bits = ((np.arange(256)[:, None] >> np.arange(8)) & 1).astype(np.uint8)
    syn = np.array([synth.pack_bits(b[None])[0] for b in bits])
    code = mld.Code(d)
    lp, _ = code.decode_dem(q, c, p, torch.tensor(syn.view(np.int64), device="cuda"))
    torch.cuda.synchronize()
    with np.errstate(divide="ignore"):
        ref = np.log(Z)
    _compare(lp.cpu().numpy(), ref)


def test_dem_independent_xz_vs_cuda_generator_d9(mld):
    """Independent X and Z flips per qubit (the case where the detector
    picture's network splits into two binary ones) at the bench size:
    65,536 syndromes, against mld_decode of the composed table (generator
    picture, exact chi) -- two different contractions of the same Z_l(s)."""
    d, B = 9, 65536
    n = d * d
    rng = np.random.default_rng(9)
    px, pz = rng.uniform(0.01, 0.12, n), rng.uniform(0.01, 0.12, n)
    q = np.concatenate([np.arange(n), np.arange(n)]).astype(np.int32)
    c = np.concatenate([np.full(n, 1), np.full(n, 2)]).astype(np.int32)
    p = np.concatenate([px, pz])
    tab = oracle.dem_qubit_table(d, q, c, p)
    np.testing.assert_allclose(tab, np.stack([(1 - px) * (1 - pz), px * (1 - pz), px * pz, (1 - px) * pz], 1),
                               atol=1e-15)
    E = synth.sample_errors(d, tab, B, seed=91)
    sy = torch.tensor(synth.syndromes_of(d, E).view(np.int64), device="cuda")
    code = mld.Code(d)
    lp, am = code.decode_dem(q, c, p, sy)
    lg, ag = code.decode(torch.tensor(tab, dtype=torch.float32, device="cuda"), sy, 32)
    torch.cuda.synchronize()
    lp, lg = lp.cpu().numpy(), lg.cpu().numpy()
    np.testing.assert_allclose(lp, lg, rtol=0, atol=2e-4)
    srt = np.sort(lg, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 1e-3
    assert np.array_equal(am.cpu().numpy()[clear], ag.cpu().numpy()[clear])
    # sampled rows against the FP64 oracle
    idx = np.random.default_rng(1).choice(B, 48, replace=False)
    ref, _ = oracle.decode(d, tab, synth.syndromes_of(d, E[idx]))
    _compare(lp[idx], ref)


def test_dem_degenerate_inputs(mld):
    d = 5
    code = mld.Code(d)
    syn = synth.syndromes_of(d, np.zeros((3, 25), np.uint8))
    syn[1, 0] = 1                                     # one flipped detector
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    # no mechanisms: only the trivial syndrome and class are possible
    lp, am = code.decode_dem([], [], [], sy)
    torch.cuda.synchronize()
    lp = lp.cpu().numpy()
    assert lp[0, 0] == 0.0 and np.isneginf(lp[0, 1:]).all()
    assert np.isneginf(lp[1]).all() and am.cpu().numpy()[0] == 0
    # empty batch
    e = torch.zeros((0, 1), dtype=torch.int64, device="cuda")
    lp0, _ = code.decode_dem([0], [1], [0.1], e)
    assert lp0.shape == (0, 4)
    # p = 1 and p = 0 mechanisms are allowed; bad ones are rejected
    code.decode_dem([0, 1], [1, 3], [1.0, 0.0], sy)
    for bad in (([25], [1], [0.1]), ([0], [0], [0.1]), ([0], [4], [0.1]), ([0], [1], [1.5]), ([0], [1], [np.nan])):
        with pytest.raises(mld.MldError):
            code.decode_dem(*bad, sy)
    big = mld.Code(13)
    with pytest.raises(mld.MldError):
        big.decode_dem([0], [1], [0.1], torch.zeros((1, 3), dtype=torch.int64, device="cuda"))


def test_dem_rerun_bit_identical(mld):
    d, B = 7, 4096
    q, c, p = _model(d, seed=70)
    E = synth.sample_errors(d, oracle.dem_qubit_table(d, q, c, p), B, seed=71)
    sy = torch.tensor(synth.syndromes_of(d, E).view(np.int64), device="cuda")
    code = mld.Code(d)
    a, _ = code.decode_dem(q, c, p, sy)
    b, _ = code.decode_dem(q, c, p, sy)
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
