"""Kac-Ward decode under independent X/Z noise (mld_decode_xz, Sec. 3.1.3)
against the oracle: the exact variable elimination (Eq. 7) element by element
at d = 3..13, the FP64 Kac-Ward oracle at d = 17 and 25 on sampled syndromes,
the generator-picture CUDA path on the same table, bit-flip noise, and the
degenerate and invalid inputs.

Tolerances. FP64: every class to 1e-8 where the oracle's exact value is within
30 nats of the leading class (beyond that the signed determinant of a class
that unlikely is below FP64's resolution of the leading one, a property of the
method). FP32 (its accuracy follows the conditioning of the matrix, which
worsens at low rates: the inputs here are sampled at rates where it is
resolved, 0.02..0.2 per qubit up to d = 13 and 0.08 at d = 17, 25): the
leading class's ln Z to 1e-4 (1e-3 at d = 25, where about 2,600 pivots round)
and the posteriors Z_l / sum Z to 1e-3; the decisions equal the oracle's
wherever its two best classes differ by more than 1e-3 in ln Z. Rare
syndromes at low rates exceed these bounds in FP32 (measured with the bench,
not asserted here)."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import kac_ward as okw

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_17230_gb300 as m
    m.load()
    return m


def _rates(d, seed, lo, hi):
    rng = np.random.default_rng(seed)
    n = d * d
    return rng.uniform(lo, hi, n).astype(np.float32), rng.uniform(lo, hi, n).astype(np.float32)


def _run(mld, code, px, pz, syn, precision):
    dpx = torch.tensor(px, device="cuda")
    dpz = None if pz is None else torch.tensor(pz, device="cuda")
    lp, am = code.decode_xz(dpx, dpz, torch.tensor(syn.view(np.int64), device="cuda"), precision)
    torch.cuda.synchronize()
    assert code.status() == 0
    return lp.cpu().numpy(), am.cpu().numpy()


def _posterior(v):
    m = v.max(axis=1, keepdims=True)
    e = np.exp(v - m)
    return e / e.sum(axis=1, keepdims=True)


def _check_fp32(lp, am, ref, ram, lead_atol=1e-4):
    rows = np.arange(len(ref))
    lead = np.argmax(ref, axis=1)
    np.testing.assert_allclose(lp[rows, lead], ref[rows, lead], rtol=0, atol=lead_atol)
    np.testing.assert_allclose(_posterior(lp), _posterior(ref), rtol=0, atol=1e-3)
    srt = np.sort(ref, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 1e-3
    np.testing.assert_array_equal(am[clear], ram[clear])


def _check_fp64(lp, am, ref, ram, atol=1e-8):
    near = ref >= ref.max(axis=1, keepdims=True) - 30.0
    np.testing.assert_allclose(lp[near], ref[near], rtol=0, atol=atol)
    srt = np.sort(ref, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 1e-6
    np.testing.assert_array_equal(am[clear], ram[clear])


@pytest.mark.parametrize("d,B", [(3, 200), (5, 97), (7, 64), (9, 40), (11, 16), (13, 8)])
def test_xz_vs_exact_oracle(mld, d, B):
    """Per-qubit rates in [0.02, 0.2], sampled errors; B not a multiple of the
    grid. FP64 and FP32 against the exact contraction."""
    px, pz = _rates(d, d, 0.02, 0.2)
    tab = okw.xz_table(px.astype(np.float64), pz.astype(np.float64))
    syn = synth.syndromes_of(d, synth.sample_errors(d, tab, B, seed=50 + d))
    ref, ram = oracle.decode(d, tab, syn)
    code = mld.Code(d)
    lp64, am64 = _run(mld, code, px, pz, syn, mld.MLD_FP64)
    _check_fp64(lp64, am64, ref, ram)
    lp32, am32 = _run(mld, code, px, pz, syn, mld.MLD_FP32)
    _check_fp32(lp32, am32, ref, ram)


@pytest.mark.parametrize("d", [3, 7, 11])
def test_bitflip_vs_exact_oracle(mld, d):
    """pz = NULL: -inf exactly where the exact contraction is zero (the l_Z = 1
    classes, and every class of a syndrome with an X-type bit), the finite
    classes equal."""
    n = d * d
    px, _ = _rates(d, 3 * d, 0.03, 0.15)
    tab = okw.xz_table(px.astype(np.float64), None)
    syn = synth.syndromes_of(d, synth.sample_errors(d, tab, 24, seed=d))
    t, _, _, _ = oracle.layout(d)
    bits = np.zeros((1, n - 1), np.uint8)
    bits[0, int(np.nonzero(t == 0)[0][-1])] = 1
    syn = np.concatenate([syn, synth.pack_bits(bits)])
    ref, ram = oracle.decode(d, tab, syn)
    code = mld.Code(d)
    for prec in (mld.MLD_FP64, mld.MLD_FP32):
        lp, am = _run(mld, code, px, None, syn, prec)
        np.testing.assert_array_equal(np.isfinite(lp), np.isfinite(ref))
        assert np.isneginf(lp[-1]).all()
        fin = np.isfinite(ref).all(axis=0)
        live = ref[:-1, :2]
        if prec == mld.MLD_FP64:
            _check_fp64(lp[:-1, :2], am[:-1], live, ram[:-1])
        else:
            _check_fp32(lp[:-1, :2], am[:-1], live, ram[:-1])
        assert not fin[2:].any()


@pytest.mark.parametrize("d,B,p", [(17, 12, 0.08), (25, 4, 0.08)])
def test_large_d_vs_kac_ward_oracle(mld, d, B, p):
    """At the distances the boundary-MPS path truncates: against the FP64
    Kac-Ward oracle (dense slogdet of the whole matrix, another drawing and
    no banding) on sampled syndromes at a uniform rate."""
    n = d * d
    px = np.full(n, p, np.float32)
    pz = np.full(n, p, np.float32)
    tab = okw.xz_table(px.astype(np.float64), pz.astype(np.float64))
    syn = synth.syndromes_of(d, synth.sample_errors(d, tab, B, seed=d))
    ref, ram = okw.decode_xz(d, px.astype(np.float64), pz.astype(np.float64), syn)
    code = mld.Code(d)
    lp64, am64 = _run(mld, code, px, pz, syn, mld.MLD_FP64)
    _check_fp64(lp64, am64, ref, ram, atol=1e-7)
    lp32, am32 = _run(mld, code, px, pz, syn, mld.MLD_FP32)
    _check_fp32(lp32, am32, ref, ram, lead_atol=1e-4 if d <= 17 else 1e-3)


def test_agrees_with_generator_sweep(mld):
    """d = 9, the bench's noise shape: the Kac-Ward kernel and the exact
    boundary-MPS sweep on the same independent X/Z table."""
    d, B = 9, 512
    px, pz = _rates(d, 77, 0.03, 0.12)
    tab = okw.xz_table(px.astype(np.float64), pz.astype(np.float64)).astype(np.float32)
    syn = synth.syndromes_of(d, synth.sample_errors(d, tab.astype(np.float64), B, seed=9))
    code = mld.Code(d)
    dsyn = torch.tensor(syn.view(np.int64), device="cuda")
    lp_mps, am_mps = code.decode(torch.tensor(tab, device="cuda"), dsyn, 16)
    lp_kw, am_kw = code.decode_xz(torch.tensor(px, device="cuda"), torch.tensor(pz, device="cuda"), dsyn)
    torch.cuda.synchronize()
    a, b = lp_mps.cpu().numpy(), lp_kw.cpu().numpy()
    rows = np.arange(B)
    lead = np.argmax(a, axis=1)
    np.testing.assert_allclose(b[rows, lead], a[rows, lead], rtol=0, atol=1e-4)
    srt = np.sort(a, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 1e-3
    np.testing.assert_array_equal(am_kw.cpu().numpy()[clear], am_mps.cpu().numpy()[clear])


def test_degenerate_and_invalid(mld):
    d = 5
    n = d * d
    code = mld.Code(d)
    px = torch.full((n,), 0.1, device="cuda")
    empty = torch.zeros((0, code.words), dtype=torch.int64, device="cuda")
    lp, am = code.decode_xz(px, px, empty)
    assert lp.shape == (0, 4)
    syn = torch.zeros((3, code.words), dtype=torch.int64, device="cuda")
    # the zero syndrome: the identity's classes lead
    lp, am = code.decode_xz(px, px, syn, mld.MLD_FP64)
    torch.cuda.synchronize()
    assert (am.cpu().numpy() == 0).all()
    # an unknown precision is refused before any launch
    out = torch.empty((3, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(mld.MldError) as e:
        mld.mld_decode_xz(code.handle, px, px, syn, 3, 7, out)
    assert e.value.status == 1
    # a rate outside (0, 1) is flagged in the status word
    bad = px.clone()
    bad[4] = 0.0
    code.decode_xz(bad, px, syn)
    torch.cuda.synchronize()
    assert code.status() == 1            # MLD_ERR_INVALID_ARG
    code2 = mld.Code(d)
    nan = px.clone()
    nan[0] = float("nan")
    code2.decode_xz(px, nan, syn)
    torch.cuda.synchronize()
    assert code2.status() == 1


def test_ln_z_sums_to_syndrome_probability(mld):
    """Sum over the four classes of Z_l = Pr(s), and over all 2^8 syndromes of
    d = 3 the probabilities sum to one (FP64)."""
    d = 3
    px, pz = _rates(d, 4, 0.05, 0.4)
    m = d * d - 1
    bits = ((np.arange(1 << m)[:, None] >> np.arange(m)[None, :]) & 1).astype(np.uint8)
    syn = synth.pack_bits(bits)
    code = mld.Code(d)
    lp, _ = _run(mld, code, px, pz, syn, mld.MLD_FP64)
    assert abs(np.exp(lp).sum() - 1.0) < 1e-9
    assert math.isfinite(lp.max())


def test_executed_flop_counter(mld):
    """The device counter of the elimination's work: positive after a decode,
    within the bound of a full window at every step (both parts), and reset by
    the read."""
    d, B = 9, 64
    n = d * d
    px, pz = _rates(d, 5, 0.05, 0.15)
    tab = okw.xz_table(px.astype(np.float64), pz.astype(np.float64))
    syn = synth.syndromes_of(d, synth.sample_errors(d, tab, B, seed=2))
    code = mld.Code(d)
    _run(mld, code, px, pz, syn, mld.MLD_FP32)      # builds the tables
    code.xz_executed_flops()
    _run(mld, code, px, pz, syn, mld.MLD_FP32)
    f = code.xz_executed_flops() / B
    # matrix order 2|E| = 184 at d = 9, band 27 / 26: per step at most 29 rows
    # times (6 + 8 * (27 + 26 + 4)) flops, two parts
    assert 0 < f <= 2 * 184 * 29 * (6 + 8 * 57)
    assert code.xz_executed_flops() == 0.0


@pytest.mark.parametrize("cutoff,atol", [(1e-7, 5e-3), (1e-9, 1e-3)])
def test_truncated_sweep_against_exact_mld(mld, cutoff, atol):
    """The truncating boundary-MPS path (chi = 32, d = 17) against exact MLD
    from the FP64 Kac-Ward path on independent X/Z noise at p = 0.10 per part:
    the decisions are equal on every syndrome; the leading class's ln Z is
    within 5e-3 at the default relative singular-value cutoff 1e-7 (dropping
    components that are small in 2-norm removes a share of the all-ones
    contraction: measured up to 2.7e-3 at d = 17 and 0.048 at d = 25 over
    thousands of syndromes) and within 1e-3 at cutoff 1e-9."""
    d, B, p = 17, 512, 0.10
    n = d * d
    px = np.full(n, p, np.float32)
    tab = okw.xz_table(px.astype(np.float64), px.astype(np.float64))
    syn = synth.syndromes_of(d, synth.sample_errors(d, tab, B, seed=91))
    code = mld.Code(d)
    exact, am_exact = _run(mld, code, px, px, syn, mld.MLD_FP64)
    code.set_svd_cutoff(cutoff)
    lp, am = code.decode(torch.tensor(tab.astype(np.float32), device="cuda"),
                         torch.tensor(syn.view(np.int64), device="cuda"), 32)
    torch.cuda.synchronize()
    assert code.status() == 0
    lp, am = lp.cpu().numpy(), am.cpu().numpy()
    rows = np.arange(B)
    lead = np.argmax(exact, axis=1)
    np.testing.assert_allclose(lp[rows, lead], exact[rows, lead], rtol=0, atol=atol)
    srt = np.sort(exact, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 1e-3
    np.testing.assert_array_equal(am[clear], am_exact[clear])


def test_fp32_against_fp64_near_threshold_d25(mld):
    """The regime the complex-FP32 path is for: d = 25, px = pz = 0.10. Over
    512 syndromes its leading-class ln Z is within 2e-3 of the FP64 path
    (measured over 4,096: max 1.1e-3) and its decisions are the FP64 ones
    wherever FP64's two best classes differ by more than 1e-3."""
    d, B, p = 25, 512, 0.10
    n = d * d
    px = np.full(n, p, np.float32)
    tab = okw.xz_table(px.astype(np.float64), px.astype(np.float64))
    syn = synth.syndromes_of(d, synth.sample_errors(d, tab, B, seed=25))
    code = mld.Code(d)
    l64, a64 = _run(mld, code, px, px, syn, mld.MLD_FP64)
    l32, a32 = _run(mld, code, px, px, syn, mld.MLD_FP32)
    rows = np.arange(B)
    lead = np.argmax(l64, axis=1)
    np.testing.assert_allclose(l32[rows, lead], l64[rows, lead], rtol=0, atol=2e-3)
    srt = np.sort(l64, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 1e-3
    np.testing.assert_array_equal(a32[clear], a64[clear])
