"""Parity of the truncating sweep (chi below the exact bond 2^floor(d/2)) with
the FP64 boundary-MPS oracle, at the sizes of the d=13, 17 and 25 workloads
(and d=15, where cutoff 0 drives bonds past the first pass's capacity).

The rank-adaptive kernel keeps k = min(chi, #{sigma > cutoff * sigma_1}) at
every cut (default cutoff 1e-7, below FP32 resolution); with cutoff 0 it keeps
min(chi, #values), the oracle's rule. Truncating columns are canonical, so
FP32 rounding (relative to the state's norm) reaches ln Z_l as ~eps Z_max/Z_l:
the bar is 1e-4 on the leading coset's ln Z and on the posterior Pr(l|s).
Expected values at d >= 13 are stored in tests/golden/ (written by
tests/golden/make_golden.py from oracle/ only).
"""
import os

import numpy as np
import pytest

import oracle
import oracle.mps as omps
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def mld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_17230_gb300 as m
    m.load()
    return m


def noise_of(d, kind):
    n = d * d
    t = synth.depolarizing(n, 0.12) if kind == "depolarizing" else synth.biased(n, 0.12, 100.0)
    return t.astype(np.float32)


def workload(d, kind, B):
    noise = noise_of(d, kind)
    E = synth.sample_errors(d, noise, B, seed=synth.config_seed(5, d, 0.12))
    return noise, E, synth.syndromes_of(d, E)


def decode(mld, d, noise, syn, chi, cutoff=None, kernel=0):
    code = mld.Code(d)
    if cutoff is not None:
        code.set_svd_cutoff(cutoff)
    code.set_truncation_kernel(kernel)
    lp, am = code.decode(torch.tensor(noise, device="cuda"), torch.tensor(syn.view(np.int64), device="cuda"), chi)
    torch.cuda.synchronize()
    st = code.status()
    flops, hist = code.executed_flops(), code.bond_histogram()
    code.close()
    assert st == 0
    return lp.cpu().numpy(), am.cpu().numpy(), flops, hist


def posterior(x):
    return np.exp(x - np.logaddexp.reduce(x, axis=1, keepdims=True))


def check_lead_and_posterior(lp, ref, tol=TOL):
    lead = np.argmax(ref, axis=1)
    rows = np.arange(len(ref))
    assert np.abs(lp[rows, lead] - ref[rows, lead]).max() <= tol
    assert np.abs(posterior(lp) - posterior(ref)).max() <= tol


def golden_large():
    rows = {}
    for line in open(os.path.join(GOLDEN, "large_mps.txt")):
        if line.startswith("#"):
            continue
        f = line.split()
        rows.setdefault((int(f[0]), int(f[1]), f[2]), []).append([float(v) for v in f[4:8]])
    return {k: np.array(v) for k, v in rows.items()}


LARGE = [(13, 32, "depolarizing", 16), (17, 32, "depolarizing", 4), (17, 64, "depolarizing", 4),
         (17, 32, "biased", 4), (17, 64, "biased", 4), (25, 32, "depolarizing", 2)]


@pytest.mark.parametrize("d,chi,kind,B", LARGE)
@pytest.mark.parametrize("cutoff", [None, 0.0])
def test_large_d_vs_fp64_mps(mld, d, chi, kind, B, cutoff):
    """d = 13, 17, 25 at chi = 32 and 64 (the scale workloads), depolarizing
    p=0.12 and biased eta=100, with the default cutoff and with cutoff 0 (the
    oracle's keep-min(chi, #values) rule, where chi = 64 keeps bonds above
    48 in the first pass, which runs with the mid capacities above chi 48)."""
    ref = golden_large()[(d, chi, kind)]
    noise, _, syn = workload(d, kind, B)
    lp, am, flops, hist = decode(mld, d, noise, syn, chi, cutoff)
    check_lead_and_posterior(lp, ref)
    assert flops > 0 and hist[1:].sum() > 0 and np.flatnonzero(hist[1:]).max() + 1 <= min(chi, 64)


def test_mid_capacity_bonds_above_48_vs_fp64_mps(mld):
    """d=13, chi=56, cutoff 0: the middle cuts keep up to 56 values, beyond the
    small capacities (bond 48), so the first pass runs with the mid ones
    (bond 64) and decodes these units itself."""
    ref = golden_large()[(13, 56, "depolarizing")]
    noise, _, syn = workload(13, "depolarizing", 2)
    lp, _, _, hist = decode(mld, 13, noise, syn, 56, 0.0)
    check_lead_and_posterior(lp, ref)
    assert hist[49:].sum() > 0                 # bonds above the small capacities occurred


@pytest.mark.parametrize("first_bond", [0, 64])
def test_bonds_above_64_vs_fp64_mps(mld, first_bond):
    """d=15, chi=72, cutoff 0: the middle cuts keep 72 values (the exact rank
    is 128). By default the first pass runs with the bond-128 capacities and
    decodes these units itself; with its capacity capped at 64
    (mld_code_set_truncation_workspace) they are handed back and decoded by
    the second, large-capacity pass. Both against the FP64 oracle."""
    ref = golden_large()[(15, 72, "depolarizing")]
    noise, _, syn = workload(15, "depolarizing", 2)
    code = mld.Code(15)
    code.set_svd_cutoff(0.0)
    code.set_truncation_kernel(1)
    code.set_truncation_workspace(first_bond)
    lp, _ = code.decode(torch.tensor(noise, device="cuda"), torch.tensor(syn.view(np.int64), device="cuda"), 72)
    torch.cuda.synchronize()
    assert code.status() == 0
    hist = code.bond_histogram()
    code.close()
    check_lead_and_posterior(lp.cpu().numpy(), ref)
    assert hist[64] > 0                        # the last bin counts kept bonds of 64 and more


def test_d17_chi128_vs_exact_oracle_64_syndromes(mld):
    """The scale workload's oracle check: d=17, chi=128 against the exact
    dense contraction on the first 64 syndromes. At p=0.12 the Schmidt
    spectra fall below 1e-7 within ~20 values, so chi=128 with the cutoff is
    within FP32 error of exact; decisions agree wherever the exact top two
    cosets differ by more than 1e-3."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "d17_exact_64.txt")) if not l.startswith("#")]
    ref = np.array([[float(v) for v in r[1:5]] for r in rows])
    noise, _, syn = workload(17, "depolarizing", 64)
    lp, am, _, _ = decode(mld, 17, noise, syn, 128)
    check_lead_and_posterior(lp, ref, 1e-3)
    top = np.sort(ref, axis=1)
    clear = top[:, -1] - top[:, -2] > 1e-3
    np.testing.assert_array_equal(am[clear], np.argmax(ref, axis=1)[clear])


@pytest.mark.parametrize("d", [17, 25])
def test_chi8_suffices_well_below_threshold(mld, d):
    """Sec. 3.2.1 reports that chi = 8 suffices at p = 5% up to d = 25: on 2,048
    depolarizing p = 0.05 syndromes the chi = 8 decisions equal the chi = 64
    ones wherever the chi = 64 top two cosets are more than 1e-3 apart, and the
    leading coset's ln Z moves by less than 1e-2."""
    n = d * d
    noise = synth.depolarizing(n, 0.05).astype(np.float32)
    syn = synth.syndromes_of(d, synth.sample_errors(d, noise, 2048, seed=synth.config_seed(5, d, 0.05)))
    lp8, am8, _, h8 = decode(mld, d, noise, syn, 8)
    lp64, am64, _, _ = decode(mld, d, noise, syn, 64)
    top = np.sort(lp64, axis=1)
    clear = top[:, -1] - top[:, -2] > 1e-3
    np.testing.assert_array_equal(am8[clear], am64[clear])
    lead = np.argmax(lp64, axis=1)
    rows = np.arange(len(syn))
    assert np.abs(lp8[rows, lead] - lp64[rows, lead]).max() < 1e-2
    assert np.flatnonzero(h8[1:]).max() + 1 <= 8


@pytest.mark.parametrize("d,chi", [(7, 4), (9, 8), (11, 16)])
@pytest.mark.parametrize("cutoff", [None, 0.0])
@pytest.mark.parametrize("kernel", [1, 2])
def test_both_truncation_kernels_small(mld, d, chi, cutoff, kernel):
    """Both truncation kernels (1: rank-adaptive, 2: fixed-shape with values
    below the cutoff written as zero) at the truncating points of the d/p
    grid, with the default cutoff and with cutoff 0, against the FP64
    boundary-MPS oracle computed here (small sizes)."""
    noise, _, syn = workload(d, "depolarizing", 8)
    ref = omps.decode_mps(d, noise.astype(np.float64), syn, chi, xl_column=d - 1)
    lp, _, _, hist = decode(mld, d, noise, syn, chi, cutoff, kernel)
    check_lead_and_posterior(lp, ref)
    if kernel == 1:                       # only the rank-adaptive kernel counts bonds
        assert 0 < np.flatnonzero(hist[1:]).max() + 1 <= chi
    else:
        assert hist.sum() == 0


def test_autotune_picks_a_truncation_kernel(mld):
    """mld_autotune on a truncating chi times the rank-adaptive kernel beside
    the fixed-shape kernel's CTA shapes and keeps the faster; decodes after
    it still match the oracle."""
    d, chi = 9, 8
    noise, _, syn = workload(d, "depolarizing", 8)
    ref = omps.decode_mps(d, noise.astype(np.float64), syn, chi, xl_column=d - 1)
    code = mld.Code(d)
    w = mld.mld_autotune(code, chi, mld.MLD_FP32, 4096)
    assert w in (1, 2, 4, 8)
    lp, _ = code.decode(torch.tensor(noise, device="cuda"), torch.tensor(syn.view(np.int64), device="cuda"), chi)
    torch.cuda.synchronize()
    assert code.status() == 0
    check_lead_and_posterior(lp.cpu().numpy(), ref)
    code.close()


def test_truncated_deterministic_and_counters(mld):
    """Units are taken from a device queue by whichever warp is free, but each
    unit is decoded by one warp in a fixed order: reruns give the same bits.
    The bond histogram counts d cuts per column pass, d + 1 passes per
    (syndrome, l_Z) unit (columns 0..d-2, then column d-1 once per l_X);
    its bin 0 counts site steps that ran in the global spill arena."""
    d, chi, B = 11, 16, 300
    noise, _, syn = workload(d, "depolarizing", B)
    a, _, fa, ha = decode(mld, d, noise, syn, chi, kernel=1)
    b, _, fb, hb = decode(mld, d, noise, syn, chi, kernel=1)
    np.testing.assert_array_equal(a, b)
    assert fa == fb and np.array_equal(ha, hb)
    finite = np.isfinite(a).any(axis=1)
    assert finite.all()
    assert ha[1:].sum() == 2 * B * d * (d + 1)      # bin 0 counts steps run in the spill arena
    assert np.flatnonzero(ha[1:]).max() + 1 <= chi


def test_svd_cutoff_and_kernel_argument_checks(mld):
    code = mld.Code(9)
    for bad in (-1e-3, 1.0, float("nan")):
        with pytest.raises(mld.MldError):
            code.set_svd_cutoff(bad)
    code.set_svd_cutoff(0.0)
    code.set_svd_cutoff(1e-6)
    for bad in (-1, 3):
        with pytest.raises(mld.MldError):
            code.set_truncation_kernel(bad)
    for ok in (0, 1, 2):
        code.set_truncation_kernel(ok)
    for bad in (-1, 1, 32, 100, 256):
        with pytest.raises(mld.MldError):
            code.set_truncation_workspace(bad)
    for ok in (0, 48, 64, 128):
        code.set_truncation_workspace(ok)
    code.close()
