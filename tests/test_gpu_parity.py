"""Parity of the CUDA decoder (through the C ABI) with the FP64 oracle.

Tolerances: |ln Z_gpu - ln Z_oracle| <= 1e-5 for the FP32 path at exact bond
dimension (chi >= 2^floor(d/2)); argmax decisions must agree except where the
oracle's two best cosets are within 1e-4 in log (a tie at FP32 resolution).
"""
import numpy as np
import pytest

import oracle
import oracle.mps as omps
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
TIE = 1e-4


@pytest.fixture(scope="module")
def mld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_17230_gb300 as m
    m.load()
    return m


_codes = {}


def code(mld, d):
    if d not in _codes:
        _codes[d] = mld.Code(d)
    return _codes[d]


def gpu_decode(mld, d, noise, syn, chi, precision=0):
    C = code(mld, d)
    nz = torch.tensor(np.asarray(noise, np.float32), device="cuda")
    sy = torch.tensor(np.asarray(syn).view(np.int64), device="cuda")
    lp, am = C.decode(nz, sy, chi, precision)
    torch.cuda.synchronize()
    assert C.status() == 0
    return lp.cpu().numpy(), am.cpu().numpy()


def check_argmax(am, ref):
    top = np.sort(ref, axis=1)
    clear = top[:, -1] - top[:, -2] > TIE
    np.testing.assert_array_equal(am[clear], np.argmax(ref, axis=1)[clear])
    # at near-ties the pick must still be one of the near-best classes
    picked = ref[np.arange(len(am)), am]
    assert np.all(picked >= top[:, -1] - TIE)


def test_d3_all_syndromes_vs_bruteforce(mld):
    d, n = 3, 9
    m = d * d - 1
    bits = ((np.arange(1 << m)[:, None] >> np.arange(m)[None, :]) & 1).astype(np.uint8)
    syn = synth.pack_bits(bits)
    noise = synth.depolarizing(n, 0.10)
    ref = np.log(oracle.bruteforce_table(d, noise))
    lp, am = gpu_decode(mld, d, noise.astype(np.float32), syn, 8)
    np.testing.assert_allclose(lp, ref, rtol=0, atol=TOL)
    check_argmax(am, ref)


def test_config_d3_1024_seed0(mld):
    d, n = 3, 9
    noise = synth.depolarizing(n, 0.10).astype(np.float32)
    E = synth.sample_errors(d, noise, 1024, seed=0)
    syn = synth.syndromes_of(d, E)
    ref, _ = oracle.decode(d, noise, syn)
    lp, am = gpu_decode(mld, d, noise, syn, 8)
    np.testing.assert_allclose(lp, ref, rtol=0, atol=TOL)
    check_argmax(am, ref)


@pytest.mark.parametrize("d", [5, 7, 9])
@pytest.mark.parametrize("p", [0.05, 0.10, 0.15, 0.19])
def test_exact_chi_vs_dense_oracle(mld, d, p):
    n = d * d
    chi = {5: 4, 7: 8, 9: 32}[d]
    noise = synth.depolarizing(n, p).astype(np.float32)
    B = 300 if d < 9 else 200           # several CTAs and a ragged tail
    E = synth.sample_errors(d, noise, B, seed=synth.config_seed(1, d, p))
    syn = synth.syndromes_of(d, E)
    ref, _ = oracle.decode(d, noise, syn)
    lp, am = gpu_decode(mld, d, noise, syn, chi)
    np.testing.assert_allclose(lp, ref, rtol=0, atol=TOL)
    check_argmax(am, ref)


@pytest.mark.parametrize("d,chi", [(5, 16), (7, 32), (9, 16), (11, 32)])
def test_more_chi_values_exact(mld, d, chi):
    n = d * d
    noise = synth.depolarizing(n, 0.12).astype(np.float32)
    E = synth.sample_errors(d, noise, 64, seed=7)
    syn = synth.syndromes_of(d, E)
    ref, _ = oracle.decode(d, noise, syn)
    lp, _ = gpu_decode(mld, d, noise, syn, chi)
    np.testing.assert_allclose(lp, ref, rtol=0, atol=TOL)


@pytest.mark.parametrize("d,chi", [(9, 8), (9, 4), (7, 4)])
def test_truncated_chi_vs_fp64_mps(mld, d, chi):
    """Below the exact bond the value is the boundary-MPS approximation: the
    FP32 kernel must match the FP64 boundary-MPS oracle with the same rule.
    Truncating columns are QR-canonicalised, and in an orthogonal gauge FP32
    rounding (relative to the state's norm) reaches ln Z_l as
    ~eps * Z_max / Z_l; the bar is therefore set on the leading coset's ln Z
    and on the posterior Pr(l|s) = Z_l / sum Z."""
    n = d * d
    noise = synth.depolarizing(n, 0.12).astype(np.float32)
    E = synth.sample_errors(d, noise, 6, seed=11)
    syn = synth.syndromes_of(d, E)
    ref = omps.decode_mps(d, noise.astype(np.float64), syn, chi, xl_column=d - 1)
    lp, _ = gpu_decode(mld, d, noise, syn, chi)
    best = np.argmax(ref, axis=1)
    np.testing.assert_allclose(lp[np.arange(len(ref)), best], ref[np.arange(len(ref)), best], rtol=0, atol=1e-4)
    post = lambda x: np.exp(x - x.max(axis=1, keepdims=True)) / np.exp(x - x.max(axis=1, keepdims=True)).sum(1, keepdims=True)
    np.testing.assert_allclose(post(lp), post(ref), rtol=0, atol=1e-4)


@pytest.mark.parametrize("d,chi,B", [(11, 16, 8), (13, 32, 2)])
def test_truncated_strongly_biased_vs_fp64_mps(mld, d, chi, B):
    """Strongly biased noise (eta = 100, p = 0.12): the blocks of a truncating
    column then hold columns many orders of magnitude below their largest
    entries, and a Householder reflector that squares unscaled entries loses
    them to underflow (this case was off by 2e-3 in ln Z before the scaled
    norms). Same bar as the depolarizing case."""
    n = d * d
    noise = synth.biased(n, 0.12, 100.0).astype(np.float32)
    E = synth.sample_errors(d, noise, B, seed=synth.config_seed(5, d, 0.12))
    syn = synth.syndromes_of(d, E)
    ref = omps.decode_mps(d, noise.astype(np.float64), syn, chi, xl_column=d - 1)
    lp, _ = gpu_decode(mld, d, noise, syn, chi)
    best = np.argmax(ref, axis=1)
    np.testing.assert_allclose(lp[np.arange(B), best], ref[np.arange(B), best], rtol=0, atol=1e-4)
    post = lambda x: np.exp(x - x.max(axis=1, keepdims=True)) / np.exp(x - x.max(axis=1, keepdims=True)).sum(1, keepdims=True)
    np.testing.assert_allclose(post(lp), post(ref), rtol=0, atol=1e-4)


def test_truncated_depolarizing_d11_vs_fp64_mps(mld):
    """Depolarizing p = 0.12 at d=11, chi=16 on 16 syndromes: small but real
    overlaps between a large and a small column must be rotated before the
    truncation (a fixed norm floor in the Jacobi sweep left them and cost
    1.4e-4 in ln Z of the leading coset)."""
    d, chi, B = 11, 16, 16
    n = d * d
    noise = synth.depolarizing(n, 0.12).astype(np.float32)
    E = synth.sample_errors(d, noise, B, seed=synth.config_seed(5, d, 0.12))
    syn = synth.syndromes_of(d, E)
    ref = omps.decode_mps(d, noise.astype(np.float64), syn, chi, xl_column=d - 1)
    lp, _ = gpu_decode(mld, d, noise, syn, chi)
    best = np.argmax(ref, axis=1)
    np.testing.assert_allclose(lp[np.arange(B), best], ref[np.arange(B), best], rtol=0, atol=1e-4)


@pytest.mark.parametrize("d,chi", [(9, 32), (13, 64)])
@pytest.mark.parametrize("prec", [0, 2])
def test_exact_strongly_biased(mld, d, chi, prec):
    """Untruncated sweep under eta = 100: entries of a block span many orders
    of magnitude, and the non-negative gauge keeps every coset to FP32
    relative accuracy."""
    n = d * d
    noise = synth.biased(n, 0.12, 100.0).astype(np.float32)
    E = synth.sample_errors(d, noise, 32, seed=synth.config_seed(9, d, 0.12))
    syn = synth.syndromes_of(d, E)
    ref, _ = oracle.decode(d, noise, syn)
    lp, am = gpu_decode(mld, d, noise, syn, chi, precision=prec)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(lp), fin)
    np.testing.assert_allclose(lp[fin], ref[fin], rtol=0, atol=TOL)
    check_argmax(am, ref)


def test_per_syndrome_depolarizing(mld):
    d = 7
    B = 257
    p = synth.per_syndrome_depolarizing(B, seed=3, lo=0.02, hi=0.18).astype(np.float32)
    E = synth.sample_errors(d, p.astype(np.float64), B, seed=3)
    syn = synth.syndromes_of(d, E)
    ref, _ = oracle.decode(d, p.astype(np.float64), syn)
    lp, am = gpu_decode(mld, d, p, syn, 8)
    np.testing.assert_allclose(lp, ref, rtol=0, atol=TOL)
    check_argmax(am, ref)


def test_nonuniform_biased_noise_table(mld):
    d, n = 7, 49
    noise = synth.lognormal_biased(n, seed=4).astype(np.float32)
    E = synth.sample_errors(d, noise, 128, seed=5)
    syn = synth.syndromes_of(d, E)
    ref, _ = oracle.decode(d, noise.astype(np.float64), syn)
    lp, am = gpu_decode(mld, d, noise, syn, 32)
    np.testing.assert_allclose(lp, ref, rtol=0, atol=TOL)
    check_argmax(am, ref)


def test_edge_cases(mld):
    d, n = 5, 25
    noise = synth.depolarizing(n, 0.1).astype(np.float32)
    C = code(mld, d)
    # B = 0 is a no-op
    nz = torch.tensor(noise, device="cuda")
    sy = torch.zeros((0, C.words), dtype=torch.int64, device="cuda")
    lp, am = C.decode(nz, sy, 4)
    assert lp.shape == (0, 4)
    # the trivial syndrome and a single syndrome
    syn = np.zeros((1, C.words), np.uint64)
    ref, _ = oracle.decode(d, noise, syn)
    lp, am = gpu_decode(mld, d, noise, syn, 4)
    np.testing.assert_allclose(lp, ref, rtol=0, atol=TOL)
    # zero-probability Paulis: p_Y = p_Z = 0 gives -inf cosets
    bf = np.zeros((n, 4), np.float32)
    bf[:, 0], bf[:, 1] = 0.9, 0.1
    E = synth.sample_errors(d, bf, 16, seed=1)
    syn = synth.syndromes_of(d, E)
    ref, _ = oracle.decode(d, bf, syn)
    lp, am = gpu_decode(mld, d, bf, syn, 4)
    assert np.array_equal(np.isneginf(lp), np.isneginf(ref))
    fin = np.isfinite(ref)
    np.testing.assert_allclose(lp[fin], ref[fin], rtol=0, atol=TOL)
    check_argmax(am, np.where(np.isfinite(ref), ref, -1e300))


def test_host_entry_point_matches_device(mld):
    d, n = 9, 81
    noise = synth.depolarizing(n, 0.15).astype(np.float32)
    E = synth.sample_errors(d, noise, 100, seed=9)
    syn = synth.syndromes_of(d, E)
    lp_d, am_d = gpu_decode(mld, d, noise, syn, 32)
    lp_h, am_h = code(mld, d).decode_host(noise, syn, 32)
    np.testing.assert_array_equal(lp_d, lp_h)
    np.testing.assert_array_equal(am_d, am_h)


def test_deterministic_rerun(mld):
    d, n = 9, 81
    noise = synth.depolarizing(n, 0.1).astype(np.float32)
    syn = synth.syndromes_of(d, synth.sample_errors(d, noise, 512, seed=2))
    a, _ = gpu_decode(mld, d, noise, syn, 32)
    b, _ = gpu_decode(mld, d, noise, syn, 32)
    np.testing.assert_array_equal(a, b)


def test_full_size_bench_config_sampled(mld):
    """The bench workload (d=9, chi=32, p=0.10, 65536 syndromes) in the same
    launch configuration; a seeded sample of 256 rows is checked against the
    oracle and every row against invariants (finite, argmax consistent)."""
    d, n, B = 9, 81, 65536
    noise = synth.depolarizing(n, 0.10).astype(np.float32)
    E = synth.sample_errors(d, noise, B, seed=synth.config_seed(1, d, 0.10))
    syn = synth.syndromes_of(d, E)
    lp, am = gpu_decode(mld, d, noise, syn, 32)
    assert np.all(np.isfinite(lp))
    assert np.array_equal(am, np.argmax(lp, axis=1))
    idx = np.random.default_rng(0).choice(B, 256, replace=False)
    ref, _ = oracle.decode(d, noise, syn[idx])
    np.testing.assert_allclose(lp[idx], ref, rtol=0, atol=TOL)
    check_argmax(am[idx], ref)


@pytest.mark.parametrize("d,chi", [(5, 4), (7, 8), (9, 32), (11, 32)])
def test_mixed_tf32_vs_oracle_and_fp32(mld, d, chi):
    """Mixed precision on the boundary-MPS kernel (split-TF32 tensor-core
    products, FP32 accumulate): within 1e-5 of the oracle and of the FP32
    path on every coset. (At d = 11 the default untruncated kernel is the
    dense-state one; the boundary-MPS kernel is selected here.)"""
    n = d * d
    noise = synth.depolarizing(n, 0.12).astype(np.float32)
    E = synth.sample_errors(d, noise, 200, seed=31)
    syn = synth.syndromes_of(d, E)
    ref, _ = oracle.decode(d, noise, syn)
    C = mld.Code(d)
    C.set_exact_kernel(1)
    nz = torch.tensor(noise, device="cuda")
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    lp32, _ = C.decode(nz, sy, chi)
    lpm, am = C.decode(nz, sy, chi, mld.MLD_MIXED_TF32)
    torch.cuda.synchronize()
    assert C.status() == 0
    lp32, lpm, am = lp32.cpu().numpy(), lpm.cpu().numpy(), am.cpu().numpy()
    np.testing.assert_allclose(lpm, ref, rtol=0, atol=TOL)
    np.testing.assert_allclose(lpm, lp32, rtol=0, atol=TOL)
    check_argmax(am, ref)
    if d not in (9, 11):                 # tensor-core products only where they pay: FP32 kernel
        assert np.array_equal(lpm, lp32)
    C.close()


def test_mixed_unsupported_cases(mld):
    d, n = 9, 81
    C = code(mld, d)
    nz = torch.tensor(synth.depolarizing(n, 0.1).astype(np.float32), device="cuda")
    sy = torch.zeros((4, C.words), dtype=torch.int64, device="cuda")
    for chi, prec in [(32, mld.MLD_MIXED_BF16), (8, mld.MLD_MIXED_TF32)]:
        with pytest.raises(mld.MldError) as e:
            C.decode(nz, sy, chi, prec)
        assert e.value.status == 2


@pytest.mark.parametrize("prec", [0, 2])
def test_d13_exact_global_workspace(mld, prec):
    """d=13 at chi=64 (untruncated): the state no longer fits a block's shared
    memory, so the persistent global-workspace mode runs; exact parity."""
    d, n = 13, 169
    noise = synth.depolarizing(n, 0.10).astype(np.float32)
    E = synth.sample_errors(d, noise, 48, seed=13)
    syn = synth.syndromes_of(d, E)
    ref, _ = oracle.decode(d, noise, syn)
    lp, am = gpu_decode(mld, d, noise, syn, 64, precision=prec)
    np.testing.assert_allclose(lp, ref, rtol=0, atol=TOL)
    check_argmax(am, ref)


@pytest.mark.parametrize("d", [9, 11, 13])
@pytest.mark.parametrize("mode", ["table", "depolarizing"])
def test_exact_kernels_dense_and_mps_vs_oracle(mld, d, mode):
    """Untruncated chi at d = 9, 11 and 13 by both kernels: the boundary-MPS
    kernel (sites at the exact cut ranks) and the dense-state kernel (the
    2^(d+2)-entry column state in shared memory, factors applied in place),
    each against the FP64 oracle, with a per-qubit table and with one
    depolarizing strength per syndrome; a ragged batch of 37 syndromes."""
    n, chi, B = d * d, 2 ** (d // 2), 37
    rng = np.random.default_rng(d)
    if mode == "table":
        noise = synth.lognormal_biased(n, seed=d).astype(np.float32)
        E = synth.sample_errors(d, noise, B, seed=d + 1)
        ref, _ = oracle.decode(d, noise.astype(np.float64), synth.syndromes_of(d, E))
        dev_noise = torch.tensor(noise, device="cuda")
        nmode = mld.MLD_NOISE_TABLE
    else:
        p = rng.uniform(0.02, 0.18, size=B).astype(np.float32)
        E = np.stack([synth.sample_errors(d, synth.depolarizing(n, float(p[b])), 1, seed=100 * d + b)[0]
                      for b in range(B)])
        # the oracle gets the rows the kernels form in FP32: (1 - p, p/3, p/3, p/3)
        rows = [np.array([np.float32(1) - p[b]] + [p[b] * np.float32(1.0 / 3.0)] * 3, np.float32)
                for b in range(B)]
        ref = np.concatenate([oracle.decode(d, np.tile(rows[b].astype(np.float64), (n, 1)),
                                            synth.syndromes_of(d, E[b:b + 1]))[0] for b in range(B)])
        dev_noise = torch.tensor(p, device="cuda")
        nmode = mld.MLD_NOISE_DEPOL
    syn = synth.syndromes_of(d, E)
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    outs = {}
    for which in (1, 2):
        C = mld.Code(d)
        C.set_exact_kernel(which)
        lp = torch.empty((B, 4), dtype=torch.float64, device="cuda")
        am = torch.empty((B,), dtype=torch.uint8, device="cuda")
        mld.mld_decode(C.handle, dev_noise, nmode, sy, B, chi, mld.MLD_FP32, lp, am)
        torch.cuda.synchronize()
        assert C.status() == 0
        outs[which] = lp.cpu().numpy()
        np.testing.assert_allclose(outs[which], ref, rtol=0, atol=TOL)
        check_argmax(am.cpu().numpy(), ref)
        C.close()


def test_exact_kernel_selector_arguments(mld):
    C = mld.Code(7)
    for bad in (-1, 3):
        with pytest.raises(mld.MldError):
            C.set_exact_kernel(bad)
    with pytest.raises(mld.MldError) as e:
        C.set_exact_kernel(2)              # no dense-state kernel at d = 7
    assert e.value.status == 2
    C.set_exact_kernel(1)
    C.set_exact_kernel(0)
    C.close()


def test_d17_truncated_close_to_exact(mld):
    """d=17 at chi=16 (truncating, global workspace): the boundary-MPS value
    is an approximation of the exact contraction (Sec. 3.2.1: small chi
    suffices well below threshold). Loose sanity bound: the leading coset is
    within 0.05 of exact at p=0.05 and the decision agrees."""
    d, n, chi = 17, 289, 16
    noise = synth.depolarizing(n, 0.05).astype(np.float32)
    E = synth.sample_errors(d, noise, 4, seed=19)
    syn = synth.syndromes_of(d, E)
    ref, _ = oracle.decode(d, noise, syn)
    lp, am = gpu_decode(mld, d, noise, syn, chi)
    best = np.argmax(ref, axis=1)
    assert np.all(np.abs(lp[np.arange(4), best] - ref[np.arange(4), best]) < 5e-2)
    assert np.array_equal(am, best)


def test_invalid_noise_reported_through_status(mld):
    """A noise row that is not a probability distribution (sum off by more
    than 1e-6, a negative or non-finite entry) or a depolarizing strength
    outside [0, 1] sets MLD_ERR_INVALID_ARG in the device status word, which
    mld_decode_status returns and clears; valid inputs leave it at MLD_OK.
    Also through the adjoint and the allocation-free entry point."""
    d, n = 5, 25
    C = mld.Code(d)
    good = synth.depolarizing(n, 0.1).astype(np.float32)
    syn = synth.syndromes_of(d, synth.sample_errors(d, good, 8, seed=3))
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    INVALID = 1
    bads = []
    t = good.copy(); t[3, 0] += 0.1; bads.append(t)                  # row sums to 1.1
    t = good.copy(); t[0, 1] = -0.01; t[0, 0] += 0.01; bads.append(t)  # negative entry, sum 1
    t = good.copy(); t[7, 2] = np.nan; bads.append(t)
    for t in bads:
        C.decode(torch.tensor(t, device="cuda"), sy, 8)
        torch.cuda.synchronize()
        assert C.status() == INVALID
        assert C.status() == 0                                         # read clears it
    C.decode(torch.tensor(good, device="cuda"), sy, 8)
    torch.cuda.synchronize()
    assert C.status() == 0
    p = np.full(8, 0.1, np.float32)
    C.decode(torch.tensor(p, device="cuda"), sy, 8)
    torch.cuda.synchronize()
    assert C.status() == 0
    p[5] = 1.5
    C.decode(torch.tensor(p, device="cuda"), sy, 8)
    torch.cuda.synchronize()
    assert C.status() == INVALID
    dn = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    up = torch.ones((8, 4), dtype=torch.float64, device="cuda")
    mld.mld_decode_grad(C.handle, torch.tensor(bads[0], device="cuda"), sy, 8, 8, up, None, dn)
    torch.cuda.synchronize()
    assert C.status() == INVALID
    lp = torch.empty((8, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(mld.MldError):
        mld.mld_decode_noalloc(C.handle, torch.tensor(bads[0], device="cuda"), mld.MLD_NOISE_TABLE, sy, 8, 8,
                               mld.MLD_FP32, lp)
    mld.mld_decode_noalloc(C.handle, torch.tensor(good, device="cuda"), mld.MLD_NOISE_TABLE, sy, 8, 8,
                           mld.MLD_FP32, lp)
