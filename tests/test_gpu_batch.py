"""Mixed batches: jobs of different d, per-syndrome noise and chi decoded by
one CUDA-graph launch (the batching row of the path), checked against the
oracle and against per-job mld_decode calls; and the CTA-shape autotuner."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHI_BY_D = {3: 16, 5: 16, 7: 16, 9: 32, 11: 32, 13: 64}


@pytest.fixture(scope="module")
def mld():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_17230_gb300 as m
    m.load()
    return m


def test_mixed_batch_graph(mld):
    rng_seed = 3
    items, host = [], []
    for d, chi in CHI_BY_D.items():
        B = 64 if d == 13 else 400
        p = synth.per_syndrome_depolarizing(B, seed=rng_seed + d, lo=0.02, hi=0.18)
        E = synth.sample_errors(d, p, B, seed=rng_seed + d)
        syn = synth.syndromes_of(d, E)
        code = mld.Code(d)
        nz = torch.tensor(p.astype(np.float32), device="cuda")
        sy = torch.tensor(syn.view(np.int64), device="cuda")
        lp = torch.full((B, 4), float("nan"), dtype=torch.float64, device="cuda")
        am = torch.zeros((B,), dtype=torch.uint8, device="cuda")
        items.append((code, nz, sy, chi, mld.MLD_MIXED_TF32, lp, am))
        host.append((d, p, syn))
    jobs = mld.make_jobs(items)
    g = mld.Graph(jobs)
    for it in items:
        it[5].fill_(float("nan"))
    g.launch()
    torch.cuda.synchronize()
    for (code, nz, sy, chi, prec, lp, am), (d, p, syn) in zip(items, host):
        assert code.status() == 0
        got = lp.cpu().numpy()
        ref, _ = oracle.decode(d, p.astype(np.float32).astype(np.float64), syn)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5)
        solo, _ = code.decode(nz, sy, chi, prec)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got, solo.cpu().numpy())
    g.close()


def test_autotune_untruncated_d13(mld):
    """d = 13, chi = 64 (untruncated): mld_autotune times the dense-state
    kernel and the boundary-MPS kernel at 2, 4, 8 and 16 resident warps per SM
    (its per-warp state is in the global workspace) and keeps the fastest
    (0 reported for the dense one); decodes after tuning match the oracle."""
    d, n, chi = 13, 169, 64
    code = mld.Code(d)
    noise = synth.depolarizing(n, 0.1).astype(np.float32)
    syn = synth.syndromes_of(d, synth.sample_errors(d, noise, 200, seed=2))
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    w = mld.mld_autotune(code, chi, mld.MLD_FP32, 2432)
    assert w in (0, 2, 4, 8, 16)
    lp, _ = code.decode(torch.tensor(noise, device="cuda"), sy, chi)
    torch.cuda.synchronize()
    assert code.status() == 0
    ref, _ = oracle.decode(d, noise, syn)
    np.testing.assert_allclose(lp.cpu().numpy(), ref, rtol=0, atol=1e-5)
    code.close()


def test_autotune_choice_is_used_and_correct(mld):
    d, n, chi = 9, 81, 32
    code = mld.Code(d)
    w = mld.mld_autotune(code, chi, mld.MLD_FP32, 4096)
    assert w in (1, 2, 4, 8)
    noise = synth.depolarizing(n, 0.1).astype(np.float32)
    syn = synth.syndromes_of(d, synth.sample_errors(d, noise, 300, seed=1))
    lp, _ = code.decode(torch.tensor(noise, device="cuda"), torch.tensor(syn.view(np.int64), device="cuda"), chi)
    torch.cuda.synchronize()
    ref, _ = oracle.decode(d, noise, syn)
    np.testing.assert_allclose(lp.cpu().numpy(), ref, rtol=0, atol=1e-5)
