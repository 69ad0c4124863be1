"""Adjoint of the sweep (mld_decode_grad) and its autograd wrapper.

Z is multilinear in the noise rows, so the oracle's exact derivative
(d ln Z / d p_{q,P} = Z with row q set to e_P, divided by Z) pins the GPU
gradient; central differences of the FP64 oracle pin the chain rule of the
conditional log-likelihood; rate recovery checks the gradient is usable for
maximum-likelihood noise estimation (Sec. 3.2.4, Eq. 10)."""
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


def _setup(d, B, seed):
    n = d * d
    noise = synth.lognormal_biased(n, seed=seed).astype(np.float32)
    E = synth.sample_errors(d, noise, B, seed=seed + 1)
    syn = synth.syndromes_of(d, E)
    return n, noise, E, syn


@pytest.mark.parametrize("d,chi", [(3, 8), (5, 4), (7, 8), (9, 16)])
def test_gradient_matches_oracle(mld, d, chi):
    n, noise, E, syn = _setup(d, 24, seed=d)
    code = mld.Code(d)
    rng = np.random.default_rng(d)
    up = rng.normal(size=(len(syn), 4))
    nz = torch.tensor(noise, device="cuda")
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    dn = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    lp = torch.zeros((len(syn), 4), dtype=torch.float64, device="cuda")
    mld.mld_decode_grad(code.handle, nz, sy, len(syn), chi, torch.tensor(up, device="cuda"), lp, dn)
    torch.cuda.synchronize()
    assert code.status() == 0
    reps = oracle.representatives(d, syn)
    lz, g = oracle.coset_dlogz(d, noise.astype(np.float64), reps.reshape(-1, n))
    np.testing.assert_allclose(lp.cpu().numpy(), lz.reshape(-1, 4), rtol=0, atol=1e-5)
    ref = np.einsum("bl,blqp->qp", up, g.reshape(len(syn), 4, n, 4))
    np.testing.assert_allclose(dn.cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())


@pytest.mark.parametrize("d,chi,B", [(5, 8, 1024), (7, 8, 1024), (9, 16, 128)])
def test_gradient_many_units_per_block(mld, d, chi, B):
    """Batches larger than the resident blocks, so that every block loops over
    several (syndrome, class) units and sums their gradients before its one
    flush: the summed gradient and every ln Z against the oracle; then the
    same launch without an upstream gradient (ln Z only, nothing added)."""
    n, noise, E, syn = _setup(d, B, seed=40 + d)
    code = mld.Code(d)
    rng = np.random.default_rng(d + 40)
    up = rng.normal(size=(B, 4))
    nz = torch.tensor(noise, device="cuda")
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    dn = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    lp = torch.zeros((B, 4), dtype=torch.float64, device="cuda")
    mld.mld_decode_grad(code.handle, nz, sy, B, chi, torch.tensor(up, device="cuda"), lp, dn)
    torch.cuda.synchronize()
    reps = oracle.representatives(d, syn)
    lz, g = oracle.coset_dlogz(d, noise.astype(np.float64), reps.reshape(-1, n))
    np.testing.assert_allclose(lp.cpu().numpy(), lz.reshape(-1, 4), rtol=0, atol=1e-5)
    ref = np.einsum("bl,blqp->qp", up, g.reshape(B, 4, n, 4))
    np.testing.assert_allclose(dn.cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
    dn0 = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    lp0 = torch.zeros((B, 4), dtype=torch.float64, device="cuda")
    mld.mld_decode_grad(code.handle, nz, sy, B, chi, None, lp0, dn0)
    torch.cuda.synchronize()
    assert code.status() == 0
    assert torch.count_nonzero(dn0).item() == 0
    np.testing.assert_allclose(lp0.cpu().numpy(), lz.reshape(-1, 4), rtol=0, atol=1e-5)


def test_gradient_rerun_bit_identical(mld):
    """The dense adjoint sums each block's units in order and the blocks'
    sums in block order: the same call twice gives the same bits."""
    d, chi, B = 7, 8, 1024
    n, noise, E, syn = _setup(d, B, seed=77)
    code = mld.Code(d)
    up = torch.tensor(np.random.default_rng(77).normal(size=(B, 4)), device="cuda")
    nz = torch.tensor(noise, device="cuda")
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    outs = []
    for _ in range(2):
        dn = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
        lp = torch.zeros((B, 4), dtype=torch.float64, device="cuda")
        mld.mld_decode_grad(code.handle, nz, sy, B, chi, up, lp, dn)
        torch.cuda.synchronize()
        outs.append((dn.cpu().numpy(), lp.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_gradient_d11_one_block_per_sm(mld):
    """d = 11: the dense adjoint with one block of 16 warps per SM (the
    states fill its shared memory; L_c is read back from the block's global
    slice), against the oracle's exact derivative."""
    d, chi, B = 11, 32, 3
    n, noise, E, syn = _setup(d, B, seed=11)
    code = mld.Code(d)
    up = np.random.default_rng(11).normal(size=(B, 4))
    nz = torch.tensor(noise, device="cuda")
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    dn = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    lp = torch.zeros((B, 4), dtype=torch.float64, device="cuda")
    mld.mld_decode_grad(code.handle, nz, sy, B, chi, torch.tensor(up, device="cuda"), lp, dn)
    torch.cuda.synchronize()
    assert code.status() == 0
    lz, g = oracle.coset_dlogz(d, noise.astype(np.float64), oracle.representatives(d, syn).reshape(-1, n))
    np.testing.assert_allclose(lp.cpu().numpy(), lz.reshape(-1, 4), rtol=0, atol=1e-5)
    ref = np.einsum("bl,blqp->qp", up, g.reshape(B, 4, n, 4))
    np.testing.assert_allclose(dn.cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())


def test_gradient_d13_global_states(mld):
    """d = 13, chi = 64 (untruncated): the states inside a column (128 KB
    each) live in the block's global slice and each thread takes four rests
    per pair step; ln Z and the gradient against the oracle's exact
    derivative, two syndromes of per-qubit lognormal biased noise."""
    d, chi, B = 13, 64, 2
    n, noise, E, syn = _setup(d, B, seed=13)
    code = mld.Code(d)
    up = np.random.default_rng(13).normal(size=(B, 4))
    nz = torch.tensor(noise, device="cuda")
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    dn = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    lp = torch.zeros((B, 4), dtype=torch.float64, device="cuda")
    mld.mld_decode_grad(code.handle, nz, sy, B, chi, torch.tensor(up, device="cuda"), lp, dn)
    torch.cuda.synchronize()
    assert code.status() == 0
    lz, g = oracle.coset_dlogz(d, noise.astype(np.float64), oracle.representatives(d, syn).reshape(-1, n))
    np.testing.assert_allclose(lp.cpu().numpy(), lz.reshape(-1, 4), rtol=0, atol=1e-5)
    ref = np.einsum("bl,blqp->qp", up, g.reshape(B, 4, n, 4))
    np.testing.assert_allclose(dn.cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
    # the autograd path at d = 13: d/dtheta of sum ln Z_l over the same units
    tab = nz.double().requires_grad_(True)
    mld.log_coset_probabilities(code, tab, sy, chi).sum().backward()
    ref1 = g.reshape(B, 4, n, 4).sum(axis=(0, 1))
    np.testing.assert_allclose(tab.grad.cpu().numpy(), ref1, rtol=1e-4, atol=1e-4 * np.abs(ref1).max())
    code.close()


def test_euler_identity_per_unit(mld):
    """sum_P p_{q,P} d ln Z / d p_{q,P} = 1 for every qubit (Z is linear in
    each row), for a single (syndrome, class) unit."""
    d, chi = 7, 8
    n, noise, E, syn = _setup(d, 3, seed=5)
    code = mld.Code(d)
    nz = torch.tensor(noise, device="cuda")
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    for unit in range(4 * len(syn)):
        up = torch.zeros((len(syn), 4), dtype=torch.float64, device="cuda")
        up.view(-1)[unit] = 1.0
        dn = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
        mld.mld_decode_grad(code.handle, nz, sy, len(syn), chi, up, None, dn)
        torch.cuda.synchronize()
        np.testing.assert_allclose((dn.cpu().numpy() * noise).sum(axis=1), 1.0, rtol=0, atol=2e-5)


def test_autograd_conditional_loglik_vs_central_differences(mld):
    """L = sum_b ln Pr(l_true | s_b) with p_I = 1 - p_X - p_Y - p_Z per qubit:
    autograd through the adjoint vs central differences (h = 1e-4) of the
    FP64 oracle."""
    d, chi = 5, 4
    n, noise, E, syn = _setup(d, 64, seed=11)
    cls = torch.tensor(synth.true_class(d, E).astype(np.int64), device="cuda")
    code = mld.Code(d)
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    theta = torch.tensor(noise[:, 1:].astype(np.float64), device="cuda", requires_grad=True)

    def table(t):
        return torch.cat([1.0 - t.sum(dim=1, keepdim=True), t], dim=1)

    lp = mld.log_coset_probabilities(code, table(theta), sy, chi)
    L = (lp.gather(1, cls[:, None]).squeeze(1) - torch.logsumexp(lp, dim=1)).sum()
    L.backward()
    grad = theta.grad.cpu().numpy()

    def L_oracle(th):
        tab = np.concatenate([1.0 - th.sum(axis=1, keepdims=True), th], axis=1)
        lpo, _ = oracle.decode(d, tab, syn)
        m = lpo.max(axis=1, keepdims=True)
        lse = m[:, 0] + np.log(np.exp(lpo - m).sum(axis=1))
        return float((lpo[np.arange(len(syn)), synth.true_class(d, E)] - lse).sum())

    th0 = noise[:, 1:].astype(np.float32).astype(np.float64)
    h = 1e-4
    rng = np.random.default_rng(0)
    for q, k in zip(rng.choice(n, 6, replace=False), rng.integers(0, 3, 6)):
        up = th0.copy(); up[q, k] += h
        dn = th0.copy(); dn[q, k] -= h
        fd = (L_oracle(up) - L_oracle(dn)) / (2 * h)
        assert abs(grad[q, k] - fd) <= 2e-3 * max(1.0, abs(fd)), (q, k, grad[q, k], fd)


def test_config4_full_batch_vs_central_differences(mld):
    """The differentiation workload itself: d=7, chi=32, per-qubit lognormal
    biased noise (median 0.05, sigma 0.5, eta ~ U[1, 10]; seed 3), 65,536
    syndromes (seed 4). The gradient of sum_b ln Pr(l_true | s_b) over the
    3 x 49 free parameters (p_I = 1 - p_X - p_Y - p_Z) from the adjoint,
    against central differences of the FP64 oracle over the same 65,536
    syndromes, for three sampled parameters.

    Under eta up to 10 the X and Y rates go down to ~0.004, so h = 1e-4 is a
    few percent of the parameter and the third-derivative error term of a
    central difference (h^2 / 6 times the third derivative) reaches ~1e-3
    relative. The differences at h and h/2 are therefore combined by
    Richardson extrapolation, (4 D(h/2) - D(h)) / 3, whose error is O(h^4);
    the adjoint must match it to 1e-4 relative, and D(h) itself to within
    its own truncation error |D(h) - extrapolation|."""
    d, chi, B = 7, 32, 65536
    n = d * d
    noise = synth.lognormal_biased(n, seed=3).astype(np.float32)
    E = synth.sample_errors(d, noise, B, seed=4)
    syn = synth.syndromes_of(d, E)
    true = synth.true_class(d, E)
    code = mld.Code(d)
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    cls = torch.tensor(true.astype(np.int64), device="cuda")
    theta = torch.tensor(noise[:, 1:].astype(np.float64), device="cuda", requires_grad=True)
    tab = torch.cat([1.0 - theta.sum(dim=1, keepdim=True), theta], dim=1)
    lp = mld.log_coset_probabilities(code, tab, sy, chi)
    L = (lp.gather(1, cls[:, None]).squeeze(1) - torch.logsumexp(lp, dim=1)).sum()
    L.backward()
    grad = theta.grad.cpu().numpy()

    def L_oracle(th):
        t = np.concatenate([1.0 - th.sum(axis=1, keepdims=True), th], axis=1)
        lpo, _ = oracle.decode(d, t, syn)
        m = lpo.max(axis=1, keepdims=True)
        lse = m[:, 0] + np.log(np.exp(lpo - m).sum(axis=1))
        return float((lpo[np.arange(B), true] - lse).sum())

    def central(th0, q, k, h):
        up = th0.copy(); up[q, k] += h
        dn = th0.copy(); dn[q, k] -= h
        return (L_oracle(up) - L_oracle(dn)) / (2 * h)

    th0 = noise[:, 1:].astype(np.float32).astype(np.float64)
    h = 1e-4
    rng = np.random.default_rng(7)
    for q, k in zip(rng.choice(n, 3, replace=False), rng.integers(0, 3, 3)):
        d1, d2 = central(th0, q, k, h), central(th0, q, k, h / 2)
        rich = (4 * d2 - d1) / 3
        assert abs(grad[q, k] - rich) <= 1e-4 * max(1.0, abs(rich)), (q, k, grad[q, k], rich, d1)
        assert abs(grad[q, k] - d1) <= 1.5 * abs(d1 - rich) + 1e-4 * max(1.0, abs(rich)), (q, k, grad[q, k], d1)
    code.close()


def test_rate_recovery_by_gradient_ascent(mld):
    """Maximum-likelihood estimation of per-qubit rates from syndromes alone
    (the marginal likelihood sum_b ln sum_l Z_l(s_b), Eq. 10): starting from a
    uniform guess, gradient ascent moves the total per-qubit rates toward
    the seeded ones."""
    d, chi = 5, 4
    n = d * d
    true = synth.lognormal_biased(n, seed=21)
    E = synth.sample_errors(d, true, 16384, seed=22)
    syn = synth.syndromes_of(d, E)
    code = mld.Code(d)
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    # parametrise the three Pauli rates per qubit through logits
    z0 = np.log(np.full((n, 3), 0.05 / 3) / (1 - 0.05))
    zt = torch.tensor(z0, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([zt], lr=0.08)

    def table(z):
        e = torch.exp(z)
        den = 1.0 + e.sum(dim=1, keepdim=True)
        return torch.cat([1.0 / den, e / den], dim=1)

    p_true = true[:, 1:].sum(axis=1)
    err0 = np.abs(table(zt).detach().cpu().numpy()[:, 1:].sum(axis=1) - p_true).mean()
    for _ in range(300):
        opt.zero_grad()
        lp = mld.log_coset_probabilities(code, table(zt), sy, chi)
        loss = -torch.logsumexp(lp, dim=1).mean()
        loss.backward()
        opt.step()
    p_fit = table(zt).detach().cpu().numpy()[:, 1:].sum(axis=1)
    err1 = np.abs(p_fit - p_true).mean()
    assert err1 < 0.5 * err0, (err0, err1)
    assert np.corrcoef(p_fit, p_true)[0, 1] > 0.5


def test_estimate_noise_d9_unlabelled(mld):
    """Large-scale estimation from unlabelled syndromes (Sec. 3.2.4, Eq. 10)
    at d = 9: full-batch Adam on -mean ln sum_l Z_l(s) over 65,536 syndromes
    drawn from per-qubit biased rates recovers them (mean total-rate error
    under a third of the uniform start's, correlation above 0.9), and the
    loss settles (the last steps change it by under 1e-4)."""
    d, chi, B = 9, 32, 65536
    n = d * d
    true = synth.lognormal_biased(n, seed=21)
    E = synth.sample_errors(d, true, B, seed=22)
    code = mld.Code(d)
    sy = torch.tensor(synth.syndromes_of(d, E).view(np.int64), device="cuda")
    tab0 = mld.noise_table_from_logits(torch.full((n, 3), np.log(0.05 / 3 / 0.95), dtype=torch.float64))
    tab, _, losses = mld.estimate_noise(code, sy, chi, steps=120, lr=0.08)
    p_true = true[:, 1:].sum(axis=1)
    err0 = np.abs(tab0.numpy()[:, 1:].sum(axis=1) - p_true).mean()
    fit = tab.cpu().numpy()[:, 1:].sum(axis=1)
    err1 = np.abs(fit - p_true).mean()
    assert err1 < err0 / 3, (err0, err1)
    assert np.corrcoef(fit, p_true)[0, 1] > 0.9
    assert losses[-1] < losses[0] and abs(losses[-1] - losses[-10]) < 1e-4, losses[-10:]
