"""The allocation-free entry point (mld_decode_noalloc) agrees with mld_decode.

Callers that cannot allocate device memory (a real-time loop that must not
stall on cudaMalloc, a process whose memory another allocator has reserved)
use mld_decode_noalloc, which keeps its scratch in a fixed device array.
This file is collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_noalloc_matches_decode_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_17230_gb300 as mld
    for d, chi in [(9, 32), (7, 8)]:
        n = d * d
        code = mld.Code(d)
        noise = synth.depolarizing(n, 0.12).astype(np.float32)
        E = synth.sample_errors(d, noise, 777, seed=d)
        syn = synth.syndromes_of(d, E)
        nz = torch.tensor(noise, device="cuda")
        sy = torch.tensor(syn.view(np.int64), device="cuda")
        ref, ref_am = code.decode(nz, sy, chi)
        torch.cuda.synchronize()
        for _ in range(2):                      # two calls in a row share the array
            lp = torch.full((len(syn), 4), float("nan"), dtype=torch.float64, device="cuda")
            am = torch.full((len(syn),), 255, dtype=torch.uint8, device="cuda")
            mld.mld_decode_noalloc(code.handle, nz, mld.MLD_NOISE_TABLE, sy, len(syn), chi, mld.MLD_FP32,
                                   lp, am, check_status=True)
            torch.cuda.synchronize()
            np.testing.assert_allclose(lp.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=TOL)
            np.testing.assert_array_equal(am.cpu().numpy(), ref_am.cpu().numpy())
        code.close()


def test_noalloc_rejects_what_it_does_not_cover():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_17230_gb300 as mld
    d = 9
    code = mld.Code(d)
    noise = torch.tensor(synth.depolarizing(d * d, 0.1).astype(np.float32), device="cuda")
    sy = torch.zeros((4, code.words), dtype=torch.int64, device="cuda")
    lp = torch.empty((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(mld.MldError) as e:               # a truncating chi needs the SVD path
        mld.mld_decode_noalloc(code.handle, noise, mld.MLD_NOISE_TABLE, sy, 4, 8, mld.MLD_FP32, lp)
    assert e.value.status == 2
    code.close()


def test_noalloc_leaves_free_device_memory_unchanged():
    """The property the entry point exists for: after one warm-up call (which
    looks up the scratch array's address), further calls with both noise
    modes, with and without the argmax, for two codes in turn, allocate no
    device memory."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_17230_gb300 as mld
    bufs = []
    for d, chi in [(5, 4), (9, 32)]:
        n = d * d
        code = mld.Code(d)
        table = synth.depolarizing(n, 0.1).astype(np.float32)
        syn = synth.syndromes_of(d, synth.sample_errors(d, table, 512, seed=d))
        bufs.append((code, chi, torch.tensor(table, device="cuda"), torch.full((512,), 0.1, device="cuda"),
                     torch.tensor(syn.view(np.int64), device="cuda"),
                     torch.empty((512, 4), dtype=torch.float64, device="cuda"),
                     torch.empty((512,), dtype=torch.uint8, device="cuda")))
    code, chi, table, depol, sy, lp, am = bufs[0]
    mld.mld_decode_noalloc(code.handle, table, mld.MLD_NOISE_TABLE, sy, 512, chi, mld.MLD_FP32, lp, am)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for code, chi, table, depol, sy, lp, am in bufs:
            mld.mld_decode_noalloc(code.handle, table, mld.MLD_NOISE_TABLE, sy, 512, chi, mld.MLD_FP32, lp, am)
            mld.mld_decode_noalloc(code.handle, depol, mld.MLD_NOISE_DEPOL, sy, 512, chi, mld.MLD_FP32, lp, None,
                                   check_status=False)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for b in bufs:
        b[0].close()
