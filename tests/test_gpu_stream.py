"""Chunked decoding to files with resume (paper_2605_17230_gb300.stream): an
interrupted job continues from its progress record and ends with the same
bits as one decode of the whole batch; another configuration is refused."""
import json

import numpy as np
import pytest

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


class Stop(Exception):
    pass


@pytest.mark.parametrize("mode", ["table", "depolarizing"])
def test_interrupted_job_resumes_to_the_same_bits(mld, tmp_path, mode):
    from paper_2605_17230_gb300 import stream
    d, chi, B, chunk = 9, 32, 5 * 1024 + 77, 1024
    n = d * d
    code = mld.Code(d)
    if mode == "table":
        table = synth.depolarizing(n, 0.1).astype(np.float32)
        syn = synth.syndromes_of(d, synth.sample_errors(d, table, B, seed=3))
        noise = torch.tensor(table, device="cuda")
        nmode = mld.MLD_NOISE_TABLE
    else:
        p = np.random.default_rng(4).uniform(0.02, 0.18, size=B).astype(np.float32)
        syn = synth.syndromes_of(d, synth.sample_errors(d, synth.depolarizing(n, 0.1), B, seed=5))
        noise = p
        nmode = mld.MLD_NOISE_DEPOL
    # reference: one decode of the whole batch
    ref_lp = torch.empty((B, 4), dtype=torch.float64, device="cuda")
    ref_am = torch.empty((B,), dtype=torch.uint8, device="cuda")
    dn = noise if nmode == mld.MLD_NOISE_TABLE else torch.tensor(p, device="cuda")
    mld.mld_decode(code.handle, dn, nmode, torch.tensor(syn.view(np.int64), device="cuda"), B, chi,
                   mld.MLD_FP32, ref_lp, ref_am)
    torch.cuda.synchronize()
    prefix = str(tmp_path / "job")
    seen = []

    def stop_after_two(start, count):
        seen.append((start, count))
        if len(seen) == 2:
            raise Stop()

    with pytest.raises(Stop):
        stream.decode_to_files(code, noise, syn, chi, prefix, chunk=chunk, noise_mode=nmode,
                               on_chunk=stop_after_two)
    with open(prefix + ".progress.json") as f:
        assert json.load(f)["done"] == 2 * chunk
    rest = []
    lp, am = stream.decode_to_files(code, noise, syn, chi, prefix, chunk=chunk, noise_mode=nmode,
                                    on_chunk=lambda s, c: rest.append((s, c)))
    assert rest[0][0] == 2 * chunk and rest[-1] == (5 * chunk, 77)
    np.testing.assert_array_equal(np.asarray(lp), ref_lp.cpu().numpy())
    np.testing.assert_array_equal(np.asarray(am), ref_am.cpu().numpy())
    # a finished job returns at once; another chi is refused
    again = []
    stream.decode_to_files(code, noise, syn, chi, prefix, chunk=chunk, noise_mode=nmode,
                           on_chunk=lambda s, c: again.append(s))
    assert again == []
    with pytest.raises(ValueError):
        stream.decode_to_files(code, noise, syn, 16, prefix, chunk=chunk, noise_mode=nmode)
    # resume=False starts over and gives the same bits
    lp2, _ = stream.decode_to_files(code, noise, syn, chi, prefix, chunk=chunk, noise_mode=nmode, resume=False)
    np.testing.assert_array_equal(np.asarray(lp2), ref_lp.cpu().numpy())
    code.close()


def test_truncated_job_resumes_to_the_same_bits(mld, tmp_path):
    """The same at a truncating chi (d=11, chi=16, rank-adaptive sweep): units
    are taken from a device queue in any order, but each is decoded by one
    warp in a fixed order, so chunks give the bits of one whole decode."""
    from paper_2605_17230_gb300 import stream
    d, chi, B, chunk = 11, 16, 1000, 384
    table = synth.depolarizing(d * d, 0.12).astype(np.float32)
    syn = synth.syndromes_of(d, synth.sample_errors(d, table, B, seed=9))
    code = mld.Code(d)
    code.set_truncation_kernel(1)
    noise = torch.tensor(table, device="cuda")
    ref, _ = code.decode(noise, torch.tensor(syn.view(np.int64), device="cuda"), chi)
    torch.cuda.synchronize()
    prefix = str(tmp_path / "trunc")
    with pytest.raises(Stop):
        def stop(start, count):
            raise Stop()
        stream.decode_to_files(code, noise, syn, chi, prefix, chunk=chunk, on_chunk=stop)
    lp, _ = stream.decode_to_files(code, noise, syn, chi, prefix, chunk=chunk)
    np.testing.assert_array_equal(np.asarray(lp), ref.cpu().numpy())
    code.close()


@pytest.mark.parametrize("bitflip", [False, True])
def test_kac_ward_job_resumes_to_the_same_bits(mld, tmp_path, bitflip):
    """decode_xz_to_files: a Kac-Ward job (d = 17, the block kernel)
    interrupted after one chunk and resumed ends with the bits of one
    decode_xz of the whole batch; a record made with other rates is refused."""
    from paper_2605_17230_gb300 import stream
    d, B, chunk = 17, 700, 256
    n = d * d
    px = torch.full((n,), 0.09, device="cuda")
    pz = None if bitflip else torch.full((n,), 0.07, device="cuda")
    pzn = np.zeros(n) if bitflip else np.full(n, 0.07)
    table = synth.independent_xz(np.full(n, 0.09), pzn)
    syn = synth.syndromes_of(d, synth.sample_errors(d, table, B, seed=17))
    code = mld.Code(d)
    ref, ram = code.decode_xz(px, pz, torch.tensor(syn.view(np.int64), device="cuda"))
    torch.cuda.synchronize()
    prefix = str(tmp_path / "kw")

    def stop(start, count):
        raise Stop()

    with pytest.raises(Stop):
        stream.decode_xz_to_files(code, px, pz, syn, prefix, chunk=chunk, on_chunk=stop)
    with open(prefix + ".progress.json") as f:
        assert json.load(f)["done"] == chunk
    lp, am = stream.decode_xz_to_files(code, px, pz, syn, prefix, chunk=chunk)
    np.testing.assert_array_equal(np.asarray(lp), ref.cpu().numpy())
    np.testing.assert_array_equal(np.asarray(am), ram.cpu().numpy())
    with pytest.raises(ValueError):
        stream.decode_xz_to_files(code, px * 0.5, pz, syn, prefix, chunk=chunk)
    code.close()
