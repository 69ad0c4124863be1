"""Host logic of the chunked decoder's progress record (no GPU): a fresh job
starts at 0, a saved count is read back, a record of another configuration is
refused, and the syndrome fingerprint tells arrays apart."""
import json
import os

import numpy as np
import pytest

from paper_2605_17230_gb300 import stream


def _config(**kw):
    c = {"d": 9, "chi": 32, "precision": 0, "noise_mode": 0, "B": 1000, "words": 2, "syndromes_sha1": "x"}
    c.update(kw)
    return c


def test_progress_roundtrip(tmp_path):
    path = str(tmp_path / "job.progress.json")
    p = stream.Progress(path, _config())
    assert not p.load() and p.done == 0
    p.save(0)
    p.save(384)
    q = stream.Progress(path, _config())
    assert q.load() and q.done == 384
    assert not os.path.exists(path + ".tmp")
    with open(path) as f:
        assert json.load(f)["done"] == 384


def test_progress_refuses_another_job(tmp_path):
    path = str(tmp_path / "job.progress.json")
    stream.Progress(path, _config()).save(10)
    for other in (_config(chi=16), _config(B=999), _config(syndromes_sha1="y")):
        with pytest.raises(ValueError):
            stream.Progress(path, other).load()


def test_progress_rejects_out_of_range_count(tmp_path):
    path = str(tmp_path / "job.progress.json")
    with open(path, "w") as f:
        json.dump({"version": stream.PROGRESS_VERSION, "config": _config(), "done": 5000}, f)
    with pytest.raises(ValueError):
        stream.Progress(path, _config()).load()


def test_fingerprint_tells_arrays_apart():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 2 ** 62, size=(10000, 2), dtype=np.int64).view(np.uint64)
    b = a.copy()
    assert stream.fingerprint(a) == stream.fingerprint(b)
    b[0, 0] ^= np.uint64(1)
    assert stream.fingerprint(a) != stream.fingerprint(b)
    c = a.copy()
    c[-1, 1] ^= np.uint64(2)
    assert stream.fingerprint(a) != stream.fingerprint(c)
    assert stream.fingerprint(a[:9999]) != stream.fingerprint(a)


def test_kac_ward_job_input_checks(tmp_path):
    """decode_xz_to_files refuses malformed syndrome arrays and chunk sizes
    before it touches the rates or a device."""
    class FakeCode:
        words, d = 2, 9
    bad_rates = object()                   # never read on these paths
    with pytest.raises(ValueError):
        stream.decode_xz_to_files(FakeCode(), bad_rates, None, np.zeros((4, 3), np.uint64), str(tmp_path / "a"))
    with pytest.raises(ValueError):
        stream.decode_xz_to_files(FakeCode(), bad_rates, None, np.zeros((4,), np.uint64), str(tmp_path / "b"))
    with pytest.raises(ValueError):
        stream.decode_xz_to_files(FakeCode(), bad_rates, None, np.zeros((4, 2), np.float32), str(tmp_path / "c"))
    with pytest.raises(ValueError):
        stream.decode_xz_to_files(FakeCode(), bad_rates, None, np.zeros((4, 2), np.uint64), str(tmp_path / "d"),
                                  chunk=0)
    assert not os.path.exists(str(tmp_path / "d.progress.json"))


def test_kac_ward_record_is_another_job(tmp_path):
    """A record written for the boundary-MPS decoder is not a Kac-Ward job's:
    the two configurations differ (method, rates), so resuming one as the
    other is refused."""
    path = str(tmp_path / "job.progress.json")
    stream.Progress(path, _config()).save(100)
    kw = {"method": "kac-ward", "d": 9, "precision": 0, "bitflip": False, "rates_sha1": "r", "B": 1000,
          "words": 2, "syndromes_sha1": "x"}
    with pytest.raises(ValueError):
        stream.Progress(path, kw).load()
