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
