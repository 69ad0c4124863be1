"""CPU-side checks of the C ABI: the library builds, loads and exports every
function declared in include/mld.h (no device calls)."""
import os
import re

import paper_2605_17230_gb300 as mld

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mld.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mld_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_what_binding_exports():
    assert _declared() == sorted(mld.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol():
    lib = mld.load()
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings():
    assert mld.mld_status_string(0) == "ok"
    assert "unsupported" in mld.mld_status_string(2)


import numpy as np
import pytest

import synth


@pytest.mark.parametrize("d", [3, 5, 9, 13, 25])
def test_host_code_layout_and_representatives(d):
    """Code construction of the library (host side, no GPU): its layout
    matches the documented convention and every representative E_{l,s} has
    syndrome s and logical class l (checked with synth's own layout)."""
    code = mld.Code(d)
    t, s, lx, lz = code.layout()
    st = synth.stabilizers(d)
    assert [x for x, _ in st] == list(t)
    for k, (_, qs) in enumerate(st):
        assert sorted(q for q in s[k] if q >= 0) == sorted(qs)
    assert list(np.flatnonzero(lx)) == [r * d for r in range(d)]
    assert list(np.flatnonzero(lz)) == list(range(d))
    E = synth.sample_errors(d, synth.depolarizing(d * d, 0.15), 128, seed=d)
    syn = synth.syndromes_of(d, E)
    reps = code.representatives(syn)
    for l in range(4):
        np.testing.assert_array_equal(synth.syndromes_of(d, reps[:, l]), syn)
        assert (synth.true_class(d, reps[:, l]) == l).all()


def test_invalid_distance_rejected():
    for d in (1, 2, 4, 27):
        with pytest.raises(mld.MldError):
            mld.Code(d)


def test_host_side_argument_checks():
    """Errors the host can see are returned before anything touches a
    device (so they run here without a GPU): bad mechanisms, sizes, chi,
    precision, noise mode, missing or misaligned pointers, distances beyond a
    path's range. B = 0 with valid arguments is a no-op."""
    import ctypes
    lib = mld.load()
    P = ctypes.c_void_p
    OK, INVALID, UNSUPPORTED = 0, 1, 2
    c5, c11, c13 = mld.Code(5), mld.Code(11), mld.Code(13)
    fake = P(4096)            # aligned, never dereferenced on these paths

    def dem(code, q, c, p, n=None, B=0):
        q = np.ascontiguousarray(q, np.int32)
        c = np.ascontiguousarray(c, np.int32)
        p = np.ascontiguousarray(p, np.float64)
        f = lambda a: a.ctypes.data_as(P)
        return lib.mld_decode_dem(P(code.handle), f(q), f(c), f(p), len(p) if n is None else n, fake, B, fake,
                                  None, None)

    assert dem(c5, [0, 24], [1, 3], [0.1, 1.0]) == OK
    assert dem(c5, [], [], []) == OK
    for q, c, p in (([25], [1], [0.1]), ([-1], [1], [0.1]), ([0], [0], [0.1]), ([0], [4], [0.1]),
                    ([0], [1], [-0.1]), ([0], [1], [1.5]), ([0], [1], [np.nan])):
        assert dem(c5, q, c, p) == INVALID, (q, c, p)
    assert dem(c5, [0], [1], [0.1], n=-1) == INVALID
    assert dem(c13, [0], [1], [0.1]) == UNSUPPORTED
    # mld_decode(code, noise, mode, syn, B, chi, precision, logP, argmax, stream)
    dec = lambda *a: lib.mld_decode(*a)
    assert dec(P(c5.handle), fake, 0, fake, 0, 8, 0, fake, None, None) == OK
    assert dec(P(c5.handle), fake, 0, fake, -1, 8, 0, fake, None, None) == INVALID
    assert dec(P(c5.handle), fake, 0, fake, 4, 0, 0, fake, None, None) == INVALID        # chi < 1
    assert dec(P(c5.handle), fake, 0, fake, 4, 8, 7, fake, None, None) == INVALID        # precision
    assert dec(P(c5.handle), fake, 5, fake, 4, 8, 0, fake, None, None) == INVALID        # noise mode
    assert dec(P(c5.handle), None, 0, fake, 4, 8, 0, fake, None, None) == INVALID        # no noise
    assert dec(P(c5.handle), P(4100), 0, fake, 4, 8, 0, fake, None, None) == INVALID     # misaligned table
    # mld_decode_grad(code, noise, syn, B, chi, dlogP, logP, dnoise, stream)
    grad = lambda *a: lib.mld_decode_grad(*a)
    assert grad(P(c5.handle), fake, fake, 0, 8, None, None, fake, None) == OK
    assert grad(P(c5.handle), fake, fake, -1, 8, None, None, fake, None) == INVALID
    assert grad(P(c5.handle), fake, fake, 4, 0, None, None, fake, None) == INVALID
    assert grad(P(c5.handle), fake, fake, 4, 8, None, None, None, None) == INVALID       # no dnoise
    c15 = mld.Code(15)
    assert grad(P(c15.handle), fake, fake, 4, 128, None, None, fake, None) == UNSUPPORTED   # d > 13


def test_wilson_interval_matches_scipy():
    """The LER intervals the bench reports: Wilson score intervals, checked
    against scipy's binomial test at several counts (including 0 and n)."""
    stats = pytest.importorskip("scipy.stats")
    import bench
    for k, n in [(0, 100), (3, 100), (50, 100), (100, 100), (17, 65536), (6000, 65536)]:
        lo, hi = bench.wilson_interval(k, n)
        ref = stats.binomtest(k, n).proportion_ci(confidence_level=0.95, method="wilson")
        assert abs(lo - ref.low) < 1e-9 and abs(hi - ref.high) < 1e-9


def test_kac_ward_host_side_argument_checks():
    """mld_decode_xz refuses what the host can see before it touches a GPU:
    an unknown precision, a negative batch, missing buffers; B = 0 is a no-op;
    the flop counter of a code that never ran the path reads zero."""
    import ctypes
    lib = mld.load()
    P = ctypes.c_void_p
    OK, INVALID = 0, 1
    fake = P(4096)            # aligned, never dereferenced on these paths
    c5 = mld.Code(5)
    xz = lib.mld_decode_xz
    h = P(c5.handle)
    assert xz(None, fake, fake, fake, 4, mld.MLD_FP32, fake, None, None) == INVALID
    assert xz(h, fake, fake, fake, 4, 7, fake, None, None) == INVALID              # precision
    assert xz(h, fake, fake, fake, 4, mld.MLD_MIXED_TF32, fake, None, None) == INVALID
    assert xz(h, fake, fake, fake, -1, mld.MLD_FP32, fake, None, None) == INVALID
    assert xz(h, fake, fake, fake, 0, mld.MLD_FP64, fake, None, None) == OK          # nothing to do
    assert xz(h, None, fake, fake, 4, mld.MLD_FP32, fake, None, None) == INVALID     # no px
    assert xz(h, fake, None, None, 4, mld.MLD_FP32, fake, None, None) == INVALID     # no syndromes
    assert xz(h, fake, fake, fake, 4, mld.MLD_FP32, None, None, None) == INVALID     # no logP
    assert c5.xz_executed_flops() == 0.0


def test_threshold_crossings_and_leading_gap():
    """The bench's curve-crossing interpolation and leading-class gap on
    hand-made inputs: two lines crossing at 0.105, curves that never cross,
    and a gap measured on the reference's leading class."""
    torch = pytest.importorskip("torch")
    import bench
    ps = [0.09, 0.10, 0.11, 0.12]
    ler = {}
    for p in ps:
        ler[(9, p)] = 0.5 * p + 0.05
        ler[(13, p)] = 1.5 * p - 0.055          # equal at p = 0.105
        ler[(17, p)] = 1.5 * p - 0.1            # below d = 13 everywhere
    cross = bench._crossings(ler, [9, 13, 17], ps)
    assert cross[0]["d"] == [9, 13] and abs(cross[0]["p_cross"] - 0.105) < 1e-12
    assert cross[1]["p_cross"] is None
    ref = torch.tensor([[-1.0, -2.0, -3.0, -4.0], [-5.0, -0.5, -9.0, -9.0]], dtype=torch.float64)
    lp = ref.clone()
    lp[0, 0] += 0.25          # the leading class of row 0
    lp[1, 2] += 7.0           # a non-leading class of row 1: not counted
    g = bench._lead_gap(lp, ref)
    assert abs(g["max"] - 0.25) < 1e-12
