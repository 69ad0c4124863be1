"""CPU-side checks of the C ABI: the library builds, loads and exports every
function declared in include/mld.h (no device calls)."""
import os
import re

import paper_2605_17230_gb300 as mld

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mld.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mld_[a-z_]+)\s*\(", src)))


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
