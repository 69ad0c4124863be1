"""FP64 CPU oracle for tensor-network MLD of the rotated surface code.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``. The decoder package never imports
it and the two share no code (only ``synth`` feeds both the same inputs).

``mld_oracle.c`` holds the exact contraction (Eq. 3/Eq. 7 of arxiv 2605.17230,
evaluated by variable elimination), brute force over all Paulis, stabiliser
group enumeration and the derivative contractions. ``mps.py`` holds the
boundary-MPS method of Sec. 3.2.1 in FP64 with numpy's QR and SVD, used to
check truncated bond dimensions. ``dem_qubit_table`` and
``dem_bruteforce_table`` state what the detector picture (Sec. 3.2.2)
computes for a code-capacity error-mechanism model. ``kac_ward.py`` evaluates
the coset sums under independent X/Z noise by Kac-Ward determinants
(Sec. 3.1.3), a second exact method.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mld_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile mld_oracle.c with gcc -O2 -fopenmp into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I, L = ctypes.c_int, ctypes.c_int64
            sig = {
                "orc_code_info": [I, P, P, P],
                "orc_layout": [I, P, P, P, P],
                "orc_destabilisers": [I, P],
                "orc_syndrome_class": [I, P, L, P, P],
                "orc_representatives": [I, P, L, P],
                "orc_coset_logz": [I, P, L, P, L, P, I],
                "orc_decode": [I, P, I, P, L, P, P, I],
                "orc_coset_dlogz": [I, P, L, P, L, P, P, I],
                "orc_bruteforce_table": [I, P, P],
                "orc_group_logz": [I, P, P, P, I],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def code_info(d: int):
    n, m, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_load().orc_code_info(d, ctypes.byref(n), ctypes.byref(m), ctypes.byref(w)), "code_info")
    return n.value, m.value, w.value


def layout(d: int):
    n, m, _ = code_info(d)
    t = np.zeros(m, np.int32)
    s = np.zeros((m, 4), np.int32)
    lx = np.zeros(n, np.uint8)
    lz = np.zeros(n, np.uint8)
    _check(_load().orc_layout(d, _p(t), _p(s), _p(lx), _p(lz)), "layout")
    return t, s, lx, lz


def destabilisers(d: int) -> np.ndarray:
    n, m, _ = code_info(d)
    T = np.zeros((m, n), np.uint8)
    _check(_load().orc_destabilisers(d, _p(T)), "destabilisers")
    return T


def syndrome_class(d: int, E: np.ndarray):
    """Syndrome bits uint8 [B][m] and class uint8 [B] of Pauli codes E [B][n]."""
    n, m, _ = code_info(d)
    E = np.ascontiguousarray(E, dtype=np.uint8).reshape(-1, n)
    bits = np.zeros((E.shape[0], m), np.uint8)
    cls = np.zeros(E.shape[0], np.uint8)
    _check(_load().orc_syndrome_class(d, _p(E), E.shape[0], _p(bits), _p(cls)), "syndrome_class")
    return bits, cls


def representatives(d: int, syn: np.ndarray) -> np.ndarray:
    """E_{l,s} for l = I, X, Z, Y: uint8 [B][4][n]."""
    n, m, w = code_info(d)
    syn = np.ascontiguousarray(syn, dtype=np.uint64).reshape(-1, w)
    reps = np.zeros((syn.shape[0], 4, n), np.uint8)
    _check(_load().orc_representatives(d, _p(syn), syn.shape[0], _p(reps)), "representatives")
    return reps


def _noise_table(d, noise, B):
    n = d * d
    noise = np.ascontiguousarray(noise, dtype=np.float64)
    if noise.ndim == 2:
        return noise.reshape(n, 4), 0
    return noise.reshape(B, n, 4), 4 * n


def coset_logz(d: int, noise, reps, threads: int = 0) -> np.ndarray:
    """ln Z of the coset of each representative (reps uint8 [B][n])."""
    n = d * d
    reps = np.ascontiguousarray(reps, dtype=np.uint8).reshape(-1, n)
    B = reps.shape[0]
    tab, stride = _noise_table(d, noise, B)
    out = np.zeros(B, np.float64)
    _check(_load().orc_coset_logz(d, _p(tab), stride, _p(reps), B, _p(out), threads), "coset_logz")
    return out


def decode(d: int, noise, syn, threads: int = 0):
    """ln Z_l(s) for l = I, X, Z, Y ([B][4], FP64) and the argmax ([B]).

    noise: [n][4] shared table, [B] depolarizing strengths, or [B][n][4].
    """
    n, m, w = code_info(d)
    syn = np.ascontiguousarray(syn, dtype=np.uint64).reshape(-1, w)
    B = syn.shape[0]
    noise = np.ascontiguousarray(noise, dtype=np.float64)
    mode = {2: 0, 1: 1, 3: 2}[noise.ndim]
    logP = np.zeros((B, 4), np.float64)
    am = np.zeros(B, np.uint8)
    _check(_load().orc_decode(d, _p(noise), mode, _p(syn), B, _p(logP), _p(am), threads), "decode")
    return logP, am


def coset_dlogz(d: int, noise, reps, threads: int = 0):
    """(ln Z [B], d ln Z / d p_{q,P} [B][n][4]) with all four entries of a row
    treated as independent variables."""
    n = d * d
    reps = np.ascontiguousarray(reps, dtype=np.uint8).reshape(-1, n)
    B = reps.shape[0]
    tab, stride = _noise_table(d, noise, B)
    lz = np.zeros(B, np.float64)
    g = np.zeros((B, n, 4), np.float64)
    _check(_load().orc_coset_dlogz(d, _p(tab), stride, _p(reps), B, _p(lz), _p(g), threads), "dlogz")
    return lz, g


def bruteforce_table(d: int, noise) -> np.ndarray:
    """Z[s][l] over all 2^m syndromes by summing Pr(E) over all 4^n Paulis."""
    n, m, _ = code_info(d)
    tab = np.ascontiguousarray(noise, dtype=np.float64).reshape(n, 4)
    Z = np.zeros((1 << m, 4), np.float64)
    _check(_load().orc_bruteforce_table(d, _p(tab), _p(Z)), "bruteforce_table")
    return Z


def group_logz(d: int, noise, rep, threads: int = 0) -> float:
    """ln of the stabiliser-group sum for the coset of one representative."""
    n = d * d
    tab = np.ascontiguousarray(noise, dtype=np.float64).reshape(n, 4)
    rep = np.ascontiguousarray(rep, dtype=np.uint8).reshape(n)
    out = ctypes.c_double()
    _check(_load().orc_group_logz(d, _p(tab), _p(rep), ctypes.byref(out), threads), "group_logz")
    return out.value


def syndrome_index(bits: np.ndarray) -> np.ndarray:
    """Integer index of syndrome bit rows (bit k -> 2^k), for small codes."""
    bits = np.asarray(bits, dtype=np.uint64)
    return (bits << np.arange(bits.shape[-1], dtype=np.uint64)).sum(axis=-1)


# --------------------------------------------------------------------------
# Code-capacity detector error models (the detector picture, Sec. 3.2.2).
# A model is a list of independent error mechanisms m: Pauli pauli[m]
# (code x + 2z: 1 = X, 2 = Z, 3 = Y) on qubit qubit[m], present with
# probability p[m]. These functions state what the detector-picture network
# contracts to; neither builds that network.

_CODE_TO_ROW = (0, 1, 3, 2)        # Pauli code x + 2z -> noise-row index (I, X, Y, Z)


def dem_qubit_table(d: int, qubit, pauli, p) -> np.ndarray:
    """Per-qubit Pauli table [n][4] (I, X, Y, Z) of a mechanism list: the
    mechanisms on one qubit are independent and compose by Pauli product
    (XOR of the codes), so the qubit's Pauli is distributed as the product
    of independent factors (1 - p_m) I + p_m P_m; mechanisms on different
    qubits are independent, so Pr(E) is the product of the rows."""
    n = d * d
    dist = np.zeros((n, 4), np.float64)            # indexed by Pauli code
    dist[:, 0] = 1.0
    for q, c, pm in zip(np.asarray(qubit, np.int64), np.asarray(pauli, np.int64), np.asarray(p, np.float64)):
        if not (0 <= q < n and 1 <= c <= 3 and 0.0 <= pm <= 1.0):
            raise ValueError(f"bad mechanism ({q}, {c}, {pm})")
        old = dist[q].copy()
        for code in range(4):
            dist[q, code] = (1.0 - pm) * old[code] + pm * old[code ^ c]
    tab = np.zeros((n, 4), np.float64)
    for code in range(4):
        tab[:, _CODE_TO_ROW[code]] = dist[:, code]
    return tab


def dem_bruteforce_table(d: int, qubit, pauli, p, chunk: int = 1 << 16) -> np.ndarray:
    """Z[s][l] over all 2^m syndromes of a mechanism list, by its definition:
    the sum over all 2^M configurations b of the mechanisms of
    prod_m p_m^{b_m} (1 - p_m)^{1 - b_m}, each configuration filed under the
    syndrome and logical class of the Pauli it produces (Eq. 3 read in the
    detector picture of Sec. 3.2.2). Small models only (M <= 22)."""
    n, m, _ = code_info(d)
    qubit = np.asarray(qubit, np.int64)
    pauli = np.asarray(pauli, np.uint8)
    p = np.asarray(p, np.float64)
    M = len(p)
    if M > 22:
        raise ValueError("too many mechanisms for enumeration")
    Z = np.zeros((1 << m, 4), np.float64)
    for lo in range(0, 1 << M, chunk):
        b = ((np.arange(lo, min(lo + chunk, 1 << M), dtype=np.int64)[:, None] >> np.arange(M)) & 1).astype(bool)
        E = np.zeros((b.shape[0], n), np.uint8)
        w = np.ones(b.shape[0], np.float64)
        for k in range(M):
            E[b[:, k], qubit[k]] ^= pauli[k]
            w *= np.where(b[:, k], p[k], 1.0 - p[k])
        bits, cls = syndrome_class(d, E)
        np.add.at(Z, (syndrome_index(bits).astype(np.int64), cls.astype(np.int64)), w)
    return Z
