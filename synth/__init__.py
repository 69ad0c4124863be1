"""Seeded synthetic inputs for rotated-surface-code decoding.

This module is the ONLY code shared by the CUDA decoder's tests/benchmarks and
the CPU oracle. It holds no decoding arithmetic: it draws Pauli errors from a
counter-based generator, turns them into syndromes, and records their true
logical class, so that both sides are fed identical inputs.

Conventions (fixed here and restated by both the library header and the
oracle, each in its own code):

* Rotated distance-d patch, d odd. Data qubit (r, c), 0 <= r, c < d, has index
  q = r*d + c.
* Plaquette (i, j), 0 <= i, j <= d, touches the data qubits (i-1, j-1),
  (i-1, j), (i, j-1), (i, j) that lie inside the patch. It is X-type when
  i+j is even and Z-type when i+j is odd. Interior plaquettes
  (1 <= i, j <= d-1) are all present; on the top/bottom rows (i in {0, d})
  only the X-type weight-2 ones, on the left/right columns (j in {0, d}) only
  the Z-type weight-2 ones. This gives n-k = d^2-1 checks (Sec. 2.1).
* Stabilizer index: present plaquettes in column-major order (j outer,
  i inner). Syndrome bit k sits in word k // 64, bit k % 64 (uint64 words).
* Logical operators: Z_L = Z on every qubit of row 0, X_L = X on every qubit
  of column 0.
* Pauli code per qubit: x + 2*z, i.e. I=0, X=1, Z=2, Y=3.
* Noise tables are [n][4] in the paper's order (p_I, p_X, p_Y, p_Z)
  (independent Pauli noise, Sec. 3.1.1).
* Logical class of an error E: l_X = <E, Z_L>, l_Z = <E, X_L> (symplectic
  products), class index l_X + 2*l_Z, i.e. order I, X, Z, Y (Sec. 2.3).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter hash: the
uniform for (seed, syndrome b, qubit q) is
``u = (h >> 11) * 2^-53`` with ``h = sm(sm(sm(seed) ^ b) ^ q)`` and ``sm`` the
SplitMix64 output function applied to its argument plus the golden gamma.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "GAMMA", "splitmix64", "uniforms", "config_seed",
    "n_qubits", "n_stabs", "syn_words", "stabilizers",
    "depolarizing", "biased", "lognormal_biased", "per_syndrome_depolarizing",
    "sample_errors", "syndromes_of", "true_class", "pack_bits",
]

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """SplitMix64 output function of (x + gamma), elementwise on uint64."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniforms(seed: int, b, q):
    """Uniform doubles in [0, 1) for counters (seed, b, q); b, q broadcast."""
    s = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    h = splitmix64(s ^ np.asarray(b, dtype=np.uint64))
    h = splitmix64(h ^ np.asarray(q, dtype=np.uint64))
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def config_seed(base: int, d: int, p: float) -> int:
    """Seed of one (d, p) point of a workload: base ^ (d << 32) ^ round(1e4 p)."""
    return (int(base) ^ (int(d) << 32) ^ int(round(1e4 * p))) & 0xFFFFFFFFFFFFFFFF


# ----------------------------------------------------------------- layout ---

def n_qubits(d: int) -> int:
    return d * d


def n_stabs(d: int) -> int:
    return d * d - 1


def syn_words(d: int) -> int:
    return (n_stabs(d) + 63) // 64


def _present(d, i, j):
    if 1 <= i <= d - 1 and 1 <= j <= d - 1:
        return True
    if i in (0, d) and 1 <= j <= d - 1 and (i + j) % 2 == 0:
        return True
    if j in (0, d) and 1 <= i <= d - 1 and (i + j) % 2 == 1:
        return True
    return False


def stabilizers(d: int):
    """List of (type, [qubits]) in stabilizer-index order; type 0 = X, 1 = Z."""
    out = []
    for j in range(d + 1):
        for i in range(d + 1):
            if not _present(d, i, j):
                continue
            qs = [r * d + c for (r, c) in ((i - 1, j - 1), (i - 1, j), (i, j - 1), (i, j))
                  if 0 <= r < d and 0 <= c < d]
            out.append((0 if (i + j) % 2 == 0 else 1, qs))
    return out


# ------------------------------------------------------------ noise models ---

def depolarizing(n: int, p: float) -> np.ndarray:
    """Depolarizing channel: p_I = 1-p, p_X = p_Y = p_Z = p/3 (Sec. 2.2)."""
    t = np.empty((n, 4), dtype=np.float64)
    t[:, 0] = 1.0 - p
    t[:, 1:] = p / 3.0
    return t


def biased(n: int, p: float, eta: float) -> np.ndarray:
    """Z-biased channel with eta = p_Z / (p_X + p_Y) and p_X = p_Y."""
    t = np.empty((n, 4), dtype=np.float64)
    pz = p * eta / (1.0 + eta)
    px = p / (2.0 * (1.0 + eta))
    t[:, 0] = 1.0 - p
    t[:, 1] = px
    t[:, 2] = px
    t[:, 3] = pz
    return t


def independent_xz(px, pz) -> np.ndarray:
    """Independent X and Z flips with per-qubit rates px, pz: the table
    (1-px)(1-pz), px(1-pz), px pz, (1-px) pz (I, X, Y, Z)."""
    px = np.asarray(px, dtype=np.float64)
    pz = np.asarray(pz, dtype=np.float64)
    return np.stack([(1 - px) * (1 - pz), px * (1 - pz), px * pz, (1 - px) * pz], axis=1)


def lognormal_biased(n: int, seed: int, median: float = 0.05, sigma: float = 0.5,
                     eta_lo: float = 1.0, eta_hi: float = 10.0) -> np.ndarray:
    """Per-qubit non-uniform biased noise: p_q = median*exp(sigma*N(0,1)) clipped
    to [1e-4, 0.45], eta_q ~ U[eta_lo, eta_hi]. Normals by Box-Muller from the
    counter generator (counters b = 0 and 1 for the pair, 2 for eta)."""
    q = np.arange(n, dtype=np.uint64)
    u1 = uniforms(seed, 0, q)
    u2 = uniforms(seed, 1, q)
    u3 = uniforms(seed, 2, q)
    g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    p = np.clip(median * np.exp(sigma * g), 1e-4, 0.45)
    eta = eta_lo + (eta_hi - eta_lo) * u3
    t = np.empty((n, 4), dtype=np.float64)
    pz = p * eta / (1.0 + eta)
    px = p / (2.0 * (1.0 + eta))
    t[:, 0] = 1.0 - p
    t[:, 1] = px
    t[:, 2] = px
    t[:, 3] = pz
    return t


def per_syndrome_depolarizing(B: int, seed: int, lo: float, hi: float) -> np.ndarray:
    """Per-syndrome depolarizing strength p_b ~ U[lo, hi] (counter q = 2^20)."""
    u = uniforms(seed, np.arange(B, dtype=np.uint64), np.uint64(1 << 20))
    return lo + (hi - lo) * u


def mechanism_model(d: int, seed: int, median: float = 0.03, sigma: float = 0.5):
    """Code-capacity error-mechanism list: an X, a Y and a Z mechanism on every
    qubit (index r*d + c; Pauli code x + 2z: X = 1, Y = 3, Z = 2), each with
    probability median*exp(sigma*N(0,1)) clipped to [1e-4, 0.3]. Normals by
    Box-Muller from the counter generator (counters b = 3 and 4, q = mechanism).
    Returns (qubit int32 [3n], pauli int32 [3n], p float64 [3n])."""
    n = d * d
    m = np.arange(3 * n, dtype=np.uint64)
    u1 = uniforms(seed, 3, m)
    u2 = uniforms(seed, 4, m)
    g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    p = np.clip(median * np.exp(sigma * g), 1e-4, 0.3)
    return (np.repeat(np.arange(n), 3).astype(np.int32), np.tile(np.array([1, 3, 2], np.int32), n), p)


def sample_mechanisms(d: int, qubit, pauli, p, B: int, seed: int, b0: int = 0) -> np.ndarray:
    """Errors E [B][n] (Pauli codes x + 2z) drawn from a mechanism list:
    mechanism m fires in sample b when uniforms(seed, b0 + b, m) < p_m, and the
    fired mechanisms' Paulis multiply (codes XOR) on their qubits."""
    n = d * d
    E = np.zeros((B, n), dtype=np.uint8)
    bs = np.arange(b0, b0 + B, dtype=np.uint64)
    for m, (q, c, pm) in enumerate(zip(qubit, pauli, p)):
        fire = uniforms(seed, bs, np.uint64(m)) < pm
        E[fire, int(q)] ^= np.uint8(c)
    return E


# -------------------------------------------------------------- sampling ---

_PAPER_TO_CODE = np.array([0, 1, 3, 2], dtype=np.uint8)   # I, X, Y, Z -> x + 2z


def sample_errors(d: int, noise, B: int, seed: int, b0: int = 0) -> np.ndarray:
    """Draw B errors, uint8 [B][n] Pauli codes.

    noise: [n][4] table shared by all errors, or [B][n][4] per error, or a
    [B] vector of depolarizing strengths. b0 offsets the syndrome counter so a
    shard of a larger batch reproduces the same errors.
    """
    n = d * d
    b = (np.arange(B, dtype=np.uint64) + np.uint64(b0))[:, None]
    q = np.arange(n, dtype=np.uint64)[None, :]
    u = uniforms(seed, b, q)                                    # [B][n]
    noise = np.asarray(noise, dtype=np.float64)
    if noise.ndim == 1:                                         # per-error depolarizing p
        p = noise[:, None]
        cum = np.stack([1.0 - p, 1.0 - p + p / 3, 1.0 - p + 2 * p / 3,
                        np.ones_like(p)], axis=-1) * np.ones((1, n, 1))
    else:
        cum = np.cumsum(noise, axis=-1)
        if cum.ndim == 2:
            cum = cum[None, :, :]
    k = (u[..., None] >= cum[..., :3]).sum(axis=-1)             # index in I,X,Y,Z
    return _PAPER_TO_CODE[k]


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """Pack uint8 [B][m] bits into uint64 [B][ceil(m/64)] (bit k -> word k//64)."""
    B, m = bits.shape
    w = (m + 63) // 64
    out = np.zeros((B, w), dtype=np.uint64)
    for k in range(m):
        out[:, k // 64] |= bits[:, k].astype(np.uint64) << np.uint64(k % 64)
    return out


def syndromes_of(d: int, E: np.ndarray) -> np.ndarray:
    """Syndromes (uint64 [B][syn_words]) of Pauli errors E (uint8 [B][n])."""
    x = (E & 1).astype(np.uint8)
    z = ((E >> 1) & 1).astype(np.uint8)
    st = stabilizers(d)
    bits = np.zeros((E.shape[0], len(st)), dtype=np.uint8)
    for k, (t, qs) in enumerate(st):
        # an X-type check anticommutes with the z-part, a Z-type with the x-part
        part = z if t == 0 else x
        bits[:, k] = np.bitwise_xor.reduce(part[:, qs], axis=1)
    return pack_bits(bits)


def true_class(d: int, E: np.ndarray) -> np.ndarray:
    """Class index l_X + 2 l_Z of each error (order I, X, Z, Y)."""
    x = (E & 1).astype(np.uint8)
    z = ((E >> 1) & 1).astype(np.uint8)
    row0 = [c for c in range(d)]                 # qubits (0, c)
    col0 = [r * d for r in range(d)]             # qubits (r, 0)
    lx = np.bitwise_xor.reduce(x[:, row0], axis=1)   # <E, Z_L>: x-part on row 0
    lz = np.bitwise_xor.reduce(z[:, col0], axis=1)   # <E, X_L>: z-part on column 0
    return (lx + 2 * lz).astype(np.uint8)
