"""GB300 (sm_103a) tensor-network maximum-likelihood decoder for the rotated
surface code: thin Python binding of the C ABI in ``include/mld.h``.

Every step of the decoding path runs in the CUDA library ``libmld.so``; this
module only marshals arguments (device pointers of torch tensors, the current
CUDA stream, host numpy buffers). There is no CPU fallback: if the library
cannot be loaded, the calls raise.

Names follow the C ABI: ``mld_code_create_rotated``, ``mld_decode``,
``mld_decode_host`` ...; ``Code`` wraps a code handle.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

__all__ = ["MLD_OK", "MLD_FP32", "MLD_MIXED_BF16", "MLD_MIXED_TF32", "MLD_FP64", "MLD_NOISE_TABLE",
           "MLD_NOISE_DEPOL", "MldError", "Code", "load", "library_path", "mld_code_create_rotated",
           "mld_decode", "mld_decode_host", "mld_decode_status", "mld_decode_launches",
           "mld_status_string", "EXPORTED_SYMBOLS", "log_coset_probabilities", "estimate_noise",
           "noise_table_from_logits", "mld_decode_xz"]

MLD_OK = 0
MLD_FP32, MLD_MIXED_BF16, MLD_MIXED_TF32, MLD_FP64 = 0, 1, 2, 3
MLD_NOISE_TABLE, MLD_NOISE_DEPOL = 0, 1

EXPORTED_SYMBOLS = ["mld_code_create_rotated", "mld_code_destroy", "mld_code_info", "mld_code_layout",
                    "mld_code_representatives",
                    "mld_decode", "mld_decode_host", "mld_decode_status", "mld_decode_launches",
                    "mld_decode_flops", "mld_decode_noalloc", "mld_decode_batch", "mld_graph_create",
                    "mld_graph_launch", "mld_graph_destroy", "mld_autotune", "mld_decode_grad",
                    "mld_decode_dem", "mld_status_string", "mld_code_set_svd_cutoff",
                    "mld_decode_executed_flops", "mld_decode_bond_histogram", "mld_measure_fp32_peak",
                    "mld_code_set_truncation_kernel", "mld_code_set_exact_kernel",
                    "mld_code_set_truncation_workspace", "mld_decode_xz",
                    "mld_decode_xz_executed_flops"]

_lib = None


class MldJob(ctypes.Structure):
    """C struct mld_job (one decode job of a mixed batch)."""
    _fields_ = [("code", ctypes.c_void_p), ("noise", ctypes.c_void_p), ("noise_mode", ctypes.c_int),
                ("syndromes", ctypes.c_void_p), ("B", ctypes.c_int64), ("chi", ctypes.c_int),
                ("precision", ctypes.c_int), ("logP", ctypes.c_void_p), ("argmax", ctypes.c_void_p)]


class MldError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {mld_status_string(status)} (status {status})")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmld.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"decoder library not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    P, I, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.mld_code_create_rotated.argtypes = [I, ctypes.POINTER(P)]
    lib.mld_code_create_rotated.restype = I
    lib.mld_code_destroy.argtypes = [P]
    lib.mld_code_destroy.restype = None
    lib.mld_code_info.argtypes = [P, P, P, P]
    lib.mld_code_info.restype = I
    lib.mld_code_layout.argtypes = [P, P, P, P, P]
    lib.mld_code_layout.restype = I
    lib.mld_code_representatives.argtypes = [P, P, L, P]
    lib.mld_code_representatives.restype = I
    lib.mld_decode.argtypes = [P, P, I, P, L, I, I, P, P, P]
    lib.mld_decode.restype = I
    lib.mld_decode_noalloc.argtypes = [P, P, I, P, L, I, I, P, P, P, I]
    lib.mld_decode_noalloc.restype = I
    lib.mld_decode_host.argtypes = [P, P, I, P, L, I, I, P, P]
    lib.mld_decode_host.restype = I
    lib.mld_decode_status.argtypes = [P]
    lib.mld_decode_status.restype = I
    lib.mld_decode_flops.argtypes = [P, I, I, ctypes.POINTER(ctypes.c_double)]
    lib.mld_decode_flops.restype = I
    lib.mld_decode_batch.argtypes = [P, I, P]
    lib.mld_decode_batch.restype = I
    lib.mld_graph_create.argtypes = [P, I, ctypes.POINTER(P)]
    lib.mld_graph_create.restype = I
    lib.mld_graph_launch.argtypes = [P, P]
    lib.mld_graph_launch.restype = I
    lib.mld_graph_destroy.argtypes = [P]
    lib.mld_graph_destroy.restype = None
    lib.mld_autotune.argtypes = [P, I, I, L, ctypes.POINTER(I)]
    lib.mld_autotune.restype = I
    lib.mld_decode_grad.argtypes = [P, P, P, L, I, P, P, P, P]
    lib.mld_decode_grad.restype = I
    lib.mld_decode_dem.argtypes = [P, P, P, P, I, P, L, P, P, P]
    lib.mld_decode_dem.restype = I
    lib.mld_decode_xz.argtypes = [P, P, P, P, L, I, P, P, P]
    lib.mld_decode_xz.restype = I
    lib.mld_decode_xz_executed_flops.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.mld_decode_xz_executed_flops.restype = I
    lib.mld_code_set_svd_cutoff.argtypes = [P, ctypes.c_double]
    lib.mld_code_set_svd_cutoff.restype = I
    lib.mld_decode_executed_flops.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.mld_decode_executed_flops.restype = I
    lib.mld_decode_bond_histogram.argtypes = [P, P]
    lib.mld_decode_bond_histogram.restype = I
    lib.mld_code_set_truncation_kernel.argtypes = [P, I]
    lib.mld_code_set_truncation_kernel.restype = I
    lib.mld_code_set_exact_kernel.argtypes = [P, I]
    lib.mld_code_set_exact_kernel.restype = I
    lib.mld_code_set_truncation_workspace.argtypes = [P, I]
    lib.mld_code_set_truncation_workspace.restype = I
    lib.mld_measure_fp32_peak.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I)]
    lib.mld_measure_fp32_peak.restype = I
    lib.mld_decode_launches.argtypes = []
    lib.mld_decode_launches.restype = I
    lib.mld_status_string.argtypes = [I]
    lib.mld_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def mld_status_string(status: int) -> str:
    return load().mld_status_string(int(status)).decode()


def _check(status, what):
    if status != MLD_OK:
        raise MldError(status, what)


def mld_code_create_rotated(d: int) -> int:
    h = ctypes.c_void_p()
    _check(load().mld_code_create_rotated(int(d), ctypes.byref(h)), "mld_code_create_rotated")
    return h.value


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def mld_decode(code, noise, noise_mode, syndromes, B, chi, precision, logP, argmax=None, stream=None):
    """C-ABI mld_decode on torch CUDA tensors (asynchronous on ``stream``,
    default: torch's current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = load().mld_decode(ctypes.c_void_p(code), _ptr(noise), int(noise_mode), _ptr(syndromes), int(B),
                           int(chi), int(precision), _ptr(logP), _ptr(argmax), ctypes.c_void_p(int(stream)))
    _check(st, "mld_decode")


def mld_decode_noalloc(code, noise, noise_mode, syndromes, B, chi, precision, logP, argmax=None, stream=None,
                       check_status=True):
    """C-ABI mld_decode_noalloc on torch CUDA tensors: no device allocation;
    scratch in the library's fixed device array (see include/mld.h)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = load().mld_decode_noalloc(ctypes.c_void_p(code), _ptr(noise), int(noise_mode), _ptr(syndromes), int(B),
                                   int(chi), int(precision), _ptr(logP), _ptr(argmax),
                                   ctypes.c_void_p(int(stream)), int(bool(check_status)))
    _check(st, "mld_decode_noalloc")


def mld_decode_host(code, noise, noise_mode, syndromes, B, chi, precision, logP, argmax=None):
    """C-ABI mld_decode_host on contiguous numpy arrays (synchronous)."""
    f = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else ctypes.c_void_p(0)
    st = load().mld_decode_host(ctypes.c_void_p(code), f(noise), int(noise_mode), f(syndromes), int(B),
                                int(chi), int(precision), f(logP), f(argmax))
    _check(st, "mld_decode_host")


def mld_decode_status(code) -> int:
    return load().mld_decode_status(ctypes.c_void_p(code))


def mld_measure_fp32_peak(seconds=1.0):
    """Sustained FP32 FMA rate of the current GPU (TFLOP/s) and its SM count."""
    t, n = ctypes.c_double(), ctypes.c_int()
    _check(load().mld_measure_fp32_peak(float(seconds), ctypes.byref(t), ctypes.byref(n)), "mld_measure_fp32_peak")
    return t.value, n.value


def mld_decode_launches() -> int:
    return load().mld_decode_launches()


class Code:
    """Rotated distance-d code handle (owns the library object)."""

    def __init__(self, d: int):
        self.d = int(d)
        self.handle = mld_code_create_rotated(self.d)
        n, m, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().mld_code_info(ctypes.c_void_p(self.handle), ctypes.byref(n), ctypes.byref(m),
                                    ctypes.byref(w)), "mld_code_info")
        self.n, self.m, self.words = n.value, m.value, w.value

    def close(self):
        if getattr(self, "handle", None):
            load().mld_code_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self):
        t = np.zeros(self.m, np.int32)
        s = np.zeros((self.m, 4), np.int32)
        lx = np.zeros(self.n, np.uint8)
        lz = np.zeros(self.n, np.uint8)
        f = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(load().mld_code_layout(ctypes.c_void_p(self.handle), f(t), f(s), f(lx), f(lz)), "mld_code_layout")
        return t, s, lx, lz

    def representatives(self, syndromes):
        """Pauli codes of E_{l,s} for l = I, X, Z, Y: uint8 [B][4][n] (host)."""
        syn = np.ascontiguousarray(syndromes, dtype=np.uint64).reshape(-1, self.words)
        out = np.zeros((syn.shape[0], 4, self.n), np.uint8)
        f = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(load().mld_code_representatives(ctypes.c_void_p(self.handle), f(syn), syn.shape[0], f(out)),
               "mld_code_representatives")
        return out

    def decode(self, noise, syndromes, chi, precision=MLD_FP32, with_argmax=True, stream=None):
        """Decode torch CUDA tensors. noise: float32 [n][4] table or [B]
        depolarizing strengths; syndromes: uint64/int64 [B][words].
        Returns (logP float64 [B][4], argmax uint8 [B] or None)."""
        import torch
        B = syndromes.shape[0]
        mode = MLD_NOISE_TABLE if noise.dim() == 2 else MLD_NOISE_DEPOL
        dev = syndromes.device
        logP = torch.empty((B, 4), dtype=torch.float64, device=dev)
        am = torch.empty((B,), dtype=torch.uint8, device=dev) if with_argmax else None
        mld_decode(self.handle, noise.contiguous(), mode, syndromes.contiguous(), B, chi, precision, logP, am,
                   stream)
        return logP, am

    def decode_host(self, noise, syndromes, chi, precision=MLD_FP32):
        """Decode numpy host arrays through the host-buffer entry point."""
        noise = np.ascontiguousarray(noise, dtype=np.float32)
        syn = np.ascontiguousarray(syndromes, dtype=np.uint64).reshape(-1, self.words)
        B = syn.shape[0]
        mode = MLD_NOISE_TABLE if noise.ndim == 2 else MLD_NOISE_DEPOL
        logP = np.zeros((B, 4), np.float64)
        am = np.zeros(B, np.uint8)
        mld_decode_host(self.handle, noise, mode, syn, B, chi, precision, logP, am)
        return logP, am

    def decode_dem(self, mech_qubit, mech_pauli, mech_p, syndromes, with_argmax=True, stream=None):
        """Detector-picture decode of a code-capacity mechanism list (numpy or
        sequences: qubit index, Pauli code x + 2z, probability) for syndromes
        on the GPU. Returns (logP float64 [B][4], argmax uint8 [B] or None)."""
        import torch
        B = syndromes.shape[0]
        dev = syndromes.device
        logP = torch.empty((B, 4), dtype=torch.float64, device=dev)
        am = torch.empty((B,), dtype=torch.uint8, device=dev) if with_argmax else None
        mld_decode_dem(self.handle, mech_qubit, mech_pauli, mech_p, syndromes.contiguous(), B, logP, am, stream)
        return logP, am

    def decode_xz(self, px, pz, syndromes, precision=MLD_FP32, with_argmax=True, stream=None):
        """Kac-Ward decode under independent X/Z noise: px, pz float32 [n]
        CUDA tensors (pz None: bit-flip noise). Returns (logP float64 [B][4],
        argmax uint8 [B] or None)."""
        import torch
        B = syndromes.shape[0]
        dev = syndromes.device
        logP = torch.empty((B, 4), dtype=torch.float64, device=dev)
        am = torch.empty((B,), dtype=torch.uint8, device=dev) if with_argmax else None
        mld_decode_xz(self.handle, px.contiguous(), None if pz is None else pz.contiguous(), syndromes.contiguous(),
                      B, precision, logP, am, stream)
        return logP, am

    def xz_executed_flops(self) -> float:
        """Flops executed by decode_xz since the last call (then reset)."""
        v = ctypes.c_double()
        _check(load().mld_decode_xz_executed_flops(ctypes.c_void_p(self.handle), ctypes.byref(v)),
               "mld_decode_xz_executed_flops")
        return v.value

    def flops(self, chi, precision=MLD_FP32) -> float:
        """Counted flops per syndrome (four classes) of the executed schedule."""
        v = ctypes.c_double()
        _check(load().mld_decode_flops(ctypes.c_void_p(self.handle), int(chi), int(precision), ctypes.byref(v)),
               "mld_decode_flops")
        return v.value

    def bond_histogram(self):
        """Kept bonds of truncating cuts since the last call: int64 [65]
        (index k; the last bin counts k >= 64); resets the device histogram."""
        h = np.zeros(65, np.int64)
        _check(load().mld_decode_bond_histogram(ctypes.c_void_p(self.handle), h.ctypes.data_as(ctypes.c_void_p)),
               "mld_decode_bond_histogram")
        return h

    def status(self) -> int:
        return mld_decode_status(self.handle)

    def set_svd_cutoff(self, rel: float):
        """Relative singular-value cutoff of truncating chi (mld_code_set_svd_cutoff)."""
        _check(load().mld_code_set_svd_cutoff(ctypes.c_void_p(self.handle), float(rel)), "mld_code_set_svd_cutoff")

    def set_exact_kernel(self, which: int):
        """Untruncated chi: 0 by d (default; the dense-state kernel at d = 11
        and 13), 1 the boundary-MPS kernel, 2 the dense-state kernel (d = 9,
        11, 13) (mld_code_set_exact_kernel)."""
        _check(load().mld_code_set_exact_kernel(ctypes.c_void_p(self.handle), int(which)),
               "mld_code_set_exact_kernel")

    def set_truncation_workspace(self, max_bond: int):
        """Bond capacity of the truncated sweep's first pass: 0 by chi
        (default), 48, 64 or 128 (mld_code_set_truncation_workspace)."""
        _check(load().mld_code_set_truncation_workspace(ctypes.c_void_p(self.handle), int(max_bond)),
               "mld_code_set_truncation_workspace")

    def set_truncation_kernel(self, which: int):
        """0: chosen per chi (default); 1: rank-adaptive; 2: fixed-shape
        (mld_code_set_truncation_kernel)."""
        _check(load().mld_code_set_truncation_kernel(ctypes.c_void_p(self.handle), int(which)),
               "mld_code_set_truncation_kernel")

    def executed_flops(self) -> float:
        """Flops executed by truncating sweeps since the last call (the
        caller synchronises first); resets the device counter."""
        v = ctypes.c_double()
        _check(load().mld_decode_executed_flops(ctypes.c_void_p(self.handle), ctypes.byref(v)),
               "mld_decode_executed_flops")
        return v.value


def make_jobs(items):
    """items: list of (Code, noise tensor, syndromes tensor, chi, precision,
    logP tensor, argmax tensor or None) on the GPU -> ctypes array of MldJob."""
    arr = (MldJob * len(items))()
    for k, (code, noise, syn, chi, prec, logP, am) in enumerate(items):
        arr[k] = MldJob(code.handle, noise.data_ptr(), MLD_NOISE_TABLE if noise.dim() == 2 else MLD_NOISE_DEPOL,
                        syn.data_ptr(), syn.shape[0], int(chi), int(prec), logP.data_ptr(),
                        am.data_ptr() if am is not None else 0)
    return arr


def mld_decode_batch(jobs, stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(load().mld_decode_batch(ctypes.cast(jobs, ctypes.c_void_p), len(jobs), ctypes.c_void_p(int(stream))),
           "mld_decode_batch")


class Graph:
    """A mixed batch captured into one CUDA graph (mld_graph_create); launch()
    decodes whatever the jobs' buffers hold."""

    def __init__(self, jobs):
        self._jobs = jobs                        # keep the job array alive
        h = ctypes.c_void_p()
        _check(load().mld_graph_create(ctypes.cast(jobs, ctypes.c_void_p), len(jobs), ctypes.byref(h)),
               "mld_graph_create")
        self.handle = h.value

    def launch(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        _check(load().mld_graph_launch(ctypes.c_void_p(self.handle), ctypes.c_void_p(int(stream))),
               "mld_graph_launch")

    def close(self):
        if getattr(self, "handle", None):
            load().mld_graph_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mld_autotune(code, chi, precision=MLD_FP32, sample_B=8192) -> int:
    w = ctypes.c_int()
    _check(load().mld_autotune(ctypes.c_void_p(code.handle), int(chi), int(precision), int(sample_B),
                               ctypes.byref(w)), "mld_autotune")
    return w.value


def mld_decode_grad(code, noise, syndromes, B, chi, dlogP, logP, dnoise, stream=None):
    """C-ABI mld_decode_grad on torch CUDA tensors (dnoise is accumulated)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(load().mld_decode_grad(ctypes.c_void_p(code), _ptr(noise), _ptr(syndromes), int(B), int(chi),
                                  _ptr(dlogP), _ptr(logP), _ptr(dnoise), ctypes.c_void_p(int(stream))),
           "mld_decode_grad")


def mld_decode_dem(code, mech_qubit, mech_pauli, mech_p, syndromes, B, logP, argmax=None, stream=None):
    """C-ABI mld_decode_dem: mechanism arrays on the host, syndromes and outputs
    torch CUDA tensors."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    q = np.ascontiguousarray(mech_qubit, dtype=np.int32)
    c = np.ascontiguousarray(mech_pauli, dtype=np.int32)
    p = np.ascontiguousarray(mech_p, dtype=np.float64)
    if not (q.shape == c.shape == p.shape and q.ndim == 1):
        raise ValueError("mechanism arrays must be 1-D and of one length")
    f = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(load().mld_decode_dem(ctypes.c_void_p(code), f(q), f(c), f(p), int(q.size), _ptr(syndromes), int(B),
                                 _ptr(logP), _ptr(argmax), ctypes.c_void_p(int(stream))), "mld_decode_dem")


def mld_decode_xz(code, px, pz, syndromes, B, precision, logP, argmax=None, stream=None):
    """C-ABI mld_decode_xz (Kac-Ward, independent X/Z noise): px, pz (or None
    for bit-flip noise), syndromes and outputs are torch CUDA tensors."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(load().mld_decode_xz(ctypes.c_void_p(code), _ptr(px), _ptr(pz), _ptr(syndromes), int(B), int(precision),
                                _ptr(logP), _ptr(argmax), ctypes.c_void_p(int(stream))), "mld_decode_xz")


def _logz_function():
    import torch

    class LogZ(torch.autograd.Function):
        """ln Z_l(s) as a differentiable function of the noise table [n][4]:
        forward through mld_decode, backward through the adjoint sweep."""

        @staticmethod
        def forward(ctx, noise, code, syndromes, chi):
            nz = noise.detach().to(torch.float32).contiguous()
            logP, _ = code.decode(nz, syndromes, chi, MLD_FP32, with_argmax=False)
            ctx.code, ctx.chi = code, chi
            ctx.save_for_backward(nz, syndromes)
            return logP

        @staticmethod
        def backward(ctx, dlogP):
            nz, syn = ctx.saved_tensors
            dnoise = torch.zeros((ctx.code.n, 4), dtype=torch.float64, device=nz.device)
            mld_decode_grad(ctx.code.handle, nz, syn, syn.shape[0], ctx.chi,
                            dlogP.detach().to(torch.float64).contiguous(), None, dnoise)
            return dnoise, None, None, None

    return LogZ


_LogZ = None


def log_coset_probabilities(code, noise, syndromes, chi):
    """Differentiable ln Z_l(s) [B][4] (float64) of a noise table [n][4]
    (torch CUDA tensor, may require grad). chi must not truncate."""
    global _LogZ
    if _LogZ is None:
        _LogZ = _logz_function()
    return _LogZ.apply(noise, code, syndromes, chi)



def noise_table_from_logits(z):
    """Per-qubit Pauli table [n][4] (I, X, Y, Z) from three logits per qubit:
    p_P = exp(z_P) / (1 + sum_P' exp(z_P')), p_I = 1 / (1 + sum_P' exp(z_P'))."""
    import torch
    e = torch.exp(z)
    den = 1.0 + e.sum(dim=1, keepdim=True)
    return torch.cat([1.0 / den, e / den], dim=1)


def estimate_noise(code, syndromes, chi, steps=200, lr=0.08, init_rate=0.05, logits=None):
    """Maximum-likelihood per-qubit Pauli rates from unlabelled syndromes
    (Sec. 3.2.4, Eq. 10): minimises L = -mean_b ln sum_l Z_l(s_b), the
    marginal likelihood of the observed syndromes, over three logits per
    qubit with Adam. Every step is one forward sweep and one adjoint sweep
    over the whole batch on the GPU (chi must not truncate).

    syndromes: int64 CUDA tensor [B][words]. Starts from the uniform table
    with total rate init_rate per qubit unless `logits` ([n][3], float64) is
    given. Returns (table [n][4] float64, logits [n][3], losses [steps])."""
    import torch
    n = code.n
    if logits is None:
        z0 = math.log(init_rate / 3.0 / (1.0 - init_rate))
        logits = torch.full((n, 3), z0, dtype=torch.float64, device=syndromes.device)
    z = logits.detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([z], lr=lr)
    losses = []
    for _ in range(steps):
        opt.zero_grad()
        lp = log_coset_probabilities(code, noise_table_from_logits(z), syndromes, chi)
        loss = -torch.logsumexp(lp, dim=1).mean()
        loss.backward()
        opt.step()
        losses.append(loss.detach())
    z = z.detach()
    hist = torch.stack(losses).cpu().numpy() if losses else np.zeros(0)
    return noise_table_from_logits(z), z, hist