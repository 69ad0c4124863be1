"""Chunked decoding of a syndrome array larger than one launch, with resume
(the boundary-MPS decode, ``decode_to_files``, and the Kac-Ward decode under
independent X/Z noise, ``decode_xz_to_files``).

Decoding is stateless per syndrome, so a long job is a sequence of chunks. The
results go to two ``.npy`` files opened as memory maps (``<prefix>.logp.npy``,
float64 [B][4], and ``<prefix>.argmax.npy``, uint8 [B]), and a small progress
file (``<prefix>.progress.json``) records how many syndromes are complete. It
is rewritten (write to a temporary file, then rename) only after a chunk's
results have been flushed, so after an interruption at any point the recorded
count never runs ahead of the stored results. A restarted job with the same
configuration continues from there; one with another configuration (code
distance, chi, precision, noise mode, batch size or syndrome fingerprint) is
refused.

The host-to-device copy of the next chunk overlaps the decode of the current
one: the syndromes are staged in two pinned buffers and copied on a stream of
their own, and the compute stream waits on the copy's event. Every chunk is one
``mld_decode`` (or ``mld_decode_xz``) call through the C ABI.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import MLD_FP32, MLD_NOISE_DEPOL, MLD_NOISE_TABLE, MldError, mld_decode, mld_decode_xz

PROGRESS_VERSION = 1


def fingerprint(syndromes: np.ndarray) -> str:
    """SHA-1 of the array's shape and of its first and last 4,096 rows."""
    h = hashlib.sha1()
    h.update(repr(tuple(syndromes.shape)).encode())
    h.update(np.ascontiguousarray(syndromes[:4096]).tobytes())
    h.update(np.ascontiguousarray(syndromes[-4096:]).tobytes())
    return h.hexdigest()


class Progress:
    """The progress record of one job: its configuration and the number of
    syndromes whose results are stored."""

    def __init__(self, path: str, config: dict):
        self.path = path
        self.config = dict(config)
        self.done = 0

    def load(self) -> bool:
        """Read an existing record. Returns False if there is none; raises
        ValueError if it belongs to another configuration."""
        if not os.path.exists(self.path):
            return False
        with open(self.path) as f:
            rec = json.load(f)
        if rec.get("version") != PROGRESS_VERSION or rec.get("config") != self.config:
            raise ValueError(f"{self.path} records another job: {rec.get('config')} != {self.config}")
        done = int(rec.get("done", 0))
        if not 0 <= done <= int(self.config["B"]):
            raise ValueError(f"{self.path}: completed count {done} outside [0, {self.config['B']}]")
        self.done = done
        return True

    def save(self, done: int) -> None:
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"version": PROGRESS_VERSION, "config": self.config, "done": int(done)}, f)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, self.path)
        self.done = int(done)


def _open_outputs(prefix: str, B: int, fresh: bool):
    mode = "w+" if fresh else "r+"
    logp = np.lib.format.open_memmap(prefix + ".logp.npy", mode=mode, dtype=np.float64, shape=(B, 4))
    am = np.lib.format.open_memmap(prefix + ".argmax.npy", mode=mode, dtype=np.uint8, shape=(B,))
    return logp, am


def decode_to_files(code, noise, syndromes: np.ndarray, chi: int, prefix: str, chunk: int = 1 << 18,
                    precision: int = MLD_FP32, noise_mode: int = MLD_NOISE_TABLE, resume: bool = True,
                    on_chunk=None):
    """Decode every row of ``syndromes`` (host uint64 [B][words], an ndarray or
    a memory map) into ``<prefix>.logp.npy`` and ``<prefix>.argmax.npy``.

    noise: a CUDA tensor [n][4] for MLD_NOISE_TABLE, or a host float32 array
    [B] of per-syndrome depolarizing strengths for MLD_NOISE_DEPOL (copied per
    chunk with the syndromes). With ``resume`` an existing progress record of
    the same job is continued; otherwise the job starts over. ``on_chunk(start,
    count)`` is called after each chunk's results and progress are stored.
    Returns the two result memory maps."""
    syndromes = np.asarray(syndromes) if not isinstance(syndromes, np.memmap) else syndromes
    if syndromes.ndim != 2 or syndromes.dtype not in (np.uint64, np.int64):
        raise ValueError("syndromes must be a uint64 array [B][words]")
    B, words = int(syndromes.shape[0]), int(syndromes.shape[1])
    if words != code.words:
        raise ValueError(f"{words} syndrome words per row, the code has {code.words}")
    if chunk < 1:
        raise ValueError("chunk must be positive")
    if noise_mode == MLD_NOISE_DEPOL:
        noise = np.ascontiguousarray(noise, dtype=np.float32)
        if noise.shape != (B,):
            raise ValueError("per-syndrome noise must be a float32 array [B]")
    elif noise_mode != MLD_NOISE_TABLE:
        raise ValueError("unknown noise mode")
    config = {"d": int(code.d), "chi": int(chi), "precision": int(precision), "noise_mode": int(noise_mode),
              "B": B, "words": words, "syndromes_sha1": fingerprint(syndromes)}
    prog = Progress(prefix + ".progress.json", config)
    have = resume and prog.load()
    logp, am = _open_outputs(prefix, B, fresh=not have)
    if not have:
        prog.save(0)
    start0 = prog.done
    if start0 >= B:
        return logp, am

    def launch(dsyn, dnoise, n, out_lp, out_am, stream):
        nz = dnoise if noise_mode == MLD_NOISE_DEPOL else noise
        mld_decode(code.handle, nz, noise_mode, dsyn, n, chi, precision, out_lp, out_am, stream)

    return _run_chunks(code, syndromes, words, chunk, prog, logp, am, launch,
                       noise if noise_mode == MLD_NOISE_DEPOL else None, on_chunk)


def decode_xz_to_files(code, px, pz, syndromes: np.ndarray, prefix: str, chunk: int = 1 << 18,
                       precision: int = MLD_FP32, resume: bool = True, on_chunk=None):
    """The same for the Kac-Ward decode under independent X/Z noise
    (``mld_decode_xz``): px, pz are CUDA float32 tensors [n] (pz None for
    bit-flip noise). The progress record also holds the method and a
    fingerprint of the rates, so a job resumed with other rates is refused."""
    syndromes = np.asarray(syndromes) if not isinstance(syndromes, np.memmap) else syndromes
    if syndromes.ndim != 2 or syndromes.dtype not in (np.uint64, np.int64):
        raise ValueError("syndromes must be a uint64 array [B][words]")
    B, words = int(syndromes.shape[0]), int(syndromes.shape[1])
    if words != code.words:
        raise ValueError(f"{words} syndrome words per row, the code has {code.words}")
    if chunk < 1:
        raise ValueError("chunk must be positive")
    h = hashlib.sha1(px.detach().cpu().numpy().tobytes())
    if pz is not None:
        h.update(pz.detach().cpu().numpy().tobytes())
    config = {"method": "kac-ward", "d": int(code.d), "precision": int(precision), "bitflip": pz is None,
              "rates_sha1": h.hexdigest(), "B": B, "words": words, "syndromes_sha1": fingerprint(syndromes)}
    prog = Progress(prefix + ".progress.json", config)
    have = resume and prog.load()
    logp, am = _open_outputs(prefix, B, fresh=not have)
    if not have:
        prog.save(0)
    if prog.done >= B:
        return logp, am
    pxc = px.contiguous()
    pzc = None if pz is None else pz.contiguous()

    def launch(dsyn, dnoise, n, out_lp, out_am, stream):
        mld_decode_xz(code.handle, pxc, pzc, dsyn, n, precision, out_lp, out_am, stream)

    return _run_chunks(code, syndromes, words, chunk, prog, logp, am, launch, None, on_chunk)


def _run_chunks(code, syndromes, words, chunk, prog, logp, am, launch, per_syn, on_chunk):
    """The chunk loop shared by both decoders: rows prog.done.. of
    ``syndromes`` in chunks, the next chunk's host-to-device copy (and its
    per-syndrome noise ``per_syn``, if any) overlapping the current decode,
    ``launch(dsyn, dnoise, n, out_logP, out_argmax, stream)`` per chunk, the
    results and the progress record stored after each."""
    import torch

    B = int(syndromes.shape[0])
    start0 = prog.done
    dev = torch.device("cuda", torch.cuda.current_device())
    n_max = min(chunk, B - start0)
    stage = [torch.empty((n_max, words), dtype=torch.int64).pin_memory() for _ in range(2)]
    dsyn = [torch.empty((n_max, words), dtype=torch.int64, device=dev) for _ in range(2)]
    if per_syn is not None:
        nstage = [torch.empty((n_max,), dtype=torch.float32).pin_memory() for _ in range(2)]
        dnoise = [torch.empty((n_max,), dtype=torch.float32, device=dev) for _ in range(2)]
    out_lp = torch.empty((n_max, 4), dtype=torch.float64, device=dev)
    out_am = torch.empty((n_max,), dtype=torch.uint8, device=dev)
    host_lp = torch.empty((n_max, 4), dtype=torch.float64).pin_memory()
    host_am = torch.empty((n_max,), dtype=torch.uint8).pin_memory()
    copy_s = torch.cuda.Stream(device=dev)
    comp_s = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    starts = list(range(start0, B, chunk))

    def prefetch(k):
        s0 = starts[k]
        n = min(chunk, B - s0)
        j = k & 1
        stage[j][:n].numpy()[:] = syndromes[s0:s0 + n].view(np.int64)
        if per_syn is not None:
            nstage[j][:n].numpy()[:] = per_syn[s0:s0 + n]
        with torch.cuda.stream(copy_s):
            dsyn[j][:n].copy_(stage[j][:n], non_blocking=True)
            if per_syn is not None:
                dnoise[j][:n].copy_(nstage[j][:n], non_blocking=True)
            copied[j].record(copy_s)

    prefetch(0)
    for k, s0 in enumerate(starts):
        n = min(chunk, B - s0)
        j = k & 1
        comp_s.wait_event(copied[j])
        launch(dsyn[j], dnoise[j] if per_syn is not None else None, n, out_lp, out_am, comp_s.cuda_stream)
        with torch.cuda.stream(comp_s):
            host_lp[:n].copy_(out_lp[:n], non_blocking=True)
            host_am[:n].copy_(out_am[:n], non_blocking=True)
        if k + 1 < len(starts):
            # the other staging buffer's last copy (chunk k-1) finished before
            # chunk k-1 was decoded, which the previous iteration waited for
            prefetch(k + 1)
        comp_s.synchronize()
        st = code.status()
        if st != 0:
            raise MldError(st, f"device status after the chunk at {s0}")
        logp[s0:s0 + n] = host_lp[:n].numpy()
        am[s0:s0 + n] = host_am[:n].numpy()
        logp.flush()
        am.flush()
        prog.save(s0 + n)
        if on_chunk is not None:
            on_chunk(s0, n)
    return logp, am
