"""Data-parallel sharding of a syndrome batch over ranks (one process per GPU).

Every (syndrome, class) contraction is independent, so the forward path has no
exchange step: rank r decodes the contiguous block ``shard_range(B, r, world)``
of the batch and the blocks are concatenated in rank order. The only reductions
are the sum of the adjoint's noise gradient (it is a sum over syndromes) and
the maximum of the per-rank step times.

``decode_sharded`` gathers results on rank 0 through the rendezvous store (host
bytes, no device collective), so a rank that raises or never reports does not
stall the others: rank 0 waits a bounded time for each block and decodes a
missing block itself. Nothing here computes any part of the decode; the
caller passes the function that does (the CUDA path in production).
"""
from __future__ import annotations

import pickle
import time
from typing import Callable, Optional

import numpy as np


def shard_range(B: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous block of a batch of B (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or B < 0:
        raise ValueError(f"bad shard request B={B} rank={rank} world={world}")
    return B * rank // world, B * (rank + 1) // world


def allreduce_sum(t, group=None):
    """Sum a tensor over ranks in place (the adjoint's noise gradient)."""
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def max_over_ranks(x: float, device=None, group=None) -> float:
    """Maximum of a host scalar over ranks (the timing rule of a weak-scaling step)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_initialized() and dist.get_world_size(group) > 1):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def decode_sharded(decode_block: Callable[[int, int], np.ndarray], B: int, rank: int, world: int, store,
                   key: str = "mld", timeout_s: float = 30.0, poll_s: float = 0.01):
    """Decode a batch of B split over ranks; rank 0 returns the whole result.

    decode_block(lo, hi) returns the rows [lo, hi) of the result (any numpy
    array with hi - lo rows). Each rank decodes its own block and posts it
    under ``key/res/<rank>`` in ``store`` (a torch.distributed Store); a block
    that fails posts ``key/fail/<rank>`` instead. Rank 0 waits up to
    ``timeout_s`` per block, then decodes any failed or missing block itself.

    Returns (result, retried_ranks) on rank 0 and (None, []) on the others.
    """
    lo, hi = shard_range(B, rank, world)
    try:
        mine = np.ascontiguousarray(decode_block(lo, hi))
        if rank != 0:
            store.set(f"{key}/res/{rank}", pickle.dumps(mine, protocol=pickle.HIGHEST_PROTOCOL))
    except Exception as e:                      # report, never leave rank 0 waiting for nothing
        mine = None
        if rank != 0:
            store.set(f"{key}/fail/{rank}", repr(e).encode())
        else:
            raise
    if rank != 0:
        return None, []
    parts, retried = [mine], []
    for r in range(1, world):
        res, fail = f"{key}/res/{r}", f"{key}/fail/{r}"
        deadline = time.monotonic() + timeout_s
        got = None
        while time.monotonic() < deadline:
            if store.check([res]):
                got = pickle.loads(store.get(res))
                break
            if store.check([fail]):
                break
            time.sleep(poll_s)
        if got is None:                          # failed or silent: decode that block here
            rlo, rhi = shard_range(B, r, world)
            got = np.ascontiguousarray(decode_block(rlo, rhi))
            retried.append(r)
        parts.append(got)
    return np.concatenate(parts, axis=0), retried


def local_store_rank_barrier(store, key: str, rank: int, world: int, timeout_s: float = 30.0,
                             poll_s: float = 0.01) -> list[int]:
    """Host-side check-in through the store: returns the ranks that did not
    check in within timeout_s (a rank learns of a departed peer before its
    next launch instead of inside a collective)."""
    store.set(f"{key}/alive/{rank}", b"1")
    deadline = time.monotonic() + timeout_s
    missing = list(range(world))
    while time.monotonic() < deadline:
        missing = [r for r in range(world) if not store.check([f"{key}/alive/{r}"])]
        if not missing:
            break
        time.sleep(poll_s)
    return missing
