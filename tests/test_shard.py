"""Multi-rank host logic of the sharded decode (CPU, gloo, world size 2).

The per-block decode in these tests is the FP64 oracle, so what is checked is
the sharding itself: the split, the merge (bit-identical to one process), the
gradient sum, the timing reduction, and the recovery of a block whose rank
raised or never reported.
"""
import os
import socket
import sys
from datetime import timedelta

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2605_17230_gb300 import shard  # noqa: E402

D, P, B = 5, 0.12, 96


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs():
    noise = synth.depolarizing(D * D, P)
    E = synth.sample_errors(D, noise, B, seed=synth.config_seed(7, D, P))
    return noise, synth.syndromes_of(D, E)


def _worker(rank, world, port, scenario):
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=timedelta(seconds=60))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world, timeout=timedelta(seconds=60))
    try:
        noise, syn = _inputs()

        def block(lo, hi):
            if scenario == "raise" and rank == 1:
                raise RuntimeError("planted failure of rank 1's block")
            lp, am = oracle.decode(D, noise, syn[lo:hi], threads=1)
            return np.concatenate([lp, am[:, None].astype(np.float64)], axis=1)

        if scenario in ("merge", "raise"):
            out, retried = shard.decode_sharded(block, B, rank, world, store, key=scenario, timeout_s=30)
            if rank == 0:
                lp, am = oracle.decode(D, noise, syn, threads=1)
                assert out.shape == (B, 5)
                assert np.array_equal(out[:, :4], lp)                   # bit-identical merge
                assert np.array_equal(out[:, 4].astype(np.uint8), am)
                assert retried == ([1] if scenario == "raise" else [])
        elif scenario == "silent":
            if rank == 1:
                return                                                 # leaves before its block
            out, retried = shard.decode_sharded(block, B, rank, world, store, key="silent", timeout_s=1.0)
            lp, _ = oracle.decode(D, noise, syn, threads=1)
            assert retried == [1] and np.array_equal(out[:, :4], lp)
        elif scenario == "grad":
            lo, hi = shard.shard_range(B, rank, world)
            reps = oracle.representatives(D, syn[lo:hi])[:, 0]
            _, g = oracle.coset_dlogz(D, noise, reps, threads=1)
            t = torch.tensor(g.sum(axis=0))
            shard.allreduce_sum(t)
            _, gf = oracle.coset_dlogz(D, noise, oracle.representatives(D, syn)[:, 0], threads=1)
            np.testing.assert_allclose(t.numpy(), gf.sum(axis=0), rtol=1e-12, atol=1e-12)
            tmax = shard.max_over_ranks(1.5 + rank)
            assert tmax == 1.5 + world - 1
        elif scenario == "checkin":
            if rank == 1:
                return
            missing = shard.local_store_rank_barrier(store, "ci", rank, world, timeout_s=1.0)
            assert missing == [1]
    finally:
        if not (scenario in ("silent", "checkin") and rank == 1):
            dist.destroy_process_group()


@pytest.fixture(scope="module", autouse=True)
def _built_oracle():
    oracle.build()


def test_shard_range_partition():
    for Bt in (0, 1, 5, 96, 65536, 1 << 20):
        for world in (1, 2, 3, 4, 8):
            ranges = [shard.shard_range(Bt, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == Bt
            for (a, b), (c, _) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


@pytest.mark.parametrize("scenario", ["merge", "raise", "silent", "grad", "checkin"])
def test_two_ranks(scenario):
    mp.start_processes(_worker, args=(2, _free_port(), scenario), nprocs=2, join=True, start_method="spawn")
