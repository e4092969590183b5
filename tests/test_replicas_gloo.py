"""Multi-GPU form of the bench: independent replicas, one instance per rank,
no collective on the data path; the only cross-rank step is the maximum of
the timings (the slowest replica sets the job's time).  Checked here with two
gloo ranks on CPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank timings: the reduction must return the maximum of each
        got = bench.reduce_max_over_ranks([1.0 + rank, 10.0 * (rank + 1), 0.5], world)
        # each replica solves its own instance: the generators are seeded by rank
        p = synth.maxcut_grid_instance(R=4, K=5, instance=rank)
        sig = float(np.sum(p.C_val * np.arange(1, p.C_val.size + 1)))
        sigs = [None] * world
        dist.all_gather_object(sigs, sig)
        out[rank] = (got, sigs)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        got, sigs = out[r]
        assert got == [2.0, 20.0, 0.5]
        assert sigs[0] != sigs[1], "the two replicas were given the same instance"
    # whole-job throughput: every rank's units over the slowest rank's time
    assert bench.replica_throughput(world, 100, 0.5) == pytest.approx(400.0)


def test_single_rank_is_identity():
    assert bench.reduce_max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
