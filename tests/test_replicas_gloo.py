"""Replica sharding across processes (one process per GPU in production): host logic tested with
two gloo ranks on CPU.  Walker ids are disjoint per rank and the accumulator reduction over
ranks equals the single-process reduction of the concatenated walkers."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1312_1282_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fake_accum(rank, W):
    g = torch.Generator().manual_seed(100 + rank)
    a = torch.zeros(W, 8, dtype=torch.float64)
    a[:, 6] = 40.0
    a[:, 0] = -5.8 * 64 * 40 + torch.randn(W, generator=g, dtype=torch.float64) * 20
    a[:, 2] = -21.0 * 64 * 40
    a[:, 3] = 15.2 * 64 * 40
    a[:, 4] = 15.1 * 64 * 40
    a[:, 5] = 15.0 * 64 * 40
    a[:, 7] = 1000.0 + rank
    return a


def _worker(rank, world, port, W, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ids = replicas.walker_ids(rank, world, W)
        gathered = [None] * world
        dist.all_gather_object(gathered, ids)
        stats = replicas.block_stats(_fake_accum(rank, W), 64)
        out[rank] = (gathered, stats)
    finally:
        dist.destroy_process_group()


def test_two_ranks_disjoint_ids_and_reduction():
    world, W = 2, 6
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, W, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    gathered, s0 = out[0]
    _, s1 = out[1]
    all_ids = sum(gathered, [])
    assert len(set(all_ids)) == world * W
    assert s0 == s1  # every rank sees the same totals
    ref = replicas.block_stats(torch.cat([_fake_accum(r, W) for r in range(world)]), 64)
    for k in ref:
        assert s0[k] == pytest.approx(ref[k], rel=1e-12)


def test_walker_ids_reject_bad_ranks():
    with pytest.raises(ValueError):
        replicas.walker_ids(2, 2, 4)
    assert replicas.walker_ids(1, 3, 4) == [4, 5, 6, 7]
