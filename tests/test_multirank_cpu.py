"""Multi-rank host logic on CPU with the gloo backend (world size 2): the
instance sharding of a batched sweep (no data-path collective) and the
max-over-ranks timing reduction of bench.py."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import lbm_cases as C


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cases = C.batched_sweep(96)
    cells = [c.cells for c in cases]
    mine = C.shard_instances(cells, world, rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = bench.max_over_ranks(1.0 + rank, world)
    out[rank] = (gathered, t, sum(cells[i] for i in mine))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_sweep_and_max_timing_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    g0, t0, load0 = out[0]
    g1, t1, load1 = out[1]
    assert g0 == g1
    a, b = g0
    assert set(a).isdisjoint(b) and sorted(a + b) == list(range(96))
    # max over ranks, as in the bench's timed region
    assert t0 == t1 == 2.0
    cells = [c.cells for c in C.batched_sweep(96)]
    assert abs(load0 - load1) <= max(cells)


def test_shard_instances_single_rank_and_errors():
    cells = [5, 3, 8, 1]
    assert C.shard_instances(cells, 1, 0) == [0, 1, 2, 3]
    with pytest.raises(ValueError):
        C.shard_instances(cells, 2, 2)
