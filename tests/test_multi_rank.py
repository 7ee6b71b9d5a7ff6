"""Multi-process logic of bench.py on CPU (gloo, world size 2).

On N GPUs every rank synthesises its own full batch from its own seed (weak scaling: rooms are
independent, no collective on the data path); the only collective is the max-reduction of the
elapsed time, and the whole-job value is all ranks' units over the slowest rank's time.  These
tests run those pieces as two gloo ranks on the host.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2304_08052_gb300 import scenes


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_s = 1.5 + rank                      # rank 1 is the slow one
        t = bench.max_over_ranks(torch, local_s, "cpu")
        seed = bench.rank_scene_seed(0, rank)
        sc = scenes.by_name("batch_256", seed)
        units = sc.B * sc.S
        value = bench.combine([units] * world, [t] * world)
        # Gather every rank's first room so rank 0 can check that the batches differ.
        mine = torch.tensor(np.concatenate([sc.dims[0], sc.src[0, 0], [sc.rt60[0]]]), dtype=torch.float64)
        allv = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(allv, mine)
        out[rank] = (t, seed, value, units, [v.tolist() for v in allv])
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        return dict(out)


def test_time_is_the_slowest_rank(two_ranks):
    assert two_ranks[0][0] == two_ranks[1][0] == 2.5


def test_ranks_draw_independent_batches(two_ranks):
    assert two_ranks[0][1] != two_ranks[1][1]
    first_rooms = two_ranks[0][4]
    assert first_rooms == two_ranks[1][4]              # both ranks saw the same gathered list
    assert not np.allclose(first_rooms[0], first_rooms[1])


def test_whole_job_value_sums_units_over_the_max_time(two_ranks):
    t, _, value, units, _ = two_ranks[0]
    assert value == pytest.approx(2 * units / t)
    assert two_ranks[1][2] == pytest.approx(value)


def test_rank_seeds_are_distinct_for_many_ranks():
    seeds = {bench.rank_scene_seed(0, r) for r in range(64)}
    assert len(seeds) == 64
