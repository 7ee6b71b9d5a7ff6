"""Multi-process logic of bench.py and of the room sharding on CPU (gloo, world size 2).

On N GPUs one batch of rooms (N seeded blocks of the workload) is split into contiguous,
cost-balanced room ranges, one per rank (paper_2304_08052_gb300/shard.py).  Every rank draws
its rooms' images with their global room index, so a shard's rows equal those of the whole
batch and no data moves between ranks; the only collectives are the timing barrier and the
max-reduction of the elapsed time.  These tests run those pieces as two gloo ranks on the host:
  * the job time is the slowest rank's time, and the job value all units over that time;
  * the partition covers every room exactly once within its stated cost bound;
  * the FP64 oracle run on each rank's shard (room_ids = global indices) equals, bit for bit,
    the same rooms of the oracle run on the whole batch.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2304_08052_gb300 import scenes, shard


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _block(name, seed):
    # a small workload block: 3 rooms, 2 sources, 3 mics, 40 images each, RIRs of 0.05-0.12 s
    return scenes.tiny(seed=seed, B=3, S=2, M=3, images=40)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        local_s = 1.5 + rank                      # rank 1 is the slow one
        t = bench.max_over_ranks(torch, local_s, "cpu")
        glob = shard.global_batch(_block, "tiny", world)
        ranges = shard.partition(shard.room_costs(glob, glob.half_len), world)
        lo, hi = ranges[rank]
        sub = glob.subset(range(lo, hi))
        op = oracle.Params(fs=sub.fs, half_len=sub.half_len)
        ref = oracle.sample(sub, op, 11, room_ids=list(range(lo, hi)))
        h = oracle.synthesize(sub, op, ref.pos, ref.g, ref.r)
        value = bench.combine([sub.B * sub.S] * world, [t] * world)
        gathered = [None] * world
        dist.all_gather_object(gathered, (lo, hi, ref.words, ref.pos, h))
        out[rank] = (t, value, sub.B * sub.S, ranges, gathered if rank == 0 else None)
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


def test_whole_job_value_sums_units_over_the_max_time(two_ranks):
    t, value, units, _, _ = two_ranks[0]
    assert value == pytest.approx(2 * units / t)


def test_ranks_agree_on_the_partition(two_ranks):
    assert two_ranks[0][3] == two_ranks[1][3]
    (lo0, hi0), (lo1, hi1) = two_ranks[0][3]
    assert lo0 == 0 and hi0 == lo1 and hi1 == 6 and hi0 > 0 and hi1 > hi0


def test_shards_equal_the_whole_batch_on_the_oracle(oracle_mod, two_ranks):
    glob = shard.global_batch(_block, "tiny", 2)
    op = oracle_mod.Params(fs=glob.fs, half_len=glob.half_len)
    ref = oracle_mod.sample(glob, op, 11)
    h = oracle_mod.synthesize(glob, op, ref.pos, ref.g, ref.r)
    rir_len, rir_off, vs_off = oracle_mod.layout(glob.rt60, glob.n_vs, glob.S, glob.M, glob.fs)
    for lo, hi, words, pos, hs in two_ranks[0][4]:
        a, b = int(vs_off[lo]), int(vs_off[hi])
        assert np.array_equal(words, ref.words[a:b])
        assert np.array_equal(pos, ref.pos[a:b])
        assert np.array_equal(hs, h[int(rir_off[lo]):int(rir_off[hi])])


@pytest.mark.parametrize("world", [1, 2, 3, 8, 64])
def test_partition_covers_every_room_once_within_the_bound(world):
    sc = scenes.large_4096(0).subset(range(500))
    costs = shard.room_costs(sc, sc.half_len)
    ranges = shard.partition(costs, world)
    assert len(ranges) == world
    assert ranges[0][0] == 0 and ranges[-1][1] == sc.B
    for (a, b), (c, _) in zip(ranges, ranges[1:]):
        assert b == c and a <= b
    bound = shard.imbalance_bound(costs, world)
    assert max(costs[a:b].sum() for a, b in ranges) <= bound * (1 + 1e-12)


def test_room_costs_follow_taps_and_samples():
    sc = scenes.batch_256(0).subset(range(4))
    c = shard.room_costs(sc, 40)
    L = np.ceil(sc.rt60.astype(np.float64) * sc.fs)
    want = sc.S * sc.M * ((sc.n_vs.astype(np.float64) + 1) * 81 + L)
    assert np.array_equal(c, want)
