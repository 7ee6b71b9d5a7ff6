"""Room shards on the GPU: sampling and synthesising rooms [k, k + n) of a batch with
room_base = k gives, bit for bit, the Philox words, image positions, reflection counts,
coefficients, RIRs, early RIRs and adjoint gradients that the whole-batch call gives those rooms
(the Philox counter carries the global room index, and every per-room computation depends only on
that room's inputs).  This is what lets rooms be split across GPUs with no data exchanged.
"""
import numpy as np
import pytest
import torch

from paper_2304_08052_gb300 import api, scenes, shard

pytestmark = pytest.mark.gpu


def _run(sc, base, seed, G=None, early=False):
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len), room_base=base)
    vs = api.sample(ds, seed=seed, words=True)
    out = api.synthesize(ds, vs, early=early)
    grads = None
    if G is not None:
        grads = api.synthesize_backward_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, G)
    torch.cuda.synchronize()
    assert ds.status() == 0
    return ds, vs, out, grads


def _check_rows(ds_full, ds_part, lo, hi, full, part):
    a, b = int(ds_full.vs_off[lo]), int(ds_full.vs_off[hi])
    vs_f, out_f = full[1], full[2]
    vs_p, out_p = part[1], part[2]
    assert torch.equal(vs_p.words, vs_f.words[a:b])
    assert torch.equal(vs_p.pos_hi, vs_f.pos_hi[a:b]) and torch.equal(vs_p.pos_lo, vs_f.pos_lo[a:b])
    assert torch.equal(vs_p.g, vs_f.g[a:b]) and torch.equal(vs_p.r, vs_f.r[lo:hi])
    o0, o1 = int(ds_full.rir_off[lo]), int(ds_full.rir_off[hi])
    outs_f = out_f if isinstance(out_f, tuple) else (out_f,)
    outs_p = out_p if isinstance(out_p, tuple) else (out_p,)
    for f, p in zip(outs_f, outs_p):
        assert torch.equal(p, f[o0:o1])


def test_shard_of_batch_256_equals_its_rows(oracle_mod):
    sc = scenes.batch_256(0)
    rng = np.random.default_rng(3)
    full = _run(sc, 0, seed=9)
    G = torch.as_tensor(rng.normal(size=full[0].rir_total).astype(np.float32), device="cuda")
    full = _run(sc, 0, seed=9, G=G, early=True)
    for lo, hi in ((0, 17), (100, 101), (131, 256)):
        sub = sc.subset(range(lo, hi))
        o0, o1 = int(full[0].rir_off[lo]), int(full[0].rir_off[hi])
        part = _run(sub, lo, seed=9, G=G[o0:o1].contiguous(), early=True)
        _check_rows(full[0], part[0], lo, hi, full, part)
        a, b = int(full[0].vs_off[lo]), int(full[0].vs_off[hi])
        gv_f, gm_f, gs_f, gr_f = full[3]
        gv_p, gm_p, gs_p, gr_p = part[3]
        assert torch.equal(gv_p, gv_f[a:b]) and torch.equal(gm_p, gm_f[lo:hi])
        assert torch.equal(gs_p, gs_f[lo:hi]) and torch.equal(gr_p, gr_f[lo:hi])


def test_partitioned_large_4096_equals_the_whole_batch():
    # The benchmark's sharding of the 4096-room, 48 kHz workload over 4 ranks, run one shard at
    # a time on one GPU: every shard's images and RIRs equal the whole batch's rows.
    sc = scenes.large_4096(0)
    full = _run(sc, 0, seed=1001)
    ranges = shard.partition(shard.room_costs(sc, sc.half_len), 4)
    for lo, hi in ranges:
        part = _run(sc.subset(range(lo, hi)), lo, seed=1001)
        _check_rows(full[0], part[0], lo, hi, full, part)
        del part
    torch.cuda.empty_cache()


def test_shard_matches_the_oracle_with_global_room_ids(oracle_mod):
    sc = scenes.grad_64(0)
    lo, hi = 40, 44
    sub = sc.subset(range(lo, hi))
    ds, vs, h, _ = _run(sub, lo, seed=5)
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sub, op, 5, room_ids=list(range(lo, hi)))
    assert np.array_equal(vs.words.cpu().numpy().view(np.uint32), ref.words)
    h_ref = oracle_mod.synthesize(sub, op, ref.pos, ref.g, ref.r)
    got = h.cpu().numpy().astype(np.float64)
    for b in range(sub.B):
        o, L = int(ds.rir_off[b]), int(ds.rir_len[b]) * sub.S * sub.M
        peak = np.abs(h_ref[o:o + L]).max()
        assert np.abs(got[o:o + L] - h_ref[o:o + L]).max() <= 1e-5 * peak
