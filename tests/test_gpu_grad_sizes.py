"""Gradient parity at the benchmarked sizes: the adjoint (fram_synthesize_backward) and the
gradient through the sampler (fram_sample_backward) run on the whole 4096-room 48 kHz batch,
the 1024-room batch with early-RIR upstream gradients and the 256-room batch, in the launch
configuration the benchmark times, and are compared on seeded samples of rooms (always
including the shortest- and longest-T60 rooms) with the FP64 oracle's analytic gradients.

The oracle draws its own images from the same seed (room_ids = the rooms' batch indices) and
gets the same float32 upstream gradients; nothing it receives comes from the GPU's outputs.
Bar: max error <= 1e-5 of the largest magnitude of that gradient (per room for image and mic
gradients, over the compared rooms for source and r gradients).
"""
import numpy as np
import pytest
import torch

from paper_2304_08052_gb300 import api, scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rooms(sc, n, seed):
    rng = np.random.default_rng(seed)
    pick = {int(np.argmin(sc.rt60)), int(np.argmax(sc.rt60))}
    while len(pick) < n:
        pick.add(int(rng.integers(sc.B)))
    return sorted(pick)


def _slices(ds, rooms):
    """Concatenated RIR-sample and image-row index arrays of `rooms` (the subset's layout)."""
    rir = np.concatenate([np.arange(int(ds.rir_off[b]), int(ds.rir_off[b + 1])) for b in rooms])
    img = np.concatenate([np.arange(int(ds.vs_off[b]), int(ds.vs_off[b + 1])) for b in rooms])
    return rir, img


def _rel_rows(got, want, offs):
    errs = []
    for a, b in zip(offs[:-1], offs[1:]):
        if b > a:
            errs.append(np.abs(got[a:b] - want[a:b]).max() / max(np.abs(want[a:b]).max(), 1e-300))
    return max(errs)


def _adjoint_vs_oracle(oracle_mod, sc, seed, n_rooms, early, tile=0):
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len, tile=tile))
    vs = api.sample(ds, seed=seed)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    G = torch.empty(ds.rir_total, device="cuda").normal_(generator=gen)
    Ge = torch.empty(ds.rir_total, device="cuda").normal_(generator=gen) if early else None
    gv, gm, gs, gr = api.synthesize_backward_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, G, Ge)
    torch.cuda.synchronize()
    assert ds.status() == 0
    rooms = _rooms(sc, n_rooms, seed)
    rir_idx, img_idx = _slices(ds, rooms)
    ri = torch.as_tensor(rir_idx, device="cuda")
    G_sub = G[ri].double().cpu().numpy()
    Ge_sub = Ge[ri].double().cpu().numpy() if early else None
    ii = torch.as_tensor(img_idx, device="cuda")
    got_v = gv[ii].double().cpu().numpy()
    rt = torch.as_tensor(rooms, device="cuda")
    got_m, got_s, got_r = (t[rt].double().cpu().numpy() for t in (gm, gs, gr))
    del G, Ge, gv
    sub = sc.subset(rooms)
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sub, op, seed, room_ids=rooms)
    rv, rm, rs, rr = oracle_mod.backward(sub, op, ref.pos, ref.g, ref.r, G_sub, Ge_sub)
    _, _, vs_off = oracle_mod.layout(sub.rt60, sub.n_vs, sub.S, sub.M, sub.fs)
    return {"vs": _rel_rows(got_v, rv, vs_off),
            "mic": max(np.abs(got_m[k] - rm[k]).max() / np.abs(rm[k]).max() for k in range(len(rooms))),
            "src": np.abs(got_s - rs).max() / np.abs(rs).max(),
            "r": np.abs(got_r - rr).max() / np.abs(rr).max()}


def test_adjoint_large_4096_sampled_rooms(oracle_mod):
    # tile 2048: the length the benchmark's tuner picks on GB300
    e = _adjoint_vs_oracle(oracle_mod, scenes.large_4096(0), 1001, 8, early=False, tile=2048)
    torch.cuda.empty_cache()
    assert max(e.values()) < TOL, e


def test_adjoint_batch_1024_with_early_rir_gradient_sampled_rooms(oracle_mod):
    e = _adjoint_vs_oracle(oracle_mod, scenes.batch_1024(0), 503, 8, early=True)
    assert max(e.values()) < TOL, e


def test_adjoint_batch_256_sampled_rooms(oracle_mod):
    e = _adjoint_vs_oracle(oracle_mod, scenes.batch_256(0), 17, 8, early=False)
    assert max(e.values()) < TOL, e


def test_sampler_adjoint_large_4096_sampled_rooms(oracle_mod):
    # fram_sample_backward over the whole batch; the compared rooms get the oracle's own synthesis
    # adjoint (float32) as upstream gradients, every other room gets zeros.
    sc = scenes.large_4096(0)
    seed = 1003
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len))
    rooms = _rooms(sc, 6, seed)
    sub = sc.subset(rooms)
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sub, op, seed, room_ids=rooms)
    _, rir_off, vs_off = oracle_mod.layout(sub.rt60, sub.n_vs, sub.S, sub.M, sub.fs)
    G = np.random.default_rng(seed).standard_normal(int(rir_off[-1]))
    up = [x.astype(np.float32) for x in oracle_mod.backward(sub, op, ref.pos, ref.g, ref.r, G, with_g=True)]
    uv, um, us, ur, ug = up
    N = ds.n_vs_total
    gv = torch.zeros((N, 3), device="cuda")
    gg = torch.zeros(N, device="cuda")
    gr = torch.zeros(sc.B, device="cuda")
    gs = torch.zeros((sc.B, sc.S, 3), device="cuda")
    gm = torch.zeros((sc.B, sc.M, 3), device="cuda")
    _, img_idx = _slices(ds, rooms)
    ii = torch.as_tensor(img_idx, device="cuda")
    rt = torch.as_tensor(rooms, device="cuda")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gv[ii] = dev(uv)
    gg[ii] = dev(ug)
    gr[rt] = dev(ur)
    gs[rt] = dev(us)
    gm[rt] = dev(um)
    out = api.sample_backward(ds, seed, gv, gg, gr, gs, gm)
    torch.cuda.synchronize()
    assert ds.status() == 0
    got = [t[rt].double().cpu().numpy() for t in out]
    want = oracle_mod.sample_backward(sub, op, seed, *(x.astype(np.float64) for x in (uv, ug, ur, us, um)),
                                      room_ids=rooms)
    for g_, w_, what in zip(got, want, ("src", "mic", "t60", "dims")):
        e = np.abs(g_ - w_).max() / max(np.abs(w_).max(), 1e-300)
        assert e <= TOL, (what, e)
