"""GPU: the tile autotuner, and the FP32 gradient against FP64 central finite differences.

The gradient workload is the 64-room, 4-mic, 1500-image scene at 16 kHz with loss
L = sum (h - y)^2 against a seeded Gaussian target y.  The GPU gradient comes from the autograd
Function (fram_synthesize_backward); the finite differences come from the FP64 oracle's own
images and forward synthesis with steps of 1e-6 m on positions and 1e-7 (relative) on r, one
room at a time (the loss separates over rooms).
"""
import numpy as np
import pytest
import torch

from paper_2304_08052_gb300 import api, scenes

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_and_auto_tile_uses_it(oracle_mod):
    sc = scenes.tiny(seed=31, B=6, S=2, M=4, images=900, t60_lo=0.3, t60_hi=0.6)
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len, tile=0))
    vs = api.sample(ds, seed=2)
    tile = api.autotune(ds, vs)
    assert tile in (256, 512, 1024, 2048)
    auto = api.synthesize(ds, vs).clone()
    ds_fix = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len, tile=tile))
    fixed = api.synthesize(ds_fix, vs)
    torch.cuda.synchronize()
    assert ds.status() == 0
    assert torch.equal(auto, fixed)


def _room_loss(oracle_mod, sc_room, op, pos, g, r, y):
    h = oracle_mod.synthesize(sc_room, op, pos, g, r)
    return float(np.sum((h - y) ** 2))


def test_gradients_match_fp64_finite_differences(oracle_mod):
    sc = scenes.grad_64(0)
    params = api.Params(fs=sc.fs, half_len=sc.half_len)
    ds = api.DeviceScene(sc, params)
    vs = api.sample(ds, seed=11)
    rng = np.random.default_rng(11)
    y = rng.normal(size=ds.rir_total).astype(np.float32)
    src = ds.src.clone().requires_grad_()
    mic = ds.mic.clone().requires_grad_()
    pos = vs.pos_hi.clone().requires_grad_()
    r = vs.r.clone().requires_grad_()
    h = api.rir(ds, src, mic, pos, r, vs.g, vs.pos_lo)
    loss = ((h - torch.as_tensor(y, device="cuda")) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    assert ds.status() == 0

    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sc, op, 11)
    step = 1e-6
    for b in (0, 17, 63):
        sub = sc.subset([b])
        sub.src = sub.src.astype(np.float64)
        sub.mic = sub.mic.astype(np.float64)
        a0, a1 = int(ds.vs_off[b]), int(ds.vs_off[b + 1])
        o0, o1 = int(ds.rir_off[b]), int(ds.rir_off[b + 1])
        yb = y[o0:o1].astype(np.float64)
        pb, gb, rb = ref.pos[a0:a1].copy(), ref.g[a0:a1], ref.r[b:b + 1].copy()
        checks = []
        for k in range(3):
            def f_src(v, k=k):
                s2 = scenes.Scene(**{**sub.__dict__})
                s2.src = sub.src.copy()
                s2.src[0, 0, k] = v
                return _room_loss(oracle_mod, s2, op, pb, gb, rb, yb)
            x0 = sub.src[0, 0, k]
            checks.append(((f_src(x0 + step) - f_src(x0 - step)) / (2 * step), src.grad[b, 0, k].item()))
            def f_mic(v, k=k):
                s2 = scenes.Scene(**{**sub.__dict__})
                s2.mic = sub.mic.copy()
                s2.mic[0, 2, k] = v
                return _room_loss(oracle_mod, s2, op, pb, gb, rb, yb)
            x0 = sub.mic[0, 2, k]
            checks.append(((f_mic(x0 + step) - f_mic(x0 - step)) / (2 * step), mic.grad[b, 2, k].item()))
            for i in (0, 700, 1499):
                def f_vs(v, k=k, i=i):
                    p2 = pb.copy()
                    p2[i, k] = v
                    return _room_loss(oracle_mod, sub, op, p2, gb, rb, yb)
                x0 = pb[i, k]
                checks.append(((f_vs(x0 + step) - f_vs(x0 - step)) / (2 * step), pos.grad[a0 + i, k].item()))
        fd = np.array([c[0] for c in checks])
        gpu = np.array([c[1] for c in checks])
        scale = np.abs(fd).max()
        assert np.max(np.abs(fd - gpu)) < 1e-5 * scale, (b, np.max(np.abs(fd - gpu)) / scale)
        def f_r(v):
            return _room_loss(oracle_mod, sub, op, pb, gb, np.array([v]), yb)
        hr = 1e-7 * rb[0]
        fd_r = (f_r(rb[0] + hr) - f_r(rb[0] - hr)) / (2 * hr)
        assert abs(fd_r - r.grad[b].item()) < 1e-5 * abs(fd_r)
