"""Gradient through the sampler on the GPU (fram_sample_backward and the adjoint's dL/dg output)
against the FP64 oracle's fo_sample_backward / fo_backward, whose chain is pinned by finite
differences of the whole oracle pipeline (test_oracle_reparam.py).

Three levels:
  * the sampler's adjoint alone: both sides get the same float32 upstream gradients (dL/dp_i,
    dL/dg_i, dL/dr and the direct source / mic gradients), so only Eq. 2-6's chain differs;
  * the adjoint's new dL/dg output against fo_backward's;
  * the whole differentiable step (api.sampled_rir: sample, synthesize, and both adjoints
    behind one torch.autograd.Function) against the oracle's pipeline on the same seed.
The bar is max-abs error <= 1e-5 of each output's largest magnitude (per room for per-image
outputs).
"""
import ctypes

import numpy as np
import pytest

from paper_2304_08052_gb300 import _lib, api, scenes

TOL = 1e-5


def _params(sc, **kw):
    return api.Params(fs=sc.fs, half_len=sc.half_len, **kw)


def _oparams(oracle_mod, sc):
    return oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _upstream(oracle_mod, sc, seed):
    """The oracle's synthesis adjoint on its own images, rounded to float32 (the common input)."""
    op = _oparams(oracle_mod, sc)
    ref = oracle_mod.sample(sc, op, seed)
    _, rir_off, _ = oracle_mod.layout(sc.rt60, sc.n_vs, sc.S, sc.M, sc.fs)
    G = np.random.default_rng(seed + 100).standard_normal(int(rir_off[-1]))
    gv, gm, gs, gr, gg = oracle_mod.backward(sc, op, ref.pos, ref.g, ref.r, G, with_g=True)
    return [x.astype(np.float32) for x in (gv, gg, gr, gs, gm)]


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["tiny", "grad_64"])
def test_sampler_adjoint_matches_the_oracle(oracle_mod, name):
    import torch
    sc = scenes.tiny(seed=51, B=3, S=2, M=4, images=300, t60_lo=0.2, t60_hi=0.5) if name == "tiny" \
        else scenes.grad_64(0)
    seed = 61
    gv, gg, gr, gs, gm = _upstream(oracle_mod, sc, seed)
    ds = api.DeviceScene(sc, _params(sc))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = api.sample_backward(ds, seed, dev(gv), dev(gg), dev(gr), dev(gs), dev(gm))
    torch.cuda.synchronize()
    assert ds.status() == 0
    got = [t.cpu().numpy() for t in out]
    ref = oracle_mod.sample_backward(sc, _oparams(oracle_mod, sc), seed, *(x.astype(np.float64)
                                                                          for x in (gv, gg, gr, gs, gm)))
    for g_, r_, what in zip(got, ref, ("src", "mic", "t60", "dims")):
        assert _rel(g_, r_) <= TOL, (what, _rel(g_, r_))


@pytest.mark.gpu
@pytest.mark.parametrize("fs,M,S,geometry,spacing,K", [
    (44100.0, 64, 1, "circular", 0.1, 63),    # the most mics the adjoint takes
    (16000.0, 2, 7, "linear", 0.3, 5),        # many sources, a short window
    (8000.0, 1, 2, "circular", 0.05, 1),      # one mic, K = 1
])
def test_sampled_rir_shapes(oracle_mod, fs, M, S, geometry, spacing, K):
    # The whole differentiable step (sample, synthesize, both adjoints) on scene shapes outside the
    # benchmark workloads, against the oracle's pipeline.
    import torch
    sc = scenes.make_batch("shape", 90 + M + S, 2, S, M, geometry, spacing, [3, 3, 2.5], [6, 5, 3.5],
                           0.1, 0.25, fs, K, images_fixed=120)
    seed = 65 + M
    ds = api.DeviceScene(sc, _params(sc))
    leaves = [t.clone().requires_grad_() for t in (ds.src, ds.mic, ds.rt60, ds.dims)]
    h, he = api.sampled_rir(ds, *leaves, seed=seed, early=True)
    G = np.random.default_rng(9).standard_normal(ds.rir_total).astype(np.float32)
    Ge = np.random.default_rng(10).standard_normal(ds.rir_total).astype(np.float32)
    loss = (h * torch.from_numpy(G).cuda()).sum() + (he * torch.from_numpy(Ge).cuda()).sum()
    loss.backward()
    torch.cuda.synchronize()
    assert ds.status() == 0
    got = [t.grad.cpu().numpy() for t in leaves]
    op = _oparams(oracle_mod, sc)
    ref = oracle_mod.sample(sc, op, seed)
    gv, gm, gs, gr, gg = oracle_mod.backward(sc, op, ref.pos, ref.g, ref.r, G.astype(np.float64),
                                             Ge.astype(np.float64), with_g=True)
    want = oracle_mod.sample_backward(sc, op, seed, gv, gg, gr, gs, gm)
    for g_, r_, what in zip(got, want, ("src", "mic", "t60", "dims")):
        assert _rel(g_, r_) <= TOL, (what, _rel(g_, r_))


@pytest.mark.gpu
def test_adjoint_reflection_count_gradient(oracle_mod):
    import torch
    sc = scenes.tiny(seed=52, B=3, S=2, M=3, images=200, t60_lo=0.1, t60_hi=0.3)
    seed = 62
    ds = api.DeviceScene(sc, _params(sc))
    vs = api.sample(ds, seed=seed)
    G = np.random.default_rng(3).standard_normal(ds.rir_total).astype(np.float32)
    Ge = np.random.default_rng(4).standard_normal(ds.rir_total).astype(np.float32)
    outs = api.synthesize_backward_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, torch.from_numpy(G).cuda(),
                                       torch.from_numpy(Ge).cuda(), want=("vs", "g"))
    gg = outs[-1].cpu().numpy()
    op = _oparams(oracle_mod, sc)
    ref = oracle_mod.sample(sc, op, seed)
    *_, gg_ref = oracle_mod.backward(sc, op, ref.pos, ref.g, ref.r, G.astype(np.float64), Ge.astype(np.float64),
                                     with_g=True)
    for b in range(sc.B):
        a0, a1 = int(ds.vs_off[b]), int(ds.vs_off[b + 1])
        assert _rel(gg[a0:a1], gg_ref[a0:a1]) <= TOL, b
    # Without the output requested, the other gradients are unchanged (bit-exact).
    gv2, = api.synthesize_backward_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, torch.from_numpy(G).cuda(),
                                       torch.from_numpy(Ge).cuda(), want=("vs",))[:1]
    assert torch.equal(gv2, outs[0])


@pytest.mark.gpu
@pytest.mark.parametrize("early", [False, True])
def test_sampled_rir_autograd_matches_the_oracle_pipeline(oracle_mod, early):
    import torch
    sc = scenes.tiny(seed=53, B=2, S=2, M=3, images=250, t60_lo=0.2, t60_hi=0.35)
    seed = 63
    ds = api.DeviceScene(sc, _params(sc))
    leaves = [t.clone().requires_grad_() for t in (ds.src, ds.mic, ds.rt60, ds.dims)]
    out = api.sampled_rir(ds, *leaves, seed=seed, early=early)
    h, he = out if early else (out, None)
    G = np.random.default_rng(7).standard_normal(ds.rir_total).astype(np.float32)
    Ge = np.random.default_rng(8).standard_normal(ds.rir_total).astype(np.float32) if early else None
    loss = (h * torch.from_numpy(G).cuda()).sum()
    if early:
        loss = loss + (he * torch.from_numpy(Ge).cuda()).sum()
    loss.backward()
    torch.cuda.synchronize()
    got = [t.grad.cpu().numpy() for t in leaves]
    op = _oparams(oracle_mod, sc)
    ref = oracle_mod.sample(sc, op, seed)
    gv, gm, gs, gr, gg = oracle_mod.backward(sc, op, ref.pos, ref.g, ref.r, G.astype(np.float64),
                                             Ge.astype(np.float64) if early else None, with_g=True)
    want = oracle_mod.sample_backward(sc, op, seed, gv, gg, gr, gs, gm)
    for g_, r_, what in zip(got, want, ("src", "mic", "t60", "dims")):
        assert _rel(g_, r_) <= TOL, (what, _rel(g_, r_))


@pytest.mark.gpu
def test_sampler_adjoint_is_deterministic_and_may_work_in_place(oracle_mod):
    import torch
    sc = scenes.tiny(seed=54, B=4, S=3, M=2, images=400, t60_lo=0.2, t60_hi=0.4)
    seed = 64
    gv, gg, gr, gs, gm = _upstream(oracle_mod, sc, seed)
    ds = api.DeviceScene(sc, _params(sc))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    a = api.sample_backward(ds, seed, dev(gv), dev(gg), dev(gr), dev(gs), dev(gm))
    b = api.sample_backward(ds, seed, dev(gv), dev(gg), dev(gr), dev(gs), dev(gm))
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    # grad_src_in / grad_mic_in aliasing the outputs.
    s_io, m_io = dev(gs), dev(gm)
    gv_d, gg_d, gr_d = dev(gv), dev(gg), dev(gr)      # held: the library keeps only the pointers
    t60, dims = torch.empty_like(a[2]), torch.empty_like(a[3])
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    _lib.check(_lib.lib().fram_sample_backward(
        ctypes.byref(ds.c_scene()), ctypes.byref(ds.params.c()), ctypes.c_uint64(seed), None, p(gv_d),
        p(gg_d), p(gr_d), p(s_io), p(m_io), p(s_io), p(m_io), p(t60), p(dims), p(ds.ws),
        ctypes.c_size_t(ds.ws_bytes), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    assert torch.equal(s_io, a[0]) and torch.equal(m_io, a[1])
    assert torch.equal(t60, a[2]) and torch.equal(dims, a[3])


@pytest.mark.gpu
def test_sampler_adjoint_bad_geometry_keeps_the_direct_gradient():
    import torch
    sc = scenes.tiny(seed=55, B=2, S=1, M=2, images=50)
    sc.rt60[1] = np.float32(0.002)       # c0 T60 = 0.69 m < the source distance
    sc.src[1, 0] = sc.mic[1].mean(axis=0) + np.array([1.5, 0, 0], np.float32)
    ds = api.DeviceScene(sc, _params(sc))
    N = ds.n_vs_total
    gv = torch.ones((N, 3), device="cuda")
    gs_in = torch.full((sc.B, sc.S, 3), 0.25, device="cuda")
    gs, gm, gt, gd = api.sample_backward(ds, 5, gv, None, None, gs_in, None)
    torch.cuda.synchronize()
    assert ds.status() & _lib.FRAM_DEV_BAD_GEOMETRY
    assert torch.equal(gs[1], gs_in[1])
    assert torch.isfinite(gs).all() and torch.isfinite(gm).all()
