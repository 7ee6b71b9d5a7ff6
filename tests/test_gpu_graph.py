"""CUDA-graph capture of the batched path: sample + synthesize (RIRs and early RIRs) with the
seed read from device memory, the adjoint and the sampler's adjoint, captured once as one graph
and replayed with new seeds written into device memory.  Every replay must equal, bit for bit,
the eager calls with the same seed (the kernels' results do not depend on scheduling), and one
replay is checked against the FP64 oracle on sampled rooms.
"""
import numpy as np
import pytest

from paper_2304_08052_gb300 import api, scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _images(torch, ds):
    n = ds.n_vs_total
    return api.Images(torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda"),
                      torch.empty(n, device="cuda"), torch.empty(ds.B, device="cuda"))


def test_graph_replays_equal_eager_calls(oracle_mod):
    import torch
    sc = scenes.batch_256(0).subset(range(24))
    params = api.Params(fs=sc.fs, half_len=sc.half_len)
    ds = api.DeviceScene(sc, params)
    vs = _images(torch, ds)
    rir = torch.empty(ds.rir_total, device="cuda")
    early = torch.empty(ds.rir_total, device="cuda")
    G = torch.from_numpy(np.random.default_rng(5).standard_normal(ds.rir_total).astype(np.float32)).cuda()
    Ge = torch.from_numpy(np.random.default_rng(6).standard_normal(ds.rir_total).astype(np.float32)).cuda()
    d_seed = torch.zeros(1, dtype=torch.int64, device="cuda")
    grads = {}

    def body():
        api.sample(ds, seed=0, d_seed=d_seed, out=vs)
        api.synthesize_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, early=True, rir=rir, early_out=early)
        gv, gm, gs, gr, gg = api.synthesize_backward_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, G, Ge,
                                                         want=("vs", "mic", "src", "r", "g"))
        grads["adjoint"] = (gv, gm, gs, gr, gg)
        grads["sampler"] = api.sample_backward(ds, 0, gv, gg, gr, gs, gm, d_seed=d_seed)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            body()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        body()

    for seed in (5, 6, 1234567890123):          # the last one uses the key's high word
        d_seed.fill_(seed)
        g.replay()
        torch.cuda.synchronize()
        assert ds.status() == 0
        got = [rir.clone(), early.clone()] + [t.clone() for t in grads["adjoint"] + tuple(grads["sampler"])]
        # eager calls on a scene object of their own
        de = api.DeviceScene(sc, params)
        ve = api.sample(de, seed=seed)
        he, hee = api.synthesize(de, ve, early=True)
        adj = api.synthesize_backward_raw(de, ve.pos_hi, ve.pos_lo, ve.g, ve.r, G, Ge,
                                          want=("vs", "mic", "src", "r", "g"))
        gv, gm, gs, gr, gg = adj
        samp = api.sample_backward(de, seed, gv, gg, gr, gs, gm)
        torch.cuda.synchronize()
        want = [he, hee] + list(adj) + list(samp)
        for k, (a, b) in enumerate(zip(got, want)):
            assert torch.equal(a, b), (seed, k)

    # The last replay's RIRs against the oracle on two rooms.
    seed = 1234567890123
    rooms = [0, 17]
    sub = sc.subset(rooms)
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sub, op, seed, room_ids=rooms)
    h_ref = oracle_mod.synthesize(sub, op, ref.pos, ref.g, ref.r)
    _, ro, _ = oracle_mod.layout(sub.rt60, sub.n_vs, sub.S, sub.M, sub.fs)
    h = got[0].cpu().numpy().astype(np.float64)
    for i, b in enumerate(rooms):
        o, n = int(ds.rir_off[b]), int(ds.rir_off[b + 1] - ds.rir_off[b])
        r = h_ref[int(ro[i]):int(ro[i]) + n]
        assert np.abs(h[o:o + n] - r).max() <= TOL * np.abs(r).max(), b
