"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, on identical seeded
inputs.  The oracle always draws its own images from the same seed -- it never receives a
value the GPU produced.

Tolerances (from the method's contract):
  * Philox words: bit-exact.  floor(g_i): exact except near-ties, |g - round(g)| < 1e-5 g,
    where FP32 and FP64 may round to different sides (they must be < 1e-4 of all images).
  * RIRs and early RIRs: max |h_gpu - h_oracle| <= 1e-5 * peak, per (room, source) RIR, with
    peak = max |h_oracle| over that RIR's channels.
  * Gradients: max error <= 1e-5 * the largest magnitude of that gradient in the room (image
    and mic gradients) or over the batch (r, source).
Sizes: small scenes span several tiles and a ragged tail; the benchmark workloads run at full
size on the GPU and are compared on seeded samples of rooms.
"""
import numpy as np
import pytest
import torch

from paper_2304_08052_gb300 import _lib, api, scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _params(sc, **kw):
    return api.Params(fs=sc.fs, half_len=sc.half_len, **kw)


def _oparams(oracle_mod, sc, **kw):
    return oracle_mod.Params(fs=sc.fs, half_len=sc.half_len, **kw)


def _gpu(sc, seed, early=False, tile=0, **kw):
    ds = api.DeviceScene(sc, _params(sc, tile=tile, **kw))
    vs = api.sample(ds, seed=seed, words=True)
    out = api.synthesize(ds, vs, early=early)
    torch.cuda.synchronize()
    assert ds.status() == 0
    return ds, vs, out


def _rir_errors(sc, rir_len, rir_off, h_gpu, h_ref, rooms_gpu, rooms_ref):
    """Per-(room, source) max error relative to that RIR's peak.  h_gpu may be a CUDA tensor:
    only the compared rooms are copied to the host."""
    errs = []
    for bg, br in zip(rooms_gpu, rooms_ref):
        L = int(rir_len[bg])
        for s in range(sc.S):
            og = int(rir_off[0][bg]) + s * sc.M * L
            orr = int(rir_off[1][br]) + s * sc.M * L
            g = h_gpu[og:og + sc.M * L]
            g = (g.cpu().numpy() if isinstance(g, torch.Tensor) else g).astype(np.float64)
            r = h_ref[orr:orr + sc.M * L]
            peak = np.abs(r).max()
            errs.append(np.abs(g - r).max() / peak)
    return np.array(errs)


def _compare_rooms(oracle_mod, sc, seed, rooms, early=False, **kw):
    ds, vs, out = _gpu(sc, seed, early=early, **kw)
    h, he = out if early else (out, None)
    sub = sc.subset(rooms) if rooms is not None else sc
    rooms = list(range(sc.B)) if rooms is None else [int(b) for b in rooms]
    op = _oparams(oracle_mod, sc, **{k: v for k, v in kw.items() if k != "tile"})
    ref = oracle_mod.sample(sub, op, seed, room_ids=rooms)
    res = oracle_mod.synthesize(sub, op, ref.pos, ref.g, ref.r, early=early)
    h_ref, he_ref = res if early else (res, None)
    _, rir_off_sub, _ = oracle_mod.layout(sub.rt60, sub.n_vs, sub.S, sub.M, sub.fs)
    e = _rir_errors(sc, ds.rir_len, (ds.rir_off, rir_off_sub), h, h_ref, rooms, range(len(rooms)))
    out = {"rir": e}
    if early:
        out["early"] = _rir_errors(sc, ds.rir_len, (ds.rir_off, rir_off_sub), he, he_ref, rooms, range(len(rooms)))
        # Eq. 9 on the GPU is an exact mask of the GPU's own h.
        assert bool(((he == h) | (he == 0)).all())
    return out, ds, vs, ref


# ------------------------------------------------------------------------------------------
# Sampler
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("name,seed", [("tiny", 3), ("single_room", 0), ("batch_256", 11)])
def test_sampler_matches_oracle(oracle_mod, name, seed):
    sc = scenes.tiny(seed=3, B=5, S=3, M=4, images=301) if name == "tiny" else scenes.by_name(name, 0)
    ds = api.DeviceScene(sc, _params(sc))
    vs = api.sample(ds, seed=seed, words=True)
    torch.cuda.synchronize()
    assert ds.status() == 0
    ref = oracle_mod.sample(sc, _oparams(oracle_mod, sc), seed)
    # Integer streams: bit-exact.
    assert np.array_equal(vs.words.cpu().numpy().view(np.uint32), ref.words)
    # Reflection coefficient (Eq. 2), stored as float.
    assert np.allclose(vs.r.cpu().numpy(), ref.r, rtol=1e-7, atol=0)
    # Distances to the array centre: exact to float-pair precision.
    pos = vs.pos_hi.double().cpu().numpy() + vs.pos_lo.double().cpu().numpy()
    cen = np.repeat(sc.mic.astype(np.float64).mean(axis=1), sc.S * sc.n_vs, axis=0)
    d_gpu = np.linalg.norm(pos - cen, axis=1)
    assert np.max(np.abs(d_gpu - ref.dist) / ref.dist) < 2e-12
    # Directions: FP32 trigonometry, tilt below 1e-6 rad.
    u_g = (pos - cen) / d_gpu[:, None]
    u_r = (ref.pos - cen) / ref.dist[:, None]
    assert np.max(np.linalg.norm(u_g - u_r, axis=1)) < 1e-6
    # Reflection counts.
    g = vs.g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - ref.g) / ref.g) < 2e-6
    # floor(g) must agree except where FP32 and FP64 sit on either side of an integer.
    mism = np.floor(g) != np.floor(ref.g)
    near_tie = np.abs(ref.g - np.round(ref.g)) < 1e-5 * ref.g
    assert np.all(near_tie[mism]) and mism.mean() < 1e-4, (mism.sum(), g.size)


def test_sampler_seed_from_device_memory(oracle_mod):
    sc = scenes.tiny(seed=2, B=3, S=2, M=2, images=50)
    ds = api.DeviceScene(sc, _params(sc))
    seed = 0x1234_5678_9ABC_DEF0
    d_seed = torch.tensor([seed], dtype=torch.int64, device="cuda")   # seed < 2^63
    a = api.sample(ds, seed=0, d_seed=d_seed, words=True)
    b = api.sample(ds, seed=seed, words=True)
    torch.cuda.synchronize()
    assert torch.equal(a.words, b.words) and torch.equal(a.pos_hi, b.pos_hi) and torch.equal(a.g, b.g)


# ------------------------------------------------------------------------------------------
# Synthesis
# ------------------------------------------------------------------------------------------
def test_tiny_exhaustive(oracle_mod):
    sc = scenes.tiny(seed=1, B=4, S=2, M=3, images=200, t60_lo=0.1, t60_hi=0.3)
    res, *_ = _compare_rooms(oracle_mod, sc, seed=5, rooms=None, early=True)
    assert res["rir"].max() < TOL, res["rir"].max()
    assert res["early"].max() < TOL


@pytest.mark.parametrize("tile", [256, 512, 2048])
def test_tiles_and_ragged_tails(oracle_mod, tile):
    # RIR lengths not multiples of the tile; several tiles per RIR.
    sc = scenes.tiny(seed=9, B=3, S=2, M=5, images=700, t60_lo=0.11, t60_hi=0.37)
    res, *_ = _compare_rooms(oracle_mod, sc, seed=2, rooms=None, tile=tile)
    assert res["rir"].max() < TOL


def test_single_room(oracle_mod):
    sc = scenes.single_room()
    res, ds, vs, ref = _compare_rooms(oracle_mod, sc, seed=0, rooms=None, early=True)
    assert res["rir"].max() < TOL and res["early"].max() < TOL


def test_batch_256_full(oracle_mod):
    sc = scenes.batch_256(0)
    res, *_ = _compare_rooms(oracle_mod, sc, seed=1, rooms=None)
    assert res["rir"].max() < TOL, np.sort(res["rir"])[-5:]


def test_batch_1024_early_sampled_rooms(oracle_mod):
    sc = scenes.batch_1024(0)
    rooms = np.random.default_rng(3).choice(sc.B, 24, replace=False)
    res, *_ = _compare_rooms(oracle_mod, sc, seed=2, rooms=rooms, early=True)
    assert res["rir"].max() < TOL and res["early"].max() < TOL


def test_large_4096_48k_sampled_rooms(oracle_mod):
    sc = scenes.large_4096(0)
    rooms = np.random.default_rng(4).choice(sc.B, 12, replace=False)
    rooms = np.concatenate([rooms, [int(np.argmax(sc.rt60)), int(np.argmin(sc.rt60))]])
    res, *_ = _compare_rooms(oracle_mod, sc, seed=3, rooms=rooms)
    assert res["rir"].max() < TOL, np.sort(res["rir"])[-5:]


@pytest.mark.parametrize("K,tile", [(1, 0), (5, 0), (16, 0), (17, 0), (33, 0), (64, 0), (100, 0), (128, 0),
                                    (128, 256)])
def test_other_half_lengths(oracle_mod, K, tile):
    # Every round count of the synthesis (one lane per tap offset: 1 to 8 rounds of 32, packed
    # in pairs with a scalar last round when odd), K = 1 (whose delta / K may leave [-1/2, 1/2]),
    # and the adjoint's path for a K without compile-time constants.  tile = 2K: a window spans
    # two tiles at most.
    sc = scenes.tiny(seed=40 + K, B=3, S=2, M=2, images=90, K=K, t60_lo=0.08, t60_hi=0.2)
    e, ds, vs, ref = _compare_rooms(oracle_mod, sc, seed=K, rooms=None, early=True, tile=tile)
    assert e["rir"].max() < TOL and e["early"].max() < TOL, (K, e["rir"].max(), e["early"].max())
    g = _grad_compare(oracle_mod, sc, seed=K, early=True)
    assert max(g.values()) < TOL, (K, g)


@pytest.mark.parametrize("fs,M,S,geometry,spacing,K,t60", [
    (8000.0, 1, 1, "circular", 0.05, 40, (0.1, 0.3)),      # one mic, low rate
    (22050.0, 64, 1, "circular", 0.1, 40, (0.05, 0.1)),    # the most mics the adjoint takes
    (44100.0, 9, 3, "linear", 0.1, 63, (0.05, 0.12)),
    (16000.0, 3, 7, "circular", 0.02, 40, (0.3, 0.5)),     # many sources
    (48000.0, 5, 2, "linear", 0.25, 63, (0.03, 0.05)),     # 1 m array: a 140-sample margin, short RIRs
])
def test_scene_shapes(oracle_mod, fs, M, S, geometry, spacing, K, t60):
    # Sample rates, array sizes and shapes, and source counts outside the benchmark workloads:
    # RIRs, early RIRs and the adjoint against the oracle on every room.
    sc = scenes.make_batch("shape", 60 + M + S, 3, S, M, geometry, spacing, [3, 3, 2.5], [6, 5, 3.5],
                           t60[0], t60[1], fs, K, images_fixed=70)
    e, ds, vs, ref = _compare_rooms(oracle_mod, sc, seed=M + S, rooms=None, early=True)
    assert e["rir"].max() < TOL and e["early"].max() < TOL, (e["rir"].max(), e["early"].max())
    g = _grad_compare(oracle_mod, sc, seed=M + S, early=True)
    assert max(g.values()) < TOL, g


def test_cartesian_float32_inputs(oracle_mod):
    # User-supplied float32 image positions (no low parts) and arbitrary g.
    sc = scenes.tiny(seed=4, B=3, S=2, M=4, images=300, t60_lo=0.2, t60_hi=0.4)
    pos, g = scenes.synthetic_vs(5, sc)
    ds = api.DeviceScene(sc, _params(sc))
    op = _oparams(oracle_mod, sc)
    r = np.array([0.93, 0.97, 0.99], np.float32)
    h = api.synthesize_raw(ds, torch.as_tensor(pos, device="cuda"), None, torch.as_tensor(g, device="cuda"),
                           torch.as_tensor(r, device="cuda"))
    torch.cuda.synchronize()
    assert ds.status() == 0
    h_ref = oracle_mod.synthesize(sc, op, pos.astype(np.float64), g.astype(np.float64), r.astype(np.float64))
    e = _rir_errors(sc, ds.rir_len, (ds.rir_off, ds.rir_off), h.cpu().numpy(), h_ref, range(sc.B), range(sc.B))
    assert e.max() < TOL


def test_integer_delay_single_tap():
    # c0 = 320 m/s at 16 kHz: 50 samples per metre; source 2 m from the mic -> t = 100.
    sc = scenes.Scene("probe", 1, 1, 1, 16000.0, 40, np.array([[10, 10, 10]], np.float32),
                      np.array([0.05], np.float32), np.array([[[1, 1, 1]]], np.float32),
                      np.array([[[3, 1, 1]]], np.float32), np.array([0], np.int32))
    ds = api.DeviceScene(sc, api.Params(fs=16000.0, half_len=40, c0=320.0))
    z = torch.zeros((0, 3), device="cuda")
    h = api.synthesize_raw(ds, z, None, torch.zeros(0, device="cuda"), torch.tensor([0.9], device="cuda"))
    h = h.cpu().numpy()
    assert abs(h[100] - 0.5) <= 0.5 * 2 ** -23
    assert np.max(np.abs(np.delete(h, 100))) < 1e-7


def test_deterministic_and_tile_independent(oracle_mod):
    sc = scenes.tiny(seed=12, B=3, S=2, M=3, images=900, t60_lo=0.2, t60_hi=0.3)
    ds = api.DeviceScene(sc, _params(sc))
    vs = api.sample(ds, seed=8)
    a = api.synthesize(ds, vs).clone()
    b = api.synthesize(ds, vs).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)                       # bit-reproducible run to run
    ds2 = api.DeviceScene(sc, _params(sc, tile=256))
    c = api.synthesize(ds2, vs)
    torch.cuda.synchronize()
    peak = a.abs().max().item()
    assert (a - c).abs().max().item() < 1e-6 * peak


def test_edge_cases(oracle_mod):
    # Rooms without images, a single mic, RIRs shorter than one tile, images far beyond the
    # RIR end (their taps fall outside [0, L) and are dropped).
    sc = scenes.tiny(seed=13, B=4, S=1, M=1, images=30, t60_lo=0.01, t60_hi=0.03)
    sc.n_vs[1] = 0
    ds = api.DeviceScene(sc, _params(sc))
    pos, g = scenes.synthetic_vs(1, sc, max_dist=40.0)
    r = np.full(sc.B, 0.95, np.float32)
    h = api.synthesize_raw(ds, torch.as_tensor(pos, device="cuda"), None, torch.as_tensor(g, device="cuda"),
                           torch.as_tensor(r, device="cuda"))
    torch.cuda.synchronize()
    assert ds.status() == 0
    op = _oparams(oracle_mod, sc)
    h_ref = oracle_mod.synthesize(sc, op, pos.astype(np.float64), g.astype(np.float64), r.astype(np.float64))
    e = _rir_errors(sc, ds.rir_len, (ds.rir_off, ds.rir_off), h.cpu().numpy(), h_ref, range(sc.B), range(sc.B))
    assert e.max() < TOL


def test_empty_batch():
    sc = scenes.tiny(seed=1, B=1, S=1, M=2, images=3)
    sc = sc.subset([])
    ds = api.DeviceScene(sc, _params(sc))
    vs = api.sample(ds, seed=1)
    h = api.synthesize(ds, vs)
    torch.cuda.synchronize()
    assert h.numel() == 0 and ds.status() == 0


def test_bad_geometry_sets_status():
    sc = scenes.tiny(seed=1, B=2, S=1, M=2, images=10)
    sc.rt60[1] = np.float32(0.002)       # c0 * T60 = 0.69 m < the source distance
    sc.src[1, 0] = sc.mic[1].mean(axis=0) + np.array([1.5, 0, 0], np.float32)
    ds = api.DeviceScene(sc, _params(sc))
    api.sample(ds, seed=1)
    torch.cuda.synchronize()
    assert ds.status() & 0x1


def test_nonfinite_image_sets_status_and_is_skipped(oracle_mod):
    # A NaN image position: the binning flags FRAM_DEV_NONFINITE and the image contributes
    # nothing; every other arrival is rendered as usual.  The oracle drops the image by giving it
    # a reflection count so large that r^g underflows to 0.
    sc = scenes.tiny(seed=3, B=2, S=1, M=2, images=30)
    ds = api.DeviceScene(sc, _params(sc))
    op = _oparams(oracle_mod, sc)
    ref = oracle_mod.sample(sc, op, 5)
    pos, g, r = ref.pos.astype(np.float32), ref.g.astype(np.float32), ref.r.astype(np.float32)
    bad = int(ds.vs_off[1]) + 7
    pos_bad = pos.copy()
    pos_bad[bad] = np.nan
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    h = api.synthesize_raw(ds, dev(pos_bad), None, dev(g), dev(r))
    torch.cuda.synchronize()
    assert ds.status() & _lib.FRAM_DEV_NONFINITE
    got = h.cpu().numpy()
    assert np.isfinite(got).all()
    g_drop = g.astype(np.float64)
    g_drop[bad] = 1.0e6
    h_ref = oracle_mod.synthesize(sc, op, pos.astype(np.float64), g_drop, r.astype(np.float64))
    e = _rir_errors(sc, ds.rir_len, (ds.rir_off, ds.rir_off), got, h_ref, range(sc.B), range(sc.B))
    assert e.max() < TOL


# ------------------------------------------------------------------------------------------
# Adjoint
# ------------------------------------------------------------------------------------------
def _grad_compare(oracle_mod, sc, seed, early, rooms=None, tile=0):
    ds = api.DeviceScene(sc, _params(sc, tile=tile))
    vs = api.sample(ds, seed=seed)
    # Seeded upstream gradients (the gradient of sum (h - y)^2 has this form for a Gaussian y);
    # the same float32 values go to both sides.
    rng = np.random.default_rng(seed)
    n = ds.rir_total
    G = rng.normal(size=n).astype(np.float32)
    Ge = rng.normal(size=n).astype(np.float32) if early else None
    gv, gm, gs, gr = api.synthesize_backward_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, torch.as_tensor(G, device="cuda"),
                                                 torch.as_tensor(Ge, device="cuda") if early else None)
    torch.cuda.synchronize()
    assert ds.status() == 0
    op = _oparams(oracle_mod, sc)
    ref = oracle_mod.sample(sc, op, seed)
    rv, rm, rs, rr = oracle_mod.backward(sc, op, ref.pos, ref.g, ref.r, G.astype(np.float64),
                                         Ge.astype(np.float64) if early else None)
    gv, gm, gs, gr = (t.double().cpu().numpy() for t in (gv, gm, gs, gr))
    errs = {}
    per_room = []
    for b in range(sc.B):
        a0, a1 = int(ds.vs_off[b]), int(ds.vs_off[b + 1])
        scale_v = np.abs(rv[a0:a1]).max() if a1 > a0 else 1.0
        per_room.append(np.abs(gv[a0:a1] - rv[a0:a1]).max() / scale_v if a1 > a0 else 0.0)
    errs["vs"] = max(per_room)
    errs["mic"] = max(np.abs(gm[b] - rm[b]).max() / np.abs(rm[b]).max() for b in range(sc.B))
    errs["src"] = np.abs(gs - rs).max() / np.abs(rs).max()
    errs["r"] = np.abs(gr - rr).max() / np.abs(rr).max()
    return errs


def test_gradients_tiny(oracle_mod):
    sc = scenes.tiny(seed=7, B=3, S=2, M=3, images=120, t60_lo=0.1, t60_hi=0.2)
    e = _grad_compare(oracle_mod, sc, seed=4, early=True)
    assert max(e.values()) < TOL, e


def test_gradients_grad_64(oracle_mod):
    sc = scenes.grad_64(0)
    e = _grad_compare(oracle_mod, sc, seed=1, early=False)
    assert max(e.values()) < TOL, e


@pytest.mark.parametrize("tile", [1024, 2048])
def test_gradients_multi_tile_items(oracle_mod, tile):
    # RIRs of 0.3-0.6 s spanning several tiles, at the default tile and at the one the benchmark's
    # tuner picks on GB300: the adjoint's items and their halos against the oracle.
    sc = scenes.tiny(seed=11, B=4, S=2, M=3, images=400, t60_lo=0.3, t60_hi=0.6)
    e = _grad_compare(oracle_mod, sc, seed=9, early=True, tile=tile)
    assert max(e.values()) < TOL, e


def test_autograd_function_matches_raw_backward(oracle_mod):
    sc = scenes.tiny(seed=8, B=2, S=2, M=3, images=80, t60_lo=0.1, t60_hi=0.15)
    ds = api.DeviceScene(sc, _params(sc))
    vs = api.sample(ds, seed=3)
    src = ds.src.clone().requires_grad_()
    mic = ds.mic.clone().requires_grad_()
    pos = vs.pos_hi.clone().requires_grad_()
    r = vs.r.clone().requires_grad_()
    h, he = api.rir(ds, src, mic, pos, r, vs.g, vs.pos_lo, early=True)
    y = torch.randn_like(h)
    loss = ((h - y) ** 2).sum() + (he ** 2).sum()
    loss.backward()
    G = (2 * (h - y)).detach()
    Ge = (2 * he).detach()
    gv, gm, gs, gr = api.synthesize_backward_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, G, Ge)
    torch.cuda.synchronize()
    assert torch.equal(pos.grad, gv) and torch.equal(mic.grad, gm)
    assert torch.equal(src.grad, gs) and torch.equal(r.grad, gr)
