"""The paper's multi-rate output path (delay_mode 1; Sec. II-B and Eq. 7-9 as printed) through
the C ABI, against the FP64 oracle's fo_synthesize_mr.

The high-rate grid turns each delay into an integer, q = ceil(D r_h fs / c0), so both sides must
decide it from the same numbers: the tests hand the oracle's own images to both, with positions
rounded to values a float pair represents exactly (hi + lo), and g and r rounded to float32.  The
GPU evaluates D and q in FP64 in the oracle's operation order, so every q is identical; the RIRs
(and early RIRs) must then agree within 1e-5 of each RIR's peak.  Host-side checks run on the CPU.
"""
import ctypes

import numpy as np
import pytest

from paper_2304_08052_gb300 import _lib, api, scenes

TOL = 1e-5


def _scene_struct(B=4, S=2, M=3, max_len=8000, nvs=400, rir_total=4 * 2 * 3 * 8000, radius=0.05):
    return _lib.FramScene(B, S, M, max_len, nvs, rir_total, radius, *([None] * 8))


def test_delay_mode_validation():
    L = _lib.lib()
    n = ctypes.c_size_t(0)
    sc = _scene_struct()
    assert L.fram_workspace_size(ctypes.byref(sc), ctypes.byref(api.Params(delay_mode=1).c()), ctypes.byref(n)) == 0
    n0 = ctypes.c_size_t(0)
    assert L.fram_workspace_size(ctypes.byref(sc), ctypes.byref(api.Params().c()), ctypes.byref(n0)) == 0
    assert n.value > n0.value                                  # room for the intermediate signals
    for bad in (dict(delay_mode=2), dict(delay_mode=-1), dict(delay_mode=1, fs=6000.0)):
        assert L.fram_workspace_size(ctypes.byref(sc), ctypes.byref(api.Params(**bad).c()),
                                     ctypes.byref(n)) == _lib.FRAM_EINVAL
    # r_l max_len must stay below 2^30 (32-bit intermediate-sample indices): r_l = 7 at 16 kHz
    long_sc = _scene_struct(max_len=(1 << 30) // 7 + 1, rir_total=4 * 2 * 3 * ((1 << 30) // 7 + 1))
    assert L.fram_workspace_size(ctypes.byref(long_sc), ctypes.byref(api.Params(delay_mode=1).c()),
                                 ctypes.byref(n)) == _lib.FRAM_EINVAL
    assert b"2^30" in L.fram_last_error()
    # the continuous mode takes that length (at tile 4096: 37,450 tiles per RIR, below 65536)
    assert L.fram_workspace_size(ctypes.byref(long_sc), ctypes.byref(api.Params(tile=4096).c()),
                                 ctypes.byref(n)) == 0


def test_backward_is_refused_in_the_multirate_mode():
    L = _lib.lib()
    fake = ctypes.c_void_p(0x1000)      # never dereferenced: the argument checks come first
    sc = _lib.FramScene(1, 1, 1, 100, 10, 100, 0.0, *([fake] * 8))
    p = api.Params(delay_mode=1)
    n = ctypes.c_size_t(0)
    assert L.fram_workspace_size(ctypes.byref(sc), ctypes.byref(p.c()), ctypes.byref(n)) == 0
    rc = L.fram_synthesize_backward(ctypes.byref(sc), ctypes.byref(p.c()), fake, None, fake, fake, fake, None,
                                    None, None, None, None, None, ctypes.c_void_p(0x100000), ctypes.c_size_t(n.value),
                                    None)
    assert rc == _lib.FRAM_EINVAL
    assert b"delay_mode" in L.fram_last_error()


def _pair_exact(pos):
    hi = pos.astype(np.float32)
    lo = (pos - hi.astype(np.float64)).astype(np.float32)
    return hi, lo, hi.astype(np.float64) + lo.astype(np.float64)


def _run(oracle_mod, sc, seed, early):
    import torch
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sc, op, seed)
    hi, lo, pos_q = _pair_exact(ref.pos)
    g32 = ref.g.astype(np.float32)
    r32 = ref.r.astype(np.float32)
    res = oracle_mod.synthesize_mr(sc, op, pos_q, g32.astype(np.float64), r32.astype(np.float64), early=early)
    h_ref, he_ref = res if early else (res, None)
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len, delay_mode=1))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = api.synthesize_raw(ds, dev(hi), dev(lo), dev(g32), dev(r32), early=early)
    torch.cuda.synchronize()
    assert ds.status() == 0
    h, he = out if early else (out, None)
    return ds, h.cpu().numpy().astype(np.float64), h_ref, (he.cpu().numpy().astype(np.float64) if early else None), he_ref


def _errors(sc, ds, h, h_ref):
    errs = []
    for b in range(sc.B):
        L = int(ds.rir_len[b])
        for s in range(sc.S):
            o = int(ds.rir_off[b]) + s * sc.M * L
            seg = slice(o, o + sc.M * L)
            peak = np.abs(h_ref[seg]).max()
            errs.append(np.abs(h[seg] - h_ref[seg]).max() / peak)
    return np.array(errs)


@pytest.mark.gpu
def test_multirate_16k_matches_the_oracle(oracle_mod):
    sc = scenes.batch_256(0).subset(range(12))
    ds, h, h_ref, _, _ = _run(oracle_mod, sc, 31, early=False)
    e = _errors(sc, ds, h, h_ref)
    assert e.max() <= TOL, e.max()


@pytest.mark.gpu
def test_multirate_48k_with_early_matches_the_oracle(oracle_mod):
    sc = scenes.tiny(seed=21, B=4, S=2, M=4, images=300, fs=48000.0, K=63, t60_lo=0.15, t60_hi=0.3)
    ds, h, h_ref, he, he_ref = _run(oracle_mod, sc, 32, early=True)
    assert _errors(sc, ds, h, h_ref).max() <= TOL
    assert _errors(sc, ds, he, he_ref).max() <= TOL


@pytest.mark.gpu
@pytest.mark.parametrize("fs,t60", [(8000.0, (0.1, 0.3)), (11025.0, (0.1, 0.2)), (22050.0, (0.05, 0.15)),
                                    (32000.0, (0.05, 0.1)), (96000.0, (0.03, 0.06)), (250000.0, (0.03, 0.04))])
def test_multirate_other_rates(oracle_mod, fs, t60):
    # Every second-resampler rate r_l = floor(sqrt(floor(1e6 / fs))) the benchmark workloads do not
    # use: 11, 9, 6, 5, 3 and 2 (16 and 48 kHz give 7 and 4), with early RIRs.
    sc = scenes.tiny(seed=int(fs) % 97, B=2, S=2, M=2, images=80, fs=fs, t60_lo=t60[0], t60_hi=t60[1])
    ds, h, h_ref, he, he_ref = _run(oracle_mod, sc, 34, early=True)
    assert _errors(sc, ds, h, h_ref).max() <= TOL
    assert _errors(sc, ds, he, he_ref).max() <= TOL


@pytest.mark.gpu
def test_multirate_tiles_and_ragged_ends(oracle_mod):
    # RIRs shorter than one tile and several tiles long; every tile length gives the same RIRs.
    sc = scenes.tiny(seed=22, B=3, S=1, M=2, images=120, fs=16000.0, t60_lo=0.02, t60_hi=0.25)
    import torch
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sc, op, 33)
    hi, lo, pos_q = _pair_exact(ref.pos)
    g32, r32 = ref.g.astype(np.float32), ref.r.astype(np.float32)
    h_ref = oracle_mod.synthesize_mr(sc, op, pos_q, g32.astype(np.float64), r32.astype(np.float64))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for tile in (256, 1024, 2048):
        ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len, delay_mode=1, tile=tile))
        h = api.synthesize_raw(ds, dev(hi), dev(lo), dev(g32), dev(r32))
        torch.cuda.synchronize()
        assert ds.status() == 0
        assert _errors(sc, ds, h.cpu().numpy().astype(np.float64), h_ref).max() <= TOL


@pytest.mark.gpu
def test_multirate_full_training_batch_on_sampled_rooms(oracle_mod):
    # The benchmark's configuration: batch_1024 (1024 rooms x 3 sources x 8 mics, 16 kHz) with early
    # RIRs in one launch.  The oracle draws every room's images (FP64), both sides get them rounded
    # to float pairs, and 6 rooms (including the longest and shortest) are compared.
    import torch
    sc = scenes.batch_1024(0)
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sc, op, 41)
    hi, lo, pos_q = _pair_exact(ref.pos)
    g32, r32 = ref.g.astype(np.float32), ref.r.astype(np.float32)
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len, delay_mode=1))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    h, he = api.synthesize_raw(ds, dev(hi), dev(lo), dev(g32), dev(r32), early=True)
    torch.cuda.synchronize()
    assert ds.status() == 0
    rooms = [int(np.argmax(sc.rt60)), int(np.argmin(sc.rt60)), 0, 333, 700, 1023]
    sub = sc.subset(rooms)
    rows = np.concatenate([np.arange(int(ds.vs_off[b]), int(ds.vs_off[b + 1])) for b in rooms])
    h_ref, he_ref = oracle_mod.synthesize_mr(sub, op, pos_q[rows], g32[rows].astype(np.float64),
                                             r32[rooms].astype(np.float64), early=True)
    rl, ro, _ = oracle_mod.layout(sub.rt60, sub.n_vs, sub.S, sub.M, sub.fs)
    hg, heg = h.cpu().numpy(), he.cpu().numpy()
    for i, b in enumerate(rooms):
        o, n = int(ds.rir_off[b]), int(ds.rir_off[b + 1] - ds.rir_off[b])
        L = int(ds.rir_len[b])
        for s in range(sc.S):
            seg_g = slice(o + s * sc.M * L, o + (s + 1) * sc.M * L)
            seg_r = slice(int(ro[i]) + s * sc.M * L, int(ro[i]) + (s + 1) * sc.M * L)
            for got, want in ((hg[seg_g], h_ref[seg_r]), (heg[seg_g], he_ref[seg_r])):
                assert np.abs(got.astype(np.float64) - want).max() <= TOL * np.abs(want).max(), (b, s)


def _piece_outputs(fs):
    """Output samples per high-pass piece, as the library cuts them: pieces of
    max(16384, 2 W) intermediate samples (W: the smallest multiple of 64 with rho^W <= 1e-9, rho
    the pole radius of the 80 Hz high-pass at r_l fs), rounded up to a multiple of 4 outputs."""
    rl = int(np.floor(np.sqrt(np.floor(1e6 / fs))))
    k = np.tan(np.pi * 80.0 / (rl * fs))
    rho = np.sqrt((1.0 - np.sqrt(2.0) * k + k * k) / (1.0 + np.sqrt(2.0) * k + k * k))
    W = (int(np.ceil(np.log(1e-9) / np.log(rho))) + 63) & ~63
    P = max(16384, 2 * W)
    return ((P + rl - 1) // rl + 3) & ~3


@pytest.mark.gpu
def test_multirate_piece_boundaries(oracle_mod):
    # RIR lengths on and next to multiples of the high-pass pieces: each piece starts its walk 12
    # groups of r_l intermediate samples before its first output from the warm-up state, so the
    # outputs on both sides of every boundary (and a last piece of one sample) must match.
    import torch
    fs = 16000.0
    Pn = _piece_outputs(fs)
    lens = [Pn - 1, Pn, Pn + 1, 2 * Pn, 2 * Pn + 1]
    B = len(lens)
    rt60 = np.array([(L - 0.5) / fs for L in lens], np.float32)
    dims = np.tile(np.array([[6.0, 5.0, 3.0]], np.float32), (B, 1))
    mic = np.tile(np.array([[[4.0, 2.5, 1.2], [4.05, 2.5, 1.2]]], np.float32), (B, 1, 1))
    src = np.tile(np.array([[[2.0, 3.0, 1.5]]], np.float32), (B, 1, 1))
    sc = scenes.Scene("pieces", B, 1, 2, fs, 40, dims, rt60, src, mic, np.full(B, 200, np.int32))
    ds, h, h_ref, he, he_ref = _run(oracle_mod, sc, 71, early=True)
    assert [int(x) for x in ds.rir_len] == lens
    assert _errors(sc, ds, h, h_ref).max() <= TOL
    assert _errors(sc, ds, he, he_ref).max() <= TOL
