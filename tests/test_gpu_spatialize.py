"""Spatialisation (fram_spatialize: FFT overlap-save convolution, SIR/SNR gains, mixture and
targets) against the FP64 oracle's direct convolution (oracle.spatialize), on the same inputs:
RIRs synthesised by the oracle (rounded to float32, the precision the library takes) and seeded
synthetic source signals.  Bar: max-abs error <= 1e-5 of each output channel's peak; gains
within 1e-5 relative.  Block lengths, chunking, ragged lengths, RIRs longer than the mixture,
single-sample RIRs and silent sources are covered; the full training-batch configuration
(batch_1024 RIRs, 4 s sources) is checked on sampled rooms.
"""
import numpy as np
import pytest

from paper_2304_08052_gb300 import api, scenes

TOL = 1e-5


def _oracle_rirs(oracle_mod, sc, seed, early=False):
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sc, op, seed)
    out = oracle_mod.synthesize(sc, op, ref.pos, ref.g, ref.r, early=early)
    return tuple(o.astype(np.float32) for o in out) if early else out.astype(np.float32)


def _chan_err(got, ref, floor=None):
    """Largest error over channels, each relative to that channel's peak (or to floor, the peak
    of the channel's untruncated convolution, where that is larger: the FFT's rounding scales
    with the whole windowed convolution, not with the samples kept)."""
    g = got.reshape(-1, got.shape[-1]).astype(np.float64)
    r = ref.reshape(-1, ref.shape[-1])
    peak = np.abs(r).max(axis=1)
    if floor is not None:
        peak = np.maximum(peak, np.asarray(floor).reshape(-1))
    return float((np.abs(g - r).max(axis=1) / np.maximum(peak, 1e-30)).max())


def _full_peaks(ds, h, signals, gains):
    """Per (room, mic): peak of sum_s g_s (h_{s,m} * x_s) over its full length (numpy)."""
    B, S, N = signals.shape
    out = np.zeros((B, ds.M))
    for b in range(B):
        L = int(ds.rir_len[b])
        for m in range(ds.M):
            acc = np.zeros(N + L - 1)
            for s in range(S):
                o = int(ds.rir_off[b]) + (s * ds.M + m) * L
                acc += gains[b, s] * np.convolve(h[o:o + L].astype(np.float64), signals[b, s].astype(np.float64))
            out[b, m] = np.abs(acc).max()
    return out


def _run(ds, rir, mx, targets=False, trir=None, **kw):
    import torch
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rir_d = dev(rir)
    trir_d = dev(trir) if trir is not None else None
    mix, tg, g = api.spatialize(ds, rir_d, dev(mx.signals), dev(mx.level_db), mx.n_speech, target_rir=trir_d,
                                targets=targets, **kw)
    torch.cuda.synchronize()
    assert api.spatialize_status(ds) == 0
    return mix.cpu().numpy(), (tg.cpu().numpy() if tg is not None else None), g.cpu().numpy()


@pytest.fixture(scope="module")
def small(oracle_mod):
    sc = scenes.tiny(seed=71, B=3, S=3, M=4, images=150, t60_lo=0.15, t60_hi=0.45)
    h, he = _oracle_rirs(oracle_mod, sc, 5, early=True)
    mx = scenes.mixtures(72, sc.B, sc.S, 9000, sc.fs)
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len))
    mix_r, tg_r, g_r = oracle_mod.spatialize(ds.rir_len, ds.rir_off, h, mx.signals, mx.n_speech, mx.level_db,
                                             target_rir=he, M=sc.M)
    return sc, ds, h, he, mx, mix_r, tg_r, g_r


@pytest.mark.gpu
@pytest.mark.parametrize("block", [4096, 8192, 16384])
def test_mixture_targets_and_gains_match_the_oracle(small, block):
    sc, ds, h, he, mx, mix_r, tg_r, g_r = small
    mix, tg, g = _run(ds, h, mx, targets=True, trir=he, block=block)
    assert _chan_err(mix, mix_r) <= TOL
    assert _chan_err(tg, tg_r) <= TOL
    np.testing.assert_allclose(g, g_r, rtol=TOL, atol=0)


@pytest.mark.gpu
def test_chunking_does_not_change_the_result(small):
    sc, ds, h, he, mx, *_ = small
    a = _run(ds, h, mx, targets=True, trir=he, chunk_rooms=1)
    b = _run(ds, h, mx, targets=True, trir=he, chunk_rooms=0)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    c = _run(ds, h, mx, targets=True, trir=he)
    for x, y in zip(a, c):
        np.testing.assert_array_equal(x, y)            # run to run


@pytest.mark.gpu
def test_reverberant_targets_sum_with_the_noise_to_the_mixture(oracle_mod, small):
    sc, ds, h, he, mx, mix_r, *_ = small
    mix, tg, g = _run(ds, h, mx, targets=True)          # targets through the same RIRs
    _, tg_r, _ = oracle_mod.spatialize(ds.rir_len, ds.rir_off, h, mx.signals, mx.n_speech, mx.level_db,
                                       target_rir=h, M=sc.M)
    assert _chan_err(tg, tg_r) <= TOL


@pytest.mark.gpu
@pytest.mark.parametrize("N", [100, 1000, 4096, 4097, 12289])
def test_ragged_mixture_lengths(oracle_mod, N):
    # RIRs from 0.02 s (320 samples) to 0.9 s (14400 samples, longer than most mixtures here).
    sc = scenes.tiny(seed=73, B=3, S=2, M=2, images=60, t60_lo=0.02, t60_hi=0.9)
    h = _oracle_rirs(oracle_mod, sc, 6)
    mx = scenes.mixtures(74, sc.B, sc.S, N, sc.fs, n_speech=1)
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len))
    mix_r, _, g_r = oracle_mod.spatialize(ds.rir_len, ds.rir_off, h, mx.signals, 1, mx.level_db, M=sc.M)
    floor = _full_peaks(ds, h, mx.signals, g_r)       # short mixtures keep only the onset
    for block in (4096, 8192):
        mix, _, g = _run(ds, h, mx, block=block)
        assert _chan_err(mix, mix_r, floor) <= TOL, (N, block)
        if N >= 1000:
            # At N = 100 (6 ms: only the direct-path onset) the mic-0 energies are tiny next to
            # the windowed convolution whose rounding they carry; the mixture check above covers it.
            np.testing.assert_allclose(g, g_r, rtol=TOL, atol=0)


@pytest.mark.gpu
def test_one_sample_mixture(oracle_mod):
    # N = 1: every kept sample is ~0 (the direct path arrives later), so levels are meaningless;
    # the mixture must still match within the rounding of its full windowed convolution.
    sc = scenes.tiny(seed=73, B=3, S=2, M=2, images=60, t60_lo=0.02, t60_hi=0.9)
    h = _oracle_rirs(oracle_mod, sc, 6)
    mx = scenes.mixtures(74, sc.B, sc.S, 1, sc.fs, n_speech=1)
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len))
    mix_r, _, g_r = oracle_mod.spatialize(ds.rir_len, ds.rir_off, h, mx.signals, 1, mx.level_db, M=sc.M)
    mix, _, g = _run(ds, h, mx)
    assert np.isfinite(mix).all() and np.isfinite(g).all()
    floor = _full_peaks(ds, h, mx.signals, np.maximum(g_r, g.astype(np.float64)))
    assert _chan_err(mix, mix_r, floor) <= TOL


@pytest.mark.gpu
def test_single_sample_rirs_and_silent_sources(oracle_mod):
    import torch
    B, S, M, N = 2, 3, 2, 5000
    sc = scenes.tiny(seed=75, B=B, S=S, M=M, images=10, t60_lo=0.1, t60_hi=0.2)
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len))
    rng = np.random.default_rng(9)
    h = rng.standard_normal(ds.rir_total).astype(np.float32)
    mx = scenes.mixtures(76, B, S, N, sc.fs)
    mx.signals[1, 1] = 0.0                           # silent second speaker in room 1
    mx.signals[0, 2] = 0.0                           # silent noise in room 0
    mix_r, _, g_r = oracle_mod.spatialize(ds.rir_len, ds.rir_off, h, mx.signals, mx.n_speech, mx.level_db, M=M)
    mix, _, g = _run(ds, h, mx)
    assert g[1, 1] == 0.0 and g[0, 2] == 0.0
    np.testing.assert_allclose(g, g_r, rtol=TOL, atol=0)
    assert _chan_err(mix, mix_r) <= TOL
    # A one-sample RIR (delta at 0, gain c) gives c x.
    sc1 = scenes.Scene("delta", 1, 1, 1, 16000.0, 40, np.array([[5, 4, 3]], np.float32),
                       np.array([2.0 ** -14], np.float32),                   # L = ceil(0.977) = 1
                       np.zeros((1, 1, 3), np.float32), np.zeros((1, 1, 3), np.float32), np.array([0], np.int32), {})
    ds1 = api.DeviceScene(sc1, api.Params())
    assert int(ds1.rir_len[0]) == 1
    sig = rng.standard_normal((1, 1, 777)).astype(np.float32)
    mx1 = scenes.Mixtures(sig, np.zeros((1, 1), np.float32), 1)
    mix1, _, g1 = _run(ds1, np.array([0.75], np.float32), mx1)
    assert g1[0, 0] == 1.0
    np.testing.assert_allclose(mix1[0, 0], 0.75 * sig[0, 0], rtol=0, atol=1e-6)


@pytest.mark.gpu
@pytest.mark.parametrize("fs,K,S,n_speech,M,N,t60", [
    (48000.0, 63, 2, 1, 3, 48000, (0.6, 1.0)),    # long RIRs: up to 12 partitions per output block
    (16000.0, 40, 1, 1, 1, 20000, (0.2, 0.4)),    # one speaker, one mic, no noise
    (16000.0, 40, 5, 3, 4, 30000, (0.1, 0.3)),    # three speakers and two noise sources
    (16000.0, 40, 8, 6, 2, 9000, (0.1, 0.2)),     # the most sources, 15 speaker pairs (four passes)
])
def test_spatialize_shapes(oracle_mod, fs, K, S, n_speech, M, N, t60):
    sc = scenes.tiny(seed=77 + S, B=2, S=S, M=M, images=100, fs=fs, K=K, t60_lo=t60[0], t60_hi=t60[1])
    h, he = _oracle_rirs(oracle_mod, sc, 8, early=True)
    mx = scenes.mixtures(78 + S, sc.B, sc.S, N, sc.fs, n_speech=n_speech)
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len))
    mix_r, tg_r, g_r = oracle_mod.spatialize(ds.rir_len, ds.rir_off, h, mx.signals, n_speech, mx.level_db,
                                             target_rir=he, M=sc.M)
    mix, tg, g = _run(ds, h, mx, targets=True, trir=he)
    assert _chan_err(mix, mix_r) <= TOL
    assert _chan_err(tg, tg_r) <= TOL
    np.testing.assert_allclose(g, g_r, rtol=TOL, atol=0)


@pytest.mark.gpu
def test_training_batch_on_sampled_rooms(oracle_mod):
    # The full configuration: batch_1024 (1024 rooms x 3 sources x 8 mics, 16 kHz) RIRs rendered
    # on the GPU, 4 s sources, the launch configuration the benchmark times; rooms 0 and 517 are
    # checked against the oracle, whose RIRs for those rooms it synthesises itself.
    import torch
    sc = scenes.batch_1024(0)
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len))
    vs = api.sample(ds, seed=11)
    rir = api.synthesize(ds, vs)
    mx = scenes.mixtures(12, sc.B, sc.S, 64000, sc.fs)
    rooms = [0, 517]
    sub = sc.subset(rooms)
    # Replace those rooms' RIRs by the oracle's (same seed, same room indices) on both sides.
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sub, op, 11, room_ids=np.array(rooms, np.int32))
    h_sub = oracle_mod.synthesize(sub, op, ref.pos, ref.g, ref.r).astype(np.float32)
    rl, ro, _ = oracle_mod.layout(sub.rt60, sub.n_vs, sub.S, sub.M, sub.fs)
    for i, b in enumerate(rooms):
        o, n = int(ds.rir_off[b]), int(ds.rir_off[b + 1] - ds.rir_off[b])
        rir[o:o + n] = torch.from_numpy(h_sub[int(ro[i]):int(ro[i + 1])]).cuda()
    mix, _, g = api.spatialize(ds, rir, torch.from_numpy(mx.signals).cuda(), torch.from_numpy(mx.level_db).cuda(),
                               mx.n_speech)
    torch.cuda.synchronize()
    assert api.spatialize_status(ds) == 0
    mix_r, _, g_r = oracle_mod.spatialize(rl, ro, h_sub, mx.signals[rooms], mx.n_speech, mx.level_db[rooms], M=sc.M)
    got = mix.cpu().numpy()[rooms]
    assert _chan_err(got, mix_r) <= TOL
    np.testing.assert_allclose(g.cpu().numpy()[rooms], g_r, rtol=TOL, atol=0)
    assert torch.isfinite(mix).all()
