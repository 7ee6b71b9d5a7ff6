"""Pins for the oracle's RIR synthesis (Eq. 1 with windowed-sinc fractional delays, Eq. 9).

None of these re-evaluates the oracle's own tap formula; each uses a property that any
correct fractional-delay windowed-sinc synthesis must have:
  * an integer delay gives exactly one nonzero tap of the stated amplitude 1/D (sinc vanishes
    at nonzero integers);
  * band-limited interpolation: a single impulse correlated with a sampled sinusoid returns
    the sinusoid at the fractional delay (this fixes the sign and origin of the delay);
  * TDOA: the DTFT phase difference between two mics of a direct-path-only RIR equals the
    geometric path difference times fs/c0 (the property the paper requires of the method);
  * superposition over images, one-sample time shift, half-sample symmetry;
  * Schroeder backward-integrated decay follows the requested T60 across rooms;
  * Eq. 9: h_e is h inside [-ceil(6 fs/1000), +ceil(50 fs/1000)] around ceil(D0 fs/c0).
A direct Python double loop (np.sinc and an explicit Hann) checks the C code on tiny
inputs as a consistency test.
"""
import numpy as np
import pytest
from scipy import stats

from paper_2304_08052_gb300 import scenes


def _one_room(src, mics, rt60=0.05, n_vs=0, dims=(20.0, 20.0, 20.0), fs=16000.0, K=40, dtype=np.float64):
    mics = np.asarray(mics, dtype)
    return scenes.Scene("probe", 1, 1, len(mics), fs, K, np.array([dims], dtype),
                        np.array([rt60], np.float32), np.array([[src]], dtype), mics[None],
                        np.array([n_vs], np.int32))


def _direct_only(oracle_mod, sc, p):
    return oracle_mod.synthesize(sc, p, np.zeros((0, 3)), np.zeros(0), np.array([0.9]))


def test_integer_delay_gives_single_tap(oracle_mod):
    p = oracle_mod.Params(fs=16000.0, half_len=40, c0=320.0)       # 50 samples per metre
    sc = _one_room([1.0, 1.0, 1.0], [[3.0, 1.0, 1.0]])             # D = 2 m -> t = 100
    h = _direct_only(oracle_mod, sc, p)
    assert h.shape == (801,)                  # ceil(float32(0.05) * 16000) = 801
    assert abs(h[100] - 0.5) < 1e-15
    others = np.delete(h, 100)
    assert np.max(np.abs(others)) < 1e-15


@pytest.mark.parametrize("frac", [0.0, 0.123, 0.37, -0.49, 0.5])
def test_fractional_delay_interpolates_sinusoids(oracle_mod, frac):
    p = oracle_mod.Params(fs=16000.0, half_len=40, c0=320.0)
    t = 160.0 + frac
    D = t / 50.0
    sc = _one_room([1.0, 1.0, 1.0], [[1.0 + D, 1.0, 1.0]], rt60=0.05)
    h = _direct_only(oracle_mod, sc, p)
    A = 1.0 / D
    n = np.arange(h.size)
    for w in (0.0, 0.05 * np.pi, 0.2 * np.pi, 0.45 * np.pi):
        got = np.sum(h * np.exp(1j * w * n)) / A
        want = np.exp(1j * w * t)
        # Hann-windowed sinc, K = 40: passband error well below 1e-2 up to 0.45 pi, while a
        # reversed delay sign or a one-sample offset errs by O(w * |frac|) or O(w).
        assert abs(got - want) < 5e-3, (w, got, want)


def test_direct_path_tdoa_matches_geometry(oracle_mod):
    p = oracle_mod.Params(fs=16000.0, half_len=40)
    mics = [[4.0 + dx, 2.5, 1.2] for dx in (-0.075, -0.025, 0.025, 0.075)]
    src = [2.0, 3.0, 1.5]
    sc = _one_room(src, mics, rt60=0.05)
    h = _direct_only(oracle_mod, sc, p).reshape(4, -1)
    n = np.arange(h.shape[1])
    w = 0.05 * np.pi                          # phase period 40 samples > any TDOA here
    H = (h * np.exp(-1j * w * n)).sum(axis=1)
    dist = np.linalg.norm(np.asarray(mics) - np.asarray(src), axis=1)
    for m in range(1, 4):
        tdoa = -np.angle(H[m] * np.conj(H[0])) / w
        assert abs(tdoa - (dist[m] - dist[0]) * p.fs / p.c0) < 2e-3


def test_superposition_over_images(oracle_mod):
    sc = scenes.tiny(seed=2, B=1, S=1, M=2, images=8)
    p = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    out = oracle_mod.sample(sc, p, seed=7)
    off = 1e7   # r**g underflows to exactly zero: the image is switched off
    g_all = out.g.copy()
    g_a = np.where(np.arange(8) < 3, out.g, off)
    g_b = np.where(np.arange(8) >= 3, out.g, off)
    g_none = np.full(8, off)
    h = {k: oracle_mod.synthesize(sc, p, out.pos, g, out.r) for k, g in
         dict(all=g_all, a=g_a, b=g_b, none=g_none).items()}
    peak = np.max(np.abs(h["all"]))
    assert np.max(np.abs(h["all"] + h["none"] - h["a"] - h["b"])) < 1e-14 * peak


def test_one_sample_time_shift(oracle_mod):
    p = oracle_mod.Params(fs=16000.0, half_len=40)
    src = np.array([1.0, 2.0, 1.5])
    mic = np.array([3.3, 2.7, 1.1])
    u = (src - mic) / np.linalg.norm(src - mic)
    sc1 = _one_room(src, [mic])
    sc2 = _one_room(src + u * p.c0 / p.fs, [mic])
    h1 = _direct_only(oracle_mod, sc1, p)
    h2 = _direct_only(oracle_mod, sc2, p)
    D1, D2 = np.linalg.norm(src - mic), np.linalg.norm(src - mic) + p.c0 / p.fs
    assert np.max(np.abs(h2[1:] * D2 - h1[:-1] * D1)) < 1e-12


def test_half_sample_delay_is_symmetric(oracle_mod):
    p = oracle_mod.Params(fs=16384.0, half_len=40, c0=256.0)        # 64 samples per metre
    sc = _one_room([1.0, 1.0, 1.0], [[1.0 + 100.5 / 64.0, 1.0, 1.0]], rt60=0.02)
    h = _direct_only(oracle_mod, sc, p)
    j = np.arange(40)
    assert np.max(np.abs(h[100 - j] - h[101 + j])) < 1e-15
    assert np.all(h[100 - j[:1]] > 0)


def test_brute_force_double_loop_tiny(oracle_mod):
    sc = scenes.tiny(seed=4, B=2, S=2, M=2, images=6)
    p = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    out = oracle_mod.sample(sc, p, seed=1)
    rir_len, rir_off, vs_off = oracle_mod.layout(sc.rt60, sc.n_vs, sc.S, sc.M, sc.fs)
    h, he = oracle_mod.synthesize(sc, p, out.pos, out.g, out.r, early=True)
    K = p.half_len
    q = p.fs / p.c0
    for b in range(sc.B):
        L = int(rir_len[b])
        for s in range(sc.S):
            ps = sc.src[b, s].astype(np.float64)
            for m in range(sc.M):
                pm = sc.mic[b, m].astype(np.float64)
                imp = [(np.linalg.norm(ps - pm), 1.0 / np.linalg.norm(ps - pm))]
                for i in range(int(sc.n_vs[b])):
                    v = vs_off[b] + s * sc.n_vs[b] + i
                    D = np.linalg.norm(out.pos[v] - pm)
                    imp.append((D, out.r[b] ** out.g[v] / D))
                ref = np.zeros(L)
                n = np.arange(L)
                for D, A in imp:
                    x = n - D * q
                    tap = np.where(np.abs(x) < K, np.sinc(x) * 0.5 * (1 + np.cos(np.pi * x / K)), 0.0)
                    ref += A * tap
                base = rir_off[b] + (s * sc.M + m) * L
                assert np.max(np.abs(h[base:base + L] - ref)) < 1e-12
                n0 = int(np.ceil(imp[0][0] * q))
                mask = (n >= n0 - 96) & (n <= n0 + 800)
                assert np.array_equal(he[base:base + L], np.where(mask, h[base:base + L], 0.0))


def test_early_window_single_room(oracle_mod):
    sc = scenes.single_room()
    p = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    out = oracle_mod.sample(sc, p, seed=0)
    h, he = oracle_mod.synthesize(sc, p, out.pos, out.g, out.r, early=True)
    h, he = h.reshape(4, -1), he.reshape(4, -1)
    for m in range(4):
        d0 = np.linalg.norm(sc.src[0, 0].astype(np.float64) - sc.mic[0, m].astype(np.float64))
        n0 = int(np.ceil(d0 * 16000 / 343.0))
        inside = np.zeros(8000, bool)
        inside[max(n0 - 96, 0):n0 + 801] = True
        assert np.array_equal(he[m][inside], h[m][inside])
        assert np.all(he[m][~inside] == 0)
        # The direct path is the strongest early arrival at its own mic.
        assert abs(np.argmax(np.abs(h[m])) - d0 * 16000 / 343.0) < 1.0


def test_schroeder_decay_tracks_requested_t60(oracle_mod):
    sc = scenes.tiny(seed=8, B=48, S=1, M=1, images=1, t60_lo=0.15, t60_hi=0.7, fs=8000.0, K=16)
    sc.n_vs[:] = np.floor(2000 * sc.rt60.astype(np.float64) + 0.5).astype(np.int32)
    p = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    out = oracle_mod.sample(sc, p, seed=3)
    h = oracle_mod.synthesize(sc, p, out.pos, out.g, out.r)
    rir_len, rir_off, _ = oracle_mod.layout(sc.rt60, sc.n_vs, 1, 1, sc.fs)
    est = []
    for b in range(sc.B):
        x = h[rir_off[b]:rir_off[b + 1]]
        edc = np.cumsum((x ** 2)[::-1])[::-1]
        edc_db = 10 * np.log10(edc / edc[0])
        sel = (edc_db <= -5) & (edc_db >= -25)
        tt = np.nonzero(sel)[0] / sc.fs
        slope = np.polyfit(tt, edc_db[sel], 1)[0]
        est.append(-60.0 / slope)
    est = np.array(est)
    rho = stats.spearmanr(est, sc.rt60).correlation
    ratio = np.median(est / sc.rt60)
    # This test pins only monotone tracking of the requested T60 across rooms (the band is wide).
    # The level of the ratio is pinned by test_oracle_envelope.py, which derives the expected
    # energy envelope from Eq. 2-6 by quadrature (about 2x T60 for this project's alpha, beta, a,
    # b, tau: Eq. 6's trend is quadratic in distance and Eq. 3 puts more images far away).
    assert rho > 0.9, rho
    assert 1.4 < ratio < 2.8, ratio
