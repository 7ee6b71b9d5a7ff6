"""Pins of the oracle's multi-rate output path (the paper's Sec. II-B and Eq. 7-9 as printed):
impulses quantised to the r_h fs grid, resampled to r_l fs, an 80 Hz high-pass, resampled to fs.

The paper names the rates but not the filters; the readings are a Kaiser-windowed (beta 5)
sinc lowpass for the polyphase resamplers and a 2nd-order Butterworth high-pass.  What pins
them here, without reusing the oracle's arithmetic:
  * the rates: the paper's formulas r_h = floor(1e6 / fs), r_l = floor(sqrt(r_h));
  * the resampling filter: scipy.signal.firwin's Kaiser windowed-sinc design (a library
    routine), times the interpolation gain `up`;
  * the high-pass: scipy.signal.butter's bilinear Butterworth design, and |H| = 1/sqrt(2) at
    80 Hz (the Butterworth closed form);
  * the whole chain: a dense pipeline on the literal high-rate impulse train -- zero-stuffing,
    full convolution and decimation by scipy.signal.upfirdn, the recursion by
    scipy.signal.lfilter -- against the oracle's sparse evaluation;
  * Eq. 7's ceil and its clamp to L - 1, and Eq. 9's mask on the high-rate grid.
"""
import math

import numpy as np
import pytest

signal = pytest.importorskip("scipy.signal")

from paper_2304_08052_gb300 import scenes


def test_rates_follow_the_paper():
    import oracle
    for fs in (8000.0, 16000.0, 22050.0, 44100.0, 48000.0):
        rh = math.floor(1e6 / fs)
        assert oracle.mr_rates(fs) == (rh, math.floor(math.sqrt(rh)))


@pytest.mark.parametrize("up,down", [(7, 62), (1, 5), (1, 7), (1, 4), (11, 125)])
def test_resample_filter_is_the_kaiser_windowed_sinc(up, down):
    import oracle
    F = oracle.resample_filter(up, down)
    mx = max(up, down)
    ref = up * signal.firwin(2 * 10 * mx + 1, 1.0 / mx, window=("kaiser", 5.0))
    np.testing.assert_allclose(F, ref, rtol=0, atol=1e-12 * up)
    assert F.sum() == pytest.approx(up, rel=1e-12)
    np.testing.assert_array_equal(F, F[::-1])


def test_highpass_is_the_butterworth_design():
    import oracle
    for fsr in (112000.0, 80000.0, 192000.0):
        b, a = oracle.hpf_coeffs(80.0, fsr)
        bs, as_ = signal.butter(2, 80.0, btype="highpass", fs=fsr)
        np.testing.assert_allclose(b, bs, rtol=1e-10)
        np.testing.assert_allclose(a, as_, rtol=1e-10)
        _, h = signal.freqz(b, a, worN=[80.0, 1e-3, 5000.0], fs=fsr)
        assert abs(h[0]) == pytest.approx(1 / math.sqrt(2), rel=1e-9)
        assert abs(h[1]) < 1e-9
        assert abs(h[2]) == pytest.approx(1.0, abs=1e-3)


def _tiny(seed, images=25, t60=0.08, fs=16000.0):
    sc = scenes.tiny(seed=seed, B=1, S=1, M=2, images=images, fs=fs, t60_lo=t60, t60_hi=t60 + 1e-6)
    return sc


def _dense_chain(q, A, Lh, fs, L):
    """The literal pipeline: impulse train at r_h fs -> upfirdn(up, down) -> lfilter -> upfirdn."""
    import oracle
    rh, rl = oracle.mr_rates(fs)
    g = math.gcd(rh, rl)
    upA, downA = rl // g, rh // g
    x = np.zeros(Lh)
    np.add.at(x, q, A)
    FA = oracle.resample_filter(upA, downA)
    HLA = (len(FA) - 1) // 2
    full = signal.upfirdn(FA, x, up=upA, down=1)          # x upsampled by upA, filtered
    Lm = -(-Lh * upA // downA)
    idx = np.arange(Lm) * downA + HLA                        # centred filter: shift by HL
    y1 = np.where(idx < len(full), full[np.minimum(idx, len(full) - 1)], 0.0)
    b, a = signal.butter(2, 80.0, btype="highpass", fs=rl * fs)
    z = signal.lfilter(b, a, y1)
    FC = oracle.resample_filter(1, rl)
    HLC = (len(FC) - 1) // 2
    fullc = np.convolve(z, FC)
    idc = np.arange(L) * rl + HLC
    return np.where(idc < len(fullc), fullc[np.minimum(idc, len(fullc) - 1)], 0.0)


@pytest.mark.parametrize("fs", [16000.0, 48000.0])
def test_sparse_chain_matches_the_dense_pipeline(oracle_mod, fs):
    sc = _tiny(3, fs=fs)
    op = oracle_mod.Params(fs=fs, half_len=40)
    ref = oracle_mod.sample(sc, op, 4)
    h = oracle_mod.synthesize_mr(sc, op, ref.pos, ref.g, ref.r)
    rh, rl = oracle_mod.mr_rates(fs)
    fh = rh * fs
    Lh = math.ceil(float(np.float32(sc.rt60[0])) * fh)
    L = math.ceil(float(np.float32(sc.rt60[0])) * fs)
    assert h.size == sc.M * L
    for m in range(sc.M):
        mic = sc.mic[0, m].astype(np.float64)
        D0 = np.linalg.norm(sc.src[0, 0].astype(np.float64) - mic)
        D = np.linalg.norm(ref.pos - mic, axis=1)
        q = np.minimum(np.ceil(np.concatenate([[D0], D]) / op.c0 * fh), Lh - 1).astype(np.int64)
        A = np.concatenate([[1.0 / D0], ref.r[0] ** ref.g / D])
        dense = _dense_chain(q, A, Lh, fs, L)
        got = h[m * L:(m + 1) * L]
        assert np.abs(got - dense).max() <= 1e-10 * np.abs(dense).max()


def test_delay_is_ceil_on_the_high_rate_grid_and_clamped(oracle_mod):
    # One source, no images: with c0 = 250 m/s, fs = 16 kHz (r_h fs = 992 kHz) and the source
    # 0.5 m from a single mic, D r_h fs / c0 = 1984 exactly: q = 1984.  Moving the source by
    # 1e-6 m pushes it to 1985.  A source beyond c0 T60 lands on L_h - 1.
    fs, c0 = 16000.0, 250.0
    op = oracle_mod.Params(fs=fs, half_len=40, c0=c0)
    rh, rl = oracle_mod.mr_rates(fs)
    fh = rh * fs
    for dist, expect in ((0.5, 1984), (0.5 + 1e-6, 1985), (30.0, None)):
        sc = scenes.Scene("one", 1, 1, 1, fs, 40, np.array([[40.0, 40.0, 40.0]], np.float32),
                          np.array([0.1], np.float32), np.array([[[1.0 + dist, 1.0, 1.0]]], np.float64),
                          np.array([[[1.0, 1.0, 1.0]]], np.float64), np.array([0], np.int32), {})
        h = oracle_mod.synthesize_mr(sc, op, np.zeros((0, 3)), np.zeros(0), np.array([0.5]))
        Lh = math.ceil(float(np.float32(0.1)) * fh)
        L = math.ceil(float(np.float32(0.1)) * fs)
        q = expect if expect is not None else Lh - 1
        dense = _dense_chain(np.array([q]), np.array([1.0 / dist]), Lh, fs, L)
        np.testing.assert_allclose(h, dense, rtol=0, atol=1e-12 / dist)
        if expect is not None:   # the neighbouring grid point gives a different RIR
            other = _dense_chain(np.array([q - 1]), np.array([1.0 / dist]), Lh, fs, L)
            assert np.abs(other - h).max() > 1e-6 / dist


def test_early_mask_is_applied_on_the_high_rate_grid(oracle_mod):
    sc = _tiny(5, images=60, t60=0.15)
    op = oracle_mod.Params(fs=16000.0, half_len=40)
    ref = oracle_mod.sample(sc, op, 6)
    h, he = oracle_mod.synthesize_mr(sc, op, ref.pos, ref.g, ref.r, early=True)
    rh, rl = oracle_mod.mr_rates(16000.0)
    fh = rh * 16000.0
    Lh = math.ceil(float(np.float32(sc.rt60[0])) * fh)
    L = math.ceil(float(np.float32(sc.rt60[0])) * 16000.0)
    for m in range(sc.M):
        mic = sc.mic[0, m].astype(np.float64)
        D0 = np.linalg.norm(sc.src[0, 0].astype(np.float64) - mic)
        D = np.linalg.norm(ref.pos - mic, axis=1)
        q = np.minimum(np.ceil(np.concatenate([[D0], D]) / op.c0 * fh), Lh - 1).astype(np.int64)
        A = np.concatenate([[1.0 / D0], ref.r[0] ** ref.g / D])
        n0 = math.ceil(D0 / op.c0 * fh)
        keep = (q >= n0 - math.ceil(6 * fh / 1000)) & (q <= n0 + math.ceil(50 * fh / 1000))
        dense = _dense_chain(q[keep], A[keep], Lh, 16000.0, L)
        got = he[m * L:(m + 1) * L]
        assert np.abs(got - dense).max() <= 1e-10 * np.abs(dense).max()
        assert keep.sum() < keep.size            # some images fall outside the window
