"""Pins of the oracle's spatialisation (Sec. IV-A: sources convolved with their RIRs, speakers
mixed at an SIR, point-source noise at an SNR; readings in fram_oracle.c).

What fixes it, without reusing its arithmetic:
  * the images: numpy.convolve (a library routine) truncated to the mixture length;
  * a delayed unit impulse as the RIR returns the signal delayed (closed form);
  * the gains: the SIR and SNR measured on the oracle's own outputs equal the requested levels
    (10 log10 of energy ratios at mic 0), and a silent source gets gain 0;
  * the mixture: speakers' targets (taken through the same RIRs) plus the noise image rebuilt
    with numpy.convolve equal the mixture;
  * targets through a second RIR set (an early-RIR-like truncation) equal g_s (h' * x_s).
"""
import numpy as np
import pytest

from paper_2304_08052_gb300 import scenes


def _ragged(seed, B, S, M, lens):
    """Decaying-noise RIRs in the library's ragged layout: room b at off[b], [S][M][L_b]."""
    rng = np.random.default_rng(seed)
    lens = np.asarray(lens, np.int32)
    off = np.zeros(B + 1, np.int64)
    off[1:] = np.cumsum(S * M * lens.astype(np.int64))
    h = np.empty(int(off[-1]))
    for b in range(B):
        L = int(lens[b])
        env = np.exp(-np.arange(L) / (0.2 * L))
        for s in range(S):
            for m in range(M):
                o = int(off[b]) + (s * M + m) * L
                h[o:o + L] = rng.standard_normal(L) * env
    return lens, off, h


def _chan(h, off, lens, M, b, s, m):
    L = int(lens[b])
    o = int(off[b]) + (s * M + m) * L
    return h[o:o + L]


@pytest.fixture(scope="module")
def case(oracle_mod):
    B, S, M, N = 3, 3, 2, 700
    lens, off, h = _ragged(1, B, S, M, [150, 333, 1000])     # one RIR longer than the mixture
    mx = scenes.mixtures(2, B, S, N, 16000.0)
    early = h.copy()
    for b in range(B):                                        # a second RIR set: first 40 taps
        for s in range(S):
            for m in range(M):
                L = int(lens[b])
                o = int(off[b]) + (s * M + m) * L
                early[o + 40:o + L] = 0.0
    mix, tg, g = oracle_mod.spatialize(lens, off, h, mx.signals, mx.n_speech, mx.level_db, target_rir=h, M=M)
    _, tge, ge = oracle_mod.spatialize(lens, off, h, mx.signals, mx.n_speech, mx.level_db, target_rir=early, M=M)
    return dict(B=B, S=S, M=M, N=N, lens=lens, off=off, h=h, early=early, mx=mx, mix=mix, tg=tg, g=g, tge=tge,
                ge=ge)


def _image(c, b, s, m, rir=None):
    h = _chan(c["h"] if rir is None else rir, c["off"], c["lens"], c["M"], b, s, m)
    x = c["mx"].signals[b, s].astype(np.float64)
    return np.convolve(h, x)[:c["N"]]


def test_speaker_targets_are_the_scaled_images(case):
    c = case
    for b in range(c["B"]):
        for s in range(c["mx"].n_speech):
            for m in range(c["M"]):
                ref = c["g"][b, s] * _image(c, b, s, m)
                np.testing.assert_allclose(c["tg"][b, s, m], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_levels_are_the_requested_sir_and_snr(case):
    c = case
    ns = c["mx"].n_speech
    for b in range(c["B"]):
        assert c["g"][b, 0] == 1.0
        e0 = np.sum(c["tg"][b, 0, 0] ** 2)
        for s in range(1, ns):
            sir = 10 * np.log10(e0 / np.sum(c["tg"][b, s, 0] ** 2))
            assert sir == pytest.approx(c["mx"].level_db[b, s], abs=1e-9)
        speech = c["tg"][b, :ns, 0].sum(axis=0)
        for s in range(ns, c["S"]):
            noise = c["g"][b, s] * _image(c, b, s, 0)
            snr = 10 * np.log10(np.sum(speech ** 2) / np.sum(noise ** 2))
            assert snr == pytest.approx(c["mx"].level_db[b, s], abs=1e-9)


def test_mixture_is_speech_plus_noise(case):
    c = case
    ns = c["mx"].n_speech
    for b in range(c["B"]):
        for m in range(c["M"]):
            ref = c["tg"][b, :ns, m].sum(axis=0)
            for s in range(ns, c["S"]):
                ref = ref + c["g"][b, s] * _image(c, b, s, m)
            np.testing.assert_allclose(c["mix"][b, m], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_targets_through_a_second_rir_set(case):
    c = case
    np.testing.assert_array_equal(c["ge"], c["g"])              # gains come from the full RIRs
    for b in range(c["B"]):
        for s in range(c["mx"].n_speech):
            for m in range(c["M"]):
                ref = c["g"][b, s] * _image(c, b, s, m, rir=c["early"])
                np.testing.assert_allclose(c["tge"][b, s, m], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_delayed_impulse_rir_delays_the_signal(oracle_mod):
    B, S, M, N, L = 1, 1, 2, 300, 64
    lens = np.array([L], np.int32)
    off = np.array([0, S * M * L], np.int64)
    h = np.zeros(S * M * L)
    h[17] = 1.0                    # mic 0: delay 17
    h[L + 63] = 0.5                # mic 1: delay 63, half amplitude
    x = np.random.default_rng(3).standard_normal((B, S, N))
    mix, _, g = oracle_mod.spatialize(lens, off, h, x, 1, np.zeros((B, S)), M=M)
    assert g[0, 0] == 1.0
    np.testing.assert_array_equal(mix[0, 0, :17], 0.0)
    np.testing.assert_allclose(mix[0, 0, 17:], x[0, 0, :N - 17], rtol=0, atol=0)
    np.testing.assert_allclose(mix[0, 1, 63:], 0.5 * x[0, 0, :N - 63], rtol=0, atol=0)


def test_silent_sources_get_zero_gain(oracle_mod):
    B, S, M, N = 1, 3, 1, 200
    lens, off, h = _ragged(4, B, S, M, [50])
    x = np.random.default_rng(5).standard_normal((B, S, N))
    x[0, 1] = 0.0
    x[0, 2] = 0.0
    mix, _, g = oracle_mod.spatialize(lens, off, h, x, 2, np.array([[0.0, 3.0, 15.0]]), M=M)
    assert g[0, 1] == 0.0 and g[0, 2] == 0.0
    np.testing.assert_allclose(mix[0, 0], np.convolve(h[:50], x[0, 0])[:N], rtol=0, atol=1e-12)


def test_invalid_arguments(oracle_mod):
    lens, off, h = _ragged(6, 1, 2, 1, [10])
    x = np.zeros((1, 2, 20))
    for ns in (0, 3):
        with pytest.raises(ValueError):
            oracle_mod.spatialize(lens, off, h, x, ns, np.zeros((1, 2)), M=1)
