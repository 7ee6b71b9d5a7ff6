"""Pins of the oracle's gradient through the sampler (reparameterised: the Philox draws of every
image held fixed, so images move with the source, the array, T60 and the room size).

The analytic chain (fo_backward for the synthesis, fo_sample_backward for Eq. 2-6) is checked
against central finite differences of the oracle's whole forward pipeline -- sample, synthesize,
L = sum G h -- with the same seed: nothing of the chain rule is reused by the reference.
"""
import numpy as np
import pytest

from paper_2304_08052_gb300 import scenes


def _scene64(sc):
    """The scene with float64 geometry, so that finite differences can perturb it finely."""
    return scenes.Scene(sc.name, sc.B, sc.S, sc.M, sc.fs, sc.half_len, sc.dims.astype(np.float64),
                        sc.rt60.astype(np.float64), sc.src.astype(np.float64), sc.mic.astype(np.float64),
                        sc.n_vs.copy(), dict(sc.meta))


def _loss(oracle_mod, sc, op, seed, G):
    ref = oracle_mod.sample(sc, op, seed)
    h = oracle_mod.synthesize(sc, op, ref.pos, ref.g, ref.r)
    return float(np.dot(G, h))


def _analytic(oracle_mod, sc, op, seed, G):
    ref = oracle_mod.sample(sc, op, seed)
    gv, gm, gs, gr, gg = oracle_mod.backward(sc, op, ref.pos, ref.g, ref.r, G, with_g=True)
    return oracle_mod.sample_backward(sc, op, seed, gv, gg, gr, gs, gm)


@pytest.fixture(scope="module")
def setup(oracle_mod):
    base = scenes.tiny(seed=41, B=2, S=2, M=3, images=80, t60_lo=0.25, t60_hi=0.35)
    sc = _scene64(base)
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    rir_len, rir_off, _ = oracle_mod.layout(base.rt60, base.n_vs, sc.S, sc.M, sc.fs)
    G = np.random.default_rng(5).standard_normal(int(rir_off[-1]))
    return sc, op, 77, G, _analytic(oracle_mod, sc, op, 77, G)


def _fd(oracle_mod, sc, op, seed, G, field, idx, eps):
    vals = []
    for sgn in (1.0, -1.0):
        s2 = _scene64(sc)
        arr = getattr(s2, field)
        arr[idx] += sgn * eps
        vals.append(_loss(oracle_mod, s2, op, seed, G))
    return (vals[0] - vals[1]) / (2 * eps)


def _check(a, f, scale):
    assert abs(a - f) <= 2e-5 * scale + 1e-9, (a, f)


def test_source_gradient_includes_the_images(oracle_mod, setup):
    sc, op, seed, G, (gs, gm, gt, gd) = setup
    scale = np.abs(gs).max()
    for idx in [(0, 0, 0), (0, 1, 2), (1, 0, 1), (1, 1, 0)]:
        _check(gs[idx], _fd(oracle_mod, sc, op, seed, G, "src", idx, 1e-6), scale)


def test_mic_gradient_includes_the_array_centre(oracle_mod, setup):
    sc, op, seed, G, (gs, gm, gt, gd) = setup
    scale = np.abs(gm).max()
    for idx in [(0, 0, 0), (0, 2, 1), (1, 1, 2)]:
        _check(gm[idx], _fd(oracle_mod, sc, op, seed, G, "mic", idx, 1e-6), scale)


def test_t60_gradient(oracle_mod, setup):
    sc, op, seed, G, (gs, gm, gt, gd) = setup
    scale = np.abs(gt).max()
    for b in range(sc.B):
        # below float32 resolution of T60: the RIR length (layout) stays fixed, the FP64 sampler moves
        _check(gt[b], _fd(oracle_mod, sc, op, seed, G, "rt60", (b,), 1e-8), scale)


def test_room_size_gradient(oracle_mod, setup):
    sc, op, seed, G, (gs, gm, gt, gd) = setup
    scale = np.abs(gd).max()
    for idx in [(0, 0), (0, 2), (1, 1)]:
        _check(gd[idx], _fd(oracle_mod, sc, op, seed, G, "dims", idx, 1e-6), scale)


def test_the_sampler_path_is_not_negligible(oracle_mod, setup):
    # Without the sampler path the source gradient is the direct path's alone; the images moving
    # with the source change it by far more than the finite-difference tolerance above.
    sc, op, seed, G, (gs, gm, gt, gd) = setup
    ref = oracle_mod.sample(sc, op, seed)
    _, _, gs_dir, _ = oracle_mod.backward(sc, op, ref.pos, ref.g, ref.r, G)
    assert np.abs(gs - gs_dir).max() > 1e-2 * np.abs(gs).max()
