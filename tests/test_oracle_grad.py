"""Pin for the oracle's analytic gradient: central finite differences of the oracle's own
forward synthesis (FP64, step 1e-6 m on positions, relative 1e-7 on r).

The loss is L = sum (h - y)^2 + sum (h_e - y_e)^2 with seeded Gaussian targets, so both the
RIR and the early-RIR paths of the gradient are exercised.  A dropped chain-rule term, a
wrong sign or a transposed mic/image index shows up as a mismatch far above the finite-
difference error (~1e-8 relative here).
"""
import numpy as np
import pytest

from paper_2304_08052_gb300 import scenes


def _loss(oracle_mod, sc, p, pos, g, r, y, ye):
    h, he = oracle_mod.synthesize(sc, p, pos, g, r, early=True)
    return np.sum((h - y) ** 2) + np.sum((he - ye) ** 2)


@pytest.fixture(scope="module")
def setup(oracle_mod):
    sc = scenes.tiny(seed=21, B=2, S=2, M=3, images=5, t60_lo=0.05, t60_hi=0.07)
    # Use FP64 copies so finite-difference steps are not rounded to float32.
    sc.src = sc.src.astype(np.float64)
    sc.mic = sc.mic.astype(np.float64)
    p = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    out = oracle_mod.sample(sc, p, seed=5)
    # Pull the images close so their windows fall inside the short RIRs.
    pos = out.pos.copy()
    for b in range(sc.B):
        c = sc.mic[b].mean(axis=0)
        sl = slice(b * sc.S * 5, (b + 1) * sc.S * 5)
        d = pos[sl] - c
        pos[sl] = c + d / np.linalg.norm(d, axis=1, keepdims=True) * np.linspace(1.0, 12.0, d.shape[0])[:, None]
    g, r = out.g.copy(), out.r.copy()
    rng = np.random.default_rng(0)
    h, he = oracle_mod.synthesize(sc, p, pos, g, r, early=True)
    y = rng.normal(size=h.shape) * 0.1
    ye = rng.normal(size=h.shape) * 0.1
    grads = oracle_mod.backward(sc, p, pos, g, r, 2 * (h - y), 2 * (he - ye))
    return sc, p, pos, g, r, y, ye, grads


def _fd(f, x0, step):
    return (f(x0 + step) - f(x0 - step)) / (2 * step)


def test_gradient_matches_central_differences(oracle_mod, setup):
    sc, p, pos, g, r, y, ye, (gv, gm, gs, gr) = setup
    L = lambda **kw: _loss(oracle_mod, kw.get("sc", sc), p, kw.get("pos", pos), g, kw.get("r", r), y, ye)
    h = 1e-6
    scale = max(np.abs(gv).max(), np.abs(gm).max(), np.abs(gs).max())
    checks = []
    for b in range(sc.B):
        for s in range(sc.S):
            for k in range(3):
                def f(v, b=b, s=s, k=k):
                    sc2 = scenes.Scene(**{**sc.__dict__})
                    sc2.src = sc.src.copy()
                    sc2.src[b, s, k] = v
                    return L(sc=sc2)
                checks.append((_fd(f, sc.src[b, s, k], h), gs[b, s, k]))
        for m in range(sc.M):
            for k in range(3):
                def f(v, b=b, m=m, k=k):
                    sc2 = scenes.Scene(**{**sc.__dict__})
                    sc2.mic = sc.mic.copy()
                    sc2.mic[b, m, k] = v
                    return L(sc=sc2)
                checks.append((_fd(f, sc.mic[b, m, k], h), gm[b, m, k]))
    for v in (0, 3, 7, 12, 19):
        for k in range(3):
            def f(val, v=v, k=k):
                pp = pos.copy()
                pp[v, k] = val
                return L(pos=pp)
            checks.append((_fd(f, pos[v, k], h), gv[v, k]))
    fd = np.array([c[0] for c in checks])
    an = np.array([c[1] for c in checks])
    assert np.max(np.abs(fd - an)) < 1e-6 * scale, np.max(np.abs(fd - an)) / scale
    for b in range(sc.B):
        def f(val, b=b):
            rr = r.copy()
            rr[b] = val
            return L(r=rr)
        fd_r = _fd(f, r[b], 1e-7 * r[b])
        assert abs(fd_r - gr[b]) < 1e-6 * max(abs(gr[b]), 1.0)


def test_gradient_is_zero_without_upstream(oracle_mod, setup):
    sc, p, pos, g, r, _, _, _ = setup
    n = oracle_mod.synthesize(sc, p, pos, g, r).size
    gv, gm, gs, gr = oracle_mod.backward(sc, p, pos, g, r, np.zeros(n), None)
    assert not gv.any() and not gm.any() and not gs.any() and not gr.any()


def test_translation_invariance_of_position_gradients(oracle_mod, setup):
    # Moving source, mics and images together leaves every distance, hence h, unchanged, so
    # the position gradients of each room sum to zero.
    sc, p, pos, g, r, y, ye, (gv, gm, gs, gr) = setup
    per = sc.S * 5
    for b in range(sc.B):
        tot = gv[b * per:(b + 1) * per].sum(axis=0) + gm[b].sum(axis=0) + gs[b].sum(axis=0)
        assert np.max(np.abs(tot)) < 1e-9 * max(np.abs(gv).max(), 1.0)
