"""The seeded input generator (scenes.py) against the workload recipes it states: room sizes,
T60 ranges, array shapes and sizes, image counts, source placement (inside the room, at least
0.3 m from the array, Sec. IV-A), and the mixture sources' levels (SIR U[-6, 6] dB, SNR
U[10, 20] dB) and speaker overlap (at least 0.5).  CPU only; no method arithmetic is involved.
"""
import numpy as np
import pytest

from paper_2304_08052_gb300 import scenes

RECIPES = {
    # name: (B, S, M, fs, K, dims_lo, dims_hi, t60 range, geometry, radius or spacing, images)
    "batch_256": (256, 1, 6, 16000.0, 40, [3, 3, 2.5], [10, 8, 4.5], (0.1, 0.7), "circular", 0.05, 4000),
    "batch_1024": (1024, 3, 8, 16000.0, 40, [3, 3, 2.5], [10, 8, 4.5], (0.1, 0.7), "circular", 0.04, 4000),
    "grad_64": (64, 1, 4, 16000.0, 40, [3, 3, 2.5], [10, 8, 4.5], (0.2, 0.6), "linear", 0.05, "1500"),
    "large_4096": (4096, 2, 16, 48000.0, 63, [3, 3, 2.5], [15, 12, 6], (0.2, 1.2), "circular", 0.10, 6000),
}


@pytest.mark.parametrize("name", sorted(RECIPES))
def test_workloads_follow_their_recipes(name):
    B, S, M, fs, K, lo, hi, t60, geometry, size, images = RECIPES[name]
    sc = scenes.CONFIGS[name](0)
    assert (sc.B, sc.S, sc.M, sc.fs, sc.half_len) == (B, S, M, fs, K)
    for a in (sc.dims, sc.rt60, sc.src, sc.mic):
        assert a.dtype == np.float32
    assert (sc.dims >= np.array(lo, np.float32)).all() and (sc.dims <= np.array(hi, np.float32)).all()
    assert (sc.rt60 >= t60[0]).all() and (sc.rt60 <= t60[1]).all()
    if isinstance(images, str):
        assert (sc.n_vs == int(images)).all()
    else:
        want = np.floor(images * sc.rt60.astype(np.float64) + 0.5).astype(np.int32)
        assert np.array_equal(sc.n_vs, want)
    mic = sc.mic.astype(np.float64)
    centre = mic.mean(axis=1)
    rel = mic - centre[:, None, :]
    if geometry == "circular":
        np.testing.assert_allclose(np.linalg.norm(rel, axis=2), size, atol=1e-5)
        assert np.abs(rel[:, :, 2]).max() < 1e-5                       # horizontal plane
        ang = np.arctan2(rel[:, :, 1], rel[:, :, 0])
        step = np.mod(np.diff(ang, axis=1), 2 * np.pi)
        np.testing.assert_allclose(step, 2 * np.pi / M, atol=1e-4)      # equally spaced, in order
    else:
        np.testing.assert_allclose(np.diff(mic[:, :, 0], axis=1), size, atol=1e-5)
        assert np.abs(np.diff(mic[:, :, 1:], axis=1)).max() < 1e-6       # along +x
    # the array point is at least 0.5 m from every wall
    assert (centre >= 0.5 - 1e-5).all() and (centre <= sc.dims - 0.5 + 1e-5).all()
    src = sc.src.astype(np.float64)
    assert (src >= 0).all() and (src <= sc.dims[:, None, :]).all()      # sources inside the room
    assert (np.linalg.norm(src - centre[:, None, :], axis=2) >= 0.3 - 1e-5).all()


def test_single_room_is_the_stated_scene():
    sc = scenes.single_room()
    assert (sc.B, sc.S, sc.M, sc.fs, sc.half_len) == (1, 1, 4, 16000.0, 40)
    np.testing.assert_array_equal(sc.dims[0], np.float32([6, 5, 3]))
    assert sc.rt60[0] == np.float32(0.5) and sc.n_vs[0] == 2000
    np.testing.assert_array_equal(sc.src[0, 0], np.float32([2, 3, 1.5]))
    np.testing.assert_allclose(sc.mic[0].mean(axis=0), [4.0, 2.5, 1.2], atol=1e-6)
    np.testing.assert_allclose(np.diff(sc.mic[0, :, 0]), 0.05, atol=1e-6)


def test_draws_are_seeded():
    a, b, c = scenes.batch_256(3), scenes.batch_256(3), scenes.batch_256(4)
    for x, y in ((a.dims, b.dims), (a.rt60, b.rt60), (a.src, b.src), (a.mic, b.mic)):
        assert np.array_equal(x, y)
    assert not np.array_equal(a.src, c.src)
    sub = a.subset([5, 2])
    assert np.array_equal(sub.src, a.src[[5, 2]]) and np.array_equal(sub.n_vs, a.n_vs[[5, 2]])


def test_mixture_sources_follow_the_recipe():
    B, S, N, fs = 40, 3, 16000, 16000.0
    mx = scenes.mixtures(9, B, S, N, fs)
    assert mx.n_speech == 2 and mx.signals.shape == (B, S, N) and mx.signals.dtype == np.float32
    np.testing.assert_allclose(np.abs(mx.signals).max(axis=2), 1.0, atol=1e-6)   # peak-normalised
    assert (mx.level_db[:, 0] == 0).all()                                         # speaker 0: reference
    assert (mx.level_db[:, 1] >= -6).all() and (mx.level_db[:, 1] <= 6).all()    # SIR
    assert (mx.level_db[:, 2] >= 10).all() and (mx.level_db[:, 2] <= 20).all()   # SNR
    active = mx.signals != 0
    both = (active[:, 0] & active[:, 1]).mean(axis=1)                            # speaker overlap ratio
    assert (both >= 0.5 - 1e-3).all() and (both <= 1.0).all()
    assert (active[:, 2].mean(axis=1) > 0.999).all()                              # noise spans the mixture
    assert np.array_equal(mx.signals, scenes.mixtures(9, B, S, N, fs).signals)
    one = scenes.mixtures(1, 2, 1, 500, fs)
    assert one.n_speech == 1 and (one.level_db == 0).all()
