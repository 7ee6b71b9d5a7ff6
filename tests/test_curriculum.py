"""T60 curriculum (the paper's "T60 curriculum training" subsection): the schedule and the batches
it draws.  The GPU test runs a first-epoch batch (the shortest RIRs) through the C ABI against the
FP64 oracle."""
import numpy as np
import pytest

from paper_2304_08052_gb300 import curriculum


def test_schedule_follows_the_paper():
    # [50, 100] ms at the first epoch, +50 ms per epoch, stopped at the required maximum.
    assert curriculum.t60_range(0, 0.7) == pytest.approx((0.05, 0.10))
    assert curriculum.t60_range(1, 0.7) == pytest.approx((0.05, 0.15))
    assert curriculum.t60_range(5, 0.7) == pytest.approx((0.05, 0.35))
    assert curriculum.t60_range(12, 0.7) == pytest.approx((0.05, 0.7))
    assert curriculum.t60_range(100, 0.7) == pytest.approx((0.05, 0.7))
    his = [curriculum.t60_range(e, 1.2)[1] for e in range(40)]
    assert all(b >= a for a, b in zip(his, his[1:]))
    assert his.index(1.2) == 22                      # 0.10 + 0.05 * 22 = 1.2


def test_schedule_rejects_bad_arguments():
    with pytest.raises(ValueError):
        curriculum.t60_range(-1, 0.7)
    with pytest.raises(ValueError):
        curriculum.t60_range(0, 0.0)


def test_batches_respect_the_range():
    for epoch in (0, 3, 30):
        lo, hi = curriculum.t60_range(epoch, 0.7)
        sc = curriculum.curriculum_batch(seed=epoch, epoch=epoch, t60_max=0.7, B=64)
        assert sc.B == 64
        assert np.all(sc.rt60 >= np.float32(lo)) and np.all(sc.rt60 <= np.float32(hi))
        np.testing.assert_array_equal(sc.n_vs, np.floor(4000.0 * sc.rt60.astype(np.float64) + 0.5))


@pytest.mark.gpu
def test_first_epoch_batch_matches_the_oracle(oracle_mod):
    import torch
    from paper_2304_08052_gb300 import api
    sc = curriculum.curriculum_batch(seed=5, epoch=0, t60_max=0.7, B=32)
    params = api.Params(fs=sc.fs, half_len=sc.half_len)
    ds = api.DeviceScene(sc, params)
    vs = api.sample(ds, seed=11)
    h = api.synthesize(ds, vs)
    torch.cuda.synchronize()
    assert ds.status() == 0
    op = oracle_mod.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle_mod.sample(sc, op, 11)
    h_ref = oracle_mod.synthesize(sc, op, ref.pos, ref.g, ref.r)
    h = h.cpu().numpy().astype(np.float64)
    for b in range(sc.B):
        L = int(ds.rir_len[b])
        o = int(ds.rir_off[b])
        seg = slice(o, o + sc.S * sc.M * L)
        peak = np.abs(h_ref[seg]).max()
        assert np.abs(h[seg] - h_ref[seg]).max() <= 1e-5 * peak
