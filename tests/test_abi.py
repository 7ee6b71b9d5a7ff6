"""Host-only checks of the C ABI: the library loads, exports every symbol include/fram.h
declares, and its host functions (layout, workspace sizing, argument validation) behave as
documented.  No call here launches GPU work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2304_08052_gb300 import _lib, api, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2304_08052_gb300 import build
    build.build()
    return _lib.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "fram.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fram_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert set(names) == set(_lib.EXPORTED), names
    for n in names:
        assert hasattr(L, n), n


def test_version_and_defaults(L):
    assert L.fram_version() == 10200
    p = _lib.FramParams()
    L.fram_default_params(ctypes.byref(p))
    assert (p.alpha, p.beta, p.a, p.b, p.tau, p.c0) == (0.25, 1.0, -2.0, 2.0, 0.25, 343.0)
    assert (p.fs, p.half_len, p.early_pre_ms, p.early_post_ms, p.tile) == (16000.0, 40, 6.0, 50.0, 0)


@pytest.mark.parametrize("name", ["single_room", "batch_256", "grad_64"])
def test_layout_matches_oracle(L, oracle_mod, name):
    sc = scenes.by_name(name, 0)
    got = api.layout(sc.rt60, sc.n_vs, sc.S, sc.M, sc.fs)
    want = oracle_mod.layout(sc.rt60, sc.n_vs, sc.S, sc.M, sc.fs)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


def test_layout_rejects_bad_scenes(L):
    with pytest.raises(_lib.FramError) as e:
        api.layout(np.array([0.5, -0.1], np.float32), np.array([10, 10], np.int32), 1, 2, 16000.0)
    assert e.value.code == _lib.FRAM_EINVAL
    with pytest.raises(_lib.FramError):
        api.layout(np.array([0.5], np.float32), np.array([-1], np.int32), 1, 2, 16000.0)
    with pytest.raises(_lib.FramError):
        api.layout(np.array([0.5], np.float32), np.array([1], np.int32), 0, 2, 16000.0)


def _scene_struct(B=4, S=2, M=3, max_len=8000, nvs=400, rir_total=4 * 2 * 3 * 8000, radius=0.05):
    return _lib.FramScene(B, S, M, max_len, nvs, rir_total, radius, *([None] * 8))


def test_workspace_size_and_param_validation(L):
    p = api.Params()
    n = ctypes.c_size_t(0)
    assert L.fram_workspace_size(ctypes.byref(_scene_struct()), ctypes.byref(p.c()), ctypes.byref(n)) == 0
    assert n.value > 0 and n.value % 256 == 0
    n2 = ctypes.c_size_t(0)
    big = _scene_struct(B=40, nvs=4000)
    assert L.fram_workspace_size(ctypes.byref(big), ctypes.byref(p.c()), ctypes.byref(n2)) == 0
    assert n2.value > n.value
    for bad in (dict(alpha=0.0), dict(beta=1.5), dict(alpha=0.5, beta=0.4), dict(tau=0.0), dict(c0=-1.0),
                dict(half_len=0), dict(half_len=129), dict(tile=300), dict(a=1.0, b=0.0)):
        q = api.Params(**bad)
        rc = L.fram_workspace_size(ctypes.byref(_scene_struct()), ctypes.byref(q.c()), ctypes.byref(n))
        assert rc == _lib.FRAM_EINVAL, bad
        assert len(L.fram_last_error()) > 0
    for bad in (dict(S=0), dict(M=0), dict(M=65), dict(B=-1)):
        s = _scene_struct(**bad)
        assert L.fram_workspace_size(ctypes.byref(s), ctypes.byref(p.c()), ctypes.byref(n)) == _lib.FRAM_EINVAL
    # room_base: the Philox room word of room 0; room_base + B must fit in 32 bits.
    for base, rc in ((0, 0), (2**32 - 4, 0), (2**32 - 3, _lib.FRAM_EINVAL), (-1, _lib.FRAM_EINVAL)):
        s = _scene_struct()
        s.room_base = base
        assert L.fram_workspace_size(ctypes.byref(s), ctypes.byref(p.c()), ctypes.byref(n)) == rc, base


def test_entry_points_reject_bad_arguments_before_any_launch(L):
    p = api.Params()
    sc = _scene_struct()
    null = ctypes.c_void_p(0)
    # Scene device arrays are null -> EINVAL, detected on the host.
    assert L.fram_sample(ctypes.byref(sc), ctypes.byref(p.c()), 0, None, null, null, null, null, null, null,
                         0, None) == _lib.FRAM_EINVAL
    assert L.fram_synthesize(ctypes.byref(sc), ctypes.byref(p.c()), null, null, null, null, null, null, null, 0,
                             None) == _lib.FRAM_EINVAL
    assert L.fram_synthesize_backward(ctypes.byref(sc), ctypes.byref(p.c()), null, null, null, null, null, null,
                                      null, null, null, null, null, null, 0, None) == _lib.FRAM_EINVAL
    assert L.fram_sample_backward(ctypes.byref(sc), ctypes.byref(p.c()), 0, None, null, null, null, null, null,
                                  null, null, null, null, null, 0, None) == _lib.FRAM_EINVAL
    assert L.fram_status(null, None, None) == _lib.FRAM_EINVAL
    # A fake (never dereferenced) device pointer set: the workspace checks fail first.
    fake = ctypes.c_void_p(0x1000)
    sc2 = _lib.FramScene(1, 1, 1, 100, 10, 100, 0.0, *([fake] * 8))
    assert L.fram_synthesize(ctypes.byref(sc2), ctypes.byref(p.c()), fake, None, fake, fake, fake, None, None, 0,
                             None) == _lib.FRAM_EWORKSPACE
    assert L.fram_synthesize(ctypes.byref(sc2), ctypes.byref(p.c()), fake, None, fake, fake, fake, None,
                             ctypes.c_void_p(0x1010), 1 << 30, None) == _lib.FRAM_EWORKSPACE   # misaligned
    n = ctypes.c_size_t(0)
    L.fram_workspace_size(ctypes.byref(sc2), ctypes.byref(p.c()), ctypes.byref(n))
    assert L.fram_synthesize(ctypes.byref(sc2), ctypes.byref(p.c()), fake, None, fake, fake, fake, None,
                             ctypes.c_void_p(0x100000), n.value - 256, None) == _lib.FRAM_EWORKSPACE


def test_auto_tile_workspace_covers_every_candidate(L):
    n_auto, n_fix = ctypes.c_size_t(0), ctypes.c_size_t(0)
    sc = _scene_struct(B=64, max_len=20000, nvs=64 * 2 * 3000)
    for tile, out in ((0, n_auto), (256, n_fix)):
        assert L.fram_workspace_size(ctypes.byref(sc), ctypes.byref(api.Params(tile=tile).c()), ctypes.byref(out)) == 0
    assert n_auto.value >= n_fix.value
    for tile in (512, 1024, 2048):
        n = ctypes.c_size_t(0)
        L.fram_workspace_size(ctypes.byref(sc), ctypes.byref(api.Params(tile=tile).c()), ctypes.byref(n))
        assert n.value <= n_auto.value


def test_spatialize_rejects_bad_arguments_on_the_host(L):
    sc = _scene_struct()
    n = ctypes.c_size_t(0)
    ok = _lib.FramSpatial(16000, 1, 0, 0, 0)
    assert L.fram_spatialize_workspace_size(ctypes.byref(sc), ctypes.byref(ok), 0, ctypes.byref(n)) == 0
    assert n.value > 0
    n_sep = ctypes.c_size_t(0)
    assert L.fram_spatialize_workspace_size(ctypes.byref(sc), ctypes.byref(ok), 1, ctypes.byref(n_sep)) == 0
    assert n_sep.value > n.value                          # room for the target-RIR spectra
    for bad in (_lib.FramSpatial(0, 1, 0, 0, 0), _lib.FramSpatial(100, 0, 0, 0, 0),
                _lib.FramSpatial(100, sc.S + 1, 0, 0, 0), _lib.FramSpatial(100, 1, 1000, 0, 0),
                _lib.FramSpatial(100, 1, 0, -1, 0)):
        assert L.fram_spatialize_workspace_size(ctypes.byref(sc), ctypes.byref(bad), 0,
                                                ctypes.byref(n)) == _lib.FRAM_EINVAL
    null = ctypes.c_void_p(0)
    assert L.fram_spatialize(ctypes.byref(sc), ctypes.byref(ok), null, null, null, null, null, null, null, null, 0,
                             None) == _lib.FRAM_EWORKSPACE


def test_binding_checks_tensors_before_handing_pointers():
    # The binding refuses what the C ABI cannot check: element type, size, device, layout.
    import torch
    from paper_2304_08052_gb300 import api
    assert api._ptr(None, 10) is None
    with pytest.raises(TypeError):
        api._ptr([1.0, 2.0], 2, name="g")
    with pytest.raises(ValueError, match="dtype"):
        api._ptr(torch.zeros(8, dtype=torch.float64), 8, name="g")
    with pytest.raises(ValueError, match="dtype"):
        api._ptr(torch.zeros(1, dtype=torch.int32), 1, api._SEED, "d_seed")
    with pytest.raises(ValueError, match="at least 9"):
        api._ptr(torch.zeros(8), 9, name="pos_hi")
    with pytest.raises(ValueError, match="CUDA"):
        api._ptr(torch.zeros(8), 8, name="rir")                  # right type and size, host memory
    with pytest.raises(ValueError, match="dtype"):
        api._ptr(torch.zeros((4, 4), dtype=torch.int64), 16, api._WORD, "words")


def test_measure_alu_rejects_bad_arguments(L):
    res = (ctypes.c_double * 4)()
    assert L.fram_measure_alu(3, 10, res, None) == _lib.FRAM_EINVAL
    assert L.fram_measure_alu(0, 0, res, None) == _lib.FRAM_EINVAL
    assert L.fram_measure_alu(0, 10, None, None) == _lib.FRAM_EINVAL
