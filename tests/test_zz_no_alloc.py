"""fram_synthesize_noalloc: synthesis for callers that cannot allocate device memory.

Some callers of this library are not allowed to call cudaMalloc: a plugin whose host
application owns every device allocation, a real-time thread that must never block on an
allocation (cudaMalloc and cudaFree can synchronise the device), or a service running in a
fixed device-memory budget.  They pass inputs and outputs they already own, and the library
uses a static 16 MiB scratch array instead of a caller workspace.  This file checks that
entry point against fram_synthesize on two calls in a row (the second call reuses scratch
left over from the first): both run the same kernels with the same tile on the same inputs and
sum every sample in a fixed order, so the outputs must be identical bit for bit.  It covers the
continuous path with and without the early RIR and the multi-rate path (delay_mode 1), and that
an oversized scene is refused before any GPU work.
It is named to run last so that a failure here never hides the other tests' results.
"""
import ctypes

import pytest
import torch

from paper_2304_08052_gb300 import _lib, api, scenes

pytestmark = pytest.mark.gpu


def _call_noalloc(ds, vs, rir, early):
    L = _lib.lib()
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    return L.fram_synthesize_noalloc(ctypes.byref(ds.c_scene()), ctypes.byref(ds.params.c()), p(vs.pos_hi),
                                     p(vs.pos_lo), p(vs.g), p(vs.r), p(rir), p(early),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _check_two_calls(ds, vs, with_early):
    res = api.synthesize(ds, vs, early=with_early)
    ref, ref_e = res if with_early else (res, None)
    torch.cuda.synchronize()
    assert ds.status() == 0
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        out_e = torch.full_like(ref, float("nan")) if with_early else None
        assert _call_noalloc(ds, vs, out, out_e) == _lib.FRAM_OK, _lib.lib().fram_last_error()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        if with_early:
            assert torch.equal(out_e, ref_e)


@pytest.mark.parametrize("with_early", [True, False])
def test_noalloc_matches_workspace_entry_point_on_two_calls(with_early):
    # The first 128 rooms of the 256-room batch: their workspace fits the 16 MiB scratch.
    sc = scenes.batch_256(0).subset(range(128))
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len))
    assert ds.ws_bytes <= 16 << 20
    vs = api.sample(ds, seed=21)
    _check_two_calls(ds, vs, with_early)


def test_noalloc_multirate_path_on_two_calls():
    sc = scenes.tiny(seed=4, B=3, S=2, M=3, images=60)
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len, delay_mode=1))
    assert ds.ws_bytes <= 16 << 20
    vs = api.sample(ds, seed=8)
    _check_two_calls(ds, vs, True)


def test_noalloc_refuses_scenes_beyond_the_static_scratch():
    L = _lib.lib()
    fake = ctypes.c_void_p(0x1000)     # never dereferenced: the size check comes first
    big = _lib.FramScene(4096, 2, 16, 57600, 34_000_000, 4096 * 2 * 16 * 57600, 0.1, *([fake] * 8))
    p = api.Params(fs=48000.0, half_len=63)
    rc = L.fram_synthesize_noalloc(ctypes.byref(big), ctypes.byref(p.c()), fake, None, fake, fake, fake, None, None)
    assert rc == _lib.FRAM_EWORKSPACE
    assert b"16 MiB" in L.fram_last_error()
