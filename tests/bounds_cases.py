"""Cases run against one build of libfram (the library FRAM_LIBRARY names, else the release
build): sample, synthesise with the early RIR, run the adjoint with early-RIR upstream
gradients and carry its gradients back through the sampler, over the half lengths, tile lengths
and scene shapes the parity tests sweep; spatialise ragged signals with targets; and run the
multi-rate path (delay_mode 1) with the early RIR at every second-resampler rate, ragged tiles and
a batch whose high-pass runs in several pieces; then print, per case, the device status bits and
a SHA-256 of every output.  tests/test_gpu_debug_bounds.py
runs it under the release build and the bounds-checking debug build and compares."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2304_08052_gb300 import api, scenes  # noqa: E402


def _digest(*tensors):
    h = hashlib.sha256()
    for t in tensors:
        h.update(t.detach().cpu().numpy().tobytes())
    return h.hexdigest()[:24]


def run_case(sc, tile, seed):
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len, tile=tile))
    vs = api.sample(ds, seed=seed)
    h, he = api.synthesize(ds, vs, early=True)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    G = torch.empty(ds.rir_total, device="cuda").normal_(generator=gen)
    Ge = torch.empty(ds.rir_total, device="cuda").normal_(generator=gen)
    gv, gm, gs, gr = api.synthesize_backward_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, G, Ge)
    # through the sampler (draws of `seed` held fixed), with a random gradient on the amplitudes
    gg = torch.empty(ds.n_vs_total, device="cuda").normal_(generator=gen)
    sb = api.sample_backward(ds, seed, gv, grad_g=gg, grad_r=gr, grad_src_in=gs, grad_mic_in=gm)
    torch.cuda.synchronize()
    return {"status": ds.status(), "out": _digest(h, he, gv, gm, gs, gr, *sb)}


def run_spatial(sc, tile, seed, n_speech, N, block):
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len, tile=tile))
    vs = api.sample(ds, seed=seed)
    h = api.synthesize(ds, vs)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.empty((ds.B, ds.S, N), device="cuda").normal_(generator=gen)
    x[:, :, N // 3:N // 3 + 700] = 0.0           # a silent stretch: zero-flagged windows
    lev = torch.empty((ds.B, ds.S), device="cuda").uniform_(-5.0, 5.0, generator=gen)
    mix, tg, gains = api.spatialize(ds, h, x, lev, n_speech, targets=True, block=block)
    torch.cuda.synchronize()
    return {"status": ds.status() | api.spatialize_status(ds), "out": _digest(mix, tg, gains)}


def run_multirate(sc, tile, seed):
    ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len, tile=tile, delay_mode=1))
    vs = api.sample(ds, seed=seed)
    h, he = api.synthesize(ds, vs, early=True)
    torch.cuda.synchronize()
    return {"status": ds.status(), "out": _digest(h, he)}


def cases():
    out = {}
    for K in (1, 5, 16, 17, 33, 64, 100, 128):
        for tile in (256, 2048):
            sc = scenes.tiny(seed=K, B=3, S=2, M=3, images=150, K=K, t60_lo=0.1, t60_hi=0.3)
            out[f"K{K}_tile{tile}"] = run_case(sc, tile, 10 + K)
    out["batch_256"] = run_case(scenes.batch_256(0), 0, 3)
    out["large_4096_64rooms"] = run_case(scenes.large_4096(0).subset(range(64)), 0, 5)
    for fs, M, S, geometry, spacing in ((44100.0, 64, 1, "circular", 0.1), (16000.0, 3, 7, "linear", 1.0),
                                        (8000.0, 1, 2, "circular", 0.05)):
        sc = scenes.make_batch("shape", M + S, 3, S, M, geometry, spacing, [3, 3, 2.5], [8, 6, 4], 0.1, 0.4, fs, 40,
                               images_fixed=300)
        out[f"shape_{int(fs)}_{M}x{S}"] = run_case(sc, 512, 7)
    # multi-rate: r_l = 2 .. 11 (250, 96, 48, 32, 22.05, 16, 11.025, 8 kHz), tiles 256 and 2048
    for fs, t60 in ((250000.0, (0.03, 0.04)), (96000.0, (0.03, 0.06)), (48000.0, (0.1, 0.2)),
                    (32000.0, (0.05, 0.1)), (22050.0, (0.05, 0.15)), (16000.0, (0.02, 0.25)),
                    (11025.0, (0.1, 0.2)), (8000.0, (0.1, 0.3))):
        sc = scenes.tiny(seed=int(fs) % 89, B=3, S=2, M=2, images=120, fs=fs, t60_lo=t60[0], t60_hi=t60[1])
        for tile in (256, 2048):
            out[f"mr_{int(fs)}_tile{tile}"] = run_multirate(sc, tile, 40 + tile % 7)
    # spatialisation: ragged signal lengths against the block, one and several speakers
    for N, block, ns in ((5000, 0, 1), (12345, 4096, 2), (3000, 8192, 2)):
        sc = scenes.tiny(seed=N % 97, B=3, S=3, M=2, images=200, t60_lo=0.1, t60_hi=0.3)
        out[f"sp_N{N}_block{block}"] = run_spatial(sc, 0, 21, ns, N, block)
    # 48 rooms of the 1024-room training batch (T60 0.1-0.7 s): up to five high-pass pieces per channel
    out["mr_batch_1024_48rooms"] = run_multirate(scenes.batch_1024(0).subset(range(48)), 0, 9)
    return out


if __name__ == "__main__":
    print(json.dumps(cases()))
