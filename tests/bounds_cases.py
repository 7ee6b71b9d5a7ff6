"""Cases run against one build of libfram (the library FRAM_LIBRARY names, else the release
build): sample, synthesise with the early RIR and run the adjoint with early-RIR upstream
gradients over the half lengths, tile lengths and scene shapes the parity tests sweep, then print,
per case, the device status bits and a SHA-256 of every output.  tests/test_gpu_debug_bounds.py
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
    torch.cuda.synchronize()
    return {"status": ds.status(), "out": _digest(h, he, gv, gm, gs, gr)}


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
    return out


if __name__ == "__main__":
    print(json.dumps(cases()))
