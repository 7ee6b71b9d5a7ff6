"""The bounds-checking debug build (paper_2304_08052_gb300/build.py, -DFRAM_DEBUG_BOUNDS) stands
in for a memory checker, which this GPU pool does not offer: in it, the synthesis and adjoint
kernels check every arrival's shared-buffer footprint, every gather window against its staged
buffer, and every work unit's image rows and RIR range before the access, the multi-rate kernels
every unit's intermediate-signal range, filter row and RIR range, the binning and gather kernels
every slot and permutation value of the sorted order, and all of them record FRAM_DEV_BOUNDS
instead of running outside a buffer.  Over the half lengths, tile lengths and
scene shapes the parity tests sweep, no guard may fire, and the outputs must equal the release
build's bit for bit (the guards change no arithmetic)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(lib_path):
    env = dict(os.environ)
    if lib_path:
        env["FRAM_LIBRARY"] = lib_path
    else:
        env.pop("FRAM_LIBRARY", None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_cases.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_no_guard_fires_and_results_match_the_release_build():
    from paper_2304_08052_gb300 import build
    debug_lib = build.build(debug_bounds=True)
    dbg = _run(debug_lib)
    rel = _run(None)
    assert set(dbg) == set(rel) and len(dbg) >= 20
    for name in dbg:
        assert dbg[name]["status"] == 0, (name, dbg[name])
        assert rel[name]["status"] == 0, (name, rel[name])
        assert dbg[name]["out"] == rel[name]["out"], name
