"""The autotuner's persistent cache (FRAM_AUTOTUNE_CACHE): a process that tunes writes its choice
to the file, keyed by the GPU's name and SM count and the workload group; a fresh process that
sets the same variable launches tile = 0 calls with the cached tile without tuning; a process
without the variable uses the library default.  Each step runs in its own process, so nothing
is carried over in memory."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = r"""
import json, sys
sys.path.insert(0, {root!r})
import torch
from paper_2304_08052_gb300 import api, scenes
sc = scenes.batch_256(0).subset(range(32))
ds = api.DeviceScene(sc, api.Params(fs=sc.fs, half_len=sc.half_len))
out = {{}}
if {tune}:
    vs = api.sample(ds, seed=3)
    out["chosen"] = api.autotune(ds, vs)
out["tile"] = api.tuned_tile(ds)
print(json.dumps(out))
"""


def _run(tmp_path, tune, cache):
    env = dict(os.environ)
    env.pop("FRAM_AUTOTUNE_CACHE", None)
    if cache is not None:
        env["FRAM_AUTOTUNE_CACHE"] = str(cache)
    code = _SCRIPT.format(root=ROOT, tune=bool(tune))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_tile_choice_persists_across_processes(tmp_path):
    cache = tmp_path / "tune.jsonl"
    a = _run(tmp_path, True, cache)
    assert a["tile"] == a["chosen"] in (256, 512, 1024, 2048)
    lines = [json.loads(x) for x in cache.read_text().splitlines() if x.strip()]
    assert len(lines) == 1 and lines[0]["tile"] == a["chosen"] and lines[0]["K"] == 40
    # Replace the recorded tile by another candidate: a fresh process must launch with it.
    other = 512 if a["chosen"] != 512 else 256
    lines[0]["tile"] = other
    cache.write_text("".join(json.dumps(x) + "\n" for x in lines))
    assert _run(tmp_path, False, cache)["tile"] == other
    # Without the variable the library default applies.
    assert _run(tmp_path, False, None)["tile"] == 1024
    # A line for another GPU model is ignored.
    lines[0]["gpu"] = "another GPU"
    cache.write_text("".join(json.dumps(x) + "\n" for x in lines))
    assert _run(tmp_path, False, cache)["tile"] == 1024
