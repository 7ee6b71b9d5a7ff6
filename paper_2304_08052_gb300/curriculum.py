"""T60 curriculum for the on-the-fly training pipeline (the paper's "T60 curriculum training"
subsection, Sec. V).

Training starts with T60 drawn from a small range, and the range's upper bound grows every epoch
until it reaches the largest T60 the pipeline must cover.  The paper's setting: [50, 100] ms in the
first epoch and +50 ms per epoch.  This module only schedules the range and draws the rooms; the
rooms then go through the same fram_sample / fram_synthesize path as any other batch.
"""
from __future__ import annotations

from . import scenes


def t60_range(epoch: int, t60_max: float, lo: float = 0.05, hi0: float = 0.10, step: float = 0.05):
    """(T60 lower, upper bound) in seconds for a 0-based epoch: [lo, hi0 + step * epoch], the upper
    bound capped at t60_max (and the lower bound at the upper one)."""
    if epoch < 0:
        raise ValueError("epoch must be >= 0")
    if not (t60_max > 0 and lo > 0 and hi0 >= lo and step >= 0):
        raise ValueError("need t60_max > 0, lo > 0, hi0 >= lo, step >= 0")
    hi = min(hi0 + step * epoch, t60_max)
    return min(lo, hi), hi


def curriculum_batch(seed: int, epoch: int, t60_max: float, B: int = 256, S: int = 1, M: int = 6,
                     geometry: str = "circular", radius: float = 0.05, dims_lo=(3.0, 3.0, 2.5),
                     dims_hi=(10.0, 8.0, 4.5), fs: float = 16000.0, K: int = 40,
                     images_per_second: float = 4000.0) -> scenes.Scene:
    """One on-the-fly batch for `epoch`: the room distribution of the 256-room workload by default,
    with T60 uniform in t60_range(epoch, t60_max) and round(images_per_second * T60) images."""
    lo, hi = t60_range(epoch, t60_max)
    return scenes.make_batch(f"curriculum_e{epoch}", seed, B, S, M, geometry, radius, list(dims_lo),
                             list(dims_hi), lo, hi, fs, K, images_per_second=images_per_second)
