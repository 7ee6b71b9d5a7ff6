"""Room sharding across GPUs: one batch of rooms split into contiguous, cost-balanced ranges.

Rooms are independent units of the method: every image of a room is drawn and rendered from
that room's own geometry (Sec. III-A to III-D), and each Philox draw is keyed by the room's
index in the batch, not by its position in a shard (fram_scene.room_base).  A rank that
samples and synthesises rooms [lo, hi) of a batch with room_base = lo therefore produces
exactly the rows the whole batch gives those rooms, and no data moves between ranks.

Cost of room b (taps plus output samples, the two terms that scale its time):
    cost_b = S M (I_b + 1)(2K + 1) + S M L_b,     L_b = ceil(T60_b fs)
partition() cuts the prefix sums of the costs at multiples of total / world, so every rank's
cost is at most total / world + max_b cost_b.
"""
from __future__ import annotations

import numpy as np


def room_costs(scene, half_len: int) -> np.ndarray:
    """Per-room cost (float64) of sampling and synthesising `scene` with half length K."""
    n_vs = np.asarray(scene.n_vs, np.float64)
    L = np.ceil(np.asarray(scene.rt60, np.float64) * float(scene.fs))
    SM = float(scene.S * scene.M)
    return SM * (n_vs + 1.0) * (2 * int(half_len) + 1) + SM * L


def partition(costs, world: int):
    """Contiguous ranges [(lo, hi)] * world covering every room once, balanced by cost: range k
    ends at the first room whose cost prefix reaches (k + 1) total / world."""
    costs = np.asarray(costs, np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    if (costs < 0).any():
        raise ValueError("costs must be >= 0")
    B = costs.shape[0]
    cum = np.concatenate([[0.0], np.cumsum(costs)])
    total = cum[-1]
    cuts = [0]
    for k in range(1, world):
        # first index j with cum[j] >= k total / world, never before the previous cut
        j = int(np.searchsorted(cum, k * total / world, side="left"))
        cuts.append(min(max(j, cuts[-1]), B))
    cuts.append(B)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def imbalance_bound(costs, world: int) -> float:
    """The largest per-rank cost partition() may give: total / world + max_b cost_b."""
    costs = np.asarray(costs, np.float64)
    return float(costs.sum() / world + (costs.max() if costs.size else 0.0))


def global_batch(factory, name: str, blocks: int):
    """A batch of `blocks` seeded blocks of a workload (block k drawn with scene seed k), as one
    scene whose room index is the global index used for the Philox draws.  factory(name, seed)
    returns a block (scenes.by_name)."""
    from . import scenes
    parts = [factory(name, k) for k in range(blocks)]
    return scenes.concat(parts, name=f"{name}x{blocks}" if blocks > 1 else name)


def shard_of(factory, name: str, world: int, rank: int, half_len: int):
    """(scene of this rank's rooms, room_base, (lo, hi), all ranges) for a batch of `world`
    blocks of workload `name` split over `world` ranks (weak scaling: about one block per rank)."""
    glob = global_batch(factory, name, world)
    ranges = partition(room_costs(glob, half_len), world)
    lo, hi = ranges[rank]
    return glob.subset(range(lo, hi)), lo, (lo, hi), ranges

