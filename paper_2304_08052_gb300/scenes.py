"""Seeded synthetic scenes: the inputs both the CUDA path and the oracle consume.

This module only draws room geometry; it holds none of the method's arithmetic (no
reflection coefficients, no image sampling, no synthesis).  Draws use numpy's PCG64
generator seeded explicitly, and every array is float32 -- the precision the library takes.

The workloads follow the paper's training distribution (Sec. IV-A: speaker-array distance
at least 0.3 m, T60 in [0.1, 0.7] s, shoebox rooms from 3x3x2.5 to 10x10x4 m) and the
benchmark workloads built on it:

  single_room()  6x5x3 m, T60 0.5 s, 16 kHz, one source at (2, 3, 1.5), 4-mic linear array
                 (5 cm spacing along +x) centred at (4, 2.5, 1.2), 2000 images, K = 40.
  batch_256()    256 rooms U[3,10]x U[3,8]x U[2.5,4.5] m, T60 U[0.1,0.7] s, 6-mic circular
                 array (radius 5 cm) >= 0.5 m from the walls, 1 source, round(4000*T60)
                 images, 16 kHz, K = 40.
  batch_1024()   as batch_256 with 1024 rooms, 8-mic circle (4 cm), 3 sources.
  grad_64()      64 rooms, 4-mic linear array (5 cm), T60 U[0.2,0.6] s, 1500 images, K = 40.
  large_4096()   4096 rooms U[3,15]x U[3,12]x U[2.5,6] m, T60 U[0.2,1.2] s, 16-mic circle
                 (10 cm), 2 sources, round(6000*T60) images, 48 kHz, K = 63.
  tiny(...)      small scenes for exhaustive CPU/GPU comparisons.

Source signals for the spatialisation (mixture) path, mixtures(...): the paper mixes two
LibriSpeech utterances and one noise recording per training example (Sec. IV-A); no dataset is
used here.  Speakers are Gaussian noise shaped by a random syllable-rate envelope (3-6 Hz) and a
random one-pole spectral tilt, active over a stretch of the mixture so that the two speakers
overlap on a fraction U[0.5, 1] of it (the paper's minimum overlap ratio of 0.5); noise is
stationary Gaussian noise with its own tilt spanning the whole mixture.  SIR ~ U[-6, 6] dB per
extra speaker and SNR ~ U[10, 20] dB per noise source, as in Sec. IV-A.

Conventions: linear arrays lie along +x centred on the array point; circular arrays lie in
the horizontal plane with mic k at angle 2*pi*k/M + psi, psi drawn per room.  A source
closer than 0.3 m to the array centre is redrawn (up to 16 attempts, then pushed radially).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Scene:
    name: str
    B: int
    S: int
    M: int
    fs: float
    half_len: int
    dims: np.ndarray     # [B,3] float32, metres
    rt60: np.ndarray     # [B] float32, seconds
    src: np.ndarray      # [B,S,3] float32
    mic: np.ndarray      # [B,M,3] float32
    n_vs: np.ndarray     # [B] int32, images per (room, source)
    meta: dict = field(default_factory=dict)

    def subset(self, rooms) -> "Scene":
        """The scene restricted to the given room indices (same order)."""
        rooms = np.asarray(rooms, dtype=np.int64)
        return Scene(self.name + f"[{len(rooms)} rooms]", len(rooms), self.S, self.M, self.fs,
                     self.half_len, self.dims[rooms].copy(), self.rt60[rooms].copy(),
                     self.src[rooms].copy(), self.mic[rooms].copy(), self.n_vs[rooms].copy(),
                     dict(self.meta, parent=self.name, rooms=rooms.tolist()))


def concat(parts, name: str = None) -> Scene:
    """One scene holding the rooms of `parts` (same S, M, fs and half length) in order."""
    if not parts:
        raise ValueError("concat needs at least one scene")
    p0 = parts[0]
    for p in parts[1:]:
        if (p.S, p.M, p.fs, p.half_len) != (p0.S, p0.M, p0.fs, p0.half_len):
            raise ValueError("concat: scenes differ in sources, mics, sample rate or half length")
    cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
    return Scene(name or p0.name, sum(p.B for p in parts), p0.S, p0.M, p0.fs, p0.half_len, cat("dims"),
                 cat("rt60"), cat("src"), cat("mic"), cat("n_vs"),
                 dict(p0.meta, blocks=[p.meta.get("seed") for p in parts]))


def _linear_array(centre, M, spacing):
    off = (np.arange(M) - (M - 1) / 2.0) * spacing
    pos = np.repeat(np.asarray(centre, np.float64)[None, :], M, axis=0)
    pos[:, 0] += off
    return pos


def _circular_array(centre, M, radius, psi):
    ang = 2.0 * np.pi * np.arange(M) / M + psi
    pos = np.repeat(np.asarray(centre, np.float64)[None, :], M, axis=0)
    pos[:, 0] += radius * np.cos(ang)
    pos[:, 1] += radius * np.sin(ang)
    return pos


def _draw_sources(rng, dims, centre, S, min_dist=0.3, tries=16):
    out = np.empty((S, 3))
    for s in range(S):
        for _ in range(tries):
            p = rng.uniform(0.0, 1.0, 3) * dims
            if np.linalg.norm(p - centre) >= min_dist:
                break
        else:
            d = p - centre
            n = np.linalg.norm(d)
            d = d / n if n > 0 else np.array([1.0, 0.0, 0.0])
            p = centre + min_dist * d
        out[s] = p
    return out


def _batch(name, seed, B, S, M, geometry, radius, dims_lo, dims_hi, t60_lo, t60_hi, fs, K,
           images_per_second=None, images_fixed=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = rng.uniform(dims_lo, dims_hi, size=(B, 3))
    rt60 = rng.uniform(t60_lo, t60_hi, size=B).astype(np.float32)
    mic = np.empty((B, M, 3))
    src = np.empty((B, S, 3))
    for b in range(B):
        centre = rng.uniform(0.5, dims[b] - 0.5)
        if geometry == "circular":
            mic[b] = _circular_array(centre, M, radius, rng.uniform(0.0, 2.0 * np.pi))
        else:
            mic[b] = _linear_array(centre, M, radius)
        src[b] = _draw_sources(rng, dims[b], mic[b].mean(axis=0), S)
    if images_fixed is not None:
        n_vs = np.full(B, images_fixed, np.int32)
    else:
        n_vs = np.floor(images_per_second * rt60.astype(np.float64) + 0.5).astype(np.int32)
    return Scene(name, B, S, M, float(fs), int(K), dims.astype(np.float32), rt60,
                 src.astype(np.float32), mic.astype(np.float32), n_vs,
                 dict(seed=seed, geometry=geometry, radius=radius))


def make_batch(name, seed, B, S, M, geometry, radius, dims_lo, dims_hi, t60_lo, t60_hi, fs, K,
               images_per_second=None, images_fixed=None) -> Scene:
    """A seeded batch of rooms: dims uniform in [dims_lo, dims_hi], T60 uniform in [t60_lo, t60_hi],
    a linear or circular array of M mics at a random position >= 0.5 m from the walls, S sources
    uniform in the room, round(images_per_second * T60) (or images_fixed) images per source."""
    return _batch(name, seed, B, S, M, geometry, radius, dims_lo, dims_hi, t60_lo, t60_hi, fs, K,
                  images_per_second=images_per_second, images_fixed=images_fixed)


def single_room() -> Scene:
    """6x5x3 m, T60 0.5 s, one source, 4-mic linear array, 2000 images, 16 kHz, K = 40."""
    mic = _linear_array([4.0, 2.5, 1.2], 4, 0.05)
    return Scene("single_room", 1, 1, 4, 16000.0, 40,
                 np.array([[6.0, 5.0, 3.0]], np.float32), np.array([0.5], np.float32),
                 np.array([[[2.0, 3.0, 1.5]]], np.float32), mic[None].astype(np.float32),
                 np.array([2000], np.int32), dict(seed=None, geometry="linear", radius=0.05))


def batch_256(seed: int = 0) -> Scene:
    return _batch("batch_256", seed, 256, 1, 6, "circular", 0.05, [3, 3, 2.5], [10, 8, 4.5],
                  0.1, 0.7, 16000, 40, images_per_second=4000)


def batch_1024(seed: int = 0) -> Scene:
    return _batch("batch_1024", seed, 1024, 3, 8, "circular", 0.04, [3, 3, 2.5], [10, 8, 4.5],
                  0.1, 0.7, 16000, 40, images_per_second=4000)


def grad_64(seed: int = 0) -> Scene:
    return _batch("grad_64", seed, 64, 1, 4, "linear", 0.05, [3, 3, 2.5], [10, 8, 4.5],
                  0.2, 0.6, 16000, 40, images_fixed=1500)


def large_4096(seed: int = 0) -> Scene:
    return _batch("large_4096", seed, 4096, 2, 16, "circular", 0.10, [3, 3, 2.5], [15, 12, 6],
                  0.2, 1.2, 48000, 63, images_per_second=6000)


def tiny(seed: int = 0, B: int = 3, S: int = 2, M: int = 3, images: int = 40, fs: float = 16000.0,
         K: int = 40, t60_lo: float = 0.05, t60_hi: float = 0.12, geometry: str = "circular",
         radius: float = 0.05) -> Scene:
    """Small scenes (short RIRs, few images) for exhaustive comparisons."""
    return _batch(f"tiny{seed}", seed, B, S, M, geometry, radius, [3, 3, 2.5], [6, 5, 3.5],
                  t60_lo, t60_hi, fs, K, images_fixed=images)


CONFIGS = {
    "single_room": single_room,
    "batch_256": batch_256,
    "batch_1024": batch_1024,
    "grad_64": grad_64,
    "large_4096": large_4096,
}


def by_name(name: str, seed: int = 0) -> Scene:
    fn = CONFIGS[name]
    return fn() if name == "single_room" else fn(seed)


def synthetic_vs(seed: int, scene: Scene, max_dist: float = 60.0):
    """Arbitrary image positions and reflection counts for the Cartesian (user-supplied)
    input path: positions uniform in direction and in distance from the array centre in
    [0.5, max_dist] m, g uniform in [1, 40].  Returns (pos [N,3] f32, g [N] f32).  This is a
    stand-in for user data, not the paper's sampler."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos, g = [], []
    for b in range(scene.B):
        c = scene.mic[b].astype(np.float64).mean(axis=0)
        n = scene.S * int(scene.n_vs[b])
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        lim = min(max_dist, 0.95 * 343.0 * float(scene.rt60[b]))
        rad = rng.uniform(0.5, lim, size=(n, 1))
        pos.append(c + rad * d)
        g.append(rng.uniform(1.0, 40.0, size=n))
    return (np.concatenate(pos).astype(np.float32) if pos else np.zeros((0, 3), np.float32),
            np.concatenate(g).astype(np.float32) if g else np.zeros(0, np.float32))


@dataclass
class Mixtures:
    signals: np.ndarray   # [B,S,N] float32, sources on the mixture's timeline
    level_db: np.ndarray  # [B,S] float32: SIR (speakers s >= 1) or SNR (noise) in dB; entry 0 unused
    n_speech: int


def _tilt(rng, x, lo, hi):
    from scipy.signal import lfilter
    return lfilter([1.0], [1.0, -rng.uniform(lo, hi)], x)     # y[n] = x[n] + a y[n-1]


def mixtures(seed: int, B: int, S: int, N: int, fs: float, n_speech: int = None) -> Mixtures:
    """Seeded synthetic sources for B examples of S sources (the last S - n_speech are noise;
    default n_speech = S - 1 when S > 1), N samples each at fs."""
    if n_speech is None:
        n_speech = S - 1 if S > 1 else 1
    rng = np.random.Generator(np.random.PCG64(seed))
    sig = np.zeros((B, S, N), np.float64)
    lev = np.zeros((B, S), np.float64)
    t = np.arange(N) / fs
    for b in range(B):
        rho = rng.uniform(0.5, 1.0)                 # overlap ratio of the first two speakers
        span = int(round(N * (1.0 + rho) / 2.0))
        for s in range(S):
            w = rng.standard_normal(N)
            if s < n_speech:
                env = np.abs(np.sin(np.pi * rng.uniform(3.0, 6.0) * t + rng.uniform(0, np.pi)))
                env *= np.sqrt(env)
                x = _tilt(rng, w, 0.3, 0.95) * env
                if n_speech > 1:
                    first = (s == 0) == (rng.uniform() < 0.5)
                    lo, hi = (0, span) if first else (N - span, N)
                    x[:lo] = 0.0
                    x[hi:] = 0.0
            else:
                x = _tilt(rng, w, 0.0, 0.8)
            sig[b, s] = x / max(np.abs(x).max(), 1e-12)
            lev[b, s] = 0.0 if s == 0 else (rng.uniform(-6.0, 6.0) if s < n_speech else rng.uniform(10.0, 20.0))
    return Mixtures(sig.astype(np.float32), lev.astype(np.float32), int(n_speech))
