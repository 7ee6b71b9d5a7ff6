"""FP64 CPU oracle for FRAM-RIR (Luo & Gu, arXiv 2304.08052) -- test infrastructure only.

This package is the slow, obviously-correct reference that the CUDA path is checked
against.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product library never does.  It shares no code with the CUDA
path: the C file ``fram_oracle.c`` restates the paper's equations in double precision and
this module only marshals numpy arrays into it.

Functions and the passages they follow:
  philox(ctr, key)            Philox4x32-10 (Salmon et al., SC'11); counter-based draws
  layout(...)                 L = ceil(T60 * fs) (Sec. III-D at the output rate), offsets
  room_stats(dims, rt60)      R = V/S (Sec. III-A), Eyring coefficient r (Eq. 2)
  sample(scene, params, seed) Eq. 3-6 and Sec. III-B: image positions and reflection counts
  synthesize(...)             Eq. 1 with windowed-sinc fractional delays; Eq. 9 early RIR
  backward(...)               analytic gradient of a loss on h (and h_e)
  sample_backward(...)        that gradient carried back through the sampler (draws held fixed)
  synthesize_mr(...)          the paper's multi-rate output path (Sec. II-B, Eq. 7-9): impulses
                              on the r_h fs grid, down to r_l fs, 80 Hz high-pass, down to fs
  mr_rates, resample_filter, hpf_coeffs   its rates and filters (readings: see fram_oracle.c)
  spatialize(...)             Sec. IV-A's use of the RIRs: signals convolved with them, mixed at
                              the given SIR / SNR, optional per-speaker targets (readings: see
                              fram_oracle.c)

Every function is pinned by tests that do not reuse its own arithmetic (see the module
docstrings of tests/test_oracle_*.py).  No function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fram_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libfram_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over rooms).  Returns the library path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("tau", ctypes.c_double), ("c0", ctypes.c_double),
                ("fs", ctypes.c_double), ("early_pre_ms", ctypes.c_double),
                ("early_post_ms", ctypes.c_double), ("half_len", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


@dataclass
class Params:
    """Method constants.  alpha, beta (Eq. 3), a, b, tau (Eq. 6) and c0 are not given in the
    paper; the defaults are this project's reading (alpha=0.25, beta=1, a=-2, b=2, tau=0.25,
    c0=343 m/s).  early_pre_ms / early_post_ms are the [-6, 50] ms of Eq. 9."""
    fs: float = 16000.0
    half_len: int = 40
    alpha: float = 0.25
    beta: float = 1.0
    a: float = -2.0
    b: float = 2.0
    tau: float = 0.25
    c0: float = 343.0
    early_pre_ms: float = 6.0
    early_post_ms: float = 50.0

    def _c(self) -> _Params:
        return _Params(self.alpha, self.beta, self.a, self.b, self.tau, self.c0, self.fs,
                       self.early_pre_ms, self.early_post_ms, int(self.half_len), 0)


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.fo_num_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().fo_num_threads())


def set_num_threads(n: int) -> None:
    _load().fo_set_num_threads(ctypes.c_int(int(n)))


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 on a batch of counters ctr [n,4] (uint32) with key [2] (uint32)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    _load().fo_philox_batch(ctypes.c_int64(ctr.shape[0]), _p(ctr), _p(key), _p(out))
    return out


def layout(rt60, n_vs, S: int, M: int, fs: float):
    """(rir_len [B] int32, rir_off [B+1] int64, vs_off [B+1] int64) with L = ceil(T60*fs)."""
    rt60 = np.ascontiguousarray(rt60, dtype=np.float32)
    n_vs = np.ascontiguousarray(n_vs, dtype=np.int32)
    B = rt60.shape[0]
    rir_len = np.empty(B, np.int32)
    rir_off = np.empty(B + 1, np.int64)
    vs_off = np.empty(B + 1, np.int64)
    rc = _load().fo_layout(ctypes.c_int32(B), ctypes.c_int32(S), ctypes.c_int32(M), ctypes.c_double(fs),
                           _p(rt60), _p(n_vs), _p(rir_len), _p(rir_off), _p(vs_off))
    if rc != 0:
        raise ValueError("oracle layout: invalid scene")
    return rir_len, rir_off, vs_off


def room_stats(dims, rt60):
    """(R, r) per room: R = V/S (Sec. III-A) and the Eyring coefficient of Eq. 2."""
    dims = _f64(dims).reshape(-1, 3)
    rt60 = _f64(rt60).reshape(-1)
    B = dims.shape[0]
    R = np.empty(B)
    r = np.empty(B)
    _load().fo_room_stats(ctypes.c_int32(B), _p(dims), _p(rt60), _p(R), _p(r))
    return R, r


@dataclass
class Sampled:
    pos: np.ndarray      # [N,3] image positions (FP64)
    g: np.ndarray        # [N] reflection counts (Eq. 6)
    r: np.ndarray        # [B] Eyring coefficient (Eq. 2)
    words: np.ndarray    # [N,4] uint32 Philox words
    dist: np.ndarray     # [N] D_i (distance to the array centre)
    x: np.ndarray        # [N] sampled x of Eq. 3
    rrmax: np.ndarray    # [B,S] RR_max (Eq. 5)
    d0: np.ndarray       # [B,S] D0


def sample(scene, params: Params, seed: int, room_ids=None) -> Sampled:
    """Sample every room/source's virtual images (Sec. III-B, III-C) in FP64.  room_ids
    (optional, [B]) are the rooms' indices in a larger batch; the draws then equal the ones
    those rooms get inside that batch."""
    B, S, M = scene.B, scene.S, scene.M
    _, _, vs_off = layout(scene.rt60, scene.n_vs, S, M, params.fs)
    N = int(vs_off[-1])
    out = Sampled(np.empty((N, 3)), np.empty(N), np.empty(B), np.empty((N, 4), np.uint32),
                  np.empty(N), np.empty(N), np.empty((B, S)), np.empty((B, S)))
    dims, rt60 = _f64(scene.dims), _f64(scene.rt60)
    src, mic = _f64(scene.src), _f64(scene.mic)
    n_vs = np.ascontiguousarray(scene.n_vs, dtype=np.int32)
    pc = params._c()
    rid = None if room_ids is None else np.ascontiguousarray(room_ids, dtype=np.int32)
    assert rid is None or rid.shape == (B,)
    rc = _load().fo_sample(ctypes.c_int32(B), ctypes.c_int32(S), ctypes.c_int32(M), _p(dims), _p(rt60),
                           _p(src), _p(mic), _p(n_vs), _p(vs_off), ctypes.byref(pc),
                           ctypes.c_uint64(seed), _p(out.pos), _p(out.g), _p(out.r), _p(out.words),
                           _p(out.dist), _p(out.x), _p(out.rrmax), _p(out.d0), _p(rid))
    if rc != 0:
        raise ValueError("oracle sample: invalid scene (c0*T60 must exceed D0) or parameters")
    return out


def _scene_arrays(scene, params: Params):
    rir_len, rir_off, vs_off = layout(scene.rt60, scene.n_vs, scene.S, scene.M, params.fs)
    return (rir_len, rir_off, vs_off, _f64(scene.src), _f64(scene.mic),
            np.ascontiguousarray(scene.n_vs, dtype=np.int32))


def synthesize(scene, params: Params, vs_pos, vs_g, r, early: bool = False):
    """FP64 RIRs (flat, ragged layout) and optionally the early RIRs of Eq. 9."""
    rir_len, rir_off, vs_off, src, mic, n_vs = _scene_arrays(scene, params)
    vs_pos, vs_g, r = _f64(vs_pos).reshape(-1, 3), _f64(vs_g).reshape(-1), _f64(r).reshape(-1)
    assert vs_pos.shape[0] == vs_off[-1] and vs_g.shape[0] == vs_off[-1] and r.shape[0] == scene.B
    rir = np.empty(int(rir_off[-1]))
    he = np.empty(int(rir_off[-1])) if early else None
    pc = params._c()
    rc = _load().fo_synthesize(ctypes.c_int32(scene.B), ctypes.c_int32(scene.S), ctypes.c_int32(scene.M),
                               _p(src), _p(mic), _p(n_vs), _p(vs_off), _p(rir_len), _p(rir_off),
                               _p(vs_pos), _p(vs_g), _p(r), ctypes.byref(pc), _p(rir), _p(he))
    if rc != 0:
        raise ValueError("oracle synthesize: invalid parameters")
    return (rir, he) if early else rir


def backward(scene, params: Params, vs_pos, vs_g, r, grad_rir, grad_early=None, with_g: bool = False):
    """Analytic FP64 gradient: (grad_vs [N,3], grad_mic [B,M,3], grad_src [B,S,3], grad_r [B])
    and, with with_g, also grad_g [N] (dL/dg_i through the amplitudes r^g_i)."""
    rir_len, rir_off, vs_off, src, mic, n_vs = _scene_arrays(scene, params)
    vs_pos, vs_g, r = _f64(vs_pos).reshape(-1, 3), _f64(vs_g).reshape(-1), _f64(r).reshape(-1)
    grad_rir = _f64(grad_rir).reshape(-1) if grad_rir is not None else None
    grad_early = _f64(grad_early).reshape(-1) if grad_early is not None else None
    N = int(vs_off[-1])
    gv = np.empty((N, 3))
    gm = np.empty((scene.B, scene.M, 3))
    gs = np.empty((scene.B, scene.S, 3))
    gr = np.empty(scene.B)
    gg = np.empty(N) if with_g else None
    pc = params._c()
    rc = _load().fo_backward(ctypes.c_int32(scene.B), ctypes.c_int32(scene.S), ctypes.c_int32(scene.M),
                             _p(src), _p(mic), _p(n_vs), _p(vs_off), _p(rir_len), _p(rir_off),
                             _p(vs_pos), _p(vs_g), _p(r), ctypes.byref(pc), _p(grad_rir), _p(grad_early),
                             _p(gv), _p(gm), _p(gs), _p(gr), _p(gg))
    if rc != 0:
        raise ValueError("oracle backward: invalid parameters")
    return (gv, gm, gs, gr, gg) if with_g else (gv, gm, gs, gr)


def sample_backward(scene, params: Params, seed: int, grad_vs, grad_g, grad_r, grad_src_dir, grad_mic_dir,
                    room_ids=None):
    """Gradients through the sampler with the draws held fixed (reparameterised): from the
    synthesis adjoint's (grad_vs, grad_g, grad_r, grad_src, grad_mic) to the total
    (grad_src [B,S,3], grad_mic [B,M,3], grad_t60 [B], grad_dims [B,3])."""
    _, _, vs_off = layout(scene.rt60, scene.n_vs, scene.S, scene.M, params.fs)
    dims, rt60, src, mic = _f64(scene.dims), _f64(scene.rt60), _f64(scene.src), _f64(scene.mic)
    n_vs = np.ascontiguousarray(scene.n_vs, dtype=np.int32)
    rid = np.ascontiguousarray(room_ids, dtype=np.int32) if room_ids is not None else None
    gs = np.empty((scene.B, scene.S, 3))
    gm = np.empty((scene.B, scene.M, 3))
    gt = np.empty(scene.B)
    gd = np.empty((scene.B, 3))
    pc = params._c()
    rc = _load().fo_sample_backward(ctypes.c_int32(scene.B), ctypes.c_int32(scene.S), ctypes.c_int32(scene.M),
                                    _p(dims), _p(rt60), _p(src), _p(mic), _p(n_vs), _p(vs_off), ctypes.byref(pc),
                                    ctypes.c_uint64(seed), _p(rid), _p(_f64(grad_vs)), _p(_f64(grad_g)),
                                    _p(_f64(grad_r)), _p(_f64(grad_src_dir)), _p(_f64(grad_mic_dir)),
                                    _p(gs), _p(gm), _p(gt), _p(gd))
    if rc != 0:
        raise ValueError("oracle sample_backward: invalid scene or parameters")
    return gs, gm, gt, gd


def mr_rates(fs: float):
    """(r_h, r_l) = (floor(1e6 / fs), floor(sqrt(r_h))) (Sec. II-B)."""
    rh, rl = ctypes.c_int32(), ctypes.c_int32()
    _load().fo_mr_rates(ctypes.c_double(fs), ctypes.byref(rh), ctypes.byref(rl))
    return rh.value, rl.value


def resample_filter(up: int, down: int) -> np.ndarray:
    """The resampling FIR for a reduced ratio up/down, centred: F[m + HL], |m| <= HL."""
    L = _load()
    L.fo_resample_filter.restype = ctypes.c_int32
    hl = L.fo_resample_filter(ctypes.c_int32(up), ctypes.c_int32(down), None)
    F = np.empty(2 * hl + 1)
    L.fo_resample_filter(ctypes.c_int32(up), ctypes.c_int32(down), _p(F))
    return F


def hpf_coeffs(fc: float, fsr: float):
    """(b, a) of the 2nd-order Butterworth high-pass (bilinear transform, pre-warped)."""
    b, a = np.empty(3), np.empty(3)
    _load().fo_hpf_coeffs(ctypes.c_double(fc), ctypes.c_double(fsr), _p(b), _p(a))
    return b, a


def synthesize_mr(scene, params: Params, vs_pos, vs_g, r, early: bool = False):
    """FP64 RIRs of the paper's multi-rate path, in the layout of synthesize()."""
    rir_len, rir_off, vs_off, src, mic, n_vs = _scene_arrays(scene, params)
    vs_pos, vs_g, r = _f64(vs_pos).reshape(-1, 3), _f64(vs_g).reshape(-1), _f64(r).reshape(-1)
    assert vs_pos.shape[0] == vs_off[-1] and vs_g.shape[0] == vs_off[-1] and r.shape[0] == scene.B
    rt60 = _f64(np.asarray(scene.rt60, dtype=np.float32))
    rir = np.empty(int(rir_off[-1]))
    he = np.empty(int(rir_off[-1])) if early else None
    pc = params._c()
    rc = _load().fo_synthesize_mr(ctypes.c_int32(scene.B), ctypes.c_int32(scene.S), ctypes.c_int32(scene.M),
                                  _p(src), _p(mic), _p(rt60), _p(n_vs), _p(vs_off), _p(rir_len), _p(rir_off),
                                  _p(vs_pos), _p(vs_g), _p(r), ctypes.byref(pc), _p(rir), _p(he))
    if rc != 0:
        raise ValueError("oracle synthesize_mr: invalid parameters or out of memory")
    return (rir, he) if early else rir


def spatialize(rir_len, rir_off, rir, signals, n_speech: int, level_db, target_rir=None, M: int = None):
    """Mixture [B,M,N], targets [B,n_speech,M,N] (None without target_rir) and gains [B,S] of
    the Sec. IV-A spatialisation: signals [B,S,N] convolved with the ragged RIR buffer (room b
    at rir_off[b], [S][M][L_b]), speakers scaled to level_db (SIR, dB) against speaker 0, noise
    sources (s >= n_speech) to level_db (SNR, dB) against the speech at mic 0."""
    x = _f64(signals)
    B, S, N = x.shape
    rir_len = np.ascontiguousarray(rir_len, dtype=np.int32)
    rir_off = np.ascontiguousarray(rir_off, dtype=np.int64)
    if M is None:
        M = int((rir_off[1] - rir_off[0]) // (S * rir_len[0])) if B else 1
    h = _f64(rir)
    ht = _f64(target_rir) if target_rir is not None else None
    lv = _f64(level_db).reshape(B, S)
    mix = np.empty((B, M, N))
    tg = np.empty((B, n_speech, M, N)) if ht is not None else None
    g = np.empty((B, S))
    rc = _load().fo_spatialize(ctypes.c_int32(B), ctypes.c_int32(S), ctypes.c_int32(M), _p(rir_len), _p(rir_off),
                               _p(h), _p(ht), ctypes.c_int64(N), _p(x), ctypes.c_int32(n_speech), _p(lv),
                               _p(mix), _p(tg), _p(g))
    if rc != 0:
        raise ValueError("oracle spatialize: invalid arguments")
    return mix, tg, g
