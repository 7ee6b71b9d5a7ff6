"""PyTorch-facing binding of libfram.  Argument marshalling only: every step of sampling,
synthesis and the adjoint runs in the library's CUDA kernels.

    from paper_2304_08052_gb300 import api, scenes
    sc = api.DeviceScene(scenes.batch_256(0), api.Params(fs=16000, half_len=40))
    vs = api.sample(sc, seed=1)                # images: pos_hi, pos_lo, g; per-room r
    rir = api.synthesize(sc, vs)               # flat ragged RIR buffer on the GPU
    h = sc.channel(rir, b=0, s=0, m=0)         # one channel
    # Differentiable path (gradients w.r.t. source, mic, image positions and r):
    src = sc.src.clone().requires_grad_()
    rir = api.rir(sc, src, sc.mic, vs.pos_hi.clone().requires_grad_(), vs.r.clone().requires_grad_(), vs.g,
                  vs.pos_lo)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import FramParams, FramScene, FramSpatial, check, lib


@dataclass
class Params:
    """Method constants (see include/fram.h).  alpha, beta, a, b, tau and c0 are not fixed by
    the paper; these are the library defaults."""
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
    tile: int = 0
    delay_mode: int = 0          # 1 = the paper's multi-rate output path (forward only)

    def c(self) -> FramParams:
        return FramParams(self.alpha, self.beta, self.a, self.b, self.tau, self.c0, self.fs,
                          self.early_pre_ms, self.early_post_ms, int(self.half_len), int(self.tile),
                          int(self.delay_mode), 0)


def layout(rt60, n_vs, S: int, M: int, fs: float):
    """Host layout through fram_layout: (rir_len [B] i32, rir_off [B+1] i64, vs_off [B+1] i64)."""
    rt60 = np.ascontiguousarray(rt60, dtype=np.float32)
    n_vs = np.ascontiguousarray(n_vs, dtype=np.int32)
    B = rt60.shape[0]
    rir_len = np.empty(B, np.int32)
    rir_off = np.empty(B + 1, np.int64)
    vs_off = np.empty(B + 1, np.int64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    check(lib().fram_layout(B, S, M, float(fs), p(rt60), p(n_vs), p(rir_len), p(rir_off), p(vs_off)))
    return rir_len, rir_off, vs_off


_F32 = (torch.float32,)
_SEED = (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ())
_WORD = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())


def _ptr(t: Optional[torch.Tensor], n: int = 0, dtypes=_F32, name: str = "tensor"):
    """The data pointer handed to libfram, after the checks the library cannot make itself: a
    contiguous CUDA tensor of the expected element type holding at least n elements (the kernels
    index up to the sizes the scene implies, so a smaller buffer would be read out of bounds)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor, got {type(t).__name__}")
    if t.dtype not in dtypes:
        raise ValueError(f"{name}: expected dtype {dtypes[0]}, got {t.dtype}")
    if t.numel() < n:
        raise ValueError(f"{name}: needs at least {n} elements, has {t.numel()}")
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name}: libfram takes contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class DeviceScene:
    """A scene resident on the GPU plus its layout and a workspace.  The workspace is
    allocated once here (by PyTorch), never by the library.  room_base is the index of room 0
    in a larger batch (a shard of that batch draws the images the whole batch gives its rooms)."""

    def __init__(self, scene, params: Params, device: str = "cuda", room_base: int = 0):
        self.scene = scene
        self.params = params
        self.room_base = int(room_base)
        self.B, self.S, self.M = int(scene.B), int(scene.S), int(scene.M)
        self.rir_len, self.rir_off, self.vs_off = layout(scene.rt60, scene.n_vs, self.S, self.M, params.fs)
        self.n_vs_total = int(self.vs_off[-1])
        self.rir_total = int(self.rir_off[-1])
        self.max_len = int(self.rir_len.max()) if self.B else 0
        mic64 = np.asarray(scene.mic, np.float64)
        cen = mic64.mean(axis=1, keepdims=True)
        self.array_radius = float(np.linalg.norm(mic64 - cen, axis=2).max()) if self.B else 0.0
        dev = torch.device(device)
        f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev)
        self.dims = f32(scene.dims)
        self.rt60 = f32(scene.rt60)
        self.src = f32(scene.src)
        self.mic = f32(scene.mic)
        self.n_vs = torch.as_tensor(np.ascontiguousarray(scene.n_vs, np.int32), device=dev)
        self.vs_off_d = torch.as_tensor(self.vs_off, device=dev)
        self.rir_len_d = torch.as_tensor(self.rir_len, device=dev)
        self.rir_off_d = torch.as_tensor(self.rir_off, device=dev)
        nbytes = ctypes.c_size_t(0)
        check(lib().fram_workspace_size(ctypes.byref(self.c_scene()), ctypes.byref(params.c()), ctypes.byref(nbytes)))
        self.ws_bytes = int(nbytes.value)
        raw = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=dev)
        off = (-raw.data_ptr()) % 256
        self._ws_raw = raw
        self.ws = raw[off:off + self.ws_bytes]

    def c_scene(self, src: Optional[torch.Tensor] = None, mic: Optional[torch.Tensor] = None,
                dims: Optional[torch.Tensor] = None, rt60: Optional[torch.Tensor] = None) -> FramScene:
        """The C scene; src, mic, dims and rt60 may be replaced by other device tensors of the
        same shapes (the layout -- RIR lengths and offsets -- stays the one made here)."""
        src = self.src if src is None else src
        mic = self.mic if mic is None else mic
        dims = getattr(self, "dims", None) if dims is None else dims
        rt60 = getattr(self, "rt60", None) if rt60 is None else rt60
        B, S, M = self.B, self.S, self.M
        cp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        return FramScene(self.B, self.S, self.M, self.max_len, self.n_vs_total, self.rir_total, self.array_radius,
                         _ptr(dims, 3 * B, name="dims"), _ptr(rt60, B, name="rt60"), _ptr(src, 3 * B * S, name="src"),
                         _ptr(mic, 3 * B * M, name="mic"),
                         cp(getattr(self, "n_vs", None)), cp(getattr(self, "vs_off_d", None)),
                         cp(getattr(self, "rir_len_d", None)), cp(getattr(self, "rir_off_d", None)),
                         getattr(self, "room_base", 0))

    def channel(self, buf: torch.Tensor, b: int, s: int, m: int) -> torch.Tensor:
        L = int(self.rir_len[b])
        o = int(self.rir_off[b]) + (s * self.M + m) * L
        return buf[o:o + L]

    def status(self) -> int:
        flags = ctypes.c_int32(0)
        rc = lib().fram_status(ctypes.c_void_p(self.ws.data_ptr()), _stream(), ctypes.byref(flags))
        if rc not in (_lib.FRAM_OK, _lib.FRAM_EDEVICE):
            check(rc)
        return int(flags.value)


@dataclass
class Images:
    pos_hi: torch.Tensor                 # [N,3]
    pos_lo: torch.Tensor                 # [N,3]
    g: torch.Tensor                      # [N]
    r: torch.Tensor                      # [B]
    words: Optional[torch.Tensor] = None  # [N,4] int32 view of the Philox words


def sample(sc: DeviceScene, seed: int = 0, d_seed: Optional[torch.Tensor] = None, words: bool = False,
           out: Optional[Images] = None, src=None, mic=None, dims=None, rt60=None) -> Images:
    """fram_sample: draw every (room, source)'s images on the GPU (src, mic, dims, rt60: optional
    replacements for the scene's own device tensors)."""
    dev = sc.dims.device
    N = sc.n_vs_total
    if out is None:
        out = Images(torch.empty((N, 3), dtype=torch.float32, device=dev),
                     torch.empty((N, 3), dtype=torch.float32, device=dev),
                     torch.empty(N, dtype=torch.float32, device=dev),
                     torch.empty(sc.B, dtype=torch.float32, device=dev),
                     torch.empty((N, 4), dtype=torch.int32, device=dev) if words else None)
    B = sc.B
    check(lib().fram_sample(ctypes.byref(sc.c_scene(src, mic, dims, rt60)), ctypes.byref(sc.params.c()),
                            ctypes.c_uint64(seed & (2**64 - 1)), _ptr(d_seed, 1, _SEED, "d_seed"),
                            _ptr(out.pos_hi, 3 * N, name="pos_hi"), _ptr(out.pos_lo, 3 * N, name="pos_lo"),
                            _ptr(out.g, N, name="g"), _ptr(out.r, B, name="r"), _ptr(out.words, 4 * N, _WORD, "words"),
                            ctypes.c_void_p(sc.ws.data_ptr()), ctypes.c_size_t(sc.ws_bytes), _stream()))
    return out


def _images(sc: DeviceScene, pos_hi, pos_lo, g, r):
    N = sc.n_vs_total
    return (_ptr(pos_hi, 3 * N, name="pos_hi"), _ptr(pos_lo, 3 * N, name="pos_lo"),
            _ptr(g, N, name="g") if g is not None else None, _ptr(r, sc.B, name="r"))


def synthesize_raw(sc: DeviceScene, pos_hi, pos_lo, g, r, src=None, mic=None, early: bool = False,
                   rir: Optional[torch.Tensor] = None, early_out: Optional[torch.Tensor] = None):
    """fram_synthesize on explicit tensors.  Returns rir or (rir, early)."""
    dev = sc.dims.device
    if rir is None:
        rir = torch.empty(sc.rir_total, dtype=torch.float32, device=dev)
    if early and early_out is None:
        early_out = torch.empty(sc.rir_total, dtype=torch.float32, device=dev)
    src = sc.src if src is None else src
    mic = sc.mic if mic is None else mic
    T = sc.rir_total
    check(lib().fram_synthesize(ctypes.byref(sc.c_scene(src, mic)), ctypes.byref(sc.params.c()),
                                *_images(sc, pos_hi, pos_lo, g, r), _ptr(rir, T, name="rir"),
                                _ptr(early_out, T, name="early_out") if early else None,
                                ctypes.c_void_p(sc.ws.data_ptr()), ctypes.c_size_t(sc.ws_bytes), _stream()))
    return (rir, early_out) if early else rir


def synthesize(sc: DeviceScene, vs: Images, early: bool = False, **kw):
    return synthesize_raw(sc, vs.pos_hi, vs.pos_lo, vs.g, vs.r, early=early, **kw)


def synthesize_backward_raw(sc: DeviceScene, pos_hi, pos_lo, g, r, grad_rir, grad_early=None, src=None, mic=None,
                            want=("vs", "mic", "src", "r")):
    """fram_synthesize_backward.  Returns (grad_vs [N,3], grad_mic [B,M,3], grad_src [B,S,3], grad_r [B]),
    plus grad_g [N] last when "g" is in `want`."""
    dev = sc.dims.device
    gg = torch.empty(sc.n_vs_total, dtype=torch.float32, device=dev) if "g" in want else None
    gv = torch.empty((sc.n_vs_total, 3), dtype=torch.float32, device=dev) if "vs" in want else None
    gm = torch.empty((sc.B, sc.M, 3), dtype=torch.float32, device=dev) if "mic" in want else None
    gs = torch.empty((sc.B, sc.S, 3), dtype=torch.float32, device=dev) if "src" in want else None
    gr = torch.empty(sc.B, dtype=torch.float32, device=dev) if "r" in want else None
    src = sc.src if src is None else src
    mic = sc.mic if mic is None else mic
    T = sc.rir_total
    check(lib().fram_synthesize_backward(ctypes.byref(sc.c_scene(src, mic)), ctypes.byref(sc.params.c()),
                                         *_images(sc, pos_hi, pos_lo, g, r), _ptr(grad_rir, T, name="grad_rir"),
                                         _ptr(grad_early, T, name="grad_early"), *_grad_outs(sc, gv, gm, gs, gr, gg),
                                         ctypes.c_void_p(sc.ws.data_ptr()), ctypes.c_size_t(sc.ws_bytes), _stream()))
    return (gv, gm, gs, gr, gg) if "g" in want else (gv, gm, gs, gr)


def _grad_outs(sc: DeviceScene, gv, gm, gs, gr, gg):
    N, B, S, M = sc.n_vs_total, sc.B, sc.S, sc.M
    return (_ptr(gv, 3 * N, name="grad_vs"), _ptr(gm, 3 * B * M, name="grad_mic"),
            _ptr(gs, 3 * B * S, name="grad_src"), _ptr(gr, B, name="grad_r"), _ptr(gg, N, name="grad_g"))


def sample_backward(sc: DeviceScene, seed: int, grad_vs, grad_g=None, grad_r=None, grad_src_in=None,
                    grad_mic_in=None, d_seed: Optional[torch.Tensor] = None, src=None, mic=None, dims=None,
                    rt60=None, out=None):
    """fram_sample_backward: carry image and r gradients back through the sampler (draws of
    `seed` held fixed).  Returns (grad_src [B,S,3], grad_mic [B,M,3], grad_t60 [B], grad_dims [B,3]),
    source and mic gradients including grad_src_in / grad_mic_in (the direct paths)."""
    dev = sc.dims.device
    if out is None:
        out = (torch.empty((sc.B, sc.S, 3), dtype=torch.float32, device=dev),
               torch.empty((sc.B, sc.M, 3), dtype=torch.float32, device=dev),
               torch.empty(sc.B, dtype=torch.float32, device=dev),
               torch.empty((sc.B, 3), dtype=torch.float32, device=dev))
    gs, gm, gt, gd = out
    N, B, S, M = sc.n_vs_total, sc.B, sc.S, sc.M
    check(lib().fram_sample_backward(ctypes.byref(sc.c_scene(src, mic, dims, rt60)), ctypes.byref(sc.params.c()),
                                     ctypes.c_uint64(seed & (2**64 - 1)), _ptr(d_seed, 1, _SEED, "d_seed"),
                                     _ptr(grad_vs, 3 * N, name="grad_vs"), _ptr(grad_g, N, name="grad_g"),
                                     _ptr(grad_r, B, name="grad_r"), _ptr(grad_src_in, 3 * B * S, name="grad_src_in"),
                                     _ptr(grad_mic_in, 3 * B * M, name="grad_mic_in"),
                                     _ptr(gs, 3 * B * S, name="grad_src"), _ptr(gm, 3 * B * M, name="grad_mic"),
                                     _ptr(gt, B, name="grad_t60"), _ptr(gd, 3 * B, name="grad_dims"),
                                     ctypes.c_void_p(sc.ws.data_ptr()), ctypes.c_size_t(sc.ws_bytes),
                                     _stream()))
    return gs, gm, gt, gd


class _FramRIR(torch.autograd.Function):
    """Differentiable synthesis: leaves src [B,S,3], mic [B,M,3], vs_pos [N,3], r [B]."""

    @staticmethod
    def forward(ctx, src, mic, vs_pos, r, g, vs_pos_lo, sc, early):
        src_c, mic_c, pos_c, r_c = (t.detach().contiguous() for t in (src, mic, vs_pos, r))
        g_c = g.detach().contiguous()
        lo_c = vs_pos_lo.detach().contiguous() if vs_pos_lo is not None else None
        out = synthesize_raw(sc, pos_c, lo_c, g_c, r_c, src=src_c, mic=mic_c, early=early)
        ctx.sc, ctx.early = sc, early
        ctx.save_for_backward(src_c, mic_c, pos_c, r_c, g_c, lo_c if lo_c is not None else torch.empty(0))
        ctx.has_lo = lo_c is not None
        return out if early else (out,)[0]

    @staticmethod
    def backward(ctx, *grads):
        src_c, mic_c, pos_c, r_c, g_c, lo_c = ctx.saved_tensors
        lo_c = lo_c if ctx.has_lo else None
        if ctx.early:
            g_rir, g_early = grads
        else:
            g_rir, g_early = grads[0], None
        g_rir = g_rir.contiguous() if g_rir is not None else None
        g_early = g_early.contiguous() if g_early is not None else None
        gv, gm, gs, gr = synthesize_backward_raw(ctx.sc, pos_c, lo_c, g_c, r_c, g_rir, g_early, src=src_c, mic=mic_c)
        return gs, gm, gv, gr, None, None, None, None


def rir(sc: DeviceScene, src, mic, vs_pos, r, g, vs_pos_lo=None, early: bool = False):
    """Differentiable RIR synthesis (autograd through fram_synthesize_backward)."""
    return _FramRIR.apply(src, mic, vs_pos, r, g, vs_pos_lo, sc, early)


class _FramSampledRIR(torch.autograd.Function):
    """Sampling and synthesis in one differentiable step: leaves src [B,S,3], mic [B,M,3],
    rt60 [B] and dims [B,3]; the draws of `seed` are held fixed (reparameterised), so the images
    move with the geometry and the gradient runs through the sampler (fram_sample_backward)."""

    @staticmethod
    def forward(ctx, src, mic, rt60, dims, sc, seed, early):
        geo = tuple(t.detach().contiguous() for t in (src, mic, rt60, dims))
        vs = sample(sc, seed, src=geo[0], mic=geo[1], rt60=geo[2], dims=geo[3])
        out = synthesize_raw(sc, vs.pos_hi, vs.pos_lo, vs.g, vs.r, src=geo[0], mic=geo[1], early=early)
        ctx.sc, ctx.seed, ctx.early = sc, seed, early
        ctx.save_for_backward(*geo, vs.pos_hi, vs.pos_lo, vs.g, vs.r)
        return out

    @staticmethod
    def backward(ctx, *grads):
        src, mic, rt60, dims, pos_hi, pos_lo, g, r = ctx.saved_tensors
        g_rir = grads[0].contiguous() if grads[0] is not None else None
        g_early = grads[1].contiguous() if ctx.early and grads[1] is not None else None
        gv, gm, gs, gr, gg = synthesize_backward_raw(ctx.sc, pos_hi, pos_lo, g, r, g_rir, g_early, src=src, mic=mic,
                                                     want=("vs", "mic", "src", "r", "g"))
        gs, gm, gt, gd = sample_backward(ctx.sc, ctx.seed, gv, gg, gr, gs, gm, src=src, mic=mic, dims=dims, rt60=rt60)
        return gs, gm, gt, gd, None, None, None


def sampled_rir(sc: DeviceScene, src, mic, rt60, dims, seed: int, early: bool = False):
    """Differentiable sample + synthesize: gradients w.r.t. source, mic, T60 and room size with
    the draws of `seed` held fixed.  RIR lengths stay those of the DeviceScene's own T60."""
    return _FramSampledRIR.apply(src, mic, rt60, dims, sc, seed, early)


def prepare(sc: DeviceScene, pos_hi, pos_lo, r, src=None, mic=None):
    """fram_prepare: per-room tables, work items and delay bins in the workspace."""
    src = sc.src if src is None else src
    mic = sc.mic if mic is None else mic
    ph, pl, _, pr = _images(sc, pos_hi, pos_lo, None, r)
    check(lib().fram_prepare(ctypes.byref(sc.c_scene(src, mic)), ctypes.byref(sc.params.c()), ph, pl, pr,
                             ctypes.c_void_p(sc.ws.data_ptr()), ctypes.c_size_t(sc.ws_bytes),
                             _stream()))


def synthesize_prepared(sc: DeviceScene, pos_hi, pos_lo, g, r, rir, early_out=None, src=None, mic=None):
    """fram_synthesize_prepared: the synthesis kernel alone, after prepare() on the same inputs."""
    src = sc.src if src is None else src
    mic = sc.mic if mic is None else mic
    T = sc.rir_total
    check(lib().fram_synthesize_prepared(ctypes.byref(sc.c_scene(src, mic)), ctypes.byref(sc.params.c()),
                                         *_images(sc, pos_hi, pos_lo, g, r), _ptr(rir, T, name="rir"),
                                         _ptr(early_out, T, name="early_out"),
                                         ctypes.c_void_p(sc.ws.data_ptr()), ctypes.c_size_t(sc.ws_bytes), _stream()))
    return rir


def synthesize_backward_prepared(sc: DeviceScene, pos_hi, pos_lo, g, r, grad_rir, grad_early=None, out=None,
                                 src=None, mic=None, grad_g=None):
    """fram_synthesize_backward_prepared: the adjoint kernels alone, after prepare()."""
    dev = sc.dims.device
    if out is None:
        out = (torch.empty((sc.n_vs_total, 3), dtype=torch.float32, device=dev),
               torch.empty((sc.B, sc.M, 3), dtype=torch.float32, device=dev),
               torch.empty((sc.B, sc.S, 3), dtype=torch.float32, device=dev),
               torch.empty(sc.B, dtype=torch.float32, device=dev))
    gv, gm, gs, gr = out
    src = sc.src if src is None else src
    mic = sc.mic if mic is None else mic
    T = sc.rir_total
    check(lib().fram_synthesize_backward_prepared(ctypes.byref(sc.c_scene(src, mic)), ctypes.byref(sc.params.c()),
                                                  *_images(sc, pos_hi, pos_lo, g, r),
                                                  _ptr(grad_rir, T, name="grad_rir"),
                                                  _ptr(grad_early, T, name="grad_early"),
                                                  *_grad_outs(sc, gv, gm, gs, gr, grad_g),
                                                  ctypes.c_void_p(sc.ws.data_ptr()), ctypes.c_size_t(sc.ws_bytes),
                                                  _stream()))
    return out


def spatialize(sc: DeviceScene, rir, signals, level_db, n_speech: int, target_rir=None, targets: bool = False,
               block: int = 0, chunk_rooms: int = 0, out=None):
    """fram_spatialize: mixture [B,M,N] of signals [B,S,N] (device, float32) through the ragged
    RIRs `rir`, speakers at level_db SIR and noise at level_db SNR (dB, [B,S]); with targets=True
    also the per-speaker targets [B,n_speech,M,N] through target_rir (default: rir).  Returns
    (mixture, targets or None, gains [B,S])."""
    dev = sc.dims.device
    if signals.dim() != 3:
        raise ValueError("signals: expected [B, S, N]")
    B, S, N = (int(v) for v in signals.shape)
    if B != sc.B or S != sc.S:
        raise ValueError(f"signals: expected [{sc.B}, {sc.S}, N], got {list(signals.shape)}")
    if not 1 <= int(n_speech) <= S:
        raise ValueError(f"n_speech must be in [1, {S}]")
    spc = FramSpatial(N, int(n_speech), int(block), int(chunk_rooms), 0)
    trir = (target_rir if target_rir is not None else rir) if targets else None
    sep = 1 if (trir is not None and trir.data_ptr() != rir.data_ptr()) else 0
    n = ctypes.c_size_t(0)
    check(lib().fram_spatialize_workspace_size(ctypes.byref(sc.c_scene()), ctypes.byref(spc), sep, ctypes.byref(n)))
    key = ("spatial", int(n.value))
    ws = getattr(sc, "_sp_ws", None)
    if ws is None or ws[0] != key:
        raw = torch.empty(int(n.value) + 256, dtype=torch.uint8, device=dev)
        off = (-raw.data_ptr()) % 256
        ws = (key, raw, raw[off:off + int(n.value)])
        sc._sp_ws = ws
    if out is None:
        out = (torch.empty((B, sc.M, N), dtype=torch.float32, device=dev),
               torch.empty((B, int(n_speech), sc.M, N), dtype=torch.float32, device=dev) if targets else None,
               torch.empty((B, S), dtype=torch.float32, device=dev))
    mix, tg, gains = out
    T, M, ns = sc.rir_total, sc.M, int(n_speech)
    check(lib().fram_spatialize(ctypes.byref(sc.c_scene()), ctypes.byref(spc), _ptr(rir, T, name="rir"),
                                _ptr(trir, T, name="target_rir"), _ptr(signals, B * S * N, name="signals"),
                                _ptr(level_db, B * S, name="level_db"), _ptr(mix, B * M * N, name="mixture"),
                                _ptr(tg, B * ns * M * N, name="targets") if targets else None,
                                _ptr(gains, B * S, name="gains"),
                                ctypes.c_void_p(ws[2].data_ptr()), ctypes.c_size_t(int(n.value)), _stream()))
    return mix, tg, gains


def spatialize_status(sc: DeviceScene) -> int:
    """Device status bits of the last fram_spatialize on this scene's spatialisation workspace."""
    flags = ctypes.c_int32(0)
    rc = lib().fram_status(ctypes.c_void_p(sc._sp_ws[2].data_ptr()), _stream(), ctypes.byref(flags))
    if rc not in (_lib.FRAM_OK, _lib.FRAM_EDEVICE):
        check(rc)
    return int(flags.value)


def algorithmic_taps(sc) -> int:
    """Windowed-sinc taps one synthesis performs: sum_b S M (I_b + 1)(2K + 1)."""
    K = int(sc.params.half_len) if isinstance(sc, DeviceScene) else int(sc.half_len)
    scene = sc.scene if isinstance(sc, DeviceScene) else sc
    return int(scene.S * scene.M * (np.asarray(scene.n_vs, np.int64) + 1).sum() * (2 * K + 1))


def autotune(sc: DeviceScene, vs: Images, rir: Optional[torch.Tensor] = None) -> int:
    """fram_autotune: time the candidate tile lengths on these inputs; later calls with
    params.tile == 0 on this kind of workload use the fastest.  Returns the chosen tile."""
    if rir is None:
        rir = torch.empty(sc.rir_total, dtype=torch.float32, device=sc.dims.device)
    out = ctypes.c_int32(0)
    check(lib().fram_autotune(ctypes.byref(sc.c_scene()), ctypes.byref(sc.params.c()),
                              *_images(sc, vs.pos_hi, vs.pos_lo, vs.g, vs.r), _ptr(rir, sc.rir_total, name="rir"),
                              ctypes.c_void_p(sc.ws.data_ptr()),
                              ctypes.c_size_t(sc.ws_bytes), _stream(), ctypes.byref(out)))
    return int(out.value)


def measure_alu(kind: int, iters: int) -> dict:
    """fram_measure_alu: throughput of one instruction kind (0 FP32 FMA, 1 packed FP32 FMA,
    2 MUFU reciprocal) on this GPU.  Returns the kernel time, SM cycles, lane operations and the
    derived lane operations per SM per clock and per second."""
    res = (ctypes.c_double * 4)()
    check(lib().fram_measure_alu(int(kind), int(iters), res, _stream()))
    ms, cyc, ops, sms = (float(v) for v in res)
    return {"ms": ms, "sm_cycles": cyc, "lane_ops": ops, "sms": int(sms),
            "per_sm_per_clock": ops / (cyc * sms), "per_s": ops / (ms * 1e-3), "clock_mhz": cyc / (ms * 1e3)}


def tuned_tile(sc: DeviceScene) -> int:
    """fram_tuned_tile: the tile length a launch with sc.params launches with."""
    out = ctypes.c_int32(0)
    check(lib().fram_tuned_tile(ctypes.byref(sc.c_scene()), ctypes.byref(sc.params.c()), ctypes.byref(out)))
    return int(out.value)
