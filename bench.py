#!/usr/bin/env python
"""Benchmark of the FRAM-RIR hot path on one GB300 (or N, one process per GPU under torchrun).

Workload (default): large_4096 -- 4096 rooms x 2 sources x 16-mic circle at 48 kHz, K = 63
(127-tap windowed sinc), round(6000 T60) images per (room, source), T60 ~ U[0.2, 1.2] s.
A step is one pass of the whole hot path over the batch:
  fwd:      fram_sample (Philox images) -> fram_synthesize (prologue, delay bins, synthesis)
  fwd+bwd:  fwd -> fram_synthesize_backward_prepared (adjoint, reusing the forward's bins)
  fwd+bwd through the sampler (reported beside): fwd+bwd with dL/dg -> fram_sample_backward
value = RIRs/s of the fwd step (one RIR = one 16-channel filter per room x source), whole job.

Also reported: taps/s; the synthesis kernel alone against the ALU roofline; the adjoint kernel
alone; an end-to-end number through host buffers; the graph-captured batched path against a
plain per-room launch loop (batch_1024 with early RIRs); the FP64 oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME] [--rooms N]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "multi-ch RIRs/s and sinc-taps/s (fwd, fwd+bwd) at 1 GB300, % of roofline"

# Algorithmic work per tap (the tap arithmetic of the paper's sum, Eq. 1 with windowed sincs):
# forward 8 FP32-pipe operations and 1 reciprocal on the MUFU (special function) pipe; adjoint
# 14 FP32 and 1 MUFU.  Per arrival (image x mic) 40 FP32 + 6 MUFU more, spread over its 2K+1 taps.
# DRAM bytes (read + write) of one synth_kernel launch per output sample, from one ncu capture
# (large_4096, first 256 rooms, 283357184 output samples: 0.0641 GB read + 1.0731 GB written);
# reported only while the synthesis source is the one that was measured (its SHA-256 prefix).
SYNTH_TRAFFIC = {"source_sha256": "96f1c3b045dc4cc7", "bytes_per_sample": (64156160 + 1072641792) / 283357184}

# Kernels of libfram per fwd step: sample_prologue, sample_kernel; room_prologue, item_scan,
# bin_images, sort_positions, item_ranges (preparation); amp_gather, synth_kernel (synthesis).
FWD_LAUNCHES = 9
FWD_FP32, BWD_FP32, ARR_FP32 = 8.0, 14.0, 40.0
TAP_MUFU, ARR_MUFU = 1.0, 6.0
FP32_LANES_PER_SM, MUFU_LANES_PER_SM = 128, 16


def combine(units_per_rank, seconds_per_rank):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return sum(units_per_rank) / max(seconds_per_rank)


def alu_peak_taps(sm_count: int, clock_hz: float, K: int, fp32_per_tap: float, fp32_lanes: float = FP32_LANES_PER_SM,
                  mufu_lanes: float = MUFU_LANES_PER_SM):
    """Taps/s the FP32 and MUFU pipes allow at `fp32_lanes` and `mufu_lanes` lane operations per SM
    per clock (nominal by default), and which pipe binds."""
    n = 2 * K + 1
    p_fp32 = sm_count * fp32_lanes * clock_hz
    p_mufu = sm_count * mufu_lanes * clock_hz
    by_fp32 = p_fp32 / (fp32_per_tap + ARR_FP32 / n)
    by_mufu = p_mufu / (TAP_MUFU + ARR_MUFU / n)
    return min(by_fp32, by_mufu), ("mufu" if by_mufu < by_fp32 else "fp32")


def measure_alu_lanes(api, seconds: float = 0.5):
    """FP32 FMA, packed FP32 FMA and MUFU reciprocal lane operations per SM per clock on this GPU
    (fram_measure_alu: a calibration run, then one of about `seconds`)."""
    out = {}
    for kind, name in ((0, "fp32_fma"), (1, "fp32x2_fma"), (2, "mufu_rcp")):
        cal = api.measure_alu(kind, 200)
        iters = max(200, int(200 * seconds * 1e3 / max(cal["ms"], 1e-3)))
        r = api.measure_alu(kind, iters)
        out[name] = {"per_sm_per_clock": r["per_sm_per_clock"], "lane_ops_per_s": r["per_s"], "ms": r["ms"],
                     "clock_mhz_from_cycles": r["clock_mhz"]}
    return out


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while a region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu_id], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _gpu_uuid(torch):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        return "0"


def _time_steps(torch, fn, steps, dist_ok, join=None):
    """Device time of `steps` calls of fn, bracketed by a barrier and synchronisations; `join`
    (optional) makes the timing stream wait for side streams before the end event."""
    if dist_ok:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    for k in range(steps):
        fn(k)
    if join is not None:
        join()
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e)
    if dist_ok:
        import torch.distributed as dist
        ms = max_over_ranks(torch, ms, "cuda")
        dist.barrier()
    return ms / 1000.0


def max_over_ranks(torch, x: float, device) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's time)."""
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(sc, seed, rooms, params):
    """The FP64 oracle as it stands, on the host cores, on `rooms` of the workload."""
    import oracle
    op = oracle.Params(fs=params.fs, half_len=params.half_len, alpha=params.alpha, beta=params.beta, a=params.a,
                       b=params.b, tau=params.tau, c0=params.c0)
    sub = sc.subset(rooms)
    t0 = time.perf_counter()
    ref = oracle.sample(sub, op, seed, room_ids=list(rooms))
    oracle.synthesize(sub, op, ref.pos, ref.g, ref.r)
    dt = time.perf_counter() - t0
    return len(rooms) * sc.S, dt, oracle.num_threads()


def run_reference(args):
    """Reference arm: the FP64 oracle on this machine's host cores, bounded samples of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2304_08052_gb300 import api, scenes
    sc = scenes.by_name(args.workload, 0)
    params = api.Params(fs=sc.fs, half_len=sc.half_len)
    per_step = args.ref_rooms
    import numpy as np
    rng = np.random.default_rng(0)
    for _ in range(args.warmup):
        cpu_baseline(sc, 1, sorted(rng.choice(sc.B, 1, replace=False).tolist()), params)
    units, secs, cores = 0, 0.0, 1
    for k in range(args.steps):
        rooms = sorted(rng.choice(sc.B, per_step, replace=False).tolist())
        u, dt, cores = cpu_baseline(sc, 100 + k, rooms, params)
        units += u
        secs += dt
    value = units / secs
    sample = f"{per_step} seeded rooms of {args.workload} per step (sample + synthesize, FP64)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RIRs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": sc.name, "rooms": sc.B, "sources": sc.S, "mics": sc.M, "fs": sc.fs,
                       "half_len": params.half_len, "rooms_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "RIRs/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "RIRs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _synth_traffic(rir_samples):
    """DRAM bytes of one synthesis launch from the recorded capture, or None if the kernel changed."""
    import hashlib
    src = os.path.join(ROOT, "paper_2304_08052_gb300", "csrc", "fram_synth.cu")
    with open(src, "rb") as f:
        if hashlib.sha256(f.read()).hexdigest()[:16] != SYNTH_TRAFFIC["source_sha256"]:
            return None
    return SYNTH_TRAFFIC["bytes_per_sample"] * rir_samples


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fused", choices=["fused", "reference"])
    ap.add_argument("--workload", default="large_4096")
    ap.add_argument("--rooms", type=int, default=0, help="first N rooms of the workload only (0 = all); "
                    "for profiler captures of a small case")
    ap.add_argument("--ref-rooms", type=int, default=8)
    ap.add_argument("--cpu-rooms", type=int, default=512)
    ap.add_argument("--cpu-rooms-1core", type=int, default=32)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the per-room comparison and the CPU baseline")
    ap.add_argument("--spatialize-rooms", type=int, default=0,
                    help="only time fram_spatialize on the first N rooms of batch_1024 (for profiling) and exit")
    ap.add_argument("--alu-only", action="store_true",
                    help="only measure the FP32 and MUFU lane rates the roofline divides by, and exit")
    ap.add_argument("--multirate-only", action="store_true",
                    help="only time the multi-rate path against the continuous one on batch_1024 (for profiling) "
                         "and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.alu_only:
        import torch

        from paper_2304_08052_gb300 import api, build
        build.build()
        with ClockSampler(_gpu_uuid(torch)) as clk:
            alu = measure_alu_lanes(api, seconds=2.0)
        print(json.dumps({"alu_only": alu, "clocks": clk.summary(),
                          "sms": torch.cuda.get_device_properties(0).multi_processor_count}), flush=True)
        return 0
    if args.multirate_only:
        import torch

        from paper_2304_08052_gb300 import api, build, scenes
        build.build()
        peaks, _ = _measured_peaks()
        print(json.dumps({"multirate_only": multirate_vs_continuous(torch, api, scenes, peaks, cpu=False,
                                                                    rooms=args.rooms)}), flush=True)
        return 0
    if args.spatialize_rooms > 0:
        import torch

        from paper_2304_08052_gb300 import api, build, scenes
        build.build()
        peaks, _ = _measured_peaks()
        print(json.dumps({"spatialize_only": spatialize_batch(torch, api, scenes, peaks, cpu_rooms=0,
                                                              rooms=args.spatialize_rooms)}), flush=True)
        return 0

    import numpy as np
    import torch

    from paper_2304_08052_gb300 import api, build, scenes, shard

    build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist_ok = world > 1
    if dist_ok:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # One batch of `world` seeded blocks of the workload (block k: scene seed k), split into
    # contiguous cost-balanced room ranges, one per rank; every rank draws its rooms' images
    # with their global room index (room_base), so its rows equal those of the whole batch.
    glob = shard.global_batch(scenes.by_name, args.workload, world)
    if args.rooms > 0:
        glob = glob.subset(range(min(args.rooms * world, glob.B)))
    ranges = shard.partition(shard.room_costs(glob, glob.half_len), world)
    room_base, hi = ranges[rank]
    sc = glob.subset(range(room_base, hi))
    params = api.Params(fs=sc.fs, half_len=sc.half_len)
    ds = api.DeviceScene(sc, params, room_base=room_base)
    job_rirs = glob.B * glob.S                  # RIRs of the whole job per step
    job_taps = api.algorithmic_taps(glob)
    N, T = ds.n_vs_total, ds.rir_total
    vs = api.Images(torch.empty((N, 3), device="cuda"), torch.empty((N, 3), device="cuda"),
                    torch.empty(N, device="cuda"), torch.empty(sc.B, device="cuda"))
    rir = torch.empty(T, device="cuda")
    G = torch.empty(T, device="cuda").normal_(generator=torch.Generator(device="cuda").manual_seed(7))
    grads = (torch.empty((N, 3), device="cuda"), torch.empty((sc.B, sc.M, 3), device="cuda"),
             torch.empty((sc.B, sc.S, 3), device="cuda"), torch.empty(sc.B, device="cuda"))
    grad_g = torch.empty(N, device="cuda")
    sgrads = (torch.empty((sc.B, sc.S, 3), device="cuda"), torch.empty((sc.B, sc.M, 3), device="cuda"),
              torch.empty(sc.B, device="cuda"), torch.empty((sc.B, 3), device="cuda"))
    taps = api.algorithmic_taps(ds)

    def fwd(k):
        api.sample(ds, seed=1000 + k, out=vs)
        api.synthesize_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, rir=rir)

    def fwd_bwd(k):
        fwd(k)
        api.synthesize_backward_prepared(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, G, None, out=grads)

    def sampler_bwd(k):
        api.sample_backward(ds, 1000 + k, grads[0], grad_g, grads[3], grads[2], grads[1], out=sgrads)

    def fwd_bwd_sampler(k):
        fwd(k)
        api.synthesize_backward_prepared(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, G, None, out=grads, grad_g=grad_g)
        sampler_bwd(k)

    api.sample(ds, seed=999, out=vs)
    tile = api.autotune(ds, vs, rir)       # picks the tile length; tile = 0 launches use it

    peaks, peak_kind = _measured_peaks()
    clock_hz = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    alu = measure_alu_lanes(api)
    # The FP32 pipe's lane rate: the better of the scalar and the packed probe (the packed one
    # issues half as many instructions, so loop overhead hides less of the pipe).
    fp32_lanes = max(alu["fp32_fma"]["per_sm_per_clock"], alu["fp32x2_fma"]["per_sm_per_clock"])
    mufu_lanes = alu["mufu_rcp"]["per_sm_per_clock"]

    for k in range(args.warmup):
        fwd_bwd_sampler(k)
    torch.cuda.synchronize()
    assert ds.status() == 0, "device status flags set"
    with ClockSampler(_gpu_uuid(torch)) as clk:
        t_fwd = _time_steps(torch, fwd, args.steps, dist_ok)
        t_fb = _time_steps(torch, fwd_bwd, args.steps, dist_ok)
        t_fbs = _time_steps(torch, fwd_bwd_sampler, args.steps, dist_ok)
        t_sb = _time_steps(torch, sampler_bwd, args.steps, False)
        # Kernels alone on the same stream, after one preparation.
        api.prepare(ds, vs.pos_hi, vs.pos_lo, vs.r)
        t_syn = _time_steps(torch, lambda k: api.synthesize_prepared(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, rir),
                            args.steps, False)
        t_bwd = _time_steps(torch, lambda k: api.synthesize_backward_prepared(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, G,
                                                                              None, out=grads), args.steps, False)
    clocks = clk.summary()
    assert ds.status() == 0, "device status flags set"

    value = args.steps * job_rirs / t_fwd
    ms_step = 1000.0 * t_fwd / args.steps
    K = params.half_len
    peak_fwd, lim_fwd = alu_peak_taps(sm_count, clock_hz, K, FWD_FP32, fp32_lanes, mufu_lanes)
    peak_bwd, lim_bwd = alu_peak_taps(sm_count, clock_hz, K, BWD_FP32, fp32_lanes, mufu_lanes)
    nom_fwd, _ = alu_peak_taps(sm_count, clock_hz, K, FWD_FP32)
    nom_bwd, _ = alu_peak_taps(sm_count, clock_hz, K, BWD_FP32)
    syn_s = t_syn / args.steps
    bwd_s = t_bwd / args.steps
    ach_fwd = taps / syn_s
    ach_bwd = taps / bwd_s
    out_bytes = 4 * T
    line = {
        "metric": METRIC, "value": value, "unit": "RIRs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": glob.name, "rooms": glob.B, "sources": sc.S, "mics": sc.M, "fs": sc.fs,
                   "half_len": K, "images": int(N), "rir_samples": int(T), "taps_per_step": job_taps,
                   "parallelism": (f"rooms split over {world} GPUs in contiguous cost-balanced ranges, global "
                                   "Philox room indices, no collective on the data path" if world > 1 else "1 GPU"),
                   "l2": f"outputs {out_bytes / 1e9:.1f} GB per step, larger than L2 (129 MB)",
                   "tile": tile, "tile_choice": "fram_autotune over 256/512/1024/2048"},
        "taps_per_s": job_taps * args.steps / t_fwd,
        "fwd_bwd": {"value": args.steps * job_rirs / t_fb, "unit": "RIRs/s",
                    "ms_per_step": 1000.0 * t_fb / args.steps, "taps_per_s": 2 * job_taps * args.steps / t_fb},
        "roofline": {"bound": "alu", "achieved": ach_fwd / 1e9, "peak": peak_fwd / 1e9, "unit": "Gtap/s",
                     "frac": ach_fwd / peak_fwd, "traffic": _synth_traffic(T),
                     "kernel": "synth_kernel (timed with amp_gather)",
                     "limit": lim_fwd, "kernel_ms": 1000.0 * syn_s, "hbm_gbs": out_bytes / syn_s / 1e9,
                     "peak_basis": "measured",
                     "peak_detail": f"{sm_count} SMs x ({fp32_lanes:.1f} FP32, {mufu_lanes:.2f} MUFU) lane ops per "
                                    f"SM per clock (measured by fram_measure_alu in this run) x "
                                    f"{clock_hz / 1e6:.0f} MHz ({peak_kind} sm_max_mhz); per tap "
                                    f"{FWD_FP32:.0f} FP32 + {TAP_MUFU:.0f} MUFU, per arrival {ARR_FP32:.0f} FP32 + "
                                    f"{ARR_MUFU:.0f} MUFU",
                     "nominal": {"peak": nom_fwd / 1e9, "frac": ach_fwd / nom_fwd,
                                 "basis": f"{FP32_LANES_PER_SM} FP32 and {MUFU_LANES_PER_SM} MUFU lanes per SM per clock"},
                     "taps_note": "taps counted as 2K+1 per arrival (the paper's window); the kernel evaluates 2K "
                                  "(the last weight is 0) and drops taps past the RIR end, about 0.8 % fewer "
                                  "on this workload"},
        "fwd_bwd_through_sampler": {
            "value": args.steps * job_rirs / t_fbs, "unit": "RIRs/s", "ms_per_step": 1000.0 * t_fbs / args.steps,
            "sample_backward_ms": 1000.0 * t_sb / args.steps,
            "sample_backward_hbm_gbs": 16.0 * N / (t_sb / args.steps) / 1e9,
            "note": "fwd -> adjoint with dL/dg -> fram_sample_backward (source, mic, T60, room-size gradients "
                    "with the draws held fixed); sample_backward reads 16 B per image"},
        "roofline_bwd": {"bound": "alu", "achieved": ach_bwd / 1e9, "peak": peak_bwd / 1e9, "unit": "Gtap/s",
                         "frac": ach_bwd / peak_bwd, "kernel": "bwd_kernel", "limit": lim_bwd,
                         "kernel_ms": 1000.0 * bwd_s, "peak_basis": "measured",
                         "nominal": {"peak": nom_bwd / 1e9, "frac": ach_bwd / nom_bwd}},
        "alu_lanes": alu,
        "gpu_launches": FWD_LAUNCHES * args.steps,
        "clocks": clocks,
    }

    if not args.no_e2e:
        line["e2e"] = e2e(torch, api, sc, params, ds, args, job_rirs, dist_ok)

    if not args.no_extras and rank == 0:
        line["graph_vs_per_room"] = graph_vs_per_room(torch, api, scenes)
        line["single_room_latency"] = single_room_latency(torch, api, scenes)
        line["multirate_vs_continuous"] = multirate_vs_continuous(torch, api, scenes, peaks)
        line["spatialize"] = spatialize_batch(torch, api, scenes, peaks)
        u, dt, cores = cpu_baseline(sc, 1, list(range(args.cpu_rooms)), params)
        line["cpu_baseline"] = {"value": u / dt, "unit": "RIRs/s", "cores": cores, "kind": "oracle",
                                "sample": f"first {args.cpu_rooms} rooms of {args.workload} (sample + synthesize, "
                                          f"FP64, {dt:.1f} s)"}
        import oracle
        threads = oracle.num_threads()
        oracle.set_num_threads(1)
        try:
            u1, dt1, _ = cpu_baseline(sc, 1, list(range(args.cpu_rooms_1core)), params)
        finally:
            oracle.set_num_threads(threads)
        line["cpu_baseline"]["single_core"] = {
            "value": u1 / dt1, "unit": "RIRs/s", "cores": 1,
            "sample": f"first {args.cpu_rooms_1core} rooms of {args.workload} (FP64, {dt1:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist_ok:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def e2e(torch, api, sc, params, ds, args, job_rirs, dist_ok, n_copy=4):
    """Same step through the public API from pinned host buffers: H2D of the scene arrays,
    fram_sample + fram_synthesize, D2H of the RIR buffer.  Pipelined: the RIRs alternate between
    two device buffers, and each step's device-to-host copy runs on n_copy side streams (one
    contiguous slice each) while the next step computes; a buffer is reused only after its copy
    has finished.  The timed region (the run's --steps, 3 to 20) ends when every copy has
    landed."""
    import numpy as np
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
            dict(dims=sc.dims, rt60=sc.rt60, src=sc.src, mic=sc.mic, n_vs=sc.n_vs.astype(np.int32),
                 vs_off=ds.vs_off, rir_len=ds.rir_len, rir_off=ds.rir_off).items()}
    dev = {"dims": ds.dims, "rt60": ds.rt60, "src": ds.src, "mic": ds.mic, "n_vs": ds.n_vs, "vs_off": ds.vs_off_d,
           "rir_len": ds.rir_len_d, "rir_off": ds.rir_off_d}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    out_host = torch.empty(ds.rir_total, dtype=torch.float32).pin_memory()
    N = ds.n_vs_total
    vs = api.Images(torch.empty((N, 3), device="cuda"), torch.empty((N, 3), device="cuda"),
                    torch.empty(N, device="cuda"), torch.empty(sc.B, device="cuda"))
    bufs = [torch.empty(ds.rir_total, device="cuda") for _ in range(2)]
    main = torch.cuda.current_stream()
    side = [torch.cuda.Stream() for _ in range(n_copy)]
    cuts = [ds.rir_total * c // n_copy for c in range(n_copy + 1)]
    done = [[None] * n_copy for _ in range(2)]

    def step(k):
        i = k % 2
        for ev in done[i]:
            if ev is not None:
                main.wait_event(ev)                # the buffer's previous copy has landed
        for name, t in host.items():
            dev[name].copy_(t, non_blocking=True)
        api.sample(ds, seed=2000 + k, out=vs)
        api.synthesize_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, rir=bufs[i])
        ready = torch.cuda.Event()
        ready.record(main)
        for c, cs in enumerate(side):
            cs.wait_event(ready)
            with torch.cuda.stream(cs):
                out_host[cuts[c]:cuts[c + 1]].copy_(bufs[i][cuts[c]:cuts[c + 1]], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(cs)
            done[i][c] = ev

    def join():
        for cs in side:
            main.wait_stream(cs)

    for k in range(args.warmup):
        step(k)
    join()
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 20))
    t = _time_steps(torch, step, steps, dist_ok, join=join)
    return {"value": steps * job_rirs / t, "unit": "RIRs/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(4 * ds.rir_total), "ms_per_step": 1000.0 * t / steps,
            "pipeline": f"2 device RIR buffers; D2H on {n_copy} side streams overlapping the next step"}


def single_room_latency(torch, api, scenes):
    """The single-room scene (6x5x3 m, 4 mics, 2000 images, 16 kHz) is latency-bound: time one
    fram_sample + fram_synthesize call at a time, each call timed on its own."""
    sc = scenes.single_room()
    params = api.Params(fs=sc.fs, half_len=sc.half_len)
    ds = api.DeviceScene(sc, params)
    N = ds.n_vs_total
    vs = api.Images(torch.empty((N, 3), device="cuda"), torch.empty((N, 3), device="cuda"),
                    torch.empty(N, device="cuda"), torch.empty(sc.B, device="cuda"))
    rir = torch.empty(ds.rir_total, device="cuda")
    for k in range(5):
        api.sample(ds, seed=k, out=vs)
        api.synthesize_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, rir=rir)
    torch.cuda.synchronize()
    ms = []
    for k in range(20):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        api.sample(ds, seed=100 + k, out=vs)
        api.synthesize_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, rir=rir)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return {"workload": "single_room (1 room x 1 source x 4 mics, 2000 images, 16 kHz, K=40)",
            "ms_median": statistics.median(ms), "ms_min": min(ms), "calls": len(ms)}


def multirate_vs_continuous(torch, api, scenes, peaks, cpu=True, rooms=0):
    """The paper's multi-rate output path (delay_mode 1: ~1 MHz impulse grid, two polyphase
    resamplers, 80 Hz high-pass) against the continuous path on batch_1024 with early RIRs:
    fram_sample + fram_synthesize per step.  The multi-rate stages stream an intermediate signal
    at r_l fs (7x the output at 16 kHz): written once by the first resampler and read once by the
    high-pass fused with the second resampler (the warm-up reads before each piece after the
    first are overhead, not counted)."""
    import math
    sc = scenes.batch_1024(0)
    if rooms > 0:
        sc = sc.subset(range(min(rooms, sc.B)))
    out = {"workload": f"batch_1024 ({sc.B} rooms x 3 src x 8 mics, 16 kHz, + early RIR)"}
    for mode in (0, 1):
        params = api.Params(fs=sc.fs, half_len=sc.half_len, delay_mode=mode)
        ds = api.DeviceScene(sc, params)
        N = ds.n_vs_total
        vs = api.Images(torch.empty((N, 3), device="cuda"), torch.empty((N, 3), device="cuda"),
                        torch.empty(N, device="cuda"), torch.empty(sc.B, device="cuda"))
        rir = torch.empty(ds.rir_total, device="cuda")
        early = torch.empty(ds.rir_total, device="cuda")

        def step(k):
            api.sample(ds, seed=500 + k, out=vs)
            api.synthesize_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, early=True, rir=rir, early_out=early)

        for k in range(3):
            step(k)
        torch.cuda.synchronize()
        t = _time_steps(torch, step, 5, False) / 5
        assert ds.status() == 0, "device status flags set"
        entry = {"ms_per_step": 1000.0 * t, "value": sc.B * sc.S / t, "unit": "RIRs/s"}
        if mode == 1:
            rh = math.floor(1e6 / sc.fs)
            rl = math.floor(math.sqrt(rh))
            inter = 2 * 4 * rl * ds.rir_total                 # RIR + early intermediate signals, bytes
            moved = 2 * inter + 2 * 4 * ds.rir_total          # 1 write + 1 read, outputs
            peak = float(peaks.get("hbm_gbs", 6800.0))
            entry["roofline"] = {"bound": "hbm", "achieved": moved / t / 1e9, "peak": peak, "unit": "GB/s",
                                 "frac": moved / t / 1e9 / peak, "bytes_per_step": moved,
                                 "note": "stream bytes of the multi-rate stages only"}
        out["continuous" if mode == 0 else "multirate"] = entry
    if not cpu:
        return out
    import oracle
    rooms = list(range(16))
    sub = sc.subset(rooms)
    op = oracle.Params(fs=sc.fs, half_len=sc.half_len)
    t0 = time.perf_counter()
    ref = oracle.sample(sub, op, 1, room_ids=rooms)
    oracle.synthesize_mr(sub, op, ref.pos, ref.g, ref.r, early=True)
    dt = time.perf_counter() - t0
    out["multirate"]["cpu_oracle"] = {"value": len(rooms) * sc.S / dt, "unit": "RIRs/s", "cores": oracle.num_threads(),
                                      "sample": f"first {len(rooms)} rooms (sample + multi-rate synthesize, FP64, {dt:.1f} s)"}
    return out


def spatialize_batch(torch, api, scenes, peaks, n_samples=64000, cpu_rooms=2, rooms=0):
    """The paper's consumer of the RIRs (Sec. IV-A): each training example is a room with two
    speakers and one point-source noise, spatialised by the room's RIRs into an 8-channel mixture
    at SIR U[-6, 6] dB and SNR U[10, 20] dB, with the speakers' early-RIR (Eq. 9) images as
    dereverberation targets.  batch_1024 (1024 rooms x 3 sources x 8 mics, 16 kHz), 4 s sources.
    Timed: fram_spatialize alone, and the whole on-the-fly step (sample + synthesize with early
    RIRs + spatialize).  Algorithmic bytes: RIRs + early RIRs + signals read, mixture + targets
    written."""
    sc = scenes.batch_1024(0)
    if rooms > 0:
        sc = sc.subset(range(min(rooms, sc.B)))
    params = api.Params(fs=sc.fs, half_len=sc.half_len)
    ds = api.DeviceScene(sc, params)
    N = ds.n_vs_total
    vs = api.Images(torch.empty((N, 3), device="cuda"), torch.empty((N, 3), device="cuda"),
                    torch.empty(N, device="cuda"), torch.empty(sc.B, device="cuda"))
    rir = torch.empty(ds.rir_total, device="cuda")
    early = torch.empty(ds.rir_total, device="cuda")
    mx = scenes.mixtures(3, sc.B, sc.S, n_samples, sc.fs)
    sig = torch.from_numpy(mx.signals).cuda()
    lev = torch.from_numpy(mx.level_db).cuda()
    out = (torch.empty((sc.B, sc.M, n_samples), device="cuda"),
           torch.empty((sc.B, mx.n_speech, sc.M, n_samples), device="cuda"), torch.empty((sc.B, sc.S), device="cuda"))

    def rirs(k):
        api.sample(ds, seed=700 + k, out=vs)
        api.synthesize_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, early=True, rir=rir, early_out=early)

    def spat(k):
        api.spatialize(ds, rir, sig, lev, mx.n_speech, target_rir=early, targets=True, out=out)

    def step(k):
        rirs(k)
        spat(k)

    for k in range(3):
        step(k)
    torch.cuda.synchronize()
    t_sp = _time_steps(torch, spat, 5, False) / 5
    t_step = _time_steps(torch, step, 5, False) / 5
    assert ds.status() == 0 and api.spatialize_status(ds) == 0, "device status flags set"
    moved = 4 * (2 * ds.rir_total + sig.numel() + out[0].numel() + out[1].numel())
    peak = float(peaks.get("hbm_gbs", 6800.0))
    res = {"workload": f"batch_1024 ({sc.B} rooms x (2 speakers + 1 noise) x 8 mics, 16 kHz), {n_samples / sc.fs:.0f} s "
                       "sources, mixture + early-RIR targets",
           "spatialize": {"ms_per_batch": 1000.0 * t_sp, "value": sc.B / t_sp, "unit": "examples/s",
                          "roofline": {"bound": "hbm", "achieved": moved / t_sp / 1e9, "peak": peak, "unit": "GB/s",
                                       "frac": moved / t_sp / 1e9 / peak, "bytes_per_batch": moved,
                                       "note": "algorithmic bytes (inputs read once, outputs written once)"}},
           "on_the_fly_step": {"ms_per_batch": 1000.0 * t_step, "value": sc.B / t_step, "unit": "examples/s",
                               "note": "sample + synthesize (RIR and early RIR) + spatialize"}}
    if cpu_rooms <= 0:
        return res
    import oracle
    rl_ = list(range(cpu_rooms))
    sub = sc.subset(rl_)
    op = oracle.Params(fs=sc.fs, half_len=sc.half_len)
    ref = oracle.sample(sub, op, 1, room_ids=rl_)
    h, he = oracle.synthesize(sub, op, ref.pos, ref.g, ref.r, early=True)
    rl, ro, _ = oracle.layout(sub.rt60, sub.n_vs, sub.S, sub.M, sub.fs)
    t0 = time.perf_counter()
    oracle.spatialize(rl, ro, h, mx.signals[rl_], mx.n_speech, mx.level_db[rl_], target_rir=he, M=sc.M)
    dt = time.perf_counter() - t0
    res["spatialize"]["cpu_oracle"] = {"value": len(rl_) / dt, "unit": "examples/s", "cores": oracle.num_threads(),
                                       "sample": f"first {len(rl_)} rooms (direct FP64 convolution, {dt:.1f} s)"}
    return res


def graph_vs_per_room(torch, api, scenes):
    """batch_1024 (1024 rooms x 3 sources x 8 mics, early RIRs): one CUDA-graph replay of
    sample + synthesize with the seed read from device memory, against a loop of plain
    per-room calls on the same GPU."""
    sc = scenes.batch_1024(0)
    params = api.Params(fs=sc.fs, half_len=sc.half_len)
    ds = api.DeviceScene(sc, params)
    N = ds.n_vs_total
    vs = api.Images(torch.empty((N, 3), device="cuda"), torch.empty((N, 3), device="cuda"),
                    torch.empty(N, device="cuda"), torch.empty(sc.B, device="cuda"))
    rir = torch.empty(ds.rir_total, device="cuda")
    early = torch.empty(ds.rir_total, device="cuda")
    d_seed = torch.zeros(1, dtype=torch.int64, device="cuda")
    seeds_host = torch.arange(1, 64, dtype=torch.int64).pin_memory()

    def body():
        api.sample(ds, seed=0, d_seed=d_seed, out=vs)
        api.synthesize_raw(ds, vs.pos_hi, vs.pos_lo, vs.g, vs.r, early=True, rir=rir, early_out=early)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            body()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        body()
    reps = 10
    for k in range(3):
        d_seed.copy_(seeds_host[k:k + 1], non_blocking=True)
        g.replay()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for k in range(reps):
        d_seed.copy_(seeds_host[3 + k:4 + k], non_blocking=True)
        g.replay()
    t1.record()
    torch.cuda.synchronize()
    t_graph = t0.elapsed_time(t1) / 1000.0 / reps
    assert ds.status() == 0

    rooms = [api.DeviceScene(sc.subset([b]), params) for b in range(sc.B)]
    bufs = []
    for d in rooms:
        n = d.n_vs_total
        bufs.append((api.Images(torch.empty((n, 3), device="cuda"), torch.empty((n, 3), device="cuda"),
                                torch.empty(n, device="cuda"), torch.empty(1, device="cuda")),
                     torch.empty(d.rir_total, device="cuda"), torch.empty(d.rir_total, device="cuda")))

    def per_room():
        for d, (v, h, he) in zip(rooms, bufs):
            api.sample(d, seed=5, out=v)
            api.synthesize_raw(d, v.pos_hi, v.pos_lo, v.g, v.r, early=True, rir=h, early_out=he)

    per_room()
    torch.cuda.synchronize()
    t0.record()
    per_room()
    t1.record()
    torch.cuda.synchronize()
    t_loop = t0.elapsed_time(t1) / 1000.0
    rirs = sc.B * sc.S
    return {"workload": "batch_1024 (1024 rooms x 3 src x 8 mics, 16 kHz, K=40, + early RIR)",
            "graph_batched": {"value": rirs / t_graph, "unit": "RIRs/s", "ms_per_batch": 1000.0 * t_graph},
            "per_room_loop": {"value": rirs / t_loop, "unit": "RIRs/s", "ms_per_batch": 1000.0 * t_loop,
                              "note": "1024 x (fram_sample + fram_synthesize) launched one room at a time"},
            "speedup": t_loop / t_graph}


if __name__ == "__main__":
    sys.exit(main())
