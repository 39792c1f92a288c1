"""Benchmark of the SRP hot path on GB300.

One step = one srp_map call (PHAT cross spectra -> critical GCC samples ->
sinc-interpolation contraction with the pair sum -> argmax) over one batch
of L = 64 STFT frames of the 3D room workload: M = 8 microphones uniform in a
0.5 m cube at the centre of a 5 x 4 x 3 m room, a 100 x 80 x 60 grid of cell
centres at 0.05 m (J = 480000 candidates, Q = 28 pairs), fs = 16 kHz,
K = 1024, N_aux = 2, FP32.  Inputs are synthetic free-field white-noise
scenes (SNR 10 dB), resident in HBM before the timed region; L2 is flushed
(256 MB write) between timed steps.

Metric: SRP cells*pairs/s = J * Q * L / step time (whole job: summed over
ranks, max time over ranks).  The conventional SRP path is timed beside it
on the same inputs; e2e times srp_map_host with pinned host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SRP cells*pairs/s (Nyquist vs conventional) at stated map error; p50/p99 ms"
UNIT = "cells*pairs/s"
WORKLOAD = dict(name="room_3d", M=8, J=480000, K=1024, L=64, n_aux=2, fs=16000.0, snr_db=10.0)
FLUSH_BYTES = 256 << 20
# The sources of the single-plan tensor-core kernels, whose DRAM traffic a
# recorded ncu capture describes.
KERNEL_SOURCES = ("srp_tc.cu", "srp_tc_common.cuh", "srp_device.cuh", "srp_gcc_mma.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")


def kernel_source_hash() -> str:
    """First 16 hex digits of the SHA-256 over the kernel sources listed in
    KERNEL_SOURCES (in that order)."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2012_09499_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(key: str):
    """DRAM bytes (read + write) per launch of kernel `key` from one ncu
    capture, as recorded in the profiles' traffic table ("key hash bytes"
    per line), or None when there is no record for the current kernel
    sources (the counters describe an older build)."""
    try:
        with open(TRAFFIC_FILE) as f:
            rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    h = kernel_source_hash()
    for r in rows:
        if len(r) >= 3 and r[0] == key and r[1] == h:
            return float(r[2])
    return None


def config_dict(Q, S):
    w = WORKLOAD
    return {
        "workload": (f"room_3d: M={w['M']} mics uniform in a 0.5 m cube centred in a 5x4x3 m "
                     f"room, 100x80x60 grid at 0.05 m (J={w['J']}), Q={Q} pairs, fs=16 kHz, "
                     f"K={w['K']}, L={w['L']} frames per step, N_aux={w['n_aux']} (S={S} "
                     f"critical samples), FP32, free-field white noise at SNR 10 dB"),
        "candidates": w["J"], "pairs": Q, "frames_per_step": w["L"], "K": w["K"],
        "n_aux": w["n_aux"], "S": S, "precision": "fp32",
        "l2": "flushed between timed steps (256 MB write)",
    }


# --------------------------------------------------------------------------
# distributed plumbing (one process per GPU; independent batches per rank)
# --------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of a float over ranks (identity when world == 1)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    QUERY = ("clocks.sm,clocks.max.sm,utilization.gpu,power.draw,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.lines, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
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

    def summary(self):
        rows = []
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) != 8:
                continue
            try:
                rows.append((float(p[0]), float(p[1]), float(p[2]), p[4:]))
            except ValueError:
                continue
        if not rows:
            return None
        loaded = [r for r in rows if r[2] >= 30.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in loaded for k, v in enumerate(r[3])
                          if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in loaded])),
                "sm_max_mhz": float(max(r[1] for r in loaded)),
                "reasons": reasons, "samples": len(loaded)}


# --------------------------------------------------------------------------
# workload
# --------------------------------------------------------------------------

def make_batches(rank: int, n: int):
    from paper_2012_09499_gb300 import synth
    cfgs = [synth.room_3d(seed=1000 * rank + s) for s in range(n)]
    # one geometry (the plan) per rank; every batch shares it
    mic, grid = cfgs[0]["mic"], cfgs[0]["grid"]
    rng = np.random.default_rng(77 + rank)
    Ys = [cfgs[0]["Y"]]
    for s in range(1, n):
        src = rng.uniform([0.3, 0.3, 0.3], [4.7, 3.7, 2.7])
        Ys.append(synth.free_field_stft(rng, mic, [src], 16000.0, 1024, 64, 10.0))
    return mic, grid, Ys


def time_steps(step, steps, warmup, flush, stream, world, timed_stage=None, name="timed"):
    """Runs warmup + steps; returns per-step device ms (CUDA events on the
    launching stream, L2 flushed before each step) and, if timed_stage is
    given, per-step ms of that stage from the library's own events.  The
    timed steps run inside the NVTX range `name` (for profiler filters)."""
    import torch
    for w in range(warmup):
        step(w)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    stage_ms = []
    torch.cuda.nvtx.range_push(name)
    t_wall = time.perf_counter()
    for k in range(steps):
        flush(k)
        ev0[k].record(stream)
        step(k)
        ev1[k].record(stream)
        if timed_stage is not None:
            stage_ms.append(timed_stage())
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    torch.cuda.nvtx.range_pop()
    ms = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    return ms, np.array(stage_ms), wall


def measured_hbm_peak():
    """HBM copy bandwidth (GB/s) measured on this machine, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


def measured_bf16_peak():
    """Dense BF16 TFLOP/s measured on this machine (burst), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "of fallback"


def bench_ours(args):
    import torch

    from paper_2012_09499_gb300 import srp

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    w = WORKLOAD
    mic, grid, Ys = make_batches(rank, 4)
    L, J = w["L"], w["J"]
    d_in = [torch.from_numpy(Y).to(dev) for Y in Ys]
    maps = torch.empty((L, J), dtype=torch.float32, device=dev)
    am = torch.empty(L, dtype=torch.int32, device=dev)
    pk = torch.empty(L, dtype=torch.float32, device=dev)
    flush_buf = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def flush(k):
        flush_buf.fill_(float(k))

    plans = {}
    for mode in ("nyquist", "conventional"):
        plans[mode] = srp.Plan(mic, grid, w["fs"], 343.0, w["K"], mode=mode, n_aux=w["n_aux"],
                               max_frames=L, host_io=2 if mode == "nyquist" else 0)
    # the conventional map on the CUDA cores too (the plain GPU path)
    plans["conventional_cuda_cores"] = srp.Plan(mic, grid, w["fs"], 343.0, w["K"],
                                                mode="conventional", max_frames=L,
                                                engine="cuda_cores")
    ny = plans["nyquist"]
    Q, S = ny.info.Q, ny.info.S

    def make_step(plan):
        def step(k):
            srp.srp_map(plan.handle, d_in[k % len(d_in)], L, maps, am, pk, stream)
        return step

    def stage_runs(plan, n=5):
        """Per-stage times from the library's own events, on n separate steps
        (L2 flushed before each).  The timed steps run with these events off:
        events between the kernels would serialise their programmatic
        launches."""
        srp.srp_set_timing(plan.handle, True)
        runs = []
        for k in range(n):
            flush(k)
            make_step(plan)(k)
            runs.append(srp.srp_stage_times(plan.handle))
        srp.srp_set_timing(plan.handle, False)
        return (np.array([r["map"] for r in runs]),
                {key: float(np.mean([r[key] for r in runs])) for key in runs[0]})

    res = {}
    with ClockSampler(local) as clk:
        for mode, plan in plans.items():
            steps = args.steps if mode == "nyquist" else max(3, min(args.steps, args.conv_steps))
            if mode == "conventional_cuda_cores":
                steps = 3
            ms, _, wall = time_steps(make_step(plan), steps, args.warmup, flush, stream, world,
                                     name=f"room_3d_{mode}")
            launches = srp.srp_last_launch_count(plan.handle) * steps
            st, stages = stage_runs(plan, 5 if mode != "conventional_cuda_cores" else 2)
            res[mode] = dict(ms=ms, stage=st, wall=wall, steps=steps, launches=launches,
                             stages=stages)
    clocks = clk.summary()

    # map error of the Nyquist approximation w.r.t. conventional on one batch
    mc = torch.empty_like(maps)
    srp.srp_map(plans["conventional"].handle, d_in[0], L, mc, am, pk, stream)
    srp.srp_map(ny.handle, d_in[0], L, maps, am, pk, stream)
    torch.cuda.synchronize()
    num = ((mc.double() - maps.double()) ** 2).sum(dim=1)
    den = (mc.double() ** 2).sum(dim=1)
    e_appr = (10.0 * torch.log10(num / den)).cpu().numpy()

    # end to end through the host entry points (pinned buffers, copies timed):
    # srp_map_host_async pipelines the copies of each step with the maps of its
    # neighbours; srp_map_host runs one step at a time
    h_in = [torch.from_numpy(Y).pin_memory() for Y in Ys]
    h_maps = [torch.empty((L, J), dtype=torch.float32).pin_memory() for _ in range(2)]
    h_am = [torch.empty(L, dtype=torch.int32).pin_memory() for _ in range(2)]
    h_pk = [torch.empty(L, dtype=torch.float32).pin_memory() for _ in range(2)]
    srp.srp_set_timing(ny.handle, False)
    e2e_steps = max(3, min(args.steps, 20))

    def host_async(k):
        srp.srp_map_host_async(ny.handle, h_in[k % 4], L, h_maps[k % 2], h_am[k % 2],
                               h_pk[k % 2], stream)

    for k in range(args.warmup):
        host_async(k)
    srp.srp_map_host_wait(ny.handle)
    barrier(world)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        host_async(k)
    srp.srp_map_host_wait(ny.handle)
    e2e_s = reduce_max((time.perf_counter() - t0) / e2e_steps, world, dev if world > 1 else None)
    for k in range(args.warmup):
        srp.srp_map_host(ny.handle, h_in[k % 4], L, h_maps[0], h_am[0], h_pk[0], stream)
    barrier(world)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        srp.srp_map_host(ny.handle, h_in[k % 4], L, h_maps[0], h_am[0], h_pk[0], stream)
    e2e_sync_s = reduce_max((time.perf_counter() - t0) / e2e_steps, world,
                            dev if world > 1 else None)
    # the same pipeline returning only each frame's maximiser and peak
    # (localisation), without the maps
    for k in range(args.warmup):
        srp.srp_map_host_async(ny.handle, h_in[k % 4], L, None, h_am[k % 2], h_pk[k % 2], stream)
    srp.srp_map_host_wait(ny.handle)
    barrier(world)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        srp.srp_map_host_async(ny.handle, h_in[k % 4], L, None, h_am[k % 2], h_pk[k % 2], stream)
    srp.srp_map_host_wait(ny.handle)
    e2e_loc_s = reduce_max((time.perf_counter() - t0) / e2e_steps, world,
                           dev if world > 1 else None)

    cells = J * Q * L
    ny_ms = reduce_max(res["nyquist"]["ms"].mean(), world, dev if world > 1 else None)
    cv_ms = reduce_max(res["conventional"]["ms"].mean(), world, dev if world > 1 else None)
    cc_ms = reduce_max(res["conventional_cuda_cores"]["ms"].mean(), world,
                       dev if world > 1 else None)
    k3_ms = float(np.mean(res["nyquist"]["stage"]))
    flops = 2.0 * J * S * L  # multiply-adds of the interpolation contraction, C_int x L
    achieved = flops / (k3_ms * 1e-3) / 1e12
    bf16_peak, peak_src = measured_bf16_peak()
    hbm_peak, hbm_src = measured_hbm_peak()
    # the GCC-sample stage (with the PHAT cross spectra): STFT frames in,
    # 16-bit operand B out (hi and lo parts for the FP32 split), and on the
    # tensor cores the plan's twiddle operand (fp16 hi and lo, N lag rows x K)
    k2_ms = float(res["nyquist"]["stages"]["gcc_samples"])
    k2_tc = bool(ny.info.gcc_tensor_cores)
    n_lag = -(-(2 * (ny.info.max_nq + w["n_aux"]) + 1) // 32) * 32
    k2_tw = 2.0 * 2.0 * n_lag * w["K"] if k2_tc else 0.0
    k2_bytes = 8.0 * L * w["M"] * (w["K"] // 2 + 1) + 2.0 * 2.0 * L * S + k2_tw

    # reduced-precision variants of the same step (Nyquist, tensor cores)
    variants = {}
    for prec, resident in (("bf16", False), ("fp16", False), ("bf16", True)):
        pl = srp.Plan(mic, grid, w["fs"], 343.0, w["K"], mode="nyquist", n_aux=w["n_aux"],
                      max_frames=L, precision=prec, resident_weights=resident)
        name = prec + ("_resident_weights" if resident else "")
        ms_v, _, _ = time_steps(make_step(pl), max(3, min(args.steps, 20)), args.warmup,
                                flush, stream, world, name=f"room_3d_{name}")
        st_v, _ = stage_runs(pl)
        variants[name] = {"ms_per_step": float(ms_v.mean()),
                          "value": world * J * Q * L / (float(ms_v.mean()) * 1e-3),
                          "map_ms": float(st_v.mean()),
                          "map_frac_of_bf16_peak": flops / (float(st_v.mean()) * 1e-3) / 1e12
                          / bf16_peak}
        if resident:  # the map streams the interpolation matrix: report it against HBM
            wb = float(pl.info.weight_bytes) + 4.0 * J * L
            variants[name]["weight_bytes"] = int(pl.info.weight_bytes)
            variants[name]["map_hbm_gbs"] = wb / (float(st_v.mean()) * 1e-3) / 1e9
        pl.close()

    conv_tc = bool(plans["conventional"].info.tensor_cores)
    conv_stages = res["conventional"]["stages"]
    for pl in plans.values():
        pl.close()
    extra = {}
    # serving first: its open-loop load generator is a host thread, whose
    # timing suffers after the batched section's large allocations are freed
    if world == 1 and not args.no_serve:
        extra["serving"] = bench_serving(args)
    if world == 1 and not args.no_batch:
        extra["batched"] = bench_batched(args, flush, stream)
    if world == 1 and not args.no_paper:
        extra["paper_setup"] = bench_paper_setup(args, flush, stream)
        extra["complexity"] = bench_complexity(args, flush, stream)
        extra["refine"] = bench_refine(args, flush, stream)
    if rank != 0:
        return
    cpu = None if args.no_cpu else cpu_baseline(mic, grid, Ys[0], w, Q, S)
    line = {
        "metric": METRIC, "value": world * cells / (ny_ms * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ny_ms,
        "p50_ms": float(np.percentile(res["nyquist"]["ms"], 50)),
        "p99_ms": float(np.percentile(res["nyquist"]["ms"], 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic free-field white-noise scenes (seeded), random array geometry",
        "config": config_dict(Q, S),
        "conventional": {
            "value": world * cells / (cv_ms * 1e-3), "ms_per_step": cv_ms,
            "steps": res["conventional"]["steps"],
            "p50_ms": float(np.percentile(res["conventional"]["ms"], 50)),
            "p99_ms": float(np.percentile(res["conventional"]["ms"], 99)),
            "map_ms": float(np.mean(res["conventional"]["stage"])),
            "engine": "tensor cores" if conv_tc else "CUDA cores",
            "cuda_cores": {"value": world * cells / (cc_ms * 1e-3), "ms_per_step": cc_ms,
                           "steps": 3,
                           "map_ms": float(np.mean(res["conventional_cuda_cores"]["stage"]))},
        },
        "speedup_nyquist_over_conventional": cv_ms / ny_ms,
        "speedup_nyquist_over_conventional_cuda_cores": cc_ms / ny_ms,
        "e_appr_db": {"median": float(np.median(e_appr)), "max": float(np.max(e_appr))},
        "map_error_bound": "FP32 path: max |map - FP64 oracle| <= 1e-4 x peak (tests)",
        "stage_ms": res["nyquist"]["stages"],
        "stage_ms_conventional": conv_stages,
        "roofline": {
            "kernel": "k_interp_tc<split> (on-chip sinc weights + tcgen05 MMA, FP32 as 3 BF16 products)",
            "bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": achieved / bf16_peak,
            "traffic": recorded_traffic("k_interp_tc_fp32_room_3d"),
            "traffic_note": ("ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch of "
                             "the current kernel sources (null if none was captured)"),
            "algorithmic": f"2*J*S*L = {flops:.4g} flop per launch (S={S} lags); "
                           f"{k3_ms:.4f} ms per launch",
            "peak_source": f"measured bf16 burst {bf16_peak:.1f} TFLOP/s ({peak_src})",
            "tensor_products_per_mac": 3,
            "tensor_pipe_frac": 3.0 * achieved / bf16_peak,
            "tensor_pipe_note": ("FP32 accuracy takes three BF16 products per multiply-add; "
                                 "tensor_pipe_frac counts them, frac counts the method's flops"),
        },
        "roofline_gcc_samples": {
            "kernel": ("k_gcc_samples_mma<split> (PHAT cross spectra + partial IDFT as an "
                       "FP16-split tcgen05 contraction)" if k2_tc else
                       "k_gcc_samples_tc<split, from STFT> (PHAT cross spectra + critical GCC "
                       "samples)"),
            "bound": "hbm", "achieved": k2_bytes / (k2_ms * 1e-3) / 1e9, "peak": hbm_peak,
            "unit": "GB/s", "frac": k2_bytes / (k2_ms * 1e-3) / 1e9 / hbm_peak,
            "traffic": recorded_traffic("k_gcc_samples_mma_fp32_room_3d" if k2_tc
                                        else "k_gcc_samples_tc_fp32_room_3d"),
            "algorithmic": (f"8*L*M*Kb STFT in + 2*2*L*S operand B out"
                            + (f" + 2*2*{n_lag}*K twiddle operand" if k2_tc else "")
                            + f" = {k2_bytes:.4g} B per launch; {k2_ms:.4f} ms per launch "
                            "(stage time by CUDA events, launch latency included)"),
            "peak_source": f"measured HBM copy {hbm_peak:.0f} GB/s ({hbm_src})",
        },
        "precision_variants": variants,
        "e2e": {"value": world * cells / e2e_s, "unit": UNIT, "ms_per_step": e2e_s * 1e3,
                "h2d_bytes_per_step": int(L * w["M"] * (w["K"] // 2 + 1) * 8),
                "d2h_bytes_per_step": int(L * J * 4 + L * 8),
                "api": "srp_map_host_async + srp_map_host_wait (pinned host buffers; every "
                       "step's input copied in and its maps, argmax and peak copied back, "
                       "overlapped with the neighbouring steps' maps)",
                "synchronous": {"value": world * cells / e2e_sync_s, "ms_per_step": e2e_sync_s * 1e3,
                                "api": "srp_map_host, one step at a time"},
                "localisation_only": {
                    "value": world * cells / e2e_loc_s, "ms_per_step": e2e_loc_s * 1e3,
                    "d2h_bytes_per_step": int(L * 8),
                    "api": "srp_map_host_async with h_maps = NULL: every step's input copied "
                           "in, its argmax and peak copied back, the maps left on the device"}},
        "gpu_launches": int(res["nyquist"]["launches"]),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    line.update(extra)
    if "serving" in extra:  # a compact copy of the serving loop's headline figures
        line["serving_summary"] = {
            k: {"maps_per_s": v["maps_per_s"], "offered_frames_per_s": v["offered_frames_per_s"],
                "p50_ms": v["p50_ms"], "p99_ms": v["p99_ms"],
                "tensor_core_streams": v["tensor_core_streams"],
                "overlapped_iterations_frac": v["overlapped_iterations_frac"]}
            for k, v in extra["serving"].items() if isinstance(v, dict) and "p99_ms" in v}
    if "batched" in extra:  # and of the batched uneven mix
        line["batched_summary"] = {
            k: {"value": v["value"], "unit": v["unit"], "ms_per_step": v["ms_per_step"],
                "stage_ms": v["stage_ms"], "roofline_frac": v["roofline"]["frac"],
                "roofline_unit": v["roofline"]["unit"]}
            for k, v in extra["batched"].items() if isinstance(v, dict) and "roofline" in v}
    print(json.dumps(line))


# --------------------------------------------------------------------------
# batched uneven instances and serving
# --------------------------------------------------------------------------

BATCH_N, BATCH_L = 256, 32
SERVE_STREAMS, SERVE_BLOCK, SERVE_RATE = 64, 8, 20000.0


def mix_inputs(n, seed):
    """n arrays of the uneven mix: M in 4..16, aperture 0.1-1 m, K in
    {512, 1024, 2048}, 2D/3D grids with J log-uniform in [10k, 500k], L = 32."""
    from paper_2012_09499_gb300 import synth
    return [synth.uneven_instance(seed + i, L=BATCH_L) for i in range(n)]


def bench_batched(args, flush, stream):
    """The uneven mix in one graph launch per step (srp_map_batch), FP32 and
    BF16, tiles chosen by the autotuner; L2 flushed between timed steps."""
    import torch

    from paper_2012_09499_gb300 import srp
    n_arrays = args.batch_arrays
    cfgs = mix_inputs(n_arrays, 1_000_000)
    d_in = [torch.from_numpy(c["Y"]).cuda() for c in cfgs]
    Js = np.array([c["grid"].shape[0] for c in cfgs], np.float64)
    Ms = np.array([c["mic"].shape[0] for c in cfgs])
    Qs = Ms * (Ms - 1) // 2
    cells = float((Js * Qs).sum() * BATCH_L)
    bf16_peak, peak_src = measured_bf16_peak()
    out = {"workload": (f"{n_arrays} arrays: M uniform in 4..16 mics in a cube of edge uniform in "
                        f"0.1-1.0 m at the centre of a 6x7x3.5 m room, K in {{512,1024,2048}} at "
                        f"16 kHz, 2D/3D cell-centre grids with J log-uniform in [10k, 500k] "
                        f"(sum J = {int(Js.sum())}), L = {BATCH_L} frames each, N_aux = 2, "
                        f"white sources at SNR 0-30 dB; one graph launch per step"),
           "arrays": n_arrays, "frames_per_array": BATCH_L, "sum_J": int(Js.sum()),
           "mean_pairs": float(Qs.mean()), "l2": "flushed between timed steps (256 MB write)"}
    L = [BATCH_L] * n_arrays
    # FP32 and BF16 generating the sinc weights on chip; BF16 again with every
    # array's interpolation matrix resident in HBM and streamed
    for name, prec, resident in (("fp32", "fp32", False), ("bf16", "bf16", False),
                                 ("bf16_resident_weights", "bf16", True)):
        plans = [srp.Plan(c["mic"], c["grid"], c["fs"], c["c"], c["K"], mode="nyquist", n_aux=2,
                          precision=prec, max_frames=BATCH_L, resident_weights=resident)
                 for c in cfgs]
        S = np.array([p.info.S for p in plans], np.float64)
        flops = float((2.0 * Js * S * BATCH_L).sum())
        Kbs = np.array([c["K"] // 2 + 1 for c in cfgs], np.float64)
        op_bytes = float((8.0 * BATCH_L * Ms * Kbs).sum() +
                         (2.0 * (2.0 if prec == "fp32" else 1.0) * BATCH_L * S).sum())
        batch = srp.Batch(plans)
        outs = batch.outputs(L, "cuda")
        maps, ams, pks = [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs]
        srp.srp_batch_tune(batch.handle, d_in, L, maps, ams, pks)

        def step(k):
            srp.srp_map_batch(batch.handle, d_in, L, maps, ams, pks, stream)

        steps = max(3, min(args.steps, args.batch_steps))
        ms, _, _ = time_steps(step, steps, args.warmup, flush, stream, 1, name=f"batched_{name}")
        srp.srp_batch_set_timing(batch.handle, True)
        st = []
        for k in range(3):
            flush(k)
            step(k)
            st.append(srp.srp_batch_stage_times(batch.handle))
        srp.srp_batch_set_timing(batch.handle, False)
        torch.cuda.synchronize()
        srp.srp_batch_poll_device_status(batch.handle)
        stage = {key: float(np.mean([x[key] for x in st])) for key in st[0]}
        info = batch.info
        peak = bf16_peak
        achieved = flops / (stage["map"] * 1e-3) / 1e12
        wbytes = float(sum(p.info.weight_bytes for p in plans))
        out[name] = {
            "value": cells / (float(ms.mean()) * 1e-3), "unit": UNIT,
            "ms_per_step": float(ms.mean()), "steps": steps,
            "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "stage_ms": stage, "gpu_launches_per_step": int(info.launches),
            "tiles": {"frames_per_item": info.tiles.frames_per_tile,
                      "stages": info.tiles.stages, "ctas_per_sm": info.tiles.ctas_per_sm,
                      "operand_a": "tmem" if info.tiles.operand_a == 1 else "smem",
                      "accumulators": info.tiles.accumulators,
                      "tuned_ms": float(info.tuned_ms)},
            "work_items": int(info.items), "persistent_ctas": int(info.ctas),
            "resident_weight_bytes": int(sum(p.info.weight_bytes for p in plans)),
            "roofline": ({"kernel": "k_map_batch_tc (persistent, streamed resident weights)",
                          "bound": "hbm",
                          "achieved": (wbytes + 4.0 * Js.sum() * BATCH_L) / (stage["map"] * 1e-3) / 1e9,
                          "peak": measured_hbm_peak()[0], "unit": "GB/s",
                          "frac": (wbytes + 4.0 * Js.sum() * BATCH_L) / (stage["map"] * 1e-3) / 1e9
                                  / measured_hbm_peak()[0],
                          "algorithmic": f"resident weights {wbytes:.4g} B + maps "
                                         f"{4.0 * Js.sum() * BATCH_L:.4g} B per launch",
                          "peak_source": f"measured HBM copy ({measured_hbm_peak()[1]})"}
                         if resident else
                         {"kernel": "k_map_batch_tc (persistent, on-chip sinc weights)",
                          "bound": "tensor", "achieved": achieved, "peak": peak,
                          "unit": "TFLOP/s", "frac": achieved / peak,
                          "tensor_products_per_mac": 3 if prec == "fp32" else 1,
                          "algorithmic": f"sum 2*J*S*L = {flops:.4g} flop per launch",
                          "peak_source": f"measured bf16 burst {bf16_peak:.1f} TFLOP/s "
                                         f"({peak_src})"}),
            "roofline_operands": {
                "kernel": "k_batch_operands (PHAT cross spectra + critical GCC samples)",
                "bound": "hbm", "unit": "GB/s", "peak": measured_hbm_peak()[0],
                "achieved": op_bytes / (stage["operands"] * 1e-3) / 1e9,
                "frac": op_bytes / (stage["operands"] * 1e-3) / 1e9 / measured_hbm_peak()[0],
                "algorithmic": f"STFT in + operand B out = {op_bytes:.4g} B per launch"},
        }
        batch.close()
        for p in plans:
            p.close()
        del outs, maps
        torch.cuda.empty_cache()
    return out


PAPER_SOURCES, PAPER_L = 16, 32


def bench_paper_setup(args, flush, stream):
    """The paper's evaluation geometry (Sec. 4) on synthetic signals: M = 6 on a
    10 cm circle, far-field half sphere at 2 degrees (J = 8101), K = 2048,
    16 white plane-wave sources at SNR -3..6 dB, 32 frames each.  Per N_aux:
    e_appr of the Nyquist map against the conventional map, the angle of each
    map's maximiser to the true direction, and the map time."""
    import torch

    from paper_2012_09499_gb300 import srp, synth
    cfgs = [synth.paper_circle_setup(3_000_000 + i, L=PAPER_L) for i in range(PAPER_SOURCES)]
    c0 = cfgs[0]
    grid = torch.from_numpy(c0["grid"]).cuda()
    truth = torch.from_numpy(np.concatenate([np.repeat(c["sources"], PAPER_L, axis=0)
                                             for c in cfgs])).cuda()
    d_in = [torch.from_numpy(c["Y"]).cuda() for c in cfgs]

    def run(mode, n_aux):
        plan = srp.Plan(c0["mic"], c0["grid"], c0["fs"], c0["c"], c0["K"], mode=mode,
                        n_aux=n_aux, far_field=True, max_frames=PAPER_L)
        maps, idx = [], []
        for x in d_in:
            m, a, _ = plan.map(x)
            maps.append(m)
            idx.append(a.long())
        t_maps = torch.empty_like(maps[0])
        t_am = torch.empty(PAPER_L, dtype=torch.int32, device="cuda")

        def step(k):
            srp.srp_map(plan.handle, d_in[k % len(d_in)], PAPER_L, t_maps, t_am, None, stream)
        ms, _, _ = time_steps(step, 10, args.warmup, flush, stream, 1, name=f"paper_{mode}_{n_aux}")
        srp.srp_poll_device_status(plan.handle)
        plan.close()
        return torch.cat(maps), torch.cat(idx), float(ms.mean())

    def angle_deg(idx):
        cosang = (grid[idx] * truth).sum(dim=1).clamp(-1.0, 1.0)
        return torch.rad2deg(torch.arccos(cosang)).cpu().numpy()

    conv, ci, conv_ms = run("conventional", 0)
    keep = slice(0, None)
    out = {"workload": (f"M = 6 on a 0.1 m circle, far-field half sphere at 2 deg (J = 8101), "
                        f"fs = 16 kHz, K = 2048, {PAPER_SOURCES} white plane-wave sources at SNR "
                        f"uniform in [-3, 6] dB, {PAPER_L} frames each"),
           "context": "paper (reverberant speech, babble): median e_appr -31.5 dB at N_aux = 0, "
                      "-34 dB at N_aux = 2; localisation gap 0.8-1.8 deg at N_aux = 0, 0 at 2",
           "conventional": {"e_local_deg_median": float(np.median(angle_deg(ci)[keep])),
                            "ms_per_32_frames": conv_ms,
                            "value": 8101 * 15 * PAPER_L / (conv_ms * 1e-3), "unit": UNIT}}
    for n_aux in range(5):
        ny, ni, ms = run("nyquist", n_aux)
        num = ((conv[keep].double() - ny[keep].double()) ** 2).sum(dim=1)
        den = (conv[keep].double() ** 2).sum(dim=1)
        e = (10.0 * torch.log10(num / den)).cpu().numpy()
        ang = angle_deg(ni)[keep]
        cosg = (grid[ni[keep]] * grid[ci[keep]]).sum(dim=1).clamp(-1.0, 1.0)
        gap = torch.rad2deg(torch.arccos(cosg)).cpu().numpy()
        out[f"nyquist_n_aux_{n_aux}"] = {
            "e_appr_db": {"median": float(np.median(e)), "q25": float(np.percentile(e, 25)),
                          "q75": float(np.percentile(e, 75))},
            "e_local_deg_median": float(np.median(ang)),
            "maximiser_gap_to_conventional_deg": {"mean": float(gap.mean()),
                                                  "frac_zero": float(np.mean(gap < 1e-3))},
            "ms_per_32_frames": ms, "value": 8101 * 15 * PAPER_L / (ms * 1e-3), "unit": UNIT}
    return out


REFINE_LEVELS, REFINE_SHRINK, REFINE_STEP = 4, 0.5, 0.1


def bench_refine(args, flush, stream):
    """Coarse-to-fine search (the refinement Sec. 3.3 leaves outside the
    paper's scope) against the full fine grid, on the same room_3d scene
    (seed 0, 64 frames, one source): (a) the Nyquist FP32 map on the
    100 x 80 x 60 grid at 0.05 m (J = 480000) and its argmax; (b) the map on
    a 25 x 20 x 15 grid at 0.2 m (J = 7500), then srp_refine around each
    frame's coarse maximiser with a 5 x 5 x 5 stencil of step 0.1 m over 4
    levels halving the step (last step 0.0125 m).  Per path: ms per step (L2
    flushed), points evaluated per frame and the median distance of the
    found point to the source."""
    import torch

    from paper_2012_09499_gb300 import srp, synth
    fine = synth.room_3d(seed=0)
    coarse = synth.room_3d(seed=0, shape=(25, 20, 15), spacing=0.2)
    assert np.array_equal(fine["Y"], coarse["Y"])
    Y = torch.from_numpy(fine["Y"]).cuda()
    L = fine["L"]
    src = fine["sources"][0]
    g = (np.arange(5) - 2.0) * REFINE_STEP
    offs = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    out = {"workload": ("room_3d seed 0 (M = 8, one source at SNR 10 dB, K = 1024, L = 64), "
                        "Nyquist FP32, N_aux = 2")}
    plans = {}
    for name, cfg in (("fine", fine), ("coarse", coarse)):
        plans[name] = srp.Plan(cfg["mic"], cfg["grid"], cfg["fs"], cfg["c"], cfg["K"],
                               mode="nyquist", n_aux=2, max_frames=L)
    am = torch.empty(L, dtype=torch.int32, device="cuda")
    pk = torch.empty(L, dtype=torch.float32, device="cuda")

    def fine_step(k):
        srp.srp_map(plans["fine"].handle, Y, L, None, am, pk, stream)
    ms_f, _, _ = time_steps(fine_step, 10, args.warmup, flush, stream, 1, name="refine_fine")
    err_f = np.linalg.norm(fine["grid"][am.cpu().numpy()] - src, axis=1)
    ref = srp.Refiner(plans["coarse"], offs, levels=REFINE_LEVELS, shrink=REFINE_SHRINK)
    xyz = torch.empty((L, 3), dtype=torch.float64, device="cuda")
    val = torch.empty(L, dtype=torch.float32, device="cuda")

    def coarse_step(k):
        srp.srp_map(plans["coarse"].handle, Y, L, None, am, pk, stream)
        srp.lib().srp_refine(ref.handle, L, am.data_ptr(), None, xyz.data_ptr(), val.data_ptr(),
                             None, srp._stream(stream))
    ms_c, _, _ = time_steps(coarse_step, 10, args.warmup, flush, stream, 1, name="refine_coarse")
    srp.srp_poll_device_status(plans["coarse"].handle)
    err_c = np.linalg.norm(xyz.cpu().numpy() - src, axis=1)
    err_0 = np.linalg.norm(coarse["grid"][am.cpu().numpy()] - src, axis=1)
    ref.close()
    for p in plans.values():
        p.close()
    out["fine_grid"] = {"ms_per_step": float(ms_f.mean()), "points_per_frame": 480000,
                        "error_m_median": float(np.median(err_f)),
                        "error_m_max": float(np.max(err_f))}
    out["coarse_plus_refine"] = {
        "ms_per_step": float(ms_c.mean()),
        "points_per_frame": 7500 + REFINE_LEVELS * offs.shape[0],
        "levels": REFINE_LEVELS, "stencil": "5 x 5 x 5", "first_step_m": REFINE_STEP,
        "last_step_m": REFINE_STEP * REFINE_SHRINK ** (REFINE_LEVELS - 1),
        "coarse_only_error_m_median": float(np.median(err_0)),
        "error_m_median": float(np.median(err_c)), "error_m_max": float(np.max(err_c))}
    out["speedup"] = float(ms_f.mean() / ms_c.mean())
    return out


COMPLEXITY_RADII = (0.025, 0.05, 0.1, 0.2, 0.3, 0.5)
COMPLEXITY_L = 64


def bench_complexity(args, flush, stream):
    """The complexity reduction factors of Sec. 3.3 against the array radius
    (the setting of Fig. 2: M = 6 on a circle, c = 340 m/s, fs = 16 kHz), from
    srp_plan_complexity, beside the measured GPU time ratios on the far-field
    half sphere at 2 degrees (J = 8101, K = 2048, K_b = 1024, N_aux = 2, FP32,
    64 frames): t_samp = the GCC-sample stage, t_int = the Nyquist map stage,
    t_conv = the conventional map stage (tensor cores).  Fig. 2's own J values
    are not in the paper's source, so R_samp is also given for J = 1e3, 1e4
    and 1e5 from the same N."""
    import torch

    from paper_2012_09499_gb300 import srp, synth
    grid = synth.half_sphere_directions(2.0)
    rng = np.random.default_rng(5)
    Kb = 1025
    Y = torch.from_numpy((rng.standard_normal((COMPLEXITY_L, 6, Kb)) +
                          1j * rng.standard_normal((COMPLEXITY_L, 6, Kb))).astype(np.complex64)).cuda()
    rows = []
    for r in COMPLEXITY_RADII:
        mic = synth.circular_array(6, r)
        row = {"radius_m": r}
        for naux in (0, 1, 2):
            d, keep = srp.make_desc(mic, grid, 16000.0, 340.0, 2048, mode="nyquist", n_aux=naux,
                                    far_field=True)
            cx = srp.srp_plan_complexity(d)
            row[f"N_aux_{naux}"] = {"N": cx["N"], "R_samp_J8101": cx["R_samp"],
                                    "R_samp_by_J": {str(J): cx["N"] / J for J in (1000, 10000, 100000)}}
            if naux == 2:
                row.update({"R_samp": cx["R_samp"], "R_int": cx["R_int"], "R": cx["R"],
                            "C_samp": cx["C_samp"], "C_int": cx["C_int"], "C_conv": cx["C_conv"]})
        t = {}
        for mode in ("nyquist", "conventional"):
            plan = srp.Plan(mic, grid, 16000.0, 340.0, 2048, mode=mode, n_aux=2, far_field=True,
                            max_frames=COMPLEXITY_L)
            srp.srp_set_timing(plan.handle)
            maps = torch.empty((COMPLEXITY_L, grid.shape[0]), dtype=torch.float32, device="cuda")
            am = torch.empty(COMPLEXITY_L, dtype=torch.int32, device="cuda")

            def step(k, plan=plan, maps=maps, am=am):
                srp.srp_map(plan.handle, Y, COMPLEXITY_L, maps, am, None, stream)
            _, st, _ = time_steps(step, 10, args.warmup, flush, stream, 1,
                                  timed_stage=lambda plan=plan: srp.srp_stage_times(plan.handle),
                                  name=f"complexity_{mode}_{r}")
            srp.srp_poll_device_status(plan.handle)
            t[mode] = {k: float(np.mean([x[k] for x in st])) for k in st[0]}
            if mode == "conventional":
                t["conv_engine"] = "tensor cores" if plan.info.tensor_cores else "cuda cores"
            plan.close()
        ts, ti, tc = t["nyquist"]["gcc_samples"], t["nyquist"]["map"], t["conventional"]["map"]
        row["measured_ms"] = {"t_samp": ts, "t_int": ti, "t_conv": tc, "conv_engine": t["conv_engine"]}
        row["measured_ratio"] = {"samp": ts / tc, "int": ti / tc, "total": (ts + ti) / tc}
        rows.append(row)
    return {"workload": ("M = 6 circle of the given radius, c = 340 m/s, fs = 16 kHz, far-field half "
                         "sphere at 2 deg (J = 8101), K = 2048 (K_b = 1024), N_aux = 2 for R and the "
                         f"timings, FP32, {COMPLEXITY_L} frames, L2 flushed between steps"),
            "radii": rows}


def serve_run(srp, plans, cfgs, rate, duration, seed):
    """Open-loop Poisson arrivals of SERVE_BLOCK-frame blocks from uniformly
    chosen streams at `rate` frames/s for `duration` s; returns latencies
    (ms, from each block's scheduled arrival) and throughput figures."""
    import threading
    srv = srp.Server(plans, device_budget_bytes=8 << 30, host_budget_bytes=2 << 30,
                     max_inflight=2)
    # warm-up outside the measured window: one block per stream, drained, so
    # that first launches (module loading, first graph launches) are not
    # charged to the requests of the timed schedule
    for s_ in range(len(plans)):
        srv.submit(s_, cfgs[s_]["Y"][:SERVE_BLOCK], tag=0)
    srv.drain(timeout_s=120.0)
    st0 = srv.stats
    rng = np.random.default_rng(seed)
    n_req = int(rate / SERVE_BLOCK * duration)
    gaps = rng.exponential(SERVE_BLOCK / rate, n_req)
    sched = np.cumsum(gaps)
    who = rng.integers(0, len(plans), n_req)
    blocks = rng.integers(0, BATCH_L // SERVE_BLOCK, n_req)
    lag = {}
    t0 = time.perf_counter()

    def submitter():
        for k in range(n_req):
            while True:
                now = time.perf_counter() - t0
                if now >= sched[k]:
                    break
                time.sleep(min(0.0005, sched[k] - now))
            s, b = int(who[k]), int(blocks[k])
            rid = srv.submit(s, cfgs[s]["Y"][b * SERVE_BLOCK:(b + 1) * SERVE_BLOCK], tag=k)
            lag[rid] = time.perf_counter() - t0 - sched[k]

    # the load generator must not be held up by the collector: no garbage
    # collection pauses and short GIL hand-overs while requests arrive
    switch = sys.getswitchinterval()
    gc_on = gc.isenabled()
    gc.disable()
    sys.setswitchinterval(1e-4)
    try:
        th = threading.Thread(target=submitter)
        th.start()
        done = []
        while th.is_alive():
            done += srv.poll(wait_ms=20)
        th.join()
        done += srv.drain(timeout_s=120.0)
    finally:
        sys.setswitchinterval(switch)
        if gc_on:
            gc.enable()
    t_end = time.perf_counter() - t0
    st = srv.stats
    srv.close()
    ok = [d for d in done if d["status"] == 0]
    lat = np.array([d["t_done"] - d["t_submit"] + 1e3 * max(0.0, lag[d["id"]]) for d in ok])
    wait = np.array([d["t_start"] - d["t_submit"] for d in ok])  # queued on the host
    run = np.array([d["t_done"] - d["t_start"] for d in ok])     # its iteration, copies included
    frames = sum(d["L"] for d in ok)
    cp = sum(d["L"] * plans[d["stream"]].info.J * plans[d["stream"]].info.Q for d in ok)
    per_iter = {d["iteration"]: d["iteration_streams"] for d in ok}
    n_iter = int(st.iterations - st0.iterations)
    return {"requests": len(done), "completed": len(ok), "frames": frames,
            "maps_per_s": frames / t_end, "cells_pairs_per_s": cp / t_end,
            "offered_frames_per_s": rate, "wall_s": t_end,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "iterations": int(st.iterations - st0.iterations),
            "queued_p50_ms": float(np.percentile(wait, 50)),
            "queued_p99_ms": float(np.percentile(wait, 99)),
            "iteration_p50_ms": float(np.percentile(run, 50)),
            "iteration_p99_ms": float(np.percentile(run, 99)),
            "mean_frames_per_iteration": frames / max(1, n_iter),
            "mean_streams_per_iteration": float(np.mean(list(per_iter.values()))),
            "max_streams_per_iteration": int(max(per_iter.values())),
            "overlapped_iterations_frac": (int(st.overlapped_iterations - st0.overlapped_iterations)
                                           / max(1, n_iter)),
            "kernel_launches": int(st.kernel_launches - st0.kernel_launches),
            "warm_up": f"one {SERVE_BLOCK}-frame block per stream, drained before the schedule",
            "device_bytes_peak": int(st.device_bytes_peak),
            "admission_waits": int(st.admission_waits),
            "submit_lag_p99_ms": float(np.percentile([1e3 * v for v in lag.values()], 99))}


def bench_serving(args):
    """64 streams of the uneven mix, 8-frame blocks arriving as a Poisson
    process at 20k frames/s in total: BF16 Nyquist, and the FP32
    conventional map beside it at the same offered load for a shorter time."""
    from paper_2012_09499_gb300 import srp
    cfgs = mix_inputs(SERVE_STREAMS, 2_000_000)
    out = {"streams": SERVE_STREAMS, "block_frames": SERVE_BLOCK,
           "offered_frames_per_s": SERVE_RATE,
           "arrivals": "Poisson (open loop), stream uniform, latency from scheduled arrival",
           "device_budget_bytes": 8 << 30, "max_inflight": 2}
    for name, mode, prec, dur in (("nyquist_bf16", "nyquist", "bf16", args.serve_seconds),
                                  ("conventional_fp32", "conventional", "fp32",
                                   min(args.serve_seconds, 1.0))):
        # Nyquist streams keep their interpolation matrices resident (built once)
        plans = [srp.Plan(c["mic"], c["grid"], c["fs"], c["c"], c["K"], mode=mode, n_aux=2,
                          precision=prec, max_frames=BATCH_L,
                          resident_weights=(mode == "nyquist")) for c in cfgs]
        res = serve_run(srp, plans, cfgs, SERVE_RATE, dur, 5)
        res["resident_weight_bytes"] = int(sum(p.info.weight_bytes for p in plans))
        res["duration_s"] = dur
        res["tensor_core_streams"] = int(sum(p.info.tensor_cores for p in plans))
        out[name] = res
        for p in plans:
            p.close()
    return out


# --------------------------------------------------------------------------
# FP64 oracle on the host cores (CPU baseline and reference arm)
# --------------------------------------------------------------------------

def oracle_step_seconds(mic, grid, Y, w, stride, frames=1):
    """Times the oracle's Nyquist path on `frames` frames and every
    `stride`-th candidate; returns (seconds extrapolated to one full step of
    L frames and J candidates, sample description, threads)."""
    from oracle import oracle
    sub = grid[::stride]
    t0 = time.perf_counter()
    x = oracle.tdoa(mic, sub, w["fs"], 343.0)
    t_tdoa = time.perf_counter() - t0  # plan-time work, not counted per step
    Nq, _ = oracle.lag_counts(mic, w["fs"], 343.0)
    t0 = time.perf_counter()
    psi = oracle.phat(Y[:frames])
    xi = oracle.gcc_samples(psi, Nq, w["n_aux"], w["K"])
    t_frame = (time.perf_counter() - t0) / frames
    t0 = time.perf_counter()
    oracle.nyquist(xi, Nq, w["n_aux"], x)
    t_interp = (time.perf_counter() - t0) / frames
    per_frame = t_frame + t_interp * (grid.shape[0] / sub.shape[0])
    desc = (f"Nyquist path on {frames} frame(s) x {sub.shape[0]} candidates (every "
            f"{stride}th), extrapolated to J={grid.shape[0]} by the exact J*S interpolation "
            f"count and to L={w['L']} frames; TDOA table ({t_tdoa:.2f} s) is plan-time")
    return per_frame * w["L"], desc, oracle.get_threads()


def cpu_baseline(mic, grid, Y, w, Q, S):
    secs, desc, threads = oracle_step_seconds(mic, grid, Y, w, stride=8, frames=2)
    return {"value": w["J"] * Q * w["L"] / secs, "unit": UNIT, "cores": threads,
            "kind": "oracle", "sample": desc}


def bench_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from oracle import oracle
    w = WORKLOAD
    mic, grid, Ys = make_batches(0, 1)
    Q = w["M"] * (w["M"] - 1) // 2
    Nq, _ = oracle.lag_counts(mic, w["fs"], 343.0)
    S = int(np.sum(2 * Nq + 2 * w["n_aux"] + 1))
    for _ in range(args.warmup):
        oracle_step_seconds(mic, grid, Ys[0], w, stride=64, frames=1)
    secs = []
    desc, threads = "", 0
    for _ in range(args.steps):
        s, desc, threads = oracle_step_seconds(mic, grid, Ys[0], w, stride=64, frames=1)
        secs.append(s)
    ms = 1e3 * float(np.mean(secs))
    value = w["J"] * Q * w["L"] / (ms * 1e-3)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic free-field white-noise scenes (seeded)", "config": config_dict(Q, S),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--conv-steps", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--batch-arrays", type=int, default=BATCH_N,
                    help="arrays of the uneven mix in the batched section (the workload is 256)")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
