#!/usr/bin/env python
"""Benchmark of the GRAPHIC ADI hot path on GB300.

One step = one full reduction (recentring shift, angle-gated median PSF
subtraction, three-shear derotation, median collapse) of one synthetic cube
of 2000 frames of 512 x 512 (padded to 1024), through the C ABI
(graphic_reduce).  Prints ONE JSON line on rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 is launched with torch.distributed.run: every rank reduces its own cube
(independent problems, no collective on the data path), the elapsed time is
the max over ranks and the value counts the frames of all ranks.

Other workloads (--workload): small (32 x 128^2 reduce), uneven (48 cubes of
mixed sizes through the batch executors and the autotuner), serve (the
serving loop alone), precision (512 x 1024^2 shift + rotation per
arithmetic, tensor-core variants), prep (master skies, sky subtraction, bad
pixels), register (centroid + Moffat fit of 2000 raw frames), photometry
(the inject / recentre / bin / reduce / aperture protocol), median /
collapse (one step of the reduction alone, for kernel captures).  --impl
reference times the CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "frames/s (1024² FFT shift+3-shear derot) & % HBM roofline; p50/p99 latency"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
FP32_LANES_PER_SM = 128     # FP32 FMA lanes per Blackwell SM (4 partitions x 32)
FALLBACK_SM_MHZ = 2070.0    # GB300 maximum SM clock


def fp32_peak(dev=0):
    """FP32 CUDA-core peak in TFLOP/s from the device's SM count
    (cudaDevAttrMultiProcessorCount), 128 FMA lanes per SM, 2 flop per FMA,
    and the maximum SM clock (MEASURED_PEAKS.json sm_max_mhz, else 2070 MHz).
    Returns (tflops, description)."""
    sms = None
    try:
        import torch
        sms = int(torch.cuda.get_device_properties(dev).multi_processor_count)
    except Exception:
        pass
    if not sms:
        sms = 152
    mhz = FALLBACK_SM_MHZ
    try:
        with open(PEAKS_FILE) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    tf = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    return tf, f"FP32 CUDA cores: {sms} SMs (device attribute) x {FP32_LANES_PER_SM} lanes x 2 flop x {mhz:.0f} MHz"

WORKLOADS = {
    "survey": dict(T=2000, n=512, seed=1,
                   desc="2000 frames of 512x512 (padded to 1024), alt-az parallactic angles (dec -30, lat -24.6, "
                        "h -1.5..+1.5 h), AR(1) speckles rho=0.99, 5 companions 10-100 px, contrast 1e-3..1e-5; "
                        "full reduce: shift, median PSF subtraction, 3-shear derotation, median collapse"),
    "small": dict(T=32, n=128, seed=0,
                  desc="32 frames of 128x128 (padded to 256), angles 0-40 deg, 2 companions; full reduce"),
}


def make_workload(name, frames=None, n=None):
    from paper_1510_04331_gb300 import synth
    w = dict(WORKLOADS[name])
    if frames:
        w["T"] = frames
    if n:
        w["n"] = n
    if name == "survey":
        return synth.survey_cube(seed=w["seed"], T=w["T"], N=w["n"])
    return synth.small_cube(seed=w["seed"], T=w["T"], N=w["n"])


def workload_desc(name, d):
    T, n = d.cube.shape[0], d.cube.shape[1]
    w = WORKLOADS[name]
    if (T, n) == (w["T"], w["n"]):
        return w["desc"]
    return f"{T} frames of {n}x{n} (padded to {2 * n}), {name} recipe; full reduce"


def max_over_ranks(value, device=None):
    """Max of a float over all ranks of the default process group (the value
    itself without one, or at world size 1)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step, steps, world, max_ms):
    """Whole-job throughput: the units all ranks processed / the slowest
    rank's elapsed time (weak scaling: fixed work per rank)."""
    return units_per_rank_step * steps * world / (max_ms / 1e3)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of a whole step of
# one kernel, from ncu captures of the current kernels: (kernel, frames, n) ->
# (bytes per step at that size, source).  Per launch = bytes / launches.
MEASURED_TRAFFIC = {
    ("adi_band_sweep", 2000, 512): (
        5.8944e9,
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of the five band-sweep launches of one median step on "
        "the 2000x512^2 survey cube itself (profiles/band_sweep_kernel_survey_2000x512.md)"),
}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# ---------------------------------------------------------------------------
# algorithmic work per kernel launch (bytes or flops), per frame of side n
# ---------------------------------------------------------------------------

def fft_flops_per_frame(kind, n):
    """Nominal 5 m log2 m flops per complex m-point FFT, forward + inverse,
    two real lines per complex transform (m = 2n)."""
    m = 2 * n
    lines = {"shift_x": n, "shift_y": n, "rot_pass1": n, "rot_pass2": m, "rot_pass3": n}[kind]
    return (lines / 2) * 2 * 5 * m * math.log2(m)


def kernel_work(kind, n, T):
    """(bound, algorithmic amount per launch-frame, unit) for one frame."""
    if kind in ("shift_x", "shift_y", "rot_pass1", "rot_pass2", "rot_pass3"):
        return "alu", fft_flops_per_frame(kind, n), "flop"
    if kind in ("adi_band_sweep", "adi_general"):
        return "hbm", 2 * n * n * 4, "B"   # reads the cube, writes the residuals
    if kind == "adi_band_prep":
        return "hbm", n * n * 4, "B"       # reads the cube
    return "hbm", n * n * 4, "B"   # collapse: read the cube once


def line_pass_roofline(kernels, n, T):
    """FP32 roofline of the five Fourier line passes together: nominal FFT
    flops of all frames over the passes' summed device time per step."""
    kinds = [k for k in ("shift_x", "shift_y", "rot_pass1", "rot_pass2", "rot_pass3") if k in kernels]
    if not kinds:
        return None
    flops = T * sum(fft_flops_per_frame(k, n) for k in kinds)
    ms = sum(kernels[k]["ms_per_step"] for k in kinds)
    if ms <= 0:
        return None
    achieved = flops / (ms / 1e3) / 1e12
    peak, src = fp32_peak()
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "flops_per_step": flops, "ms_per_step": ms,
            "peak_source": src, "kernels": kinds}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu_id)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid_or_index(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return dev


# ---------------------------------------------------------------------------
# oracle CPU baseline (a bounded sample of the same workload)
# ---------------------------------------------------------------------------

def cpu_baseline(d, budget_s=15.0):
    import oracle
    T, n = d.cube.shape[0], d.cube.shape[1]
    nt = oracle.num_threads()
    k = max(1, min(T, nt))
    fr = np.linspace(0, T - 1, k).astype(int)
    c64 = d.cube[fr].astype(np.float64)
    t0 = time.perf_counter()
    sh = oracle.shift(c64, d.dx[fr], d.dy[fr])
    t1 = time.perf_counter()
    oracle.rotate(sh, -d.parang[fr])
    t2 = time.perf_counter()
    per_frame_geom = (t2 - t0) / k
    # median stages on a few pixels of the whole cube
    rng = np.random.default_rng(0)
    npix = max(1, nt)
    pix = rng.choice(n * n, npix, replace=False)
    c64_all = d.cube.astype(np.float64)
    t3 = time.perf_counter()
    oracle.adi_subtract(c64_all, d.parang, d.fwhm, d.n_fwhm, d.edges, pixels=pix)
    t4 = time.perf_counter()
    per_pix_adi = (t4 - t3) / npix
    # scale the pixel sample up if the first round was short
    extra = max(0.0, budget_s - (t4 - t0))
    if extra > 1.0 and per_pix_adi > 0:
        more = int(min(extra / per_pix_adi * 0.8, 64 * npix))
        if more >= 1:
            pix2 = rng.choice(n * n, more, replace=False)
            t5 = time.perf_counter()
            oracle.adi_subtract(c64_all, d.parang, d.fwhm, d.n_fwhm, d.edges, pixels=pix2)
            t6 = time.perf_counter()
            per_pix_adi = ((t4 - t3) + (t6 - t5)) / (npix + more)
            npix += more
    t7 = time.perf_counter()
    cp = rng.choice(n * n, min(n * n, 4096), replace=False)
    oracle.collapse_median(c64_all, pixels=cp)
    t8 = time.perf_counter()
    per_pix_col = (t8 - t7) / cp.size
    sec_per_cube = per_frame_geom * T + (per_pix_adi + per_pix_col) * n * n
    return {
        "value": T / sec_per_cube, "unit": "frames/s", "cores": nt, "kind": "oracle",
        "sample": (f"FP64 oracle throughout, extrapolated: shift + 3-shear rotation timed on {k} of {T} frames "
                   f"({per_frame_geom:.3f} s/frame), median PSF subtraction on {npix} of {n * n} pixels x {T} "
                   f"frames ({per_pix_adi:.4f} s/pixel) and median collapse on {cp.size} pixels, each scaled "
                   f"linearly to the whole {T}x{n}x{n} cube"),
        "sec_per_cube": sec_per_cube,
    }


# ---------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return 0
    name = args.workload
    d = make_workload(name, args.frames, args.n)
    T, n = d.cube.shape[0], d.cube.shape[1]
    vals = []
    # each step is one bounded oracle sample; the whole run stays within a few minutes
    budget = min(args.ref_budget, max(2.0, 150.0 / (args.warmup + args.steps)))
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(d, budget_s=budget)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = statistics.median(vals)
    sec = T / v
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(name, d), "frames": T, "n": n, "m": 2 * n},
        "cpu_baseline": {"value": v, "unit": "frames/s", "cores": cb["cores"], "kind": "oracle",
                         "sample": cb["sample"] + "; each step times one such sample"},
        "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_1510_04331_gb300 import graphic

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    name = args.workload
    d = make_workload(name, args.frames, args.n)
    T, n = d.cube.shape[0], d.cube.shape[1]
    NN = n * n
    ctx = graphic.Context(local_rank)
    stream = torch.cuda.current_stream(dev)
    cube = torch.from_numpy(d.cube).to(dev)
    work = torch.empty_like(cube)
    out = torch.empty((n, n), dtype=torch.float32, device=dev)

    # optional time gate: frames taken at hour angles linear over the sequence
    # (the alt-az recipe's -1.5 .. +1.5 h), reference frames within t_max hours
    times = np.linspace(-1.5, 1.5, T) if args.t_max else None

    def step():
        ctx.graphic_reduce(cube, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges, work=work, out=out, times=times,
                           t_max=args.t_max)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    sampler = ClockSampler(gpu_uuid_or_index(local_rank)) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.4)
    ctx.profile(True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(args.steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    prof = ctx.profile_read()
    ctx.profile(False)
    clocks = sampler.stop() if sampler else None
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = max_over_ranks(evs[0].elapsed_time(evs[-1]), dev)
    value = job_throughput(T, args.steps, world, total_ms)

    # e2e: host buffers through graphic_reduce_host, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        host = torch.from_numpy(d.cube).pin_memory()
        hout = torch.empty((n, n), dtype=torch.float32).pin_memory()
        ne = max(2, min(args.steps, args.e2e_steps))
        for _ in range(2):
            ctx.graphic_reduce_host(host, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges, out_host=hout)
        barrier()
        t0 = time.perf_counter()
        for _ in range(ne):
            ctx.graphic_reduce_host(host, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges, out_host=hout)
        el = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": job_throughput(T, ne, world, el * 1e3), "unit": "frames/s", "h2d_bytes_per_step": T * NN * 4,
               "d2h_bytes_per_step": NN * 4, "steps": ne}

    if rank != 0:
        return 0
    # per-kernel table and the dominant kernel's roofline
    hbm_peak, peak_src = peaks()
    kernels = {}
    for kname, (ms, cnt) in prof.items():
        if cnt == 0:
            continue
        kernels[kname] = {"ms_per_step": ms / args.steps, "launches_per_step": cnt / args.steps,
                          "avg_launch_ms": ms / cnt}
    ktot = sum(k["ms_per_step"] for k in kernels.values())
    for k in kernels.values():
        k["share"] = k["ms_per_step"] / ktot if ktot else None
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    kd = kernels[dom]
    frames_per_launch = T / kd["launches_per_step"]
    bound, per_frame, unit = kernel_work(dom, n, T)
    amount = per_frame * frames_per_launch
    avg_s = kd["avg_launch_ms"] / 1e3
    if bound == "hbm":
        achieved = amount / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": None, "kernel": dom, "peak_source": peak_src + " (copy, MEASURED_PEAKS.json hbm_gbs)"
                if peak_src == "measured" else "fallback 6.8 TB/s",
                "algorithmic_per_launch": amount}
    else:
        achieved = amount / avg_s / 1e12
        fpk, fsrc = fp32_peak(local_rank)
        roof = {"bound": "alu", "achieved": achieved, "peak": fpk, "unit": "TFLOP/s",
                "frac": achieved / fpk, "traffic": None, "kernel": dom, "peak_source": fsrc,
                "algorithmic_per_launch": amount}
    mt = MEASURED_TRAFFIC.get((dom, T, n))
    if mt:
        roof["traffic"] = mt[0] / kd["launches_per_step"]
        roof["traffic_source"] = mt[1]
    # whole-step HBM roofline (algorithmic 7 n^2 4 B per frame)
    alg_bytes = 7 * NN * 4 * T
    step_s = statistics.median(step_ms) / 1e3
    whole = {"algorithmic_bytes_per_step": alg_bytes, "achieved_gbs": alg_bytes / step_s / 1e9,
             "frac_of_hbm": alg_bytes / step_s / 1e9 / hbm_peak}
    line_fp32 = line_pass_roofline(kernels, n, T)
    srt = sorted(step_ms)
    p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc(name, d) + (f"; reference frames within {args.t_max} h (time gate)"
                                                          if args.t_max else ""), "frames": T, "n": n, "m": 2 * n,
                   "l2": "inputs larger than L2 (cube %.2f GB per rank)" % (T * NN * 4 / 1e9),
                   "parallelism": f"{world} independent cubes (one per GPU)"},
        "latency_ms": {"p50": statistics.median(step_ms), "p99": p99, "min": srt[0], "max": srt[-1]},
        "roofline": roof,
        "line_passes_fp32": line_fp32,
        "whole_step_hbm": whole,
        "kernels": kernels,
        "gpu_launches": int(round(sum(k["launches_per_step"] for k in kernels.values()) * args.steps)),
        "clocks": clocks,
        "e2e": e2e,
    }
    del cube, work
    torch.cuda.empty_cache()
    if not args.no_serve and world == 1:
        line["serving"] = run_serving(local_rank, n_req=args.serve_requests, max_active=args.serve_max_active)
    if not args.no_extra and world == 1:
        # the uneven-batch and precision workloads, a few steps each, under the same clock
        line["uneven"] = measure_uneven(local_rank, rank, steps=5, warmup=3, tune=True)
        line["precision"] = measure_precision(local_rank, rank, steps=5, warmup=3)
    if not args.no_cpu_baseline and world == 1:
        cb = cpu_baseline(d, budget_s=args.ref_budget)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    elif not args.no_cpu_baseline:
        line["cpu_baseline"] = None
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# precision variant: 512 frames of 1024 x 1024 (2048-point lines), shift + 3-shear rotation
# ---------------------------------------------------------------------------

def tc_gemm_flops_per_frame(n=1024):
    """Tensor-core flops one frame of side n costs in the precision variant:
    per 2048-point transform two radix-16 stages (128 x 32 x 32) and one
    radix-8 stage (256 x 16 x 16), three split products each, two
    transforms (forward, inverse) per line pair."""
    per_transform = 3 * 2 * (2 * 128 * 32 * 32 + 256 * 16 * 16)
    pairs = n // 2 * 4 + n   # shift x, shift y, rotation 1, 3 (n / 2 pairs each), rotation 2 (n pairs)
    return 2 * per_transform * pairs


def bf16_peak():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), "measured (cuBLAS bf16 burst, MEASURED_PEAKS.json)"
    except Exception:
        return 1900.0, "fallback 1.9 PFLOP/s"


def measure_precision(local_rank, rank, steps, warmup, frames=None):
    """Each step: shift then rotate every frame of a 512 x 1024 x 1024 cube
    (the geometric steps of the reduction at 2048-point lines), once per
    arithmetic; errors of each step against the FP64 oracle on sampled
    frames of the survey recipe at this size.  Returns a dict."""
    import torch
    import oracle
    from paper_1510_04331_gb300 import graphic, synth

    torch.cuda.set_device(local_rank)
    T, n = (frames or 512), 1024
    gen = torch.Generator(device="cuda").manual_seed(3 + rank)
    cube = torch.randn((T, n, n), generator=gen, device="cuda")
    out = torch.empty_like(cube)
    rng = np.random.default_rng(3)
    dx, dy = rng.uniform(-0.5, 0.5, T), rng.uniform(-0.5, 0.5, T)
    th = -synth.altaz_parang(T)
    names = {graphic.PREC_FP32: "fp32", graphic.PREC_BF16X3: "bf16x3", graphic.PREC_FP16X3: "fp16x3"}
    res = {}
    sampler = ClockSampler(gpu_uuid_or_index(local_rank)) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.4)
    for prec, name in names.items():
        ctx = graphic.Context(local_rank)
        ctx.set_precision(prec)

        def step():
            ctx.graphic_shift(cube, dx, dy, out=out)
            ctx.graphic_rotate(out, th, out=out)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        ctx.profile(True)
        ms = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        prof = ctx.profile_read()
        ctx.profile(False)
        ctx.close()
        med = statistics.median(ms)
        kern = {k: {"ms_per_step": v[0] / steps, "launches_per_step": v[1] / steps}
                for k, v in prof.items() if v[1]}
        res[name] = {"ms_p50": med, "frames_per_s": T / (med / 1e3), "kernels": kern}
    clocks = sampler.stop() if sampler else None
    del cube, out
    torch.cuda.empty_cache()
    # per-step error against the FP64 oracle on 2 frames of the survey recipe at n = 1024
    d = synth.make_cube(2, n, seed=3, parang=synth.altaz_parang(2), peak=1e5, rho=0.99,
                        edges=synth.default_edges(n))
    x64 = d.cube.astype(np.float64)
    ex, ey, et = np.array([0.31, -0.47]), np.array([-0.22, 0.44]), np.array([37.7, -101.3])
    ref_s = oracle.shift(x64, ex, ey)
    ref_r = oracle.rotate(ref_s, et)
    peak_in = float(np.abs(d.cube).max())
    for prec, name in names.items():
        ctx = graphic.Context(local_rank)
        ctx.set_precision(prec)
        xs = ctx.graphic_shift(torch.from_numpy(d.cube).cuda(), ex, ey)
        e_s = float(np.abs(xs.cpu().numpy() - ref_s).max() / peak_in)
        xr = ctx.graphic_rotate(torch.from_numpy(ref_s.astype(np.float32)).cuda(), et)
        e_r = float(np.abs(xr.cpu().numpy() - ref_r).max() / peak_in)
        ctx.close()
        res[name]["error_vs_fp64_oracle"] = {"shift": e_s, "rotate": e_r, "unit": "max abs / frame peak"}
    tc_flops = tc_gemm_flops_per_frame(n) * T
    bpk, bsrc = bf16_peak()
    best_tc = min(("bf16x3", "fp16x3"), key=lambda k: res[k]["ms_p50"])
    ach = tc_flops / (res[best_tc]["ms_p50"] / 1e3) / 1e12
    fp32_flops = T * sum(fft_flops_per_frame(k, n) for k in ("shift_x", "shift_y", "rot_pass1", "rot_pass2",
                                                                "rot_pass3"))
    fpk, fsrc = fp32_peak(local_rank)
    return {
        "frames": T, "n": n, "steps": steps, "warmup": warmup, "best_tensor_core": best_tc,
        "workload": f"{T} frames of 1024x1024 padded to 2048, shift U(-0.5,0.5) px + derotation by "
                    "alt-az angles; errors on 2 frames of the survey recipe (peak 1e5)",
        "variants": res,
        "tensor_vs_fp32_frames_per_s": res[best_tc]["frames_per_s"] / res["fp32"]["frames_per_s"],
        "roofline": {"bound": "tensor", "achieved": ach, "peak": bpk, "unit": "TFLOP/s", "frac": ach / bpk,
                     "traffic": None, "kernel": f"line_pass_tc ({best_tc}), GEMM flops executed",
                     "peak_source": bsrc, "algorithmic_per_launch": tc_flops},
        "fp32_roofline": {"bound": "alu", "achieved": fp32_flops / (res["fp32"]["ms_p50"] / 1e3) / 1e12,
                          "peak": fpk, "unit": "TFLOP/s", "peak_source": fsrc,
                          "frac": fp32_flops / (res["fp32"]["ms_p50"] / 1e3) / 1e12 / fpk},
        "clocks": clocks,
    }


def run_precision(args, rank, world, local_rank):
    r = measure_precision(local_rank, rank, args.steps, args.warmup, args.frames)
    best = r["best_tensor_core"]
    line = {
        "metric": "frames/s, 1024x1024 shift + 3-shear rotation (2048-point lines), per arithmetic",
        "value": r["variants"][best]["frames_per_s"], "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["variants"][best]["ms_p50"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": best, "data": "synthetic",
        "config": {"workload": r["workload"], "frames": r["frames"], "n": r["n"],
                   "l2": "inputs larger than L2 (%.1f GB)" % (r["frames"] * r["n"] ** 2 * 4 / 1e9)},
        "variants": r["variants"], "roofline": r["roofline"], "fp32_roofline": r["fp32_roofline"],
        "clocks": r["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# image-quality pre-processing (Sect. 3.2) of the survey-sized cube
# ---------------------------------------------------------------------------

def run_prep(args, rank, world, local_rank):
    """Each step: 20 master skies (each the masked median of 50 dithered sky
    frames), the subtraction of the nearest sky from 2000 science frames of
    512 x 512, the bad pixel map of a master dark (C = 5) and the
    neighbour-median correction of the 2000 frames (0.1 % hot pixels and
    3 x 3 clumps, plus NaN from the masks)."""
    import torch
    from paper_1510_04331_gb300 import graphic

    torch.cuda.set_device(local_rank)
    T, n, ns, nsf = (args.frames or 2000), 512, 20, 50
    gen = torch.Generator(device="cuda").manual_seed(5 + rank)
    sci = torch.randn((T, n, n), generator=gen, device="cuda") * 10.0 + 100.0
    skyf = torch.randn((nsf, n, n), generator=gen, device="cuda") * 3.0 + 100.0
    dark = torch.randn((n, n), generator=gen, device="cuda")
    rng = np.random.default_rng(5)
    hot = rng.choice(n * n, n * n // 1000, replace=False)
    dark.view(-1)[torch.from_numpy(hot).cuda()] = 100.0
    for (r0, c0) in rng.integers(10, n - 10, (5, 2)):
        dark[r0:r0 + 3, c0:c0 + 3] = 100.0
    mx, my = rng.uniform(100, 400, nsf), rng.uniform(100, 400, nsf)
    frame_t = np.linspace(0.0, 1.0, T)
    sky_t = np.linspace(0.0, 1.0, ns)
    ctx = graphic.Context(local_rank)
    skies = torch.empty((ns, n, n), device="cuda")
    out = torch.empty_like(sci)

    def step(ev=None):
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(5)] if ev is not None else None
        if marks:
            marks[0].record()
        for j in range(ns):
            ctx.graphic_sky_median(skyf, mx, my, 30.0, out=skies[j])
        if marks:
            marks[1].record()
        ctx.graphic_sky_subtract(sci, skies, frame_t, sky_t, out=out)
        if marks:
            marks[2].record()
        m = ctx.graphic_bad_pixel_map(dark, 5.0)
        if marks:
            marks[3].record()
        ctx.graphic_bad_pixel_fix(out, m)
        if marks:
            marks[4].record()
            ev.append(marks)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        step(evs)
    torch.cuda.synchronize()
    names = ["sky_median_x20", "sky_subtract", "bad_pixel_map", "bad_pixel_fix"]
    per = {k: statistics.median(e[i].elapsed_time(e[i + 1]) for e in evs) for i, k in enumerate(names)}
    tot = statistics.median(e[0].elapsed_time(e[4]) for e in evs)
    hbm, _ = peaks()
    sub_bytes = 2 * T * n * n * 4
    line = {
        "metric": "frames/s, image-quality pre-processing (master skies, sky subtraction, bad pixels)",
        "value": T / (tot / 1e3), "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{T} science frames of {n}x{n}, {ns} master skies of {nsf} masked frames, "
                               "bad pixel map of a master dark (0.1 % hot pixels, 3x3 clumps), correction",
                   "frames": T, "n": n},
        "stages_ms": per,
        "roofline": {"bound": "hbm", "kernel": "sky_subtract", "achieved": sub_bytes / (per["sky_subtract"] / 1e3) / 1e9,
                     "peak": hbm, "unit": "GB/s",
                     "frac": sub_bytes / (per["sky_subtract"] / 1e3) / 1e9 / hbm, "traffic": None,
                     "algorithmic_per_launch": sub_bytes},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


REG_PARAMS = dict(R=16, min_size=4, max_size=400, w=10)   # thresh = 0.1 x the star's peak


def run_register(args, rank, world, local_rank):
    """Each step: registration (Sect. 3.1) of 2000 raw frames of 512 x 512 --
    per frame the brightest-seeded patch centroid and the Moffat fit by
    Levenberg-Marquardt (FP64) -- through graphic_register.  The frames are
    200 distinct seeded star frames (star dithered +-60 px, 10 % AO-loss
    frames) repeated 10 times; the 1 GB cube exceeds L2, so every step reads
    it from HBM.  Centres are checked against the FP64 oracle on the 200
    distinct frames."""
    import torch
    import oracle
    from paper_1510_04331_gb300 import graphic, synth

    torch.cuda.set_device(local_rank)
    T, n, nd = (args.frames or 2000), 512, 200
    d = synth.star_frames(nd, n, seed=13 + rank, jitter=60.0, lost=0.1)
    base = torch.from_numpy(d.cube).cuda()
    cube = base.repeat((T + nd - 1) // nd, 1, 1)[:T].contiguous()
    thresh = 0.1 * d.peak
    ctx = graphic.Context(local_rank)
    out = torch.empty((T, 8), dtype=torch.float64, device="cuda")
    it = torch.empty(T, dtype=torch.int32, device="cuda")

    def step():
        ctx.graphic_register(cube, thresh, REG_PARAMS["R"], REG_PARAMS["min_size"], REG_PARAMS["max_size"],
                             REG_PARAMS["w"], out=out, iters=it)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_uuid_or_index(local_rank)) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1) / args.steps
    ctx.profile(True)
    for _ in range(3):
        step()
    prof = ctx.profile_read()
    ctx.profile(False)
    t_arg = prof["register_argmax"][0] / max(1, prof["register_argmax"][1])
    t_fit = prof["register_fit"][0] / max(1, prof["register_fit"][1])
    got = out[:nd].cpu().numpy()
    want_f, want_x, want_y, want_fw = oracle.register(d.cube, thresh, **REG_PARAMS)
    m = want_f
    parity = {"found_equal": bool(np.array_equal(got[:, 0] == 1.0, want_f)),
              "max_abs_centre_px": float(np.abs(np.r_[got[m, 1] - want_x[m], got[m, 2] - want_y[m]]).max()),
              "max_rel_fwhm": float(np.abs(got[m, 3] / want_fw[m] - 1.0).max()),
              "max_abs_centre_vs_truth_px": float(np.abs(np.r_[got[m, 1] - d.x[m], got[m, 2] - d.y[m]]).max())}
    hbm, src = peaks()
    arg_bytes = T * n * n * 4
    line = {
        "metric": "frames/s, registration (centroid + Moffat Levenberg-Marquardt fit, FP64)",
        "value": T / (ms / 1e3), "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{T} raw frames of {n}x{n} (200 distinct seeded star frames x10, dither +-60 px, "
                               f"10 % lost), R={REG_PARAMS['R']}, w={REG_PARAMS['w']}, size "
                               f"{REG_PARAMS['min_size']}..{REG_PARAMS['max_size']}, thresh 0.1 peak",
                   "frames": T, "n": n, "l2": "cube 1 GB > L2"},
        "kernels_ms": {"register_argmax": t_arg, "register_fit": t_fit},
        "lm_iterations_mean": float(it.float().mean().item()),
        "roofline": {"bound": "hbm", "kernel": "frame_argmax", "achieved": arg_bytes / (t_arg / 1e3) / 1e9,
                     "peak": hbm, "unit": "GB/s", "frac": arg_bytes / (t_arg / 1e3) / 1e9 / hbm,
                     "traffic": None, "peak_source": src, "algorithmic_per_launch": arg_bytes},
        "parity_vs_oracle": parity,
        "clocks": clocks,
        "gpu_launches": 2 * args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


PHOT_COMPANIONS = [   # (separation arcsec, position angle deg, delta mag), the Table 1 grid
    (1.0, 30.0, 8.0), (3.0, 110.0, 8.0), (3.0, 250.0, 10.0), (5.0, 190.0, 8.0), (5.0, 330.0, 10.0)]
PIXEL_SCALE_ARCSEC = 0.02719   # NACO L27 camera


def run_photometry(args, rank, world, local_rank):
    """The photometric-accuracy and binning protocol of Sect. 4.2-4.3 on a
    synthetic 2-hour sequence (2000 raw frames of 512 x 512, 120 deg of
    field rotation: alt-az angles at dec -33.4, lat -24.6, h -1..+1 h, the
    survey speckle recipe, no companions in the data): registration of the
    raw frames (centres, Moffat alpha / beta, star flux I0), then for bins
    of 1, 10 and 50 frames: companions injected into a copy of the raw
    frames at 1, 3, 5 arcsec (Delta mag 8 and 10, the star's fitted PSF and
    flux), recentring by the registered centres, median binning, the full
    reduction with the bins' mean angles, aperture photometry (radius 1
    FWHM) at the derotated positions.  Recovered flux = aperture in the
    reduced image / aperture of the same companion injected alone."""
    import torch
    from paper_1510_04331_gb300 import graphic, synth

    torch.cuda.set_device(local_rank)
    T, n = (args.frames or 2000), 512
    pa = synth.altaz_parang(T, dec_deg=-33.4, h0_h=-1.0, h1_h=1.0)
    d = synth.make_cube(T, n, 21 + rank, parang=pa, peak=1e5, rho=0.99, companions=[],
                        edges=synth.default_edges(n), name="photometry")
    raw = torch.from_numpy(d.cube).cuda()
    del d.cube
    ctx = graphic.Context(local_rank)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    e0, e1 = ev(), ev()
    reg = ctx.graphic_register(raw, 0.1 * 1e5, 16, 4, 400, 10)      # warm-up (module load, attributes)
    e0.record()
    reg = ctx.graphic_register(raw, 0.1 * 1e5, 16, 4, 400, 10)
    e1.record()
    torch.cuda.synchronize()
    t_reg = e0.elapsed_time(e1)
    r = reg.cpu().numpy()
    keep = np.nonzero(r[:, 0] == 1.0)[0]
    if len(keep) < T:
        raw = raw[torch.from_numpy(keep).cuda()].contiguous()
    x0, y0, alpha, beta, i0 = r[keep, 1], r[keep, 2], r[keep, 5], r[keep, 6], r[keep, 4]
    pa = pa[keep]
    Tk = len(keep)
    star_flux = float(np.median(i0))
    seps = np.array([c[0] / PIXEL_SCALE_ARCSEC for c in PHOT_COMPANIONS])
    pa0 = np.array([c[1] for c in PHOT_COMPANIONS])
    flux = star_flux * 10.0 ** (-0.4 * np.array([c[2] for c in PHOT_COMPANIONS]))
    xs, ys = n / 2 + seps * np.cos(np.radians(pa0)), n / 2 + seps * np.sin(np.radians(pa0))
    r_ap = d.fwhm
    half = 16
    alone = torch.zeros((1, n, n), device="cuda")
    ctx.graphic_inject(alone, [0.0], [n / 2], [n / 2], seps, pa0, flux, [float(np.median(alpha))],
                       [float(np.median(beta))], half)
    ref = ctx.graphic_aperture(alone[0], xs, ys, r_ap)
    dx, dy = n / 2 - x0, n / 2 - y0
    results = {}
    for B in (1, 10, 50):
        if B > 1:
            # the binning kernel alone, timed by the library's per-kernel events
            xs_ = ctx.graphic_shift(raw, dx, dy)
            ctx.graphic_bin_median(xs_, B)
            ctx.profile(True)
            ctx.graphic_bin_median(xs_, B)
            bin_ms = ctx.profile_read()["bin_median"][0]
            ctx.profile(False)
            del xs_
        times = []
        for rep in range(max(1, args.steps)):
            x = raw.clone()
            torch.cuda.synchronize()
            e0.record()
            ctx.graphic_inject(x, pa, x0, y0, seps, pa0, flux, alpha, beta, half)
            if B == 1:
                img = ctx.graphic_reduce(x, dx, dy, pa, d.fwhm, d.n_fwhm, d.edges)
            else:
                x = ctx.graphic_shift(x, dx, dy)
                xb = ctx.graphic_bin_median(x, B)
                z = np.zeros(xb.shape[0])
                img = ctx.graphic_reduce(xb, z, z, graphic.bin_mean(pa, B), d.fwhm, d.n_fwhm, d.edges)
            ap = ctx.graphic_aperture(img, xs, ys, r_ap)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            del x
        results[B] = {"ms": statistics.median(times),
                      "recovered_percent": [round(100.0 * v, 1) for v in (ap / ref)]}
        if B > 1:
            G = (Tk + B - 1) // B
            nbytes = (Tk + G) * n * n * 4
            hbm, _ = peaks()
            results[B]["bin_median"] = {"ms": bin_ms, "bytes": nbytes, "gbs": nbytes / (bin_ms / 1e3) / 1e9,
                                        "frac_of_hbm": nbytes / (bin_ms / 1e3) / 1e9 / hbm}
    table = {f"bin {B}": results[B]["recovered_percent"] for B in results}
    line = {
        "metric": "frames/s, photometric protocol (inject, recentre, median PSF reduction, aperture), no binning",
        "value": Tk / (results[1]["ms"] / 1e3), "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": 0, "ms_per_step": results[1]["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{T} raw frames of {n}x{n}, 120 deg rotation in 2 h (dec -33.4), survey speckles, "
                               "companions at 1/3/5 arcsec, Delta mag 8/10, bins 1/10/50",
                   "frames": T, "kept_frames": Tk, "n": n, "aperture_radius_px": r_ap},
        "registration_ms": t_reg,
        "companions": [{"sep_arcsec": c[0], "pa0_deg": c[1], "delta_mag": c[2]} for c in PHOT_COMPANIONS],
        "recovered_flux_percent": table,
        "protocol_ms": {f"bin {B}": results[B]["ms"] for B in results},
        "bin_median_kernel": {f"bin {B}": results[B]["bin_median"] for B in results if B > 1},
        "paper_table1_percent": {"no binning": [60, 81, 106, 71, 72], "10 frame bins": [52, 63, 93, 59, 20],
                                 "50 frame bins": [61, 66, 101, 60, 52]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# serving loop: Poisson arrivals of full reductions, sizes from the uneven mix
# ---------------------------------------------------------------------------

SERVE_SIDES = (64, 128, 256, 512, 1024)


def serve_requests(seed, n_req, t_range=(16, 400)):
    """Request shapes and parameters: side from SERVE_SIDES, frame count
    uniform in t_range, alt-az parallactic angles resampled to the frame
    count, recentring shifts U(-0.5, 0.5) px, FWHM 4 px, 1.5 FWHM gate."""
    from paper_1510_04331_gb300 import synth
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_req):
        n = int(rng.choice(SERVE_SIDES))
        T = int(rng.integers(t_range[0], t_range[1] + 1))
        out.append(dict(n=n, T=T, dx=rng.uniform(-0.5, 0.5, T), dy=rng.uniform(-0.5, 0.5, T),
                        parang=synth.altaz_parang(T), fwhm=4.0, n_fwhm=1.5, edges=synth.default_edges(n)))
    return out


def _pct(v, q):
    s = sorted(v)
    return s[min(len(s) - 1, max(0, int(math.ceil(q * len(s))) - 1))]


def run_serving(local_rank, n_req=200, rates=(20.0, 200.0, 2000.0), seed=4, max_active=64):
    """Each rate: the same Poisson arrival sequence served (a) by the serving
    loop (graphic_server: admission by device memory, cross-request
    batching) and (b) by plain sequential per-request reductions
    (graphic_reduce_host in arrival order).  Latency = completion - arrival."""
    import queue as _queue

    import torch
    from paper_1510_04331_gb300 import graphic

    reqs = serve_requests(seed, n_req)
    tmax = max(r["T"] for r in reqs)
    gen = torch.Generator().manual_seed(seed)
    pool = {}
    for n in sorted({r["n"] for r in reqs}):
        pool[n] = torch.randn((tmax, n, n), generator=gen, dtype=torch.float32).pin_memory()
    inputs = [pool[r["n"]][:r["T"]] for r in reqs]
    frames = sum(r["T"] for r in reqs)
    in_bytes = sum(r["T"] * r["n"] * r["n"] * 4 for r in reqs)
    results = []
    for rate in rates:
        arr = np.cumsum(np.random.default_rng(seed + int(rate)).exponential(1.0 / rate, n_req))
        row = {"rate_per_s": rate}
        # (a) serving loop
        with graphic.Server(local_rank, max_active=max_active) as srv:
            for r, x in list(zip(reqs, inputs))[:3]:    # warm-up: graphs, plans
                srv.wait(srv.submit(x, r["dx"], r["dy"], r["parang"], r["fwhm"], r["n_fwhm"], r["edges"]))
            ids = [None] * n_req
            ready = threading.Event()

            def submitter():
                t0 = time.perf_counter()
                for i, (r, x) in enumerate(zip(reqs, inputs)):
                    dt = t0 + arr[i] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    ids[i] = srv.submit(x, r["dx"], r["dy"], r["parang"], r["fwhm"], r["n_fwhm"], r["edges"])
                ready.set()

            th = threading.Thread(target=submitter)
            th.start()
            infos = []
            for i in range(n_req):
                while ids[i] is None:
                    time.sleep(0.0002)
                infos.append(srv.wait(ids[i])[1])
            th.join()
            st = srv.stats()
        bad = [x for x in infos if x["status"] != 0]
        lat = [(x["t_done"] - x["t_submit"]) * 1e3 for x in infos]
        span = max(x["t_done"] for x in infos) - min(x["t_submit"] for x in infos)
        row["server"] = {"frames_per_s": frames / span, "p50_ms": statistics.median(lat), "p99_ms": _pct(lat, 0.99),
                         "span_s": span, "failed": len(bad),
                         "mean_batch": st["batch_items"] / max(1, st["batch_launches"]),
                         "max_batch": st["max_batch_items"], "max_resident": st["max_resident"],
                         "iterations": st["iterations"], "device_bytes_peak": st["device_bytes_peak"]}
        # (b) sequential per-request reductions in arrival order
        ctx = graphic.Context(local_rank)
        outs = {n: torch.empty((n, n), dtype=torch.float32).pin_memory() for n in pool}
        for r, x in list(zip(reqs, inputs))[:3]:
            ctx.graphic_reduce_host(x, r["dx"], r["dy"], r["parang"], r["fwhm"], r["n_fwhm"], r["edges"],
                                    out_host=outs[r["n"]])
        q = _queue.Queue()
        t_arr = [0.0] * n_req
        t_done = [0.0] * n_req

        def worker():
            while True:
                i = q.get()
                if i is None:
                    return
                r = reqs[i]
                ctx.graphic_reduce_host(inputs[i], r["dx"], r["dy"], r["parang"], r["fwhm"], r["n_fwhm"],
                                        r["edges"], out_host=outs[r["n"]])
                t_done[i] = time.perf_counter()

        wt = threading.Thread(target=worker)
        wt.start()
        t0 = time.perf_counter()
        for i in range(n_req):
            dt = t0 + arr[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            t_arr[i] = time.perf_counter()
            q.put(i)
        q.put(None)
        wt.join()
        ctx.close()
        lat = [(t_done[i] - t_arr[i]) * 1e3 for i in range(n_req)]
        span = max(t_done) - min(t_arr)
        row["sequential"] = {"frames_per_s": frames / span, "p50_ms": statistics.median(lat),
                             "p99_ms": _pct(lat, 0.99), "span_s": span}
        row["speedup_frames_per_s"] = row["server"]["frames_per_s"] / row["sequential"]["frames_per_s"]
        results.append(row)
    return {"requests": n_req, "frames": frames, "input_bytes": in_bytes, "seed": seed, "max_active": max_active,
            "mix": "sides from {64,128,256,512,1024}, 16-400 frames (seeded), alt-az angles resampled per request, "
                   "full reduce each (shift, median PSF subtraction, derotation, collapse)",
            "host_inputs": "pinned host memory, copied in and the result copied out inside each request",
            "rates": results}


# ---------------------------------------------------------------------------
# uneven batches: 48 cubes, sides 64..1024, 16..400 frames, shift + rotation
# ---------------------------------------------------------------------------

def measure_uneven(local_rank, rank, steps, warmup, tune=True):
    """The 48-cube uneven batch (shift + rotation of every frame) through
    the per-cube, persistent and grouped executors, after the autotuner
    (unless tune is False).  Returns a dict."""
    import torch
    from paper_1510_04331_gb300 import graphic, synth

    torch.cuda.set_device(local_rank)
    spec = synth.uneven_spec(seed=3 + rank)
    gen = torch.Generator(device="cuda").manual_seed(1234 + rank)
    cubes = [torch.randn((T, n, n), generator=gen, device="cuda") for (n, T, _, _, _) in spec]
    outs = [torch.empty_like(c) for c in cubes]
    dx = [sp[2] for sp in spec]
    dy = [sp[3] for sp in spec]
    th = [sp[4] for sp in spec]
    frames = sum(sp[1] for sp in spec)
    ctx = graphic.Context(local_rank)
    tuned = None
    if tune:
        t0 = time.perf_counter()
        sched, t_pc, t_ps, t_gr = ctx.graphic_autotune(cubes, dx, dy, th, outs=outs)
        tuned = {"schedule": sched, "best_per_cube_ms": t_pc, "best_persistent_ms": t_ps, "best_grouped_ms": t_gr,
                 "tuning_s": time.perf_counter() - t0}
    res = {}
    modes = ((graphic.BATCH_PER_CUBE, "per_cube"), (graphic.BATCH_PERSISTENT, "persistent"),
             (graphic.BATCH_GROUPED, "grouped"))
    for mode, name in modes:
        for _ in range(warmup):
            ctx.graphic_batch_geom(cubes, dx, dy, th, outs=outs, mode=mode)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.graphic_batch_geom(cubes, dx, dy, th, outs=outs, mode=mode)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[name] = {"ms_p50": statistics.median(ms), "frames_per_s": frames / (statistics.median(ms) / 1e3)}
    batched = "grouped" if ctx.schedule()["batch_mode"] == graphic.BATCH_GROUPED else "persistent"
    ctx.close()
    nbytes = sum(c.numel() for c in cubes) * 4
    del cubes, outs
    torch.cuda.empty_cache()
    # algorithmic flops of the batch (nominal 5 m log2 m per complex line transform, both ways)
    flops = 0.0
    for (n, T, _, _, _) in spec:
        flops += T * sum(fft_flops_per_frame(k, n) for k in ("shift_x", "shift_y", "rot_pass1", "rot_pass2",
                                                              "rot_pass3"))
    bs = res[batched]["ms_p50"] / 1e3
    fpk, fsrc = fp32_peak(local_rank)
    return {
        "workload": "48 cubes, sides from {64,128,256,512,1024}, 16-400 frames each (seeded), shifts "
                    "U(-2,2) px, rotations U(0,360) deg", "frames": frames, "steps": steps, "warmup": warmup,
        "sides": [sp[0] for sp in spec], "counts": [sp[1] for sp in spec], "input_bytes": nbytes,
        "batched_mode": batched, "modes": res,
        "speedup_batched_vs_per_cube": res["per_cube"]["ms_p50"] / res[batched]["ms_p50"],
        "speedup_persistent_vs_per_cube": res["per_cube"]["ms_p50"] / res["persistent"]["ms_p50"],
        "autotune": tuned,
        "roofline": {"bound": "alu", "achieved": flops / bs / 1e12, "peak": fpk, "unit": "TFLOP/s",
                     "frac": flops / bs / 1e12 / fpk, "traffic": None, "kernel": "batch_" + batched,
                     "peak_source": fsrc, "algorithmic_per_launch": flops},
    }


def run_uneven(args, rank, world, local_rank):
    r = measure_uneven(local_rank, rank, args.steps, args.warmup, tune=not args.no_tune)
    b = r["batched_mode"]
    line = {
        "metric": "frames/s, uneven batch (shift + 3-shear rotation)", "value": r["modes"][b]["frames_per_s"],
        "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["modes"][b]["ms_p50"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": r["workload"], "frames": r["frames"], "sides": r["sides"], "counts": r["counts"],
                   "l2": "inputs larger than L2 (%.1f GB)" % (r["input_bytes"] / 1e9)},
        "batched_mode": b, "modes": r["modes"],
        "speedup_batched_vs_per_cube": r["speedup_batched_vs_per_cube"],
        "autotune": r["autotune"], "roofline": r["roofline"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_stage(args, rank, world, local_rank):
    """One step of the reduction alone on the survey recipe cube (resident
    on the device): `median` = the median PSF subtraction, `collapse` = the
    median collapse.  For kernel captures of a single step."""
    import torch
    from paper_1510_04331_gb300 import graphic

    torch.cuda.set_device(local_rank)
    d = make_workload("survey", args.frames, args.n)
    T, n = d.cube.shape[0], d.cube.shape[1]
    x = torch.from_numpy(d.cube).cuda()
    work = torch.empty_like(x) if args.workload == "median" else None
    img = torch.empty((n, n), dtype=torch.float32, device="cuda")
    ctx = graphic.Context(local_rank)

    def step():
        if args.workload == "median":
            ctx.graphic_adi_subtract(x, d.parang, d.fwhm, d.n_fwhm, d.edges, out=work)
        else:
            ctx.graphic_collapse_median(x, out=img)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ms = []
    ctx.profile(True)
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    prof = ctx.profile_read()
    ctx.profile(False)
    med = statistics.median(ms)
    nbytes = (2 if args.workload == "median" else 1) * T * n * n * 4
    hbm, src = peaks()
    line = {
        "metric": f"ms per call, {args.workload} step alone", "value": med, "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": med, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc("survey", d) + f"; {args.workload} step only", "frames": T, "n": n},
        "kernels": {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                    for k, v in prof.items() if v[1]},
        "hbm": {"algorithmic_bytes": nbytes, "gbs": nbytes / (med / 1e3) / 1e9,
                "frac": nbytes / (med / 1e3) / 1e9 / hbm, "peak_source": src},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="survey",
                    choices=sorted(WORKLOADS) + ["uneven", "serve", "precision", "prep", "register", "photometry",
                                                 "median", "collapse"])
    ap.add_argument("--no-tune", action="store_true", help="uneven workload: skip the autotuner")
    ap.add_argument("--frames", type=int, default=None, help="override the workload's frame count")
    ap.add_argument("--n", type=int, default=None, help="override the workload's frame side")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=15.0, help="seconds of oracle work per sample")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the uneven-batch and precision sub-measurements of the default line")
    ap.add_argument("--t-max", type=float, default=None,
                    help="time gate of the median PSF: reference frames within this many hours")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-max-active", type=int, default=64)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "uneven":
        return run_uneven(args, rank, world, local_rank)
    if args.workload in ("median", "collapse"):
        return run_stage(args, rank, world, local_rank)
    if args.workload == "precision":
        return run_precision(args, rank, world, local_rank)
    if args.workload == "prep":
        return run_prep(args, rank, world, local_rank)
    if args.workload == "register":
        return run_register(args, rank, world, local_rank)
    if args.workload == "photometry":
        return run_photometry(args, rank, world, local_rank)
    if args.workload == "serve":
        import torch
        torch.cuda.set_device(local_rank)
        sv = run_serving(local_rank, n_req=args.serve_requests, max_active=args.serve_max_active)
        top = sv["rates"][-1]
        line = {"metric": "frames/s, serving loop (full reduction requests)", "value": top["server"]["frames_per_s"],
                "unit": "frames/s", "n_gpus": world, "steps": 1, "warmup": 3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "serving: %d requests, Poisson arrivals, rates %s req/s" %
                                       (sv["requests"], [r["rate_per_s"] for r in sv["rates"]])},
                "serving": sv}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        return run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
