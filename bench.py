#!/usr/bin/env python
"""Benchmark of GB300 filter-bank correlation (one JSON line on stdout).

Headline workload: the precision configuration -- a 512x512x32 U[-1,1) input
correlated 'valid' against 256 filters of 5x5x32 drawn N(0, 1/800), giving a
508x508x256 output -- computed in split-BF16 (hi*hi + hi*lo + lo*hi on the
tcgen05 tensor cores, FP32 accumulation), reported next to the FP32 direct
kernel and plain BF16 on the same inputs.  One step = one forward call (BF16
split pre-pass + correlation kernel), inputs resident in HBM; the working set
(34 MB in, 264 MB out) exceeds the 129 MB L2, so no flush is needed between
steps.  GFLOP/s count 2*H'*W'*N*fh*fw*D per step (algorithmic FLOPs).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (no collective
on the data path); rank 0 prints the line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "filter-bank correlation GFLOP/s and % of roofline, split-BF16 vs FP32 at <=1e-5 rel err"
UNIT = "GFLOP/s"
HEADLINE_MODE = "bf16x3"


# ----------------------------------------------------------------------------- helpers
def load_peaks(sm_count: int) -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    src = "measured"
    try:
        with open(path) as f:
            pk = json.load(f)
    except Exception:
        pk = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
              "sm_max_mhz": 2070.0}
        src = "fallback"
    mhz = float(pk.get("sm_max_mhz", 2070.0))
    return {
        "source": src,
        "hbm_gbs": float(pk["hbm_gbs"]),
        "bf16_tflops": float(pk["bf16_tflops"]),
        "bf16_tflops_sustained": float(pk.get("bf16_tflops_sustained", pk["bf16_tflops"])),
        "sm_max_mhz": mhz,
        # FP32 FMA peak: SMs x 128 FP32 lanes x 2 FLOP x max SM clock
        "fp32_tflops": sm_count * 128 * 2 * mhz * 1e6 / 1e12,
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed loop runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="fbc_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(power) if power else None}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    """The slowest rank's value (replicas are timed together; the job ends
    when the last one does)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, ms: float, world: int) -> float:
    """Whole-job throughput of `world` independent replicas that each processed
    `units_per_rank` units, timed by the slowest rank (`ms`)."""
    return world * units_per_rank / (ms * 1e-3)


def time_loop(torch, fn, steps, warmup, world, flush=None):
    """W warm-up calls, then K timed calls bracketed by barrier + synchronize.
    Returns milliseconds per step (max over ranks).  With `flush`, every step is
    timed by its own event pair and L2 is flushed between steps outside them."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    if flush is None:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
    else:
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for a, b in evs:
            flush()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    barrier(world)
    return max_over_ranks(ms, world)


def make_flush(torch):
    buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def flush():
        buf.zero_()
    return flush


def workload_by_name(name):
    from paper_0911_3456_gb300 import inputs
    if name == "precision":
        return inputs.workload_precision()
    if name == "precision384":
        # the same recipe at 384x384x32 (output 148 MB, still above the L2 size),
        # used for detailed profiler captures
        rng = np.random.default_rng(3)
        x = inputs.uniform(rng, (384, 384, 32), -1.0, 1.0)
        w = inputs.normal(rng, (256, 5, 5, 32), var=1.0 / 800.0)
        return inputs.Workload("precision_384x384x32_256x5x5x32", x, w)
    if name == "paper_row1":
        return inputs.workload_paper_row1_clamp()
    if name == "small":
        return inputs.workload_small_f32()
    raise ValueError(name)


def l2_note(wl, out_shape):
    inb = wl.x.nbytes + wl.w.nbytes
    outb = int(np.prod(out_shape)) * 4
    if inb + outb > 129e6:
        return (f"no flush: {inb / 1e6:.0f} MB in + {outb / 1e6:.0f} MB out per step exceed the "
                f"129 MB L2")
    return f"working set {(inb + outb) / 1e6:.0f} MB fits in L2; back-to-back steps reuse it"


# ----------------------------------------------------------------------------- CPU oracle leg
def oracle_rows_sample(wl, rows, r0=None):
    """The oracle on `rows` consecutive output rows of the workload (a bounded
    sample); returns (rows start, FP64 output slab, seconds, cores)."""
    import oracle
    Ho = wl.out_shape[0]
    fh = wl.w.shape[1]
    if r0 is None:
        r0 = (Ho - rows) // 2
    slab = wl.x[r0:r0 + rows + fh - 1]
    t = time.perf_counter()
    y = oracle.fwd(slab, wl.w)
    dt = time.perf_counter() - t
    return r0, y, dt, oracle.max_threads()


def cpu_baseline(wl, target_s=12.0):
    """Time the oracle on a sample of output rows sized for about target_s
    (at most the whole output).  The oracle spreads output rows over its
    threads, so the per-row time is calibrated on two rows per thread."""
    import oracle
    Ho, Wo, N = wl.out_shape
    _, fh, fw, D = wl.w.shape
    row_flops = 2 * Wo * N * fh * fw * D
    k = max(1, min(Ho, 2 * oracle.max_threads()))
    _, _, dtk, cores = oracle_rows_sample(wl, k)
    rows = max(1, min(Ho, int(target_s * k / max(dtk, 1e-6))))
    r0, y, dt, cores = oracle_rows_sample(wl, rows)
    gflops = rows * row_flops / dt / 1e9
    single = oracle_single_core(wl, dt / rows * cores, min(2.0, target_s / 4))
    return {"value": gflops, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{rows} consecutive output rows (from row {r0}) of {Ho}: "
                      f"{rows * Wo * N} outputs, FP64 nested loops, OpenMP over rows",
            "seconds": dt, "single_core": single}, (r0, y)


def oracle_single_core(wl, row_s_guess, target_s):
    """The oracle on one thread over a slab of consecutive output rows sized
    for about target_s (from a per-row time guess), extrapolated linearly to the
    whole output and labelled as extrapolated."""
    import oracle
    Ho, Wo, N = wl.out_shape
    _, fh, fw, D = wl.w.shape
    row_flops = 2 * Wo * N * fh * fw * D
    rows = max(1, min(Ho, int(target_s / max(row_s_guess, 1e-6))))
    oracle.set_threads(1)
    try:
        r0, _, dt, _ = oracle_rows_sample(wl, rows)
    finally:
        oracle.set_threads(0)
    return {"value": rows * row_flops / dt / 1e9, "unit": UNIT, "cores": 1, "rows": rows, "seconds": dt,
            "whole_output_seconds_extrapolated": dt / rows * Ho,
            "note": f"{rows} consecutive output rows (from row {r0}) of {Ho} on one thread, "
                    "extrapolated linearly to the whole output"}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle timed as the reference arm on the headline workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_0911_3456_gb300 import inputs
    wl = inputs.workload_precision()
    Ho, Wo, N = wl.out_shape
    _, fh, fw, D = wl.w.shape
    per_point = 2 * fh * fw * D
    rng = np.random.default_rng(0)
    # calibrate points per second, then size each step so K + W steps take ~90 s
    idx = np.stack([rng.integers(0, Ho, 20000), rng.integers(0, Wo, 20000), rng.integers(0, N, 20000)], 1)
    t = time.perf_counter()
    oracle.fwd_points(wl.x, wl.w, idx)
    rate = 20000 / max(time.perf_counter() - t, 1e-6)
    budget = 90.0 / (args.steps + args.warmup)
    npts = int(max(256, min(2_000_000, rate * budget)))
    idx = np.stack([rng.integers(0, Ho, npts), rng.integers(0, Wo, npts), rng.integers(0, N, npts)], 1)
    for _ in range(args.warmup):
        oracle.fwd_points(wl.x, wl.w, idx)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.fwd_points(wl.x, wl.w, idx)
    dt = (time.perf_counter() - t) / args.steps
    value = npts * per_point / dt / 1e9
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl.name, "sample_points_per_step": npts},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{npts} random output elements of {Ho}x{Wo}x{N} per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def sampled_error(y_gpu_rows, ref_rows, scale=None):
    d = np.abs(y_gpu_rows.astype(np.float64) - ref_rows).max()
    s = np.abs(ref_rows).max() if scale is None else scale
    return float(d / s)


def measured_traffic(info, workload):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
    plan's correlation kernel, from profiles/traffic.json: entries are keyed by the
    hash of the generated kernel source, so a kernel changed since its capture
    (or a different tuned variant) finds none and reports null."""
    fwd = info.get("fwd", {})
    h = fwd.get("source_hash") or fwd.get("detail", {}).get("source_hash")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "traffic.json")
    if not h or not os.path.exists(path):
        return None, None
    with open(path) as f:
        entry = json.load(f).get(h)
    if not entry or entry.get("workload") != workload:
        return None, None
    return int(entry["dram_bytes_per_launch"]), entry.get("profile")


def fp32_fma_probe(sm_count: int, iters: int = 5000) -> dict:
    """The FP32 multiply-add rate the GPU sustains (the library's register-only
    probe, scalar FMAs and packed pairs), beside the nominal FP32 peak; run
    outside every timed region.  A failure is reported, not raised."""
    import ctypes
    from paper_0911_3456_gb300 import _capi as C
    lib = C.load()
    out = {"iters": iters}
    for name, pk in (("scalar", 0), ("packed", 1)):
        t, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
        st = lib.fbcorr_fp32_fma_probe(pk, iters, ctypes.byref(t), ctypes.byref(ms))
        if st != 0:
            return {"unavailable": f"{C.STATUS_NAMES.get(st, st)}: {C.last_error()}"}
        out[f"{name}_tflops"] = t.value
        out[f"{name}_ms"] = ms.value
    best = max(out["scalar_tflops"], out["packed_tflops"])
    # the SM clock at which 128 lanes x 2 FLOP per SM would give the best rate
    out["implied_sm_mhz"] = best * 1e12 / (sm_count * 128 * 2) / 1e6
    return out


def link_rate(torch, h2d_bytes, d2h_bytes, reps=5):
    """The host link measured on the e2e byte counts: one cudaMemcpyAsync per
    direction between page-locked host memory and the device (torch copy_),
    timed by CUDA events; each direction alone, and both at once on two
    streams (the link is full duplex, so that is the floor of a step that moves
    both).  Medians of `reps` runs."""
    hsrc = torch.empty(h2d_bytes, dtype=torch.uint8).pin_memory()
    ddst = torch.empty(h2d_bytes, dtype=torch.uint8, device="cuda")
    dsrc = torch.empty(d2h_bytes, dtype=torch.uint8, device="cuda")
    hdst = torch.empty(d2h_bytes, dtype=torch.uint8).pin_memory()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def alone(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s1)
        with torch.cuda.stream(s1):
            fn()
        e1.record(s1)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def duplex():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record(s1)
        s2.wait_event(e0)
        with torch.cuda.stream(s1):
            ddst.copy_(hsrc, non_blocking=True)
        e1.record(s1)
        with torch.cuda.stream(s2):
            hdst.copy_(dsrc, non_blocking=True)
        e2.record(s2)
        torch.cuda.synchronize()
        return max(e0.elapsed_time(e1), e0.elapsed_time(e2))

    h2d = statistics.median(alone(lambda: ddst.copy_(hsrc, non_blocking=True)) for _ in range(reps))
    d2h = statistics.median(alone(lambda: hdst.copy_(dsrc, non_blocking=True)) for _ in range(reps))
    both = statistics.median(duplex() for _ in range(reps))
    return {"h2d_gbs": h2d_bytes / (h2d * 1e-3) / 1e9, "d2h_gbs": d2h_bytes / (d2h * 1e-3) / 1e9,
            "h2d_ms": h2d, "d2h_ms": d2h, "duplex_ms": both,
            "how": "one cudaMemcpyAsync per direction, pinned host memory, CUDA events, median of "
                   f"{reps}; duplex = both directions at once on two streams"}


def run_ours(args):
    import torch
    from paper_0911_3456_gb300 import inputs
    from paper_0911_3456_gb300.api import Plan, BatchPlan

    world, rank, local = dist_setup()
    props = torch.cuda.get_device_properties(local)
    peaks = load_peaks(props.multi_processor_count)
    wl = workload_by_name(args.workload)
    flops = wl.flops
    x = torch.from_numpy(wl.x).cuda()
    w = torch.from_numpy(wl.w).cuda()

    # clocks: sampled from before the auto-tuning (which runs this plan's
    # kernels for seconds) to the end of the timed steps, so that a short timed
    # region still has samples under the same load
    clocks = ClockSampler(local)
    clocks.start()
    mode = args.mode
    plans = {}
    for m in dict.fromkeys([mode, "f32", "bf16", "bf16x3"]):
        if args.quick and m != mode:
            continue
        try:
            p = Plan(wl.x.shape, wl.w.shape, m, wl.clamp)
            if args.spec and m == mode:
                p.set_variant(args.spec)
            elif not args.no_tune:
                p.autotune()
            plans[m] = p
        except Exception as e:   # a mode the library cannot run is reported, not hidden
            if m == mode:
                raise
            plans[m] = e
    plan = plans[mode]
    y = torch.empty(plan.out_shape, device="cuda")

    # ---- headline: device-resident inputs, K back-to-back steps.  FP32: one
    # kernel per step, timed per launch by events inside the timed region.  The
    # tensor-core modes launch the operand split and the correlation kernel as
    # its programmatic dependent, which overlap; an event between steps holds the
    # next pair back, so the device time of a step is taken from the event pair
    # around the K timed steps.
    per_launch = mode == "f32"
    if per_launch:
        plan.profile(args.steps)
    ms = time_loop(torch, lambda: plan.forward(x, w, y), args.steps, args.warmup, world)
    clk = clocks.stop()
    clk["window"] = "plan auto-tuning, warm-up and the timed steps"
    if per_launch:
        kern_ms = plan.profile_read()
        plan.profile(0)
        kern_avg = float(np.mean(kern_ms)) if kern_ms else None
    else:
        kern_avg = ms
    value = replica_throughput(flops, ms, world) / 1e9
    info = plan.info()
    launches_per_step = int(info["fwd"].get("launches", 1))

    # roofline of the dominant kernel (the correlation kernel)
    if mode == "f32":
        peak = peaks["fp32_tflops"]
        roof = {"bound": "alu", "peak": peak, "unit": "TFLOP/s",
                "peak_note": "FP32 FMA: SMs x 128 lanes x 2 x max SM clock"}
    else:
        peak = peaks["bf16_tflops_sustained"] if args.steps * ms > 1000 else peaks["bf16_tflops"]
        roof = {"bound": "tensor", "peak": peak, "unit": "TFLOP/s",
                "peak_note": f"cuBLAS bf16 {'sustained' if args.steps * ms > 1000 else 'burst'}, "
                             f"{peaks['source']}"}
    achieved = flops / (kern_avg * 1e-3) / 1e12 if kern_avg else None
    traffic, traffic_src = measured_traffic(info, wl.name)
    roof.update({"achieved": achieved, "frac": (achieved / peak) if achieved else None,
                 "traffic": traffic, "kernel_ms": kern_avg,
                 "algorithmic_flops_per_launch": flops})
    if traffic_src:
        roof["traffic_profile"] = traffic_src
    if mode != "f32":
        roof["kernel_note"] = ("device time per step of the BF16 operand split and the correlation kernel "
                               "(launched as its programmatic dependent; they overlap), from the events "
                               "around the timed steps")
    if mode == "bf16x3" and achieved:
        # split BF16 spends three BF16 products per algorithmic multiply-add, so its
        # own ceiling in algorithmic FLOPs is a third of the BF16 peak
        roof["tensor_issued_tflops"] = 3 * achieved
        roof["peak_split_bf16x3"] = peak / 3
        roof["frac_of_split_peak"] = 3 * achieved / peak

    # ---- e2e through the C ABI from page-locked host buffers: fbcorr_forward_host
    # copies x and w in and y out every step, banded so that the transfers
    # overlap the compute; the same byte counts are also timed as plain copies
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(wl.x).pin_memory()
        wh = torch.from_numpy(wl.w).pin_memory()
        yh = torch.empty(plan.out_shape, dtype=torch.float32).pin_memory()

        def e2e_step():
            plan.forward_host(xh, wh, yh, bands=args.bands)

        k_e2e = max(3, min(args.steps, 100))
        ms_e2e = time_loop(torch, e2e_step, k_e2e, max(3, args.warmup), world)
        torch.cuda.synchronize()
        e2e_diff = float((yh - y.cpu()).abs().max() / y.abs().max())
        h2d_b, d2h_b = int(wl.x.nbytes + wl.w.nbytes), int(np.prod(plan.out_shape) * 4)
        e2e = {"value": world * flops / (ms_e2e * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms_e2e,
               "steps": k_e2e, "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b,
               "call": "fbcorr_forward_host", "bands": args.bands or "auto",
               "max_rel_diff_vs_device_forward": e2e_diff}
        try:
            link = link_rate(torch, h2d_b, d2h_b)
            link["e2e_frac_of_duplex_copy"] = link["duplex_ms"] / ms_e2e
            e2e["link"] = link
        except Exception as ex:   # reported, never fatal to the line
            e2e["link"] = {"unavailable": str(ex)}

    # ---- the same step back to back for about --sustained-s seconds (clocks
    # sampled during it), rated against the sustained BF16 peak
    sustained = None
    if args.sustained_s > 0 and not args.quick:
        n_s = max(args.steps, int(args.sustained_s * 1e3 / max(ms, 1e-3)))
        sc = ClockSampler(local)
        sc.start()
        ms_s = time_loop(torch, lambda: plan.forward(x, w, y), n_s, 3, world)
        sclk = sc.stop()
        sustained = {"steps": n_s, "seconds": n_s * ms_s / 1e3, "ms_per_step": ms_s,
                     "gflops": world * flops / (ms_s * 1e-3) / 1e9, "clocks": sclk}
        if mode != "f32":
            pk_s = peaks["bf16_tflops_sustained"]
            a_s = flops / (ms_s * 1e-3) / 1e12
            sustained["frac_of_sustained_peak"] = a_s / pk_s
            if mode == "bf16x3":
                sustained["frac_of_split_sustained_peak"] = 3 * a_s / pk_s

    detail = {"headline_plan": info}
    accuracy = None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # CPU oracle on a bounded sample; the same sample gives the error of every mode
        cpu, (r0, ref) = cpu_baseline(wl, target_s=args.cpu_seconds)
        rows = ref.shape[0]
        errs = {}
        for m, p in plans.items():
            if isinstance(p, Exception):
                errs[m] = f"unavailable: {p}"
                continue
            yy = p.forward(x, w)
            torch.cuda.synchronize()
            errs[m] = sampled_error(yy[r0:r0 + rows].cpu().numpy(), ref)
        accuracy = {"max_rel_err_vs_fp64_oracle": errs,
                    "definition": "max|y - y_oracle| / max|y_oracle| over the sample",
                    "sample_rows": [int(r0), int(r0 + rows)], "gates": {"f32": 1e-5, "bf16x3": 1e-5, "bf16": 1e-2}}

    # ---- the same workload in the other modes (kernel + step times)
    modes = {}
    summary = None
    if not args.quick:
        for m, p in plans.items():
            if isinstance(p, Exception):
                modes[m] = {"unavailable": str(p)}
                continue
            if m == "f32":
                p.profile(50)
            ms_m = time_loop(torch, lambda p=p: p.forward(x, w, y), 50, 3, world)
            if m == "f32":
                km = p.profile_read()
                p.profile(0)
                k_avg = float(np.mean(km)) if km else None
            else:
                k_avg = ms_m   # split + dependent correlation kernel, per step
            pk = peaks["fp32_tflops"] if m == "f32" else peaks["bf16_tflops"]
            modes[m] = {"gflops": flops / (ms_m * 1e-3) / 1e9, "ms_per_step": ms_m,
                        "kernel_ms": k_avg,
                        "kernel_frac_of_peak": (flops / (k_avg * 1e-3) / 1e12 / pk) if k_avg else None,
                        "peak_tflops": pk, "spec": p.info()["fwd"].get("spec")}
        detail["modes_same_workload"] = modes
        if "gflops" in modes.get("f32", {}) and "gflops" in modes.get(mode, {}):
            detail["speedup_vs_fp32_direct"] = modes[mode]["gflops"] / modes["f32"]["gflops"]
        detail.update(secondary(torch, args, world, peaks))
        try:
            detail["fp32_fma_probe"] = fp32_fma_probe(props.multi_processor_count)
        except Exception as e:   # reported, never fatal to the line
            detail["fp32_fma_probe"] = {"unavailable": str(e)}
        summary = summarize(detail, modes, mode)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": mode, "data": "synthetic",
            "config": {"workload": wl.name, "input": list(wl.x.shape), "bank": list(wl.w.shape),
                       "output": list(plan.out_shape), "mode": mode, "flops_per_step": flops,
                       "l2": l2_note(wl, plan.out_shape),
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "clocks": clk, "gpu_launches": launches_per_step * args.steps,
            "accuracy": accuracy, "sustained": sustained,
            "e2e": e2e, "cpu_baseline": cpu, "peaks": peaks, "summary": summary,
        }
        full = dict(line, detail=detail)
        if args.detail_out:
            with open(args.detail_out, "w") as f:
                json.dump(full, f, indent=1)
        print(json.dumps({"detail": detail}), file=sys.stderr, flush=True)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def summarize(detail, modes, mode):
    """The figures of the secondary workloads that the printed line keeps (the
    full record goes to --detail-out and stderr)."""
    def r3(v):
        return None if v is None else float(f"{v:.4g}")

    out = {"modes": {m: {"gflops": r3(v.get("gflops")), "kernel_frac_of_peak": r3(v.get("kernel_frac_of_peak")),
                         "spec": v.get("spec")} for m, v in modes.items() if "gflops" in v}}
    if "speedup_vs_fp32_direct" in detail:
        out["modes"][f"{mode}_speedup_vs_fp32_direct"] = r3(detail["speedup_vs_fp32_direct"])
    for key, name in (("small_128x128x8_16x9x9x8", "small_f32"), ("paper_row1_256x256x8_64x9x9x8_clamp",
                                                                     "paper_row1_clamp_f32")):
        v = detail.get(key)
        if v:
            out[name] = {k: r3(v.get(k)) if k != "tuned_spec" else v.get(k)
                         for k in ("default_gflops", "heuristic_gflops", "tuned_gflops", "boost_percent",
                                   "search_gain_percent", "tuned_frac_of_fp32_peak", "tuned_spec")}
            if v.get("stream"):
                out[name]["stream_gflops"] = r3(v["stream"]["gflops"])
                out[name]["stream_frac_of_fp32_peak"] = r3(v["stream"]["frac_of_fp32_peak"])
    if detail.get("paper_table_fp32"):
        out["paper_table_fp32"] = [{"shape": f"{'x'.join(map(str, r['input']))}/{'x'.join(map(str, r['bank']))}",
                                    "default": r3(r["default_gflops"]), "heuristic": r3(r["heuristic_gflops"]),
                                    "tuned": r3(r["tuned_gflops"]), "boost_percent": r3(r["boost_percent"]),
                                    "search_gain_percent": r3(r["search_gain_percent"])}
                                   for r in detail["paper_table_fp32"]]
    fb = detail.get("fwdbwd_256x256x16_64x7x7x16")
    if fb:
        out["fwdbwd_f32"] = {k: r3(fb[k]) for k in ("fwd_gflops", "dx_gflops", "dw_gflops", "fwd_bwd_gflops",
                                                     "fwd_bwd_frac_of_fp32_peak")}
    b = detail.get("batch64_uneven")
    if b:
        out["batch64_f32"] = {"gflops": r3(b["gflops"]), "frac_of_fp32_peak": r3(b["frac_of_fp32_peak"]),
                              "launches_per_step": b["launches_per_step"]}
    c = detail.get("cascade_3layer_256x256x8")
    if c:
        out["cascade_gflops"] = {m: r3(c[m]["gflops"]) for m in ("f32", "bf16x3") if m in c}
    nn = detail.get("nn_search_4096_patches_8x8")
    if nn:
        last = nn[-1]
        out["nn_search"] = {"neighbors": last["neighbors"], "ms": r3(last["ms"]),
                            "pairs_per_s": r3(last["pairs_per_s"]), "status": last["status"]}
    fma = detail.get("fp32_fma_probe")
    if fma and "packed_tflops" in fma:
        out["fp32_fma_probe_tflops"] = r3(max(fma["scalar_tflops"], fma["packed_tflops"]))
    return out


def stream_of_forwards(torch, p, x, w, y, flops, world, peaks, copies=128, replays=8):
    """A small workload as a stream of forwards: `copies` distinct (x, w, y)
    sets, together larger than L2, so every forward reads its operands from HBM;
    one forward per set captured in a CUDA graph and the graph replayed, so the
    launches queue on the device (the direct kernels are programmatic dependents:
    each one launches while the previous finishes) instead of waiting on the
    host.  Milliseconds per forward = event time of the replays / forwards."""
    xs = [x.clone() for _ in range(copies)]
    wsr = [w.clone() for _ in range(copies)]
    ys = [torch.empty_like(y) for _ in range(copies)]
    set_mb = copies * (x.numel() + w.numel() + y.numel()) * 4 / 1e6
    for i in range(copies):            # one eager pass: warm-up outside the capture
        p.forward(xs[i], wsr[i], ys[i])
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            for i in range(copies):
                p.forward(xs[i], wsr[i], ys[i])
    ms = time_loop(torch, graph.replay, replays, 3, world) / copies
    same = bool(torch.equal(ys[0], ys[-1]))
    return {"ms": ms, "gflops": flops / ms / 1e6, "frac_of_fp32_peak": flops / ms / 1e9 / peaks["fp32_tflops"],
            "forwards": copies * replays, "buffer_sets": copies, "buffer_mb": round(set_mb, 1),
            "l2": f"no flush: {copies} buffer sets ({set_mb:.0f} MB) cycled, larger than the 129 MB L2",
            "outputs_identical": same, "launch": "one CUDA graph of one forward per set, replayed"}


def boost_entry(torch, wl, world, flush, peaks):
    """One FP32 workload with the prebuilt default kernel, the generated kernel
    with the model's untimed tile (heuristic) and the tuned kernel, each timed
    with an L2 flush between steps; a workload under 1 GFLOP also as a stream of
    forwards over cold buffer sets."""
    from paper_0911_3456_gb300.api import Plan
    x = torch.from_numpy(wl.x).cuda()
    w = torch.from_numpy(wl.w).cuda()
    p = Plan(wl.x.shape, wl.w.shape, "f32", wl.clamp)
    y = torch.empty(p.out_shape, device="cuda")
    p.set_variant("default")
    ms_def = time_loop(torch, lambda: p.forward(x, w, y), 30, 3, world, flush)
    p.set_variant("heuristic")
    heur_spec = p.info()["fwd"].get("spec")
    ms_heur = time_loop(torch, lambda: p.forward(x, w, y), 30, 3, world, flush)
    p.autotune()
    ms_tuned = time_loop(torch, lambda: p.forward(x, w, y), 30, 3, world, flush)
    e = {"default_gflops": wl.flops / ms_def / 1e6, "heuristic_gflops": wl.flops / ms_heur / 1e6,
         "tuned_gflops": wl.flops / ms_tuned / 1e6,
         "boost_percent": 100.0 * (ms_def / ms_tuned - 1.0),
         "search_gain_percent": 100.0 * (ms_heur / ms_tuned - 1.0),
         "tuned_frac_of_fp32_peak": wl.flops / ms_tuned / 1e9 / peaks["fp32_tflops"],
         "tuned_ms_per_launch": ms_tuned, "l2": "flushed between steps, one event pair per step",
         "heuristic_spec": heur_spec, "tuned_spec": p.info()["fwd"].get("spec")}
    if wl.flops < 1e9:
        e["stream"] = stream_of_forwards(torch, p, x, w, y, wl.flops, world, peaks)
    return e


def small_only(args):
    """The first configuration alone (128x128x8 input, 16 filters 9x9x8, FP32):
    default, heuristic and tuned kernels with an L2 flush between steps, and the
    tuned kernel as a stream of forwards over cold buffer sets; one JSON line."""
    import torch
    from paper_0911_3456_gb300 import inputs
    world, rank, local = dist_setup()
    peaks = load_peaks(torch.cuda.get_device_properties(0).multi_processor_count)
    wl = inputs.workload_small_f32()
    e = boost_entry(torch, wl, world, make_flush(torch), peaks)
    if rank == 0:
        print(json.dumps({"metric": "FP32 forward GFLOP/s", "value": e["stream"]["gflops"], "unit": "GFLOP/s",
                          "higher_is_better": True, "config": {"workload": wl.name}, "small": e}), flush=True)
    return 0


def secondary(torch, args, world, peaks):
    """Other workloads of the method, each timed with an L2 flush between steps."""
    from paper_0911_3456_gb300 import inputs
    from paper_0911_3456_gb300.api import Plan
    flush = make_flush(torch)
    out = {}
    for name, wl in (("small_128x128x8_16x9x9x8", inputs.workload_small_f32()),
                     ("paper_row1_256x256x8_64x9x9x8_clamp", inputs.workload_paper_row1_clamp())):
        out[name] = boost_entry(torch, wl, world, flush, peaks)
    # the paper's own table shapes: default (prebuilt generic), heuristic (the
    # generated kernel with the model's tile, not searched) and tuned; the
    # table's "Default", "RTCG auto-tuned" and "Boost" columns measured here,
    # and tuned over heuristic, the gain of the search itself
    table = []
    for row in range(len(inputs.PAPER_TABLE_SHAPES)):
        wl = inputs.workload_paper_table(row)
        x = torch.from_numpy(wl.x).cuda()
        w = torch.from_numpy(wl.w).cuda()
        p = Plan(wl.x.shape, wl.w.shape, "f32")
        y = torch.empty(p.out_shape, device="cuda")
        p.set_variant("default")
        ms_def = time_loop(torch, lambda: p.forward(x, w, y), 20, 3, world, flush)
        p.set_variant("heuristic")
        heur_spec = p.info()["fwd"].get("spec")
        ms_heur = time_loop(torch, lambda: p.forward(x, w, y), 20, 3, world, flush)
        p.autotune()
        ms_tuned = time_loop(torch, lambda: p.forward(x, w, y), 20, 3, world, flush)
        table.append({"input": list(wl.x.shape), "bank": list(wl.w.shape),
                      "default_gflops": wl.flops / ms_def / 1e6, "heuristic_gflops": wl.flops / ms_heur / 1e6,
                      "tuned_gflops": wl.flops / ms_tuned / 1e6,
                      "boost_percent": 100.0 * (ms_def / ms_tuned - 1.0),
                      "search_gain_percent": 100.0 * (ms_heur / ms_tuned - 1.0),
                      "heuristic_spec": heur_spec,
                      "tuned_frac_of_fp32_peak": wl.flops / ms_tuned / 1e9 / peaks["fp32_tflops"],
                      "tuned_spec": p.info()["fwd"].get("spec")})
        del x, w, y, p
    out["paper_table_fp32"] = table

    wl = inputs.workload_differentiation()
    x = torch.from_numpy(wl.x).cuda()
    w = torch.from_numpy(wl.w).cuda()
    g = torch.from_numpy(wl.g).cuda()
    p = Plan(wl.x.shape, wl.w.shape, "f32")
    p.autotune()
    y = torch.empty(p.out_shape, device="cuda")

    def fb():
        p.forward(x, w, y)
        p.backward(x, w, g)
    ms_f = time_loop(torch, lambda: p.forward(x, w, y), 30, 3, world, flush)
    ms_dx = time_loop(torch, lambda: p.backward(x, w, g, need_dw=False), 30, 3, world, flush)
    ms_dw = time_loop(torch, lambda: p.backward(x, w, g, need_dx=False), 30, 3, world, flush)
    ms_fb = time_loop(torch, fb, 30, 3, world, flush)
    fp = peaks["fp32_tflops"]
    out["fwdbwd_256x256x16_64x7x7x16"] = {
        "fwd_gflops": wl.flops / ms_f / 1e6, "dx_gflops": wl.flops / ms_dx / 1e6,
        "dw_gflops": wl.flops / ms_dw / 1e6, "fwd_bwd_gflops": 3 * wl.flops / ms_fb / 1e6,
        "ms_fwd": ms_f, "ms_dx": ms_dx, "ms_dw": ms_dw, "ms_fwd_bwd": ms_fb,
        "fwd_bwd_frac_of_fp32_peak": 3 * wl.flops / ms_fb / 1e9 / fp,
        "plan": p.info()}
    # three-layer cascade: bank -> fused non-linearity (snippet epilogue) -> next bank
    from paper_0911_3456_gb300.cascade import Cascade, Layer
    cx, cbanks = inputs.workload_cascade()
    xd = torch.from_numpy(cx).cuda()
    wds = [torch.from_numpy(b).cuda() for b in cbanks]
    nl = ["y > 0.f ? y : 0.f", "fminf(fmaxf(y, 0.f), 1.f)", None]   # threshold, saturation, linear
    casc = {}
    for mode in ("f32", "bf16x3"):
        cas = Cascade(cx.shape, [Layer(b.shape[0], b.shape[1], b.shape[2], e) for b, e in zip(cbanks, nl)], mode)
        cas.autotune()
        outs = [torch.empty(pl.out_shape, device="cuda") for pl in cas.plans]
        ms_c = time_loop(torch, lambda: cas.forward(xd, wds, outs), 30, 3, world, flush)
        casc[mode] = {"gflops": cas.flops / ms_c / 1e6, "ms": ms_c,
                      "specs": [pl.info()["fwd"].get("spec") for pl in cas.plans]}
    out["cascade_3layer_256x256x8"] = {"layers": [list(b.shape) for b in cbanks],
                                       "nonlinearities": nl, "flops": cas.flops, **casc}
    del xd, wds, outs

    # exact nearest-neighbour search (Sec. 6.4): 4096 8x8 patches against the
    # paper's neighbour counts; the paper's GTX 295 seconds are context only
    from paper_0911_3456_gb300.api import NNPlan
    paper_gtx295_s = {4096: 0.089, 16384: 0.299, 65536: 1.146, 262144: 4.508, 1048576: 17.989}
    nn_rows = []
    for m in inputs.NN_NEIGHBORS:
        tq, nq = inputs.nn_patches(n_neighbors=m)
        td, nd = torch.from_numpy(tq).cuda(), torch.from_numpy(nq).cuda()
        plan_nn = NNPlan(tq.shape[0], m, tq.shape[1])
        res = {}

        def nn_step():
            res["out"] = plan_nn.search(td, nd)
        ms_nn = time_loop(torch, nn_step, 10, 3, world)
        row = {"targets": tq.shape[0], "neighbors": m, "dim": tq.shape[1], "ms": ms_nn,
               "pairs_per_s": tq.shape[0] * m / (ms_nn * 1e-3), "gflops_3_per_coord": plan_nn.flops / ms_nn / 1e6,
               "paper_gtx295_s": paper_gtx295_s.get(m), "status": plan_nn.device_status()}
        nn_rows.append(row)
        del td, nd, plan_nn, res
    out["nn_search_4096_patches_8x8"] = nn_rows

    # the 64-image uneven batch: one persistent launch replayed from a CUDA graph
    out["batch64_uneven"] = measure_batch(torch, world, flush, fp, 20, 3)
    return out


def measure_batch(torch, world, flush, fp, steps, warmup):
    """The 64-image uneven batch (per-image tiles auto-tuned on this GPU): one
    persistent launch per step, replayed from a CUDA graph, L2 flushed between
    steps."""
    from paper_0911_3456_gb300 import inputs
    from paper_0911_3456_gb300.api import BatchPlan
    bw = inputs.workload_batch()
    t0 = time.perf_counter()
    old_at = os.environ.get("FBCORR_AUTOTUNE")
    os.environ["FBCORR_AUTOTUNE"] = "1"          # per-variant tiles measured on this GPU
    try:
        bp = BatchPlan([it.x.shape for it in bw.items], [it.w.shape for it in bw.items])
    finally:
        if old_at is None:
            os.environ.pop("FBCORR_AUTOTUNE", None)
        else:
            os.environ["FBCORR_AUTOTUNE"] = old_at
    t_plan = time.perf_counter() - t0
    xs = [torch.from_numpy(it.x).cuda() for it in bw.items]
    wss = [torch.from_numpy(it.w).cuda() for it in bw.items]
    ys = [torch.empty(it.out_shape, device="cuda") for it in bw.items]
    ms_b = time_loop(torch, lambda: bp.forward(xs, wss, ys), steps, warmup, world, flush)
    binfo = bp.info()
    return {
        "gflops": bw.flops / ms_b / 1e6, "ms": ms_b, "flops": bw.flops,
        "frac_of_fp32_peak": bw.flops / ms_b / 1e9 / fp, "launches_per_step": binfo["launches"],
        "work_items": binfo["work_items"], "grid": binfo["grid"], "variants": len(binfo["variants"]),
        "plan_seconds_incl_tuning": t_plan, "tiles": [v["spec"] for v in binfo["variants"]]}


def batch_only(args):
    """The 64-image uneven batch alone: W warm-up and K timed steps (one
    persistent launch each); one JSON line."""
    import torch
    world, rank, local = dist_setup()
    peaks = load_peaks(torch.cuda.get_device_properties(0).multi_processor_count)
    steps = min(args.steps, 50)
    res = measure_batch(torch, world, make_flush(torch), peaks["fp32_tflops"], steps, args.warmup)
    if rank == 0:
        print(json.dumps({"metric": "batched FP32 forward GFLOP/s", "value": res["gflops"] * world,
                          "unit": "GFLOP/s", "higher_is_better": True, "steps": steps, "warmup": args.warmup,
                          "config": {"workload": "batch64_uneven", "l2": "flushed between steps"},
                          "batch": res}), flush=True)
    return 0


def nn_only(args):
    """The nearest-neighbour search alone: 4096 8x8 patches against args.nn
    neighbours (split BF16 screening, exact FP32 re-ranking), W warm-up and K
    timed searches; one JSON line."""
    import torch
    from paper_0911_3456_gb300 import inputs
    from paper_0911_3456_gb300.api import NNPlan
    world, rank, local = dist_setup()
    t, n = inputs.nn_patches(n_neighbors=args.nn)
    td, nd = torch.from_numpy(t).cuda(), torch.from_numpy(n).cuda()
    p = NNPlan(t.shape[0], args.nn, t.shape[1])
    steps = min(args.steps, 50)
    ms = time_loop(torch, lambda: p.search(td, nd), steps, args.warmup, world)
    if rank == 0:
        print(json.dumps({"metric": "exact nearest-neighbour search time", "value": ms, "unit": "ms",
                          "higher_is_better": False, "steps": steps, "warmup": args.warmup,
                          "pairs_per_s": t.shape[0] * args.nn / (ms * 1e-3), "status": p.device_status(),
                          "config": {"workload": f"nn_{t.shape[0]}x{args.nn}x{t.shape[1]}",
                                     "data": "synthetic 1/f-image 8x8 patches"}}), flush=True)
    return 0


def fwdbwd_only(args):
    """The differentiation workload alone (256x256x16 input, 64 filters 7x7x16,
    FP32): forward, dL/dx, dL/dw and the three together, each timed over K steps
    with an L2 flush between steps (its 20 MB working set fits in L2); one JSON line."""
    import torch
    from paper_0911_3456_gb300 import inputs
    from paper_0911_3456_gb300.api import Plan
    world, rank, local = dist_setup()
    peaks = load_peaks(torch.cuda.get_device_properties(0).multi_processor_count)
    flush = make_flush(torch)
    wl = inputs.workload_differentiation()
    x = torch.from_numpy(wl.x).cuda()
    w = torch.from_numpy(wl.w).cuda()
    g = torch.from_numpy(wl.g).cuda()
    p = Plan(wl.x.shape, wl.w.shape, "f32")
    if not args.no_tune:
        p.autotune()
    y = torch.empty(p.out_shape, device="cuda")
    steps = min(args.steps, 50)

    def fb():
        p.forward(x, w, y)
        p.backward(x, w, g)
    ms = {"fwd": time_loop(torch, lambda: p.forward(x, w, y), steps, args.warmup, world, flush),
          "dx": time_loop(torch, lambda: p.backward(x, w, g, need_dw=False), steps, args.warmup, world, flush),
          "dw": time_loop(torch, lambda: p.backward(x, w, g, need_dx=False), steps, args.warmup, world, flush),
          "fwd_bwd": time_loop(torch, fb, steps, args.warmup, world, flush)}
    if rank == 0:
        fp = peaks["fp32_tflops"]
        print(json.dumps({"metric": "FP32 forward + backward GFLOP/s", "value": 3 * wl.flops / ms["fwd_bwd"] / 1e6,
                          "unit": "GFLOP/s", "higher_is_better": True, "steps": steps, "warmup": args.warmup,
                          "ms": ms, "gflops": {k: (3 if k == "fwd_bwd" else 1) * wl.flops / v / 1e6
                                                for k, v in ms.items()},
                          "frac_of_fp32_peak": 3 * wl.flops / ms["fwd_bwd"] / 1e9 / fp,
                          "config": {"workload": wl.name, "l2": "flushed between steps"},
                          "plan": p.info()}), flush=True)
    return 0


def cascade_only(args):
    """The synthetic three-layer cascade alone (bank -> fused non-linearity
    snippet -> next bank across the previous output), in --mode f32 or
    bf16x3, K steps with an L2 flush between steps; one JSON line."""
    import torch
    from paper_0911_3456_gb300 import inputs
    from paper_0911_3456_gb300.cascade import Cascade, Layer
    world, rank, local = dist_setup()
    cx, cbanks = inputs.workload_cascade()
    xd = torch.from_numpy(cx).cuda()
    wds = [torch.from_numpy(b).cuda() for b in cbanks]
    nl = ["y > 0.f ? y : 0.f", "fminf(fmaxf(y, 0.f), 1.f)", None]   # threshold, saturation, linear
    mode = args.mode if args.mode in ("f32", "bf16x3", "bf16") else "f32"
    cas = Cascade(cx.shape, [Layer(b.shape[0], b.shape[1], b.shape[2], e) for b, e in zip(cbanks, nl)], mode)
    if not args.no_tune:
        cas.autotune()
    outs = [torch.empty(pl.out_shape, device="cuda") for pl in cas.plans]
    steps = min(args.steps, 50)
    ms = time_loop(torch, lambda: cas.forward(xd, wds, outs), steps, args.warmup, world, make_flush(torch))
    if rank == 0:
        print(json.dumps({"metric": "three-layer cascade GFLOP/s", "value": cas.flops / ms / 1e6, "unit": "GFLOP/s",
                          "higher_is_better": True, "steps": steps, "warmup": args.warmup, "ms": ms, "mode": mode,
                          "config": {"workload": "cascade_256x256x8", "layers": [list(b.shape) for b in cbanks],
                                     "nonlinearities": nl, "l2": "flushed between steps"},
                          "specs": [pl.info()["fwd"].get("spec") for pl in cas.plans]}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["f32", "bf16", "bf16x3"], default=HEADLINE_MODE)
    ap.add_argument("--quick", action="store_true", help="headline only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--bands", type=int, default=0, help="bands of the e2e host pipeline (0: automatic)")
    ap.add_argument("--spec", default=None,
                    help="forward variant of the headline plan instead of auto-tuning (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", choices=["precision", "precision384", "paper_row1", "small"],
                    default="precision")
    ap.add_argument("--detail-out", default=None,
                    help="write the full detail record (every secondary workload, plans) to this JSON file")
    ap.add_argument("--sustained-s", type=float, default=1.0,
                    help="seconds of the back-to-back sustained headline loop (0: skip)")
    ap.add_argument("--nn", type=int, default=0,
                    help="time only the nearest-neighbour search against this many neighbours")
    ap.add_argument("--fwdbwd", action="store_true",
                    help="the differentiation workload alone (forward, dL/dx, dL/dw)")
    ap.add_argument("--batch", action="store_true",
                    help="the 64-image uneven batch alone (one persistent launch per step)")
    ap.add_argument("--small", action="store_true",
                    help="the first configuration alone (flushed steps and a stream of forwards)")
    ap.add_argument("--cascade", action="store_true",
                    help="the three-layer cascade alone (--mode f32 or bf16x3)")
    args = ap.parse_args()
    if args.small:
        return small_only(args)
    if args.cascade:
        if args.warmup < 3:
            args.warmup = 3
        return cascade_only(args)
    if args.fwdbwd:
        if args.warmup < 3:
            args.warmup = 3
        return fwdbwd_only(args)
    if args.batch:
        if args.warmup < 3:
            args.warmup = 3
        return batch_only(args)
    if args.nn:
        if args.warmup < 3:
            args.warmup = 3
        return nn_only(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
