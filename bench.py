#!/usr/bin/env python3
"""Benchmark of the FSI hot path on B300: acc+grad pair interactions per second.

Workload (default): N = 2^20 Plummer stars with a Kroupa IMF plus 16 black holes of
50-100 Msun in the core, Henon units, speed of light c = 1e4 (PN1.0 pair terms for every
pair with a black hole), mixed precision.  One step = one complete FSI cycle of the whole
set (Sect. 2.1, Eq. fsi-cycle) wrapped in PN1.0 half-kicks (Sect. 3.9):
    PN(h/2)  kick h/6 [acc pass]  drift h/2  acc pass  kick 2h/3 with a + h^2/24 G
    [grad pass]  drift h/2  kick h/6 [acc pass]  PN(h/2)
i.e. 3 acceleration passes and 1 gradient pass over all N(N-1) ordered pairs.

Metric: acc+grad pair interactions per second, one interaction = one acceleration pair
term (20 flops) plus one gradient pair term (36 flops); a step therefore counts
N(N-1) (3*20 + 36) / 56 interactions.

Usage:  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica (the pair sum of one
cluster does not need more than one B300); value = total interactions of all ranks / the
slowest rank's time.
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
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_2210_02472_b300 import inputs  # noqa: E402

METRIC = "acc+grad pair interactions/s at N=2^20 (mixed precision, FSI cycle with PN1.0)"
UNIT = "interactions/s"
FLOP_ACC, FLOP_GRAD = 20, 36
FLOP_PAIR = FLOP_ACC + FLOP_GRAD
FP32_LANES, SM_MAX_MHZ = 128, 2032.0      # FP32 lanes per SM; B300 maximum SM clock
# FP64: B300's listed rate (1.25 TFLOP/s) over 148 SMs at 2.032 GHz is ~4 flop per SM per
# clock, i.e. two FP64 FMA lanes per SM; the FP64 peak below is that rate times the SM count
# the device reports times the maximum SM clock.
FP64_FLOP_PER_SM_CLK = 4
CPU_ROWS = 4096
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant
# kernel (per pass: both kernels of a pass that takes two), from one one-pass ncu capture
# of this benchmark's own workload (`--tuning A,G --steps 1 --warmup 3` with the kernel's
# variant, mean of the cycle's three acceleration passes).  Keyed by
# (kernel label, workload, N); a kernel changed since the capture must drop its entry, and
# any other configuration reports null.
DRAM_TRAFFIC = {("sym_mixed_v2_kernel<acc, I=5, far>", "kroupa1m_bh16", 1048592): 201.9e6,
                ("sym_mixed_x2_kernel<acc, I=8, MINB=1> + sym_diag_ff_kernel", "kroupa1m_bh16",
                 1048592): 301.0e6}


def step_interactions(n: int) -> float:
    pairs = float(n) * float(n - 1)
    return pairs * (3 * FLOP_ACC + FLOP_GRAD) / FLOP_PAIR


def sm_count(device=None) -> int:
    """Streaming multiprocessors of the device, as the driver reports them."""
    import torch
    return int(torch.cuda.get_device_properties(device if device is not None else 0).multi_processor_count)


def fp32_peak_tflops(sms: int, mhz: float = SM_MAX_MHZ) -> float:
    return sms * FP32_LANES * 2 * mhz * 1e6 / 1e12


def fp64_peak_tflops(sms: int, mhz: float = SM_MAX_MHZ) -> float:
    return sms * FP64_FLOP_PER_SM_CLK * mhz * 1e6 / 1e12


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    try:
        return json.loads(p.read_text())
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


CPU_ROW_SEED, CPU_FIELD_SEED = 4242, 4243


def cpu_baseline(c, rows: int, threads: int):
    """The FP64 CPU oracle, as it stands, on a seeded sample of `rows` active particles
    against all N sources: acc and grad pair sums.  Returns interactions/s and an info dict
    that also holds the sample's rows and the oracle's sums (for the accuracy check of the
    GPU results on the same rows)."""
    import oracle
    oracle.set_threads(threads)
    A = inputs.random_subset(c.n, rows, CPU_ROW_SEED)
    accg = inputs.random_field(c.n, CPU_FIELD_SEED)
    t0 = time.perf_counter()
    a = oracle.acc(c.pos, c.mass, A, None)
    t1 = time.perf_counter()
    g = oracle.grad(c.pos, c.mass, accg, A, None)
    t2 = time.perf_counter()
    pairs = float(rows) * (c.n - 1)
    inter = pairs * (FLOP_ACC + FLOP_GRAD) / FLOP_PAIR
    return inter / (t2 - t0), {"acc_s": t1 - t0, "grad_s": t2 - t1, "rows": A, "acc": a, "grad": g,
                               "sample": f"{rows} seeded active rows x all {c.n} sources, "
                                         f"acc + grad (FP64 oracle)"}


def error_stats(got, ref):
    """Distribution of |d v| / |v| over the columns of (3, n) arrays."""
    d = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    return {"rows": int(d.size), "median": float(np.median(d)), "p99": float(np.percentile(d, 99)),
            "p99.9": float(np.percentile(d, 99.9)), "max": float(d.max()),
            "frac_above_1e-7": float(np.mean(d > 1e-7))}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("FSI_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
        return rank, ws, local, dist
    return rank, ws, local, None


def reduce_max(value: float, dist, device=None) -> float:
    """Max of a per-rank float over all ranks (identity without a process group).  Uses a
    CPU tensor with gloo and a device tensor with NCCL."""
    if dist is None:
        return float(value)
    import torch
    on_cpu = dist.get_backend() == "gloo" or device is None
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device="cpu" if on_cpu else device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world_size: int, t_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world_size / t_max


def run_reference(args):
    rank, ws, local, dist = dist_init()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    c = inputs.workload(args.workload)
    threads = os.cpu_count() or 1
    rows = max(16, args.ref_rows)
    for _ in range(args.warmup):
        cpu_baseline(c, 16, threads)
    vals, times = [], []
    info = None
    for _ in range(args.steps):
        v, info = cpu_baseline(c, rows, threads)
        vals.append(v)
        times.append(info["acc_s"] + info["grad_s"])
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": c.n, "oracle": "plain FP64 C, OpenMP over rows"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": info["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def fp64_passes(F, c, pos, mass, dev, flush, sms, peak_mhz):
    """The FP64 half of the metric on the same set: one same-set acceleration pass and one
    force-gradient pass over all N(N-1) ordered pairs (fsi_accel_grad, FP64 context), each
    timed by the library's event pair around its launch, L2 flushed before.  Pipe fraction
    against the FP64 peak of this device (SM count queried, FP64 FMA rate per SM, maximum
    SM clock) and against the library's FP64 FMA probe."""
    import torch
    N = c.n
    ctx = F.Context("fp64")
    F.fsi_reserve(ctx, N, N)
    sub = torch.arange(0, min(N, 16384), dtype=torch.int32, device=dev)
    F.fsi_accel_grad(ctx, pos, None, mass, sub, sub)          # warm-up of the same kernels
    torch.cuda.synchronize()
    flush.zero_()
    F.fsi_profile(ctx, True)
    e0, e1 = _timed_events(None)
    e0.record()
    F.fsi_accel_grad(ctx, pos, None, mass)
    e1.record()
    torch.cuda.synchronize()
    prof = F.fsi_profile_read(ctx)
    F.fsi_profile(ctx, False)
    if F.fsi_sync_status(ctx) != F.FSI_OK:
        raise SystemExit("device error in the FP64 passes")
    t = e0.elapsed_time(e1) / 1e3
    probe = probe_peak_tflops(F, 1)
    ctx.close()
    pairs = float(N) * (N - 1)
    peak = fp64_peak_tflops(sms, peak_mhz)
    out = {"workload": "same set as the cycle", "n": N,
           "passes": "one same-set acc pass + one grad pass (fsi_accel_grad), FP64 pair terms",
           "value": pairs / t, "unit": "acc+grad interactions/s", "s_per_acc_grad": t,
           "peak_tflops": peak,
           "peak_basis": f"{sms} SMs x {FP64_FLOP_PER_SM_CLK} FP64 flop per SM per clock x "
                         f"{peak_mhz:.0f} MHz",
           "probe_tflops": probe}
    tot_fl, tot_s = 0.0, 0.0
    for k, fl in (("acc", FLOP_ACC), ("grad", FLOP_GRAD)):
        nl, ms = prof[k]
        ach = pairs * fl / (ms / max(nl, 1) / 1e3) / 1e12
        tot_fl += pairs * fl
        tot_s += ms / 1e3
        out[k] = {"ms_per_launch": ms / max(nl, 1), "launches": nl, "achieved_tflops": ach,
                  "frac": ach / peak, "frac_of_probe": ach / probe}
    out["frac"] = tot_fl / tot_s / 1e12 / peak     # acc + grad together
    return out


def run_fsi(args):
    import torch
    rank, ws, local, dist = dist_init()
    torch.cuda.set_device(local)
    from paper_2210_02472_b300 import fsi as F

    c = inputs.workload(args.workload)
    if args.n:
        c = inputs.plummer(args.n, inputs.SEED_BASE + 3, imf="kroupa", n_bh=16)
    N = c.n
    dev = torch.device("cuda", local)
    pos0 = torch.as_tensor(c.pos).to(dev)
    vel0 = torch.as_tensor(c.vel).to(dev)
    mass = torch.as_tensor(c.mass).to(dev)
    bh = torch.as_tensor(c.is_bh.astype(np.uint8)).to(dev)
    pos, vel = pos0.clone(), vel0.clone()
    h = 1.0 / 1024
    cl = 1e4
    ctx = F.Context(args.precision, c=cl)
    F.fsi_reserve(ctx, N, N)
    if args.tuning:
        tuning = tuple(int(x) for x in args.tuning.split(","))
        F.fsi_set_tuning(ctx, *tuning)
    else:
        tuning = F.fsi_autotune(ctx, pos, mass, n=N, reps=1)   # variant per kernel kind
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step():
        F.fsi_step(ctx, pos, vel, mass, h, nsteps=1, is_bh=bh)

    e0 = F.fsi_energy(ctx, pos, vel, mass).sum().item() if not args.no_energy else None
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if F.fsi_sync_status(ctx) != F.FSI_OK:
        raise SystemExit(f"device error after warm-up: {F._lib.fsi_last_error()}")

    # ---- device-timed region (inputs resident in HBM)
    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    F.fsi_profile(ctx, True)
    F.fsi_far_stats(ctx, reset=True)
    n0 = F.fsi_launch_count()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                       # L2 flush between steps (outside the events)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = F.fsi_launch_count() - n0 - 0
    clocks = sampler.stop()
    prof = F.fsi_profile_read(ctx)
    F.fsi_profile(ctx, False)
    far_v, near_v = F.fsi_far_stats(ctx)
    if F.fsi_sync_status(ctx) != F.FSI_OK:
        raise SystemExit("device error in the timed region")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    e1 = F.fsi_energy(ctx, pos, vel, mass).sum().item() if not args.no_energy else None
    t_dev = reduce_max(sum(step_ms) / 1e3, dist, dev)
    inter = step_interactions(N) * args.steps
    value = job_value(inter, ws, t_dev)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    hpos = torch.as_tensor(c.pos).pin_memory()
    hvel = torch.as_tensor(c.vel).pin_memory()
    opos = torch.empty_like(hpos).pin_memory()
    ovel = torch.empty_like(hvel).pin_memory()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pos.copy_(hpos, non_blocking=True)
        vel.copy_(hvel, non_blocking=True)
        step()
        opos.copy_(pos, non_blocking=True)
        ovel.copy_(vel, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = reduce_max(time.perf_counter() - t0, dist, dev)
    e2e_value = job_value(step_interactions(N) * e2e_steps, ws, t_e2e)
    bytes_io = 2 * 3 * N * 8

    # ---- roofline of the dominant pair kernel (FP32 pipe bound for the mixed path)
    kinds = {"acc": FLOP_ACC, "grad": FLOP_GRAD}
    dom = max(kinds, key=lambda k: prof[k][1])
    nl, ms = prof[dom]
    achieved = (float(N) * (N - 1) * kinds[dom]) / (ms / nl / 1e3) / 1e12
    sms = sm_count(dev)
    peak_mhz = clocks.get("sm_max_mhz") or SM_MAX_MHZ
    peak = fp32_peak_tflops(sms, peak_mhz) if args.precision == "mixed" else fp64_peak_tflops(sms, peak_mhz)
    var = tuning[0 if dom == "acc" else 1]
    if var & 128 and var & 512:
        kname = f"sym_mixed_x2_kernel<{dom}, I={var & 15}, MINB=1, NT=384>"
    elif var & 128:
        kname = f"sym_mixed_x2_kernel<{dom}, I={var & 15}, MINB={1 if var & 16 else 2}>"
    if var & 128 and dom == "acc" and args.precision == "mixed" and N >= 196608:
        # the pass's time includes the float-float kernel of the pairs inside each i-block
        kname += " + sym_diag_ff_kernel"
    elif var & 32:
        kname = f"sym_mixed_v2_kernel<{dom}, I={var & 15}{', far' if var & 64 else ''}>"
    else:
        kname = f"sym_pair_kernel<{args.precision}, {dom}, I={var & 15}>"
    traffic = DRAM_TRAFFIC.get((kname, args.workload if not args.n else "", N))
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                "traffic_basis": ("DRAM bytes per launch, one ncu capture of this workload"
                                  if traffic else None),
                "sm_count": sms,
                "peak_basis": (f"{sms} SMs (device query) x 128 FP32 lanes x 2 flop x {peak_mhz:.0f} MHz "
                               "(max SM clock)" if args.precision == "mixed" else
                               f"{sms} SMs (device query) x {FP64_FLOP_PER_SM_CLK} FP64 flop per SM "
                               f"per clock x {peak_mhz:.0f} MHz (max SM clock)"),
                "per_kernel_ms": {k: prof[k][1] / max(prof[k][0], 1) for k in prof},
                "per_kernel_launches": {k: prof[k][0] for k in prof}}
    if clocks.get("sm_mhz"):
        roofline["frac_at_median_clock"] = achieved / (
            fp32_peak_tflops(sms, clocks["sm_mhz"]) if args.precision == "mixed"
            else fp64_peak_tflops(sms, clocks["sm_mhz"]))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": N, "precision": args.precision,
                   "step": "one FSI cycle of all N + PN1.0 half-kicks (3 acc + 1 grad pair passes)",
                   "c": cl, "h": h, "l2": "flushed between steps (256 MB write)",
                   "tuning": {"acc_variant": tuning[0], "grad_variant": tuning[1]},
                   "far_tile_visits": {"far": far_v, "near": near_v,
                                       "far_fraction": far_v / max(far_v + near_v, 1)},
                   "parallelism": f"replicas x{ws}"},
        "wall_s": wall, "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bytes_io,
                "d2h_bytes_per_step": bytes_io, "steps": e2e_steps},
        "roofline": roofline, "clocks": clocks,
    }
    # ---- energy drift over the warm-up and timed cycles (FP64 energy, outside the timing)
    if e1 is not None:
        line["energy"] = {"cycles": args.warmup + args.steps, "h": h, "E0": e0,
                          "rel_drift": abs((e1 - e0) / e0),
                          "what": "|E1 - E0| / |E0| of the FP64 energy of all N (T + W) before "
                                  "the warm-up and after the timed cycles"}
    if rank == 0 and args.precision == "mixed" and not args.no_fp64:
        line["fp64"] = fp64_passes(F, c, pos0, mass, dev, flush, sms, peak_mhz)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        # the kernels' sums at the initial state, for the accuracy check on the oracle's rows
        ga = F.fsi_accel(ctx, pos0, mass).cpu().numpy()
        gg = F.fsi_grad(ctx, pos0, mass, torch.as_tensor(
            inputs.random_field(N, CPU_FIELD_SEED)).to(dev)).cpu().numpy()
        v, info = cpu_baseline(c, args.cpu_rows, threads)
        v1, info1 = cpu_baseline(c, args.cpu_rows_1t, 1)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": info["sample"],
                                "value_1thread": v1, "sample_1thread": info1["sample"]}
        rows = info["rows"]
        line["accuracy"] = {
            "against": "the FP64 oracle on the cpu_baseline sample (same-set passes of the "
                       "benchmark's kernels at the initial state; gradient with a seeded field)",
            "acc": error_stats(ga[:, rows], info["acc"]),
            "grad": error_stats(gg[:, rows], info["grad"])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def _timed_events(stream):
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_ensemble(args):
    """512 independent clusters, N log-uniform in [64, 8192], Kroupa IMF, mixed precision:
    one persistent launch of `--batch-steps` FSI cycles per call, replayed from a CUDA graph."""
    import torch
    from paper_2210_02472_b300 import fsi as F
    torch.cuda.set_device(0)
    cat, off = inputs.ensemble(512, 64, 8192, inputs.SEED_BASE + 5)
    sizes = np.diff(off).astype(np.float64)
    pairs = float((sizes * (sizes - 1)).sum())
    S = args.batch_steps
    per_call = pairs * ((1 + 2 * S) * FLOP_ACC + S * FLOP_GRAD) / FLOP_PAIR
    dev = torch.device("cuda", 0)
    m = torch.as_tensor(cat.mass).to(dev)
    ctx = F.Context(args.precision)
    b = F.Batch(ctx, off, max_steps=S)
    # autotune: particles per thread x resident CTAs per SM (or fixed by --batch-tuning)
    best = None
    fixed = [tuple(int(x) for x in args.batch_tuning.split(","))] if args.batch_tuning else None
    combos = fixed or [(ipt, cps) for ipt in ((1, 2, 4, 6, 8) if args.precision == "mixed" else (1, 2))
                       for cps in (1, 2, 0) if not (ipt == 8 and cps == 2)]   # ipt 4, 6, 8: symmetric
    for ipt, cps in combos:
        F.fsi_batch_set_tuning(ctx, b, ipt, cps)
        p, v = torch.as_tensor(cat.pos).to(dev), torch.as_tensor(cat.vel).to(dev)
        F.fsi_batch_step(ctx, b, p, v, m, 1e-3, S)
        e0, e1 = _timed_events(None)
        e0.record()
        F.fsi_batch_step(ctx, b, p, v, m, 1e-3, S)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        if best is None or t < best[0]:
            best = (t, F.fsi_batch_get_tuning(b))
    F.fsi_batch_set_tuning(ctx, b, *best[1])
    p, v = torch.as_tensor(cat.pos).to(dev), torch.as_tensor(cat.vel).to(dev)
    # per-cluster energies (FP64 pair sums) before and after every replayed cycle
    members = [torch.arange(off[k], off[k + 1], dtype=torch.int32, device=dev)
               for k in range(len(off) - 1)]

    def energies():
        return np.array([float(F.fsi_energy(ctx, p, v, m, P=ids).sum()) for ids in members])

    e_start = energies()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    n_cap = F.fsi_launch_count()
    with torch.cuda.graph(g, stream=s):
        F.fsi_batch_step(ctx, b, p, v, m, 1e-3, S, stream=s)
    kernels_per_replay = F.fsi_launch_count() - n_cap      # kernel nodes of the graph
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sampler = ClockSampler(0)
    sampler.start()
    F.fsi_batch_stats(b, reset=True)
    F.fsi_batch_item_stats(b, reset=True)
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = _timed_events(None)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    wait_ns, life_ns, ctas = F.fsi_batch_stats(b)
    item_stats = F.fsi_batch_item_stats(b)
    de = np.abs((energies() - e_start) / e_start)
    assert F.fsi_sync_status(ctx) == F.FSI_OK
    t = sum(ms) / 1e3
    # idle: CTA time spent waiting for other CTAs' phases, plus CTAs out of work before the
    # launch ended, over the launch's whole CTA capacity (CTAs x elapsed time)
    cap_ns = ctas * t * 1e9
    idle = {"fraction": 1.0 - (life_ns - wait_ns) / cap_ns, "phase_waits": wait_ns / cap_ns,
            "tail": 1.0 - life_ns / cap_ns, "ctas": ctas}
    # busy CTA time by work-item kind (symmetric form), as fractions of the CTA capacity
    busy = {k: {"fraction": ns / cap_ns, "items": n}
            for k, (ns, n) in zip(("own_pairs", "two_blocks", "pack_apply"), item_stats)}
    value = per_call * args.steps / t
    ach = value * FLOP_PAIR / 1e12
    peak = fp32_peak_tflops(sm_count(dev)) if args.precision == "mixed" else fp64_peak_tflops(sm_count(dev))
    line = {
        "metric": "ensemble acc+grad pair interactions/s (512 clusters, N in [64, 8192])",
        "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": "ensemble512", "clusters": 512, "n_total": int(off[-1]),
                   "pairs_per_pass": pairs, "fsi_cycles_per_launch": S,
                   "launch": "one persistent kernel per call, replayed from a CUDA graph",
                   "tuning": {"ipt": best[1][0], "ctas_per_sm": best[1][1]},
                   "l2": "flushed between launches (256 MB write)"},
        "gpu_launches": kernels_per_replay * args.steps,
        "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                     "frac": ach / peak, "traffic": None,
                     "kernel": "batch_sym_kernel" if best[1][0] == 4 else "batch_kernel"},
        "idle": idle, "busy": busy,
        # fixed h, no softening: a few of the smallest clusters meet close encounters the
        # step does not resolve (the oracle's own FSI gives |dE/E| ~ 1-10 on them)
        "energy": {"fsi_cycles": (args.warmup + args.steps) * S, "h": 1e-3,
                   "median_rel_error": float(np.median(de)),
                   "p90_rel_error": float(np.percentile(de, 90)), "max_rel_error": float(de.max()),
                   "clusters_above_1e-3": int((de > 1e-3).sum())},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    b.close()
    ctx.close()
    return 0


def run_vjp(args):
    """N = 16384 equal-mass Plummer, FP64, 200 FSI steps of h = 1e-3, L = sum |x|^2;
    gradient w.r.t. (x0, v0, m) by the checkpointed adjoint (every 20 steps), timed
    against the forward; central finite differences on a few components."""
    import math
    import torch
    from paper_2210_02472_b300 import fsi as F
    from paper_2210_02472_b300.autodiff import fsi_rollout
    torch.cuda.set_device(0)
    c = inputs.workload("plummer16k")
    dev = torch.device("cuda", 0)
    h, steps = 1e-3, args.vjp_steps
    ctx = F.Context("fp64")
    x = torch.as_tensor(c.pos).to(dev).requires_grad_(True)
    v = torch.as_tensor(c.vel).to(dev).requires_grad_(True)
    m = torch.as_tensor(c.mass).to(dev).requires_grad_(True)
    # warm-up (untimed): one checkpoint segment and its adjoint, so that neither timed pass
    # pays for first-use set-up (module loading, kernel attributes, workspace allocation)
    xw, vw, mw = (t.detach().clone().requires_grad_(True) for t in (x, v, m))
    pw, _ = fsi_rollout(ctx, xw, vw, mw, h, 20, ckpt_every=20)
    (pw * pw).sum().backward()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p, _ = fsi_rollout(ctx, x, v, m, h, steps, ckpt_every=20)
    L = (p * p).sum()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    L.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    grads = [x.grad.cpu().numpy(), v.grad.cpu().numpy(), m.grad.cpu().numpy()]

    def final(px, pv, pm):
        P, V = torch.as_tensor(px).to(dev), torch.as_tensor(pv).to(dev)
        F.fsi_step(ctx, P, V, torch.as_tensor(pm).to(dev), h, nsteps=steps)
        return P.cpu().numpy()

    rng = np.random.default_rng(20221009)
    fd = []
    for t in range(args.fd_components):
        which = t % 3
        k, i = int(rng.integers(3)), int(rng.integers(c.n))
        arrs = [c.pos.copy(), c.vel.copy(), c.mass.copy()]
        idx = (i,) if which == 2 else (k, i)
        step = 1e-4 * arrs[2][i] if which == 2 else 1e-6
        arrs[which][idx] += step
        fp = final(*arrs)
        arrs[which][idx] -= 2 * step
        fm = final(*arrs)
        d = math.fsum(((fp * fp) - (fm * fm)).ravel()) / (2 * step)
        an = float(grads[which][idx])
        fd.append({"var": "xvm"[which], "index": [int(q) for q in idx], "fd": d, "vjp": an,
                   "rel_diff": abs(d - an) / max(abs(an), 1e-300)})
    line = {
        "metric": "adjoint (VJP) of a 200-step FSI rollout: backward / forward time",
        "value": (t2 - t1) / (t1 - t0), "unit": "ratio", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": 1e3 * (t2 - t0), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "plummer16k", "n": c.n, "steps": steps, "h": h, "ckpt_every": 20,
                   "loss": "sum |x_final|^2"},
        "forward_s": t1 - t0, "backward_s": t2 - t1, "finite_differences": fd,
        "max_rel_diff": max([q["rel_diff"] for q in fd], default=None),
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# The softened equal-mass long run of Sect. 5.2 in Henon units: 161000 stars of 0.5 Msun
# (M = 80500 Msun), half-mass radius 3.1 pc, softening length 1e-3 pc, interval 1e-3 Myr,
# eta 0.2 (free fall, fly-by) and 0.1 (jerk, gradient).  Plummer: r_h = a / (2^{2/3} - 1)^{1/2}
# with a = 3 pi / 16, so the length unit is 3.1 pc / r_h and the time unit
# (L^3 / (G M))^{1/2} with G = 4.4985e-3 pc^3 / (Msun Myr^2).
SOFT_RH_NB = (3.0 * math.pi / 16.0) / math.sqrt(2.0 ** (2.0 / 3.0) - 1.0)
SOFT_LUNIT_PC = 3.1 / SOFT_RH_NB
SOFT_TUNIT_MYR = math.sqrt(SOFT_LUNIT_PC ** 3 / (4.4985e-3 * 80500.0))
SOFT_EPS = 1e-3 / SOFT_LUNIT_PC
SOFT_TAU = 1e-3 / SOFT_TUNIT_MYR


def run_hhs(args):
    """HHS intervals: N = 65536 Plummer with a Kroupa IMF, eps = 0, tau0 = 1/64 (default);
    with --workload plummer161k the softened equal-mass long run (Sect. 5.2 setup), which
    reports the energy error of every interval."""
    import torch
    from paper_2210_02472_b300 import fsi as F
    torch.cuda.set_device(0)
    wl = args.workload if args.workload != "kroupa1m_bh16" or args.hhs_pn else "kroupa64k"
    c = inputs.workload(wl) if not args.n else inputs.plummer(args.n, inputs.SEED_BASE + 2, imf="kroupa")
    dev = torch.device("cuda", 0)
    pos, vel = torch.as_tensor(c.pos).to(dev), torch.as_tensor(c.vel).to(dev)
    mass = torch.as_tensor(c.mass).to(dev)
    bh = torch.as_tensor(c.is_bh.astype(np.uint8)).to(dev)
    cl = 1e4 if args.hhs_pn else 0.0
    soft = wl == "plummer161k"
    tau = SOFT_TAU if soft else args.tau
    kw = dict(eps2=SOFT_EPS ** 2, eta_ff=0.2, eta_fb=0.2, eta_jerk=0.1, eta_grad=0.1) if soft else {}
    ctx = F.Context(args.precision, c=cl, wide_ctas=args.wide_ctas,
                    hhs_small_max=args.hhs_small_max, order_min=args.order_min,
                    hhs_grid_max=args.hhs_grid_max, **kw)
    if args.tuning:
        F.fsi_set_tuning(ctx, *[int(v) for v in args.tuning.split(",")])
    energy = lambda: float(F.fsi_energy(ctx, pos, vel, mass).cpu().numpy().sum())
    warm = 1 if args.warmup > 0 else 0
    if warm:
        # one untimed interval on a copy of the state, so that the timed intervals pay no
        # first-use set-up (module loading, kernel attributes, workspace) and still start
        # from the workload's initial state
        pw, vw = pos.clone(), vel.clone()
        F.fsi_hhs_interval(ctx, pw, vw, mass, tau, is_bh=bh if cl > 0 else None)
        torch.cuda.synchronize()
        del pw, vw
    e0 = energy()
    F.fsi_work_stats(ctx, reset=True)
    if args.grid_profile:
        F.fsi_profile(ctx, True)
        F.fsi_grid_stats(ctx, reset=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    levels, per_interval, t_int = [], [], 0.0
    ek = e0
    for _ in range(args.intervals):
        ti = time.perf_counter()
        code = F.fsi_hhs_interval(ctx, pos, vel, mass, tau, is_bh=bh if cl > 0 else None)
        levels.append(F.fsi_level_stats(ctx))
        if soft:
            torch.cuda.synchronize()
            t_int += time.perf_counter() - ti
            e = energy()                 # outside the interval timing
            per_interval.append(abs((e - ek) / ek))
            ek = e
    torch.cuda.synchronize()
    t = t_int if soft else time.perf_counter() - t0
    acc_p, grad_p = F.fsi_work_stats(ctx)
    grid_profile = None
    if args.grid_profile:
        ns, ph = F.fsi_grid_stats(ctx)
        F.fsi_profile(ctx, False)
        F.fsi_profile_read(ctx)
        kinds = ["time_steps", "split", "inter_level_kick", "fsi_pass", "one_cta_recursion",
                 "gradient_criteria", "set_up", "pn_kick"]
        grid_profile = {k: {"ms_per_interval": ns[q] / 1e6 / args.intervals,
                            "phases_per_interval": ph[q] / args.intervals}
                        for q, k in enumerate(kinds) if ph[q]}
    e1 = energy()
    inter = (acc_p * FLOP_ACC + grad_p * FLOP_GRAD) / FLOP_PAIR
    line = {
        "metric": f"HHS acc+grad pair interactions/s ({wl}, tau0 = {tau:g})",
        "value": inter / t, "unit": UNIT, "n_gpus": 1, "steps": args.intervals, "warmup": warm,
        "ms_per_step": 1e3 * t / args.intervals, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": wl, "n": c.n, "tau": tau, "intervals": args.intervals, "c": cl,
                   "wide_ctas": args.wide_ctas, "hhs_small_max": args.hhs_small_max,
                   "hhs_grid_max": args.hhs_grid_max,
                   "order_min": args.order_min,
                   "tuning": args.tuning or "default",
                   **({"eps2": SOFT_EPS ** 2, "eta": "ff 0.2, fb 0.2, jerk 0.1, gradient 0.1",
                       "units": f"length {SOFT_LUNIT_PC:.4f} pc, time {SOFT_TUNIT_MYR:.4f} Myr"}
                      if soft else {})},
        "level_counts": levels, "rel_energy_error": abs((e1 - e0) / e0),
        "rel_energy_error_per_interval": per_interval or None,
        "mean_rel_energy_error_per_interval": float(np.mean(per_interval)) if per_interval else None,
        "acc_pairs": acc_p, "grad_pairs": grad_p, "maxlevel_status": code,
    }
    if grid_profile is not None:
        # wall clock of CTA 0 per phase kind of the cooperative-launch recursions
        line["grid_phase_profile"] = grid_profile
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def probe_peak_tflops(F, mode: int) -> float:
    """FMA throughput of this GPU measured by the library's probe (0: FP32, 1: FP64,
    2: packed FP32x2): best of 3 launches of 8 CTAs per SM."""
    import torch
    blocks = sm_count() * 8
    iters = 400 if mode == 1 else 20000
    sink = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    F.fsi_fma_probe(mode, blocks, iters, sink)
    best = 0.0
    for _ in range(3):
        e0, e1 = _timed_events(None)
        e0.record()
        fl = F.fsi_fma_probe(mode, blocks, iters, sink)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, fl / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def run_accgrad(args):
    """One same-set acceleration pass plus one force-gradient pass over all N(N-1) ordered
    pairs (fsi_accel_grad), the acc+grad throughput at N = 2^20, in either precision;
    each pass against the FMA peak of its pipe measured by the probe in the same run."""
    import torch
    from paper_2210_02472_b300 import fsi as F
    torch.cuda.set_device(0)
    c = inputs.workload(args.workload)
    if args.n:
        c = inputs.plummer(args.n, inputs.SEED_BASE + 3, imf="kroupa", n_bh=16)
    N = c.n
    dev = torch.device("cuda", 0)
    pos = torch.as_tensor(c.pos).to(dev)
    mass = torch.as_tensor(c.mass).to(dev)
    ctx = F.Context(args.precision)
    if args.tuning:
        F.fsi_set_tuning(ctx, *(int(x) for x in args.tuning.split(",")))
    tuning = F.fsi_get_tuning_for(ctx, N)
    # warm-up on a 2^16 subset (same kernels), then the full set
    sub = torch.arange(0, min(N, 65536), dtype=torch.int32, device=dev)
    for _ in range(max(1, args.warmup)):
        F.fsi_accel_grad(ctx, pos, None, mass, sub, sub)
    torch.cuda.synchronize()
    peak_fp32 = probe_peak_tflops(F, 0)
    peak_fp64 = probe_peak_tflops(F, 1)
    sampler = ClockSampler(0)
    sampler.start()
    F.fsi_profile(ctx, True)
    e0, e1 = _timed_events(None)
    e0.record()
    for _ in range(args.steps):
        F.fsi_accel_grad(ctx, pos, None, mass)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof = F.fsi_profile_read(ctx)
    F.fsi_profile(ctx, False)
    assert F.fsi_sync_status(ctx) == F.FSI_OK
    t = e0.elapsed_time(e1) / 1e3
    pairs = float(N) * (N - 1)
    value = pairs * args.steps / t
    peak = peak_fp32 if args.precision == "mixed" else peak_fp64
    kern = {}
    for k, fl in (("acc", FLOP_ACC), ("grad", FLOP_GRAD)):
        nl, ms = prof[k]
        ach = pairs * fl / (ms / nl / 1e3) / 1e12
        kern[k] = {"ms_per_launch": ms / nl, "launches": nl, "achieved_tflops": ach,
                   "frac_of_probe_peak": ach / peak,
                   "frac_of_nominal": ach / (fp32_peak_tflops(sm_count(dev)) if args.precision == "mixed"
                                             else fp64_peak_tflops(sm_count(dev)))}
    line = {
        "metric": f"acc+grad pair interactions/s at N={N} ({args.precision}, one acc + one grad pass)",
        "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload if not args.n else f"plummer_kroupa_bh16_{N}", "n": N,
                   "precision": args.precision, "tuning": list(tuning),
                   "flops": "acc pair 20, grad pair 36"},
        "probe_peaks_tflops": {"fp32": peak_fp32, "fp64": peak_fp64},
        "kernels": kern, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_update(args):
    """The fused kick/drift update (fsi_kick_drift, FP64) on a state larger than L2:
    N = --update-n particles (default 2^25: x, v and a are 805 MB each), every particle
    (contiguous SoA rows) and a sorted half of them through an id list (the gather/scatter
    pattern of a level set).  Algorithmic bytes: read a, v, x and write v, x (120 B per
    particle) + 4 B per id; reported against the measured HBM copy bandwidth.  Each case
    times max(--steps, 400) launches."""
    import torch
    from paper_2210_02472_b300 import fsi as F
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    N = args.update_n
    g = torch.Generator(device=dev)
    g.manual_seed(inputs.SEED_BASE + 7)
    pos = torch.rand((3, N), dtype=torch.float64, device=dev, generator=g)
    vel = torch.rand((3, N), dtype=torch.float64, device=dev, generator=g)
    acc_all = torch.rand((3, N), dtype=torch.float64, device=dev, generator=g)
    keep = torch.rand(N, device=dev, generator=g) < 0.5
    ids = torch.nonzero(keep).flatten().to(torch.int32).contiguous()
    acc_ids = torch.rand((3, ids.numel()), dtype=torch.float64, device=dev, generator=g)
    ctx = F.Context("fp64")
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs") or 6400.0)
    res = {}
    sampler = ClockSampler(0)
    steps = max(args.steps, 400)        # >= ~0.25 s timed, so the 200 ms clock samples see it
    for name, idx, acc, bpp in (("all", None, acc_all, 120.0), ("ids", ids, acc_ids, 124.0)):
        n = N if idx is None else idx.numel()
        for _ in range(max(3, args.warmup)):
            F.fsi_kick_drift(ctx, pos, vel, acc, 1e-9, 1e-9, idx=idx)
        torch.cuda.synchronize()
        if name == "all":
            sampler.start()
        e0, e1 = _timed_events(None)
        e0.record()
        for _ in range(steps):
            F.fsi_kick_drift(ctx, pos, vel, acc, 1e-9, 1e-9, idx=idx)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / steps
        gbs = bpp * n / t / 1e9
        res[name] = {"n": n, "ms_per_launch": 1e3 * t, "particles_per_s": n / t,
                     "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / hbm}
    clocks = sampler.stop()
    assert F.fsi_sync_status(ctx) == F.FSI_OK
    a = res["all"]
    line = {
        "metric": f"kick+drift particle updates/s (N = {N}, FP64 state, contiguous)",
        "value": a["particles_per_s"], "unit": "particles/s", "n_gpus": 1, "steps": steps,
        "warmup": max(3, args.warmup), "ms_per_step": a["ms_per_launch"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"state_{N}", "n": N, "bytes_per_particle": "120 (124 with ids)",
                   "l2": "inputs 805 MB per array, > L2"},
        "roofline": {"bound": "hbm", "achieved": a["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                     "frac": a["frac_of_measured_hbm"], "traffic": None,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks.get("hbm_gbs") else "fallback"},
        "id_list": res["ids"], "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_sharded(args):
    """The i-sharded FSI cycle (paper_2210_02472_b300.shard) of the headline workload over
    all ranks: every rank kicks, drifts and sums the pairs of its slice of the set, with
    NCCL all-gathers of the positions after drifts and of the accelerations before the
    gradient pass; with --shard-pairs the same-set passes are split by pairs instead (every
    rank a share of the unordered pairs for both particles, the shares all-reduced, every
    rank kicking and drifting the whole set).  Strong scaling: the total work (one set of
    N) is fixed; value = the set's interactions per step / the slowest rank's time."""
    import torch
    rank, ws, local, dist = dist_init()
    torch.cuda.set_device(local)
    from paper_2210_02472_b300 import fsi as F
    from paper_2210_02472_b300.shard import Exchange, LibfsiCompute, ShardedFSI

    c = inputs.workload(args.workload)
    if args.n:
        c = inputs.plummer(args.n, inputs.SEED_BASE + 3, imf="kroupa", n_bh=16)
    N = c.n
    dev = torch.device("cuda", local)
    pos = torch.as_tensor(c.pos).to(dev)
    vel = torch.as_tensor(c.vel).to(dev)
    mass = torch.as_tensor(c.mass).to(dev)
    bh = torch.as_tensor(c.is_bh.astype(np.uint8)).to(dev)
    h, cl = 1.0 / 1024, 1e4
    ctx = F.Context(args.precision, c=cl)
    F.fsi_reserve(ctx, N, N)
    sh = ShardedFSI(LibfsiCompute(ctx), Exchange(), pairs=args.shard_pairs)

    def step():
        sh.step(pos, vel, mass, h, nsteps=1, c=cl, is_bh=bh)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if F.fsi_sync_status(ctx) != F.FSI_OK:
        raise SystemExit("device error after warm-up")
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    n0 = F.fsi_launch_count()
    for k in range(args.steps):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = F.fsi_launch_count() - n0
    clocks = sampler.stop()
    if F.fsi_sync_status(ctx) != F.FSI_OK:
        raise SystemExit("device error in the timed region")
    t_dev = reduce_max(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dist, dev)
    value = step_interactions(N) * args.steps / t_dev
    line = {
        "metric": METRIC + ", i-sharded over ranks", "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": N, "precision": args.precision,
                   "step": ("one FSI cycle of all N + PN1.0 half-kicks, the same-set passes "
                            "split by pairs (shares of the symmetric kernel, all-reduced)"
                            if args.shard_pairs else
                            "one FSI cycle of all N + PN1.0 half-kicks, receivers sharded over "
                            "ranks (one-sided pair passes over each rank's slice)"),
                   "c": cl, "h": h,
                   "parallelism": f"{'pair' if args.shard_pairs else 'i'}-sharded x{ws}"},
        "gpu_launches": launches, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fsi", choices=["fsi", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="kroupa1m_bh16")
    ap.add_argument("--n", type=int, default=0, help="override N (stars) for quick runs")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-rows", type=int, default=CPU_ROWS)
    ap.add_argument("--ref-rows", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows-1t", type=int, default=256,
                    help="rows of the single-thread oracle sample of cpu_baseline")
    ap.add_argument("--no-fp64", action="store_true",
                    help="cycle mode: skip the FP64 acc + grad passes of the line's fp64 object")
    ap.add_argument("--no-energy", action="store_true",
                    help="cycle mode: skip the FP64 energies before and after the cycles")
    ap.add_argument("--tuning", default="", help="fixed pair-kernel variants 'acc,grad' "
                    "(see fsi_set_tuning); default: autotune on a 2^18 sample")
    ap.add_argument("--mode", default="cycle",
                    choices=["cycle", "ensemble", "vjp", "hhs", "accgrad", "update", "sharded"],
                    help="cycle: the headline FSI-cycle benchmark; the others measure the "
                         "ensemble, adjoint and HHS workloads and one acc + grad pass")
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--batch-tuning", default="", help="ensemble mode: fixed 'ipt,ctas_per_sm' "
                    "(ipt 4 = symmetric form) instead of the autotuning sweep")
    ap.add_argument("--vjp-steps", type=int, default=200)
    ap.add_argument("--fd-components", type=int, default=3)
    ap.add_argument("--intervals", type=int, default=1)
    ap.add_argument("--update-n", type=int, default=1 << 25,
                    help="update mode: particles in the state (default 2^25)")
    ap.add_argument("--tau", type=float, default=1.0 / 64)
    ap.add_argument("--hhs-pn", action="store_true", help="HHS mode: PN1.0 on (c = 1e4)")
    ap.add_argument("--wide-ctas", type=int, default=0, help="HHS mode: fsi_params.wide_ctas "
                    "(0 = 32, -1 = tiled passes only)")
    ap.add_argument("--hhs-small-max", type=int, default=0, help="HHS mode: fsi_params.hhs_small_max")
    ap.add_argument("--order-min", type=int, default=0, help="HHS mode: fsi_params.order_min")
    ap.add_argument("--hhs-grid-max", type=int, default=0, help="HHS mode: fsi_params.hhs_grid_max")
    ap.add_argument("--shard-pairs", action="store_true",
                    help="sharded mode: split the same-set passes by pairs, not by receivers")
    ap.add_argument("--grid-profile", action="store_true",
                    help="HHS mode: phase profile of the cooperative-launch recursions (fsi_grid_stats)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "ensemble":
        return run_ensemble(args)
    if args.mode == "vjp":
        return run_vjp(args)
    if args.mode == "hhs":
        return run_hhs(args)
    if args.mode == "accgrad":
        return run_accgrad(args)
    if args.mode == "update":
        return run_update(args)
    if args.mode == "sharded":
        return run_sharded(args)
    return run_fsi(args)


if __name__ == "__main__":
    sys.exit(main())
