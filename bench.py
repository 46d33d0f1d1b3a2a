#!/usr/bin/env python
"""Benchmark of the FCBM-EC hot path on one GB300 (or N replicas).

Workload (the 3D elastostatic configuration): 128^3 periodic box, horizon
delta = 3 grid spacings, body = cube [3, 125)^3 minus a centred ball of radius
32, linearized state-based solid with E = 1, nu = 0.25, clamp (chi_Omega = 0,
w = 0) on the three node layers at the x1-low face, body-force layer
b1 = sigma/delta (sigma = 1e-3) on the three layers at the x1-high face.
One step = one complete static solve from u = 0 to a relative FP64 residual of
1e-8: FP32 FFT-convolution CG with FP64 inner products inside FP64 iterative
refinement (pd_solve_static). The plan's pass configuration is picked by the
library's autotuner timing the solver's own CG iterations
(pd_plan_autotune_solve) before the warm-up, unless --no-autotune.

Metric: force evaluations x nodes per second (each CG iteration and each FP64
residual is one evaluation of the PD operator on all 128^3 nodes), plus the
solve time and the HBM roofline fraction of the dominant FFT pass.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
Under torchrun (N > 1) every rank solves its own copy (replicas: the problem
does not shard) and rank 0 prints one JSON line.

--workload force measures one FP32 bond-model force evaluation (pd_force) on
an n^3 box (--n, e.g. 128/256/512; cube minus a centred ball, delta = 3) for the
scale sweep, with per-pass times and roofline fractions.

--workload batched measures the batched form instead: 64 uneven 2D bond-model
specimens (sides 256..1024 padded to powers of two, delta 3..5, elliptical
cutouts, seeded loads) solved to a relative FP64 residual of 1e-8 by dynamic
relaxation (FP32 FFT passes, FP64 refinement) in one CUDA-graph launch per
step (pd_solve_dr_batched); metric = relaxation steps x specimen nodes per
second.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PD force evals x nodes/sec (FCBM-EC static solve to 1e-8 rel. residual)"
UNIT = "node-evals/s"
N_GRID = 128
DELTA = 3.0
RTOL = 1e-8


def workload_config(n):
    return {
        "workload": f"3D linearized state-based PD elastostatic solve, {n}^3 box, cube minus centred ball "
                    f"r={n // 4}, delta=3, E=1, nu=0.25, clamp on x1-low face via EC, body-force layer "
                    f"b1=sigma/delta (sigma=1e-3) on x1-high face, FP32 FFT CG + FP64 refinement to 1e-8",
        "grid": [n, n, n],
        "delta_cells": DELTA,
        "rtol": RTOL,
        "l2": "working set > L2 (solver vectors, spectra, boundary field ~0.4 GB) and 256 MB L2 flush "
              "between steps",
    }


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = os.path.join("/tmp", f"pd_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.uuid and parts[1] != self.uuid:
                    continue
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
# committed ncu summaries; None when the kernel changed after the capture.
MEASURED_TRAFFIC = {
    "plane_fwd": (143.3e6, "profiles/cg_iteration_kernels_static_solve_128cube.md"),
    "rows_inv": (101.2e6, "profiles/cg_iteration_kernels_static_solve_128cube.md"),
    "last_axis": (42.3e6, "profiles/cg_iteration_kernels_static_solve_128cube.md"),
    "rows_fwd": (146.4e6, "profiles/cg_iteration_kernels_static_solve_128cube.md"),
    "force256_rows_fwd": (368.0e6, "profiles/force_eval_256cube.md"),
    "force256_last_axis": (495.4e6, "profiles/force_eval_256cube.md"),
    "force256_rows_inv": (563.5e6, "profiles/force_eval_256cube.md"),
}


def max_over_ranks(value, world, device=None):
    """The largest of one float per rank (a replicated job takes as long as its
    slowest rank); `value` itself when there is one rank."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, t_max_ms):
    """Whole-job throughput: every rank processes units_per_rank in the job time."""
    return world * units_per_rank / (t_max_ms * 1e-3)


def pass_bytes(kind, N, nbound, d=3, nc=6):
    """Algorithmic bytes of one launch of each FP32 pass of the fused CG
    iteration (d = 3 components; a packed half spectrum holds 4 bytes per node).
      rows_fwd : read e, r, p, q (16d), mask bits (1); write e, r, p (12d) and
                 d spectra (4d)
      cols_x2  : read + write d spectra
      last_axis: read + write d spectra, folded kernel table (nc floats per
                 folded mode, (n/2+1)^3 ~ N/8 modes)
      rows_inv : read d spectra (4d), p, r (8d), mask bits (1); write q (4d);
                 boundary list (32 B per boundary node) and p there (4d)
      plane_fwd, plane_inv: the same bytes as rows_fwd, rows_inv (their x2
                 transforms stay in shared memory)"""
    per_node = {
        "rows_fwd": 32 * d + 1,
        "plane_fwd": 32 * d + 1,
        "cols_x2": 8 * d,
        "last_axis": 8 * d + nc * 4 / 8.0,
        "rows_inv": 16 * d + 1,
        "plane_inv": 16 * d + 1,
    }[kind]
    extra = (32 + 4 * d) * nbound if kind in ("rows_inv", "plane_inv") else 0
    return per_node * N + extra


def run_native(args, rank, world):
    import torch

    from paper_2105_06055_gb300 import build as pd_build
    from paper_2105_06055_gb300 import inputs, pd

    if rank == 0 or world == 1:
        pd_build.build()
    if world > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    n = args.n
    cfg = inputs.cube_with_cavity(n=n)
    shape = cfg["shape"]
    N = n ** 3
    prob = pd.Problem(shape=shape, delta=DELTA, model=pd.PD_LIN_STATE, E=1.0, nu=0.25, fp64=False)
    chi = torch.tensor(cfg["chi"], device=dev)
    chi_om = torch.tensor(cfg["chi_omega"], device=dev)
    plan = pd.Plan(prob, chi, chi_om)
    if args.plane_mask is not None:
        plan.set_plane_passes(args.plane_mask)
    if args.tuning:
        plan.set_tuning(*[int(v) for v in args.tuning.split(",")])
        tuning = plan.tuning
    else:
        tuning = None if args.no_autotune else plan.autotune(solve=True)
    b = torch.tensor(cfg["b"], dtype=torch.float64, device=dev)
    u = torch.zeros((3,) + shape, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def one_solve():
        u.zero_()
        it, rel, st = plan.solve_static(u, b, None, rtol=RTOL, max_iter=50000)
        if st != 0:
            raise RuntimeError(f"solve did not converge: rel {rel}")
        return it, rel

    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()
    # one untimed profiled solve: per-pass event times of every pass kind and
    # the dominant kind (the timed region below carries no profiling events)
    plan.profile(True)
    one_solve()
    torch.cuda.synchronize()
    calib = plan.profile_read()
    plan.profile(False)
    dom_name = max(calib.items(), key=lambda kv: kv[1][0])[0]
    # one inverse row or plane pass per force evaluation
    evals_per_solve = calib["rows_inv"][1] + calib.get("plane_inv", (0.0, 0))[1]

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    launches0 = plan.launch_count
    times = []
    its = []
    rels = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, rel = one_solve()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        its.append(it)
        rels.append(rel)
    clocks = sampler.stop()
    launches = plan.launch_count - launches0
    evals_per_step = float(evals_per_solve)
    total_ms = sum(times)
    t_max = max_over_ranks(total_ms, world, dev)
    value = job_rate(evals_per_step * args.steps * N, world, t_max)

    # dominant pass: its average launch time from CUDA events recorded on the
    # plan's stream around every launch of that kind, over two more solves
    plan.profile(True, kinds=[dom_name])
    for _ in range(2):
        flush.fill_(1.0)
        one_solve()
    torch.cuda.synchronize()
    dom_ms, dom_n = plan.profile_read()[dom_name]
    plan.profile(False)
    peak, peak_kind = load_peaks()
    bytes_alg = pass_bytes(dom_name, N, plan.boundary_nodes)
    traffic = MEASURED_TRAFFIC.get(dom_name, (None, None))
    t_launch = dom_ms / dom_n * 1e-3
    # the fraction counts the bytes the kernel really moves: the measured DRAM
    # traffic where a capture of the current kernel exists, never more than the
    # algorithmic bytes
    bytes_used = min(bytes_alg, traffic[0]) if traffic[0] else bytes_alg
    achieved = bytes_used / t_launch / 1e9
    t_eval_ms = total_ms / (evals_per_step * args.steps)
    m2 = 25.0 * N / (t_eval_ms * 1e-3) / (peak * 1e9)

    # end to end through the public API with host buffers: every step copies b
    # in and u out (pinned host memory), the same L2 flush before each step
    b_host = torch.tensor(cfg["b"], dtype=torch.float64).pin_memory()
    u_host = torch.empty((3,) + shape, dtype=torch.float64).pin_memory()
    e2e_times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.copy_(b_host, non_blocking=True)
        one_solve()
        u_host.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = world * evals_per_step * N / statistics.mean(e2e_times)

    result = None
    if rank == 0:
        result = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t_max / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 FFT convolutions + f64 residuals/inner products",
            "data": "synthetic (seeded geometry and load, no dataset)",
            "config": dict(workload_config(n), parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
            "static_solve_ms": t_max / args.steps,
            "cg_iterations_per_solve": statistics.mean(its),
            "force_evals_per_solve": evals_per_step,
            "final_rel_residual": max(rels),
            "ms_per_force_eval": t_eval_ms,
            "m2_end_to_end_hbm_frac": m2,
            "passes_ms_per_launch": {k: (v[0] / v[1] if v[1] else None) for k, v in calib.items()},
            "passes_note": "per-pass times from one untimed profiled solve (all passes bracketed by events); "
                           "the timed steps carry no profiling events",
            "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak,
                         "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic[0], "traffic_source": traffic[1],
                         "algorithmic_bytes_per_launch": bytes_alg,
                         "frac_algorithmic": bytes_alg / t_launch / 1e9 / peak,
                         "launch_us": 1e6 * t_launch,
                         "bytes_note": "frac uses min(measured DRAM traffic, algorithmic bytes) per launch; "
                                       "launch_us from CUDA events on the plan's stream over two solves"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(b_host.numel() * 8),
                    "d2h_bytes_per_step": int(u_host.numel() * 8)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "tuning": tuning,
            # halves of the CG iteration that ran as plane passes (bit 0 forward, bit 1 inverse)
            "plane_passes": (1 if calib.get("plane_fwd", (0, 0))[1] else 0) | (2 if calib.get("plane_inv", (0, 0))[1] else 0),
        }
    plan.close()
    return result, cfg


FORCE_PASS_BYTES = {  # algorithmic bytes per node of each FP32 pass of the bond force (d = 3)
    "rows_fwd": 25.0,   # read u (12), chi (1); write 3 packed spectra (12)
    "cols_x2": 24.0,    # read + write 3 spectra
    "last_axis": 27.0,  # read + write 3 spectra, folded kernel table (6 floats per N/8 modes)
    "rows_inv": 25.0,   # read 3 spectra (12), chi (1); write L (12); + 44 B per boundary node
}


def force_point(n, steps, warmup, tuning_arg="", no_autotune=False, e2e=True):
    """One FP32 bond-model force evaluation (pd_force) on an n^3 box: median
    event time over `steps` evaluations (L2 flushed between them), per-pass
    event times and their algorithmic-byte fractions of the measured peak."""
    import torch

    from paper_2105_06055_gb300 import inputs, pd

    dev = torch.device("cuda")
    shape = (n, n, n)
    N = n ** 3
    chi = inputs.cube_with_ball_mask(n)
    u = inputs.separable_modes(shape, 4, max(n // 16, 2), 1e-3, seed=n, kmin=max(n // 32, 1)) * chi
    plan = pd.Plan(pd.Problem(shape=shape, delta=DELTA, fp64=False), torch.tensor(chi, device=dev))
    if tuning_arg:
        plan.set_tuning(*[int(v) for v in tuning_arg.split(",")])
        tuning = plan.tuning
    else:
        tuning = None if no_autotune else plan.autotune()
    ud = torch.tensor(u, device=dev)
    L = torch.empty_like(ud)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.force(ud, L=L)
    torch.cuda.synchronize()
    plan.profile(True)
    for _ in range(max(steps, 3)):
        plan.force(ud, L=L)
    torch.cuda.synchronize()
    prof = plan.profile_read()
    plan.profile(False)
    launches0 = plan.launch_count
    sampler = ClockSampler(None)
    sampler.start()
    times = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.force(ud, L=L)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    launches = plan.launch_count - launches0
    peak, peak_kind = load_peaks()
    nb = plan.boundary_nodes
    passes = {}
    for k, (ms, cnt) in prof.items():
        if not cnt:
            continue
        per = ms / cnt
        byt = FORCE_PASS_BYTES[k] * N + (44 * nb if k == "rows_inv" else 0)
        passes[k] = {"us": 1e3 * per, "algorithmic_bytes": byt, "frac_of_measured_peak": byt / (per * 1e-3) / 1e9 / peak}
        meas = MEASURED_TRAFFIC.get(f"force{n}_{k}")
        if meas:
            # DRAM bytes of a committed capture of this pass at this size, over the live event time
            passes[k]["dram_bytes_measured"] = meas[0]
            passes[k]["frac_measured_bytes"] = meas[0] / (per * 1e-3) / 1e9 / peak
    t_ms = statistics.median(times)
    out = {"n": n, "ms_per_eval": t_ms, "node_evals_per_s": N / (t_ms * 1e-3), "passes": passes,
           "m2_end_to_end_hbm_frac": 25.0 * N / (t_ms * 1e-3) / (peak * 1e9), "gpu_launches": int(launches),
           "clocks": clocks, "tuning": tuning, "boundary_nodes": nb, "peak": peak, "peak_source": peak_kind}
    if e2e:
        # end to end: host u -> device, force, device L -> host
        u_host = torch.tensor(u).pin_memory()
        L_host = torch.empty_like(u_host).pin_memory()
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ud.copy_(u_host, non_blocking=True)
            plan.force(ud, L=L)
            L_host.copy_(L, non_blocking=True)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        out["e2e"] = {"value": N / statistics.median(ts), "unit": UNIT, "h2d_bytes_per_step": int(u_host.numel() * 4),
                      "d2h_bytes_per_step": int(L_host.numel() * 4)}
    plan.close()
    del flush
    torch.cuda.empty_cache()
    return out


def run_force(args):
    from paper_2105_06055_gb300 import build as pd_build

    pd_build.build()
    n = args.n
    N = n ** 3
    pt = force_point(n, args.steps, args.warmup, args.tuning, args.no_autotune)
    passes = pt["passes"]
    dom = max(passes, key=lambda k: passes[k]["us"] * (2 if k == "cols_x2" else 1))
    traffic = MEASURED_TRAFFIC.get(f"force{n}_{dom}", (None, None))
    t_ms = pt["ms_per_eval"]
    return {
        "metric": f"PD force evals x nodes/sec (3D bond force evaluation, {n}^3)",
        "value": N / (t_ms * 1e-3),
        "unit": UNIT,
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded separable smooth field, no dataset)",
        "config": {"workload": f"3D linearized bond-based PD force evaluation (pd_force), {n}^3 box, cube minus "
                               f"centred ball r={n // 4}, delta=3, E=1", "grid": [n, n, n],
                   "l2": "256 MB L2 flush between steps"},
        "passes": passes,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": passes[dom]["algorithmic_bytes"] /
                     (passes[dom]["us"] * 1e-6) / 1e9, "peak": pt["peak"], "peak_source": pt["peak_source"],
                     "unit": "GB/s", "frac": passes[dom]["frac_of_measured_peak"], "traffic": traffic[0],
                     "traffic_source": traffic[1]},
        "m2_end_to_end_hbm_frac": pt["m2_end_to_end_hbm_frac"],
        "e2e": pt["e2e"],
        "gpu_launches": pt["gpu_launches"],
        "clocks": pt["clocks"],
        "tuning": pt["tuning"],
        "boundary_nodes": pt["boundary_nodes"],
    }


def fracture_point(steps=200, warmup=50):
    """The 2D dynamic-fracture workload (1024 x 512 nodes, delta = 4, pre-notch,
    traction layers, critical stretch s0 = 1e-3 given to the library, FP32,
    W by the horizon sum): milliseconds per velocity-Verlet step with bond
    breaking, timed with CUDA events over `steps` steps after `warmup`."""
    import torch

    from paper_2105_06055_gb300 import inputs, pd

    dev = torch.device("cuda")
    cfg = inputs.notched_plate(n1=1024, n2=512, delta=4.0, sigma=1.0)
    shape = cfg["shape"]
    plan = pd.Plan(pd.Problem(shape=shape, delta=4.0, rho=1.0, s0=1e-3, nu=1.0 / 3.0, fp64=False),
                   torch.tensor(cfg["chi"], device=dev))
    plan.set_energy_mode(True)
    b = torch.tensor(cfg["b"] * (0.242 * math.sqrt(plan.critical_energy)), dtype=torch.float32, device=dev)
    u = torch.zeros((2,) + shape, dtype=torch.float32, device=dev)
    v = torch.zeros_like(u)
    lam = torch.tensor(cfg["lam"], device=dev)
    dt = 0.8 * plan.stable_dt
    plan.step_verlet(u, v, lam, b, None, dt=dt, nsteps=warmup)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = plan.launch_count
    torch.cuda.synchronize()
    e0.record(stream)
    broken = plan.step_verlet(u, v, lam, b, None, dt=dt, nsteps=steps, count_broken=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    N = shape[0] * shape[1]
    out = {"ms_per_step": ms, "node_steps_per_s": N / (ms * 1e-3), "steps": steps, "after_warmup_steps": warmup,
           "broken_nodes_in_timed_steps": broken, "launches_per_step": (plan.launch_count - l0) / steps,
           "workload": "1024x512 pre-notched plate, delta=4, s0=1e-3, FP32, W by horizon sum"}
    plan.close()
    return out


def run_batched(args):
    import numpy as np
    import torch

    from paper_2105_06055_gb300 import build as pd_build
    from paper_2105_06055_gb300 import inputs, pd

    pd_build.build()
    dev = torch.device("cuda")
    cfgs = inputs.batched_specimens(count=args.specimens, seed=0)

    def t(a, dt=torch.float64):
        return torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)

    probs = [pd.Problem(shape=c["shape"], delta=c["delta"], nu=1.0 / 3.0, fp64=False) for c in cfgs]
    batch = pd.Batch(probs, [t(c["chi"], torch.uint8) for c in cfgs], [t(c["chi_omega"], torch.uint8) for c in cfgs])
    t0 = time.perf_counter()
    tuning = batch.autotune()
    tune_s = time.perf_counter() - t0
    us = [torch.zeros((2,) + c["shape"], dtype=torch.float64, device=dev) for c in cfgs]
    bs = [t(c["b"]) for c in cfgs]
    nodes = [c["shape"][0] * c["shape"][1] for c in cfgs]

    def one():
        for u in us:
            u.zero_()
        its, rels, sts = batch.solve_dr(us, bs, rtol=RTOL, max_iter=2000000, raise_on_fail=False)
        if any(s != 0 for s in sts):
            raise RuntimeError(f"batched solve: statuses {sorted(set(sts))}")
        return its, rels

    for _ in range(args.warmup):
        one()
    stream = torch.cuda.current_stream()
    launches0 = sum(p.launch_count for p in batch.plans)
    sampler = ClockSampler(None)
    sampler.start()
    times, steps = [], []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its, rels = one()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        steps.append(sum(i * n for i, n in zip(its, nodes)))
    clocks = sampler.stop()
    launches = sum(p.launch_count for p in batch.plans) - launches0
    total_s = sum(times) * 1e-3
    value = sum(steps) / total_s
    peak, peak_kind = load_peaks()
    out = {
        "metric": "PD force evals x nodes/sec (batched FCBM-EC, dynamic relaxation to 1e-8 rel. residual)",
        "value": value,
        "unit": UNIT,
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": sum(times) / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 FFT convolutions + f64 residuals/inner products",
        "data": "synthetic (seeded geometry and load, no dataset)",
        "config": {"workload": f"{len(cfgs)} uneven 2D linearized bond-based specimens, sides 256..1024 padded to "
                               f"powers of two, delta 3..5, elliptical cutouts, clamp + body-force layer, "
                               f"adaptive dynamic relaxation + FP64 refinement to 1e-8, one graph launch",
                   "box_nodes": int(sum(nodes)), "specimens": len(cfgs),
                   "l2": "working set ~10 GB > L2"},
        "relaxation_steps_per_solve": [int(i) for i in its],
        "final_rel_residual_max": max(rels),
        "autotune_s": tune_s,
        "tuning": sorted({tuple(sorted(d.items())) for d in tuning}),
        "m2_end_to_end_hbm_frac": 17.0 * value / (peak * 1e9),
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    batch.close()
    return out


def oracle_threads(t):
    import oracle
    oracle.set_threads(t)


def oracle_sample(n, nevals, threads=None, min_seconds=0.0):
    """Time the FP64 oracle's state-based force on the same workload (host cores):
    at least nevals evaluations, and more until min_seconds have passed."""
    import numpy as np

    import oracle
    from paper_2105_06055_gb300 import inputs

    oracle.build()
    if threads:
        oracle.set_threads(threads)
    cfg = inputs.cube_with_cavity(n=n)
    ka, cb, _ = oracle.lps_constants(1.0, 0.25, 1.0, DELTA)
    u = inputs.sine_modes(cfg["shape"], 4, 1e-3, 3, 5)
    t0 = time.perf_counter()
    k = 0
    while k < nevals or time.perf_counter() - t0 < min_seconds:
        oracle.force_lps(u, cfg["chi"], 1.0, DELTA, ka, cb)
        k += 1
    dt = time.perf_counter() - t0
    N = n ** 3
    return k * N / dt, oracle.num_threads(), dt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", "--grid", dest="n", type=int, default=N_GRID)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="static", choices=["static", "batched", "force"])
    ap.add_argument("--no-autotune", action="store_true", help="skip the pass autotuner (built-in tile heuristic)")
    ap.add_argument("--plane-mask", type=int, default=None, metavar="M",
                    help="static solve: halves of the CG iteration run as fused x1-x2 plane passes (bit 0 forward, "
                         "bit 1 inverse; 0 = row and column passes; default: the library's)")
    ap.add_argument("--tuning", default="", metavar="ROWS,WX2,WLAST,SCHED[,STAGES[,STAGES_INV]]",
                    help="pin a pass configuration instead of autotuning (e.g. the one a tuned run reported)")
    ap.add_argument("--specimens", type=int, default=64)
    ap.add_argument("--no-sweep", dest="sweep", action="store_false",
                    help="skip the 256^3 / 512^3 force-evaluation keys of the default run")
    ap.add_argument("--profile-solve", type=int, default=0, metavar="K",
                    help="no timing: build the workload and run one solve capped at K CG iterations "
                         "(a short, deterministic target for ncu captures)")
    args = ap.parse_args()

    if args.profile_solve:
        import torch

        from paper_2105_06055_gb300 import build as pd_build
        from paper_2105_06055_gb300 import inputs, pd
        pd_build.build()
        cfg = inputs.cube_with_cavity(n=args.n)
        dev = torch.device("cuda")
        plan = pd.Plan(pd.Problem(shape=cfg["shape"], delta=DELTA, model=pd.PD_LIN_STATE, nu=0.25, fp64=False),
                       torch.tensor(cfg["chi"], device=dev), torch.tensor(cfg["chi_omega"], device=dev))
        if args.plane_mask is not None:
            plan.set_plane_passes(args.plane_mask)
        if args.tuning:
            plan.set_tuning(*[int(v) for v in args.tuning.split(",")])
        elif not args.no_autotune:
            plan.autotune(solve=True)
        u = torch.zeros((3,) + cfg["shape"], dtype=torch.float64, device=dev)
        it, rel, _ = plan.solve_static(u, torch.tensor(cfg["b"], dtype=torch.float64, device=dev), None,
                                       rtol=RTOL, max_iter=args.profile_solve, raise_on_fail=False)
        torch.cuda.synchronize()
        print(json.dumps({"profile_solve_iterations": it, "rel_residual": rel}))
        plan.close()
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        # the reference arm is the FP64 oracle on the host cores; rank 0 only
        if rank != 0:
            return
        if args.workload != "static":
            print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm times the static workload only "
                                                                  f"(asked for --workload {args.workload})"}))
            return
        value, cores, dt = oracle_sample(args.n, 1)  # warm-up (page-in, thread spin-up)
        samples = []
        for _ in range(args.warmup - 1 if args.warmup > 1 else 0):
            oracle_sample(args.n, 1)
        t_all = 0.0
        for _ in range(args.steps):
            v, cores, dt = oracle_sample(args.n, 1)
            samples.append(v)
            t_all += dt
        value = statistics.mean(samples)
        out = {
            "impl": "reference",
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": args.gpus,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic (seeded geometry and load, no dataset)",
            "config": workload_config(args.n),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one FP64 direct-sum state-based force evaluation of the {args.n}^3 "
                                       f"workload per step (the solve's unit of work)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(out))
        return

    if args.workload == "batched":
        print(json.dumps(run_batched(args)))
        return
    if args.workload == "force":
        print(json.dumps(run_force(args)))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    result, cfg = run_native(args, rank, world)
    if rank == 0 and args.sweep:
        # the force evaluation at the larger grids of the scale sweep (extra keys;
        # the headline stays the static solve)
        sweep = {}
        for n in (256, 512):
            pt = force_point(n, 5, 3, "", args.no_autotune, e2e=False)
            sweep[f"{n}^3"] = {k: pt[k] for k in ("ms_per_eval", "node_evals_per_s", "passes",
                                                  "m2_end_to_end_hbm_frac", "tuning")}
        result["force_sweep"] = sweep
        result["fracture_step"] = fracture_point()
        # the batched workload (64 uneven 2D specimens, one graph launch per solve), one timed solve
        bargs = argparse.Namespace(specimens=args.specimens, warmup=1, steps=1)
        bt = run_batched(bargs)
        result["batched"] = {k: bt[k] for k in ("value", "unit", "ms_per_step", "relaxation_steps_per_solve",
                                                "final_rel_residual_max", "autotune_s", "gpu_launches")}
        result["batched"]["config"] = bt["config"]
    if rank == 0:
        if not args.no_cpu_baseline:
            v, cores, dt = oracle_sample(args.n, 2, min_seconds=2.0)
            k = int(round(v * dt / args.n ** 3))
            result["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                      "sample": f"{k} FP64 direct-sum state-based force evaluations of the "
                                                f"{args.n}^3 workload ({dt:.1f} s on {cores} threads)"}
            # the same on one host core (one evaluation)
            v1, _, dt1 = oracle_sample(args.n, 1, threads=1)
            oracle_threads(cores)
            result["cpu_baseline"]["value_1_core"] = v1
            result["cpu_baseline"]["sample_1_core"] = (f"1 FP64 direct-sum evaluation of the {args.n}^3 workload on "
                                                       f"one thread ({dt1:.1f} s)")
        print(json.dumps(result))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
