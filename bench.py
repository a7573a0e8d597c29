#!/usr/bin/env python
"""Benchmark of the HB-UGKS pseudo-time iteration on GB300 (one JSON line on rank 0).

A step is one pseudo-time iteration of HB-UGKS over every cell, discrete velocity and sub-time level of
the workload (face moments, interface parameters, macro update, micro update, residual).  The default
workload is the large thermally driven cavity: 128x128 cells, 64x64 velocities, Shakhov Pr 2/3, bottom wall
T0 (1 + 0.5 sin wt), Kn 0.05, St 5, N_H 5 (N_T 11), FP32-split storage (5.9 GB of distribution state, far
larger than L2, so no flush is needed between timed steps).  The metric is cell.velocity.level updates/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

--impl reference times the FP64 CPU oracle (the method written plainly from the paper, as it stands) on every
usable host core, each core iterating its own bounded sample of the same workload: the same velocity grid, N_T
and parameters on an 8x8-cell cavity (the metric is per update, so the sample's rate is the workload's).
With torchrun (N > 1) every rank runs its own replica of the workload (the path has no data exchange
between cases); value counts the updates of all ranks over the slowest rank's time.
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

METRIC = "HB-UGKS cell*velocity*level updates/s"
# ncu DRAM bytes (read + write) per update of one k4_cells launch on the 64x64-cell, 64x64-velocity, N_T = 11
# thermal cavity, by micro-update variant (tile x, tile y, velocity blocks per CTA); see profiles/
K4_TRAFFIC_64 = {(4, 2, 2): 19.2881}
UNIT = "updates/s"


def workloads():
    """Workload name -> factory of the list of cases iterated together by one handle."""
    from paper_2605_03479_gb300 import inputs as I
    return {
        "thermal128_v64_nh5_fp32split": lambda: [I.config5(precision=1)],
        "thermal128_v64_nh5_fp64": lambda: [I.config5(precision=0)],
        "thermal64_v48_nh3_fp32split": lambda: [I.config3(precision=1)],
        # the large thermal cavity's velocity grid, levels and physics on 64 x 64 cells (a profiling size)
        "thermal64_v64_nh5_fp32split": lambda: [I.make_case("thermal64_v64_nh5", 64, 64, kn=0.05, st=5.0, nh=5,
                                                            pr=2.0 / 3.0, drive="thermal", amp=0.5, precision=1)],
        "thermal64_v48_nh3_fp64": lambda: [I.config3(precision=0)],
        "shear32_v24_nh1_fp64": lambda: [I.config1()],
        "shear64tanh_v32_nh1_sweep12_fp64": lambda: I.config2_cases(),
        "batch48_fp32split": lambda: I.config4_cases(precision=1),
        # the paper's shear cavities (Sec 3.1.1): aspect 0.5, 1, 2 on 90-row wall-refined meshes, 28 x 28
        # Gauss-Hermite velocities, Kn 0.1, St 30, N_H 1, in one handle
        "paper_shear_A0.5_1_2_gh28_st30_fp32split":
            lambda: [I.paper_shear_case(0.1, 30.0, a, precision=1) for a in (0.5, 1.0, 2.0)],
        "paper_shear_A0.5_1_2_gh28_st30_fp64":
            lambda: [I.paper_shear_case(0.1, 30.0, a, precision=0) for a in (0.5, 1.0, 2.0)],
        "paper_thermal90_v64_nh2_fp32split": lambda: [I.paper_thermal_case(0.1, 2.0, precision=1)],
    }


def with_precision(cases, precision):
    import copy
    out = []
    for c in cases:
        d = copy.deepcopy(c)
        d.precision = precision
        out.append(d)
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def smi_device(local: int) -> str:
    """The nvidia-smi id (index or UUID) of the process's CUDA device `local`: CUDA_VISIBLE_DEVICES renumbers
    the devices a process sees, nvidia-smi does not."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    items = [x.strip() for x in vis.split(",") if x.strip()]
    if items and 0 <= local < len(items):
        return items[local]
    return str(local)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = smi_device(gpu_index)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", self.idx, "-lms", "100"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.15)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            return None
        sms, maxs, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxs.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms)}


def oracle_sample(case_full):
    """The oracle's bounded sample of the workload: same velocity grid, N_T and physics on 8x8 cells."""
    from paper_2605_03479_gb300 import inputs as I
    c = I.make_case("sample8x8", 8, case_full.nu, kn=case_full.kn, st=case_full.st, nh=case_full.n_harmonics,
                    pr=case_full.pr, drive="rest", half_width=case_full.umax)
    c.walls = [list(w) for w in case_full.walls]
    return c


def _oracle_worker(case_full, steps, warmup, min_seconds, barrier, out):
    """One process of the CPU leg: the oracle, as it stands, iterating its own copy of the sample."""
    from oracle import oracle as O
    from paper_2605_03479_gb300 import inputs as I
    c = oracle_sample(case_full)
    P = O.Problem(c)
    W, h, b = I.initial_state(c)
    for _ in range(warmup):
        O.iterate(P, W, h, b, 1)
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    n = 0
    while n < steps or (time.perf_counter() - t0) < min_seconds:
        O.iterate(P, W, h, b, 1)
        n += 1
    out.put((n, time.perf_counter() - t0))


def usable_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def run_oracle(case_full, steps, warmup, min_seconds=0.0, procs=1):
    """The oracle on `procs` host cores: that many processes (started with spawn, so none inherits a CUDA
    context) each iterate their own copy of the 8x8-cell sample, started together behind a barrier.  Returns the
    aggregate updates/s (sum over processes), the seconds per iteration of the slowest process, the number of
    iterations each ran (the smallest), and a description of the sample."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()                                   # compile once before the workers load it
    c = oracle_sample(case_full)
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    bar = ctx.Barrier(procs) if procs > 1 else None
    ps = [ctx.Process(target=_oracle_worker, args=(case_full, steps, warmup, min_seconds, bar, out))
          for _ in range(procs)]
    for p in ps:
        p.start()
    res = [out.get() for _ in ps]
    for p in ps:
        p.join()
    ups = sum(c.updates_per_iteration() * n / dt for n, dt in res)
    sec = max(dt / n for n, dt in res)
    n_min = min(n for n, _ in res)
    sample = (f"{procs} process(es), each iterating its own {c.nx}x{c.ny}-cell cavity with the workload's "
              f"{c.nu}x{c.nv} velocity grid, N_T {c.nt}, Kn {c.kn:g}, St {c.st:g}, Pr {c.pr:.3g}, same walls; "
              f">= {n_min} iterations each, {c.updates_per_iteration()} updates per iteration")
    return ups, sec, n_min, sample


def sample_config(case_full, procs):
    c = oracle_sample(case_full)
    return {"cells": [c.nx, c.ny], "velocities": [c.nu, c.nv], "n_levels": c.nt,
            "updates_per_step_per_process": c.updates_per_iteration(), "processes": procs}


def host_info() -> dict:
    """The host the CPU baseline ran on: architecture, usable and logical cores, CPU model (lscpu's model name,
    which aarch64 kernels do not print in /proc/cpuinfo)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip().lower() == "model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    key = line.split(":")[0].strip().lower()
                    if key in ("model name", "cpu model", "hardware", "cpu part"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"machine": platform.machine(), "nproc": os.cpu_count(), "usable_cores": usable_cores(), "cpu": model}


def slowest_rank_ms(ms: float, dist, device) -> float:
    """The job's step time: the maximum over ranks (every rank runs a replica; the job ends with the slowest)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_updates_per_s(updates_per_rank_step: int, world: int, ms: float) -> float:
    """Whole-job throughput: the updates of all ranks per step over the slowest rank's step time."""
    return updates_per_rank_step * world / (ms * 1e-3)


def describe(name, cases, upd, world):
    par = f"replicas{world}" if world > 1 else "single"
    if len(cases) == 1:
        c = cases[0]
        return {"workload": name, "cells": [c.nx, c.ny], "velocities": [c.nu, c.nv], "n_levels": c.nt, "kn": c.kn,
                "st": c.st, "pr": c.pr, "updates_per_step": upd, "parallelism": par,
                "l2": "state larger than L2 (no flush needed)"}
    return {"workload": name, "cases": len(cases), "cells": sorted({c.nx for c in cases}),
            "velocities": sorted({c.nu for c in cases}), "n_levels": sorted({c.nt for c in cases}),
            "kn": [min(c.kn for c in cases), max(c.kn for c in cases)],
            "st": [min(c.st for c in cases), max(c.st for c in cases)], "updates_per_step": upd,
            "parallelism": par, "l2": "state larger than L2 (no flush needed)"}


def time_to_residual(args, cases):
    """Wall-clock time until every case's level-0 density residual is <= args.ttr, FP32-split and FP64 GPU
    paths from the same start (rest), with the iteration counts.  A path that has not converged within the
    budget is extrapolated from its own time per iteration and the other path's iteration count (the two
    paths follow the same residual history), and flagged so."""
    import numpy as np
    import torch
    from paper_2605_03479_gb300 import hbugks as hb
    res_out = {}
    for prec, key in ((1, "fp32split"), (0, "fp64")):
        cs = with_precision(cases, prec)
        for c in cs:
            c.spectral_implicit = args.spectral_implicit
        s = hb.Solver(cs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its = np.zeros(len(cs), dtype=np.int64)
        while True:
            rc, it, res = s.iterate(250, tol_rho=args.ttr)
            its += it
            el = time.perf_counter() - t0
            budget = args.ttr_budget if prec == 1 or args.ttr_budget_fp64 is None else args.ttr_budget_fp64
            if rc != hb.NOT_CONVERGED or el > budget:
                break
        res_out[key] = {"seconds": el, "iterations": int(its.max()), "status": hb.status_string(rc),
                        "converged": rc == hb.OK, "residual": float(res[:, 0].max()),
                        "seconds_per_iteration": el / max(int(its.max()), 1), "extrapolated": False}
        s.destroy()
    a, b = res_out["fp32split"], res_out["fp64"]
    for x, y in ((a, b), (b, a)):
        if not x["converged"] and y["converged"]:
            x["seconds"] = x["seconds_per_iteration"] * y["iterations"]
            x["extrapolated"] = True
    # mixed precision: FP32-split to the target, then FP64 finishing iterations from its state
    # (hbugks_copy_state), which bring every harmonic of U, V, T, tau_xy to the FP64 result within 1e-5
    mixed = None
    if a["converged"] and args.ttr_finish > 0:
        cs32 = with_precision(cases, 1)
        cs64 = with_precision(cases, 0)
        for c in cs32 + cs64:
            c.spectral_implicit = args.spectral_implicit
        s32, s64 = hb.Solver(cs32), hb.Solver(cs64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while True:
            rc, it, res = s32.iterate(250, tol_rho=args.ttr)
            if rc != hb.NOT_CONVERGED or time.perf_counter() - t0 > args.ttr_budget:
                break
        t_32 = time.perf_counter() - t0
        for k in range(len(cases)):
            s64.copy_state_from(k, s32, k)
        s64.iterate(args.ttr_finish)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        mixed = {"seconds": el, "fp32split_seconds": t_32, "fp64_finish_iterations": args.ttr_finish,
                 "converged": rc == hb.OK}
        s32.destroy()
        s64.destroy()
    line = {"metric": "time to level-0 density residual", "tol": args.ttr, "unit": "s", "workload": args.workload,
            "cases": len(cases), "fp32split": a, "fp64": b, "fp32split_fp64_finish": mixed,
            "speedup_fp32split_over_fp64": b["seconds"] / a["seconds"] if a["seconds"] > 0 else None,
            "speedup_mixed_over_fp64": b["seconds"] / mixed["seconds"] if mixed else None,
            "spectral_source": "new iterate (implicit)" if args.spectral_implicit else "old iterate (as printed)",
            "higher_is_better": False, "data": "synthetic", "start": "rest on every level"}
    print(json.dumps(line), flush=True)


def td_steps_per_period(c) -> int:
    """Steps per forcing period of explicit time-domain UGKS at the case's CFL number: the largest global step
    CFL / max_i nu_i (Eq. nu_conv at rest, u_max + sqrt(gamma R T0)), rounded so that a period holds a whole
    number of steps."""
    import numpy as np
    ut = c.umax + math.sqrt(c.gamma * 0.5)
    vt = c.vmax + math.sqrt(c.gamma * 0.5)
    dx, dy = np.diff(c.xnodes), np.diff(c.ynodes)
    nu = ut / dx.min() + vt / dy.min()
    return int(math.ceil((2 * math.pi / c.st) / (c.cfl / nu)))


def hb_versus_td(args):
    """Wall-clock time for the density residual of Eq. benchmark_residuals to drop args.hb_vs_td orders below
    its first valid value: HB-UGKS (R_HB over pseudo-time iterations, level 0) against explicit time-domain
    UGKS on the same mesh, velocity grid, fluxes and walls (R_TD between consecutive periods at the same
    phase), from rest.  The comparison the paper reports (Sec 3.1), on this GPU."""
    import numpy as np
    import torch
    from paper_2605_03479_gb300 import hbugks as hb
    from paper_2605_03479_gb300 import inputs as I
    orders, budget, atol = args.hb_vs_td, args.ttr_budget, args.hb_vs_td_abs
    sts = [float(x) for x in args.hb_vs_td_st.split(",")]
    runs = [(d, st, 1 if d == "shear" else 2) for d in args.hb_vs_td_drives.split(",") for st in sts]

    def mk(drive, st, nh):
        if args.hb_vs_td_mesh == "paper":
            # the paper's own cavities (Sec 3.1.1, 3.2): 90 rows refined to 0.001 H at every wall; lid
            # 0.0015 cos(wt) with 28 x 28 Gauss-Hermite velocities at Kn 0.1; top wall T0 (1 + 0.3 cos wt)
            # with the 64 x 64 midpoint grid
            if drive == "shear":
                c = I.paper_shear_case(0.1, st, 1.0, nh=nh, precision=args.precision)
            else:
                c = I.paper_thermal_case(0.1, st, nh=nh, precision=args.precision)
        else:
            # the paper's two cavities (Sec 3.1, 3.2) on a coarse uniform mesh: lid U_a cos(wt); top wall
            # T0 (1 + 0.3 cos wt), N_H = 2
            c = I.make_case(f"{drive}32_v24", 32, 24, kn=0.1, st=st, nh=nh, pr=1.0 if drive == "shear" else 2 / 3,
                            drive="shear" if drive == "shear" else "rest", amp=0.01, precision=args.precision)
            if drive == "thermal":
                c.walls[I.TOP][7] = 0.3                  # T_re: 0.3 T0 cos(theta)
        c.spectral_implicit = args.spectral_implicit if nh > 0 else 0
        return c

    for drive, st, nh in runs:
        out = {}
        # harmonic balance
        c = mk(drive, st, nh)
        s = hb.Solver(c)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, r1, r, t_rel, t_abs = 0, 0.0, 0.0, None, None
        chunk = 64
        while True:
            s.iterate(chunk)
            its += chunk
            h_ = s.residual_history(0, chunk)[:, 0]
            if r1 == 0.0 and np.any(h_ > 0):
                r1 = float(h_[h_ > 0][0])
            r = float(h_[-1])
            el = time.perf_counter() - t0
            if t_rel is None and r1 > 0 and r <= r1 * 10.0 ** (-orders):
                t_rel = (el, its)
            if t_abs is None and its > chunk and r <= atol:
                t_abs = (el, its)
            if (t_rel and t_abs) or (t_abs and args.hb_vs_td_abs_only) or el > budget or not np.isfinite(r):
                break
        out["hb"] = {"seconds_to_relative_drop": t_rel[0] if t_rel else None,
                     "iterations_to_relative_drop": t_rel[1] if t_rel else None,
                     "seconds_to_absolute": t_abs[0] if t_abs else None,
                     "iterations_to_absolute": t_abs[1] if t_abs else None,
                     "first_residual": r1, "last_residual": r, "iterations_run": its, "n_levels": c.nt,
                     "updates_per_iteration": c.updates_per_iteration()}
        s.destroy()
        # explicit time domain
        c = mk(drive, st, 0)
        c.td_steps = M = td_steps_per_period(c)
        s = hb.Solver(c)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prev = s.get_W(0)[0, :, 0].copy()
        periods, r1, r, t_rel, t_abs = 0, 0.0, 0.0, None, None
        while True:
            s.iterate(M)
            periods += 1
            rho = s.get_W(0)[0, :, 0]
            r = float(np.sqrt(np.mean((rho - prev) ** 2)))
            prev = rho.copy()
            if r1 == 0.0 and r > 0:
                r1 = r
            el = time.perf_counter() - t0
            if t_rel is None and r1 > 0 and r <= r1 * 10.0 ** (-orders):
                t_rel = (el, periods)
            if t_abs is None and periods > 1 and r <= atol:
                t_abs = (el, periods)
            if (t_rel and t_abs) or (t_abs and args.hb_vs_td_abs_only) or el > budget or not np.isfinite(r):
                break
        out["td"] = {"seconds_to_relative_drop": t_rel[0] if t_rel else None,
                     "periods_to_relative_drop": t_rel[1] if t_rel else None,
                     "seconds_to_absolute": t_abs[0] if t_abs else None,
                     "periods_to_absolute": t_abs[1] if t_abs else None,
                     "steps_per_period": M, "first_residual": r1, "last_residual": r, "periods_run": periods,
                     "updates_per_step": c.updates_per_iteration()}
        s.destroy()
        ratio = lambda k: (out["td"][k] / out["hb"][k]) if out["td"][k] and out["hb"][k] else None
        line = {"metric": "wall time to a density-residual drop, HB-UGKS vs explicit time-domain UGKS",
                "orders": orders, "absolute": atol, "unit": "s",
                "case": (f"{drive} cavity {c.nx}x{c.ny} cells ({args.hb_vs_td_mesh} mesh), {c.nu}x{c.nv} velocities, "
                         f"Kn {c.kn:g}, St {st:g}, N_H {nh}"),
                "dtype": "f32-split" if args.precision else "f64",
                "hb_spectral_source": "new iterate (implicit)" if args.spectral_implicit else "old iterate (as printed)",
                "hb": out["hb"], "td": out["td"],
                "speedup_hb_over_td_relative": ratio("seconds_to_relative_drop"),
                "speedup_hb_over_td_absolute": ratio("seconds_to_absolute"),
                "paper_speedup": {"shear St 2": 1.4, "shear St 30": 9.0, "thermal St 2": 1.06, "thermal St 30": 8.26},
                "data": "synthetic", "start": "rest"}
        print(json.dumps(line), flush=True)


def batch_versus_single(args, cases):
    """The cases of a multi-case workload iterated together in one handle, and each case alone in a handle of
    its own, one after another: device time per iteration (CUDA events, after the warm-up) and updates/s of
    both ways over the same cases, from rest."""
    import torch
    from paper_2605_03479_gb300 import hbugks as hb
    stream = torch.cuda.current_stream()
    W_ = max(args.warmup, 3)

    def per_iteration_ms(cs):
        s = hb.Solver(cs, stream=stream)
        s.init_uniform(-1, 1.0, 0.0, 0.0, 1.0)
        s.enqueue_iterations(W_)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.enqueue_iterations(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        s.destroy()
        return e0.elapsed_time(e1) / args.steps

    upd = sum(c.updates_per_iteration() for c in cases)
    batch_ms = per_iteration_ms(cases)
    single_ms = [per_iteration_ms([c]) for c in cases]
    line = {"mode": "batch_vs_single", "workload": args.workload, "cases": len(cases), "steps": args.steps,
            "warmup": W_, "updates_per_iteration": upd,
            "batch": {"ms_per_iteration": batch_ms, "updates_per_s": upd / (batch_ms * 1e-3)},
            "one_by_one": {"ms_per_iteration": sum(single_ms), "updates_per_s": upd / (sum(single_ms) * 1e-3),
                           "slowest_case_ms": max(single_ms)},
            "batch_speedup": sum(single_ms) / batch_ms, "data": "synthetic", "start": "rest"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="thermal128_v64_nh5_fp32split")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--loop-mode", type=int, default=0,
                    help="0: device-side loop (default); 1: host-launched graphs of 16 iterations, whose kernels "
                         "profilers list one by one (they do not list kernels inside conditional graph nodes)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ttr", type=float, default=0.0,
                    help="time to this level-0 density residual, FP32-split against FP64 (one JSON line)")
    ap.add_argument("--ttr-budget", type=float, default=600.0, help="seconds per precision for --ttr")
    ap.add_argument("--ttr-budget-fp64", type=float, default=None, help="seconds for the FP64 path (default: same)")
    ap.add_argument("--ttr-finish", type=int, default=300,
                    help="--ttr: FP64 iterations that finish the mixed-precision run (0: skip that run)")
    ap.add_argument("--hb-vs-td", type=float, default=0.0,
                    help="orders of residual drop: time HB-UGKS against explicit time-domain UGKS (one JSON line per case)")
    ap.add_argument("--precision", type=int, default=0, help="precision of --hb-vs-td (0 FP64, 1 FP32-split)")
    ap.add_argument("--hb-vs-td-abs", type=float, default=1e-8, help="absolute density residual for --hb-vs-td")
    ap.add_argument("--hb-vs-td-st", default="2,30", help="Strouhal numbers for --hb-vs-td")
    ap.add_argument("--hb-vs-td-mesh", choices=("coarse32", "paper"), default="coarse32",
                    help="--hb-vs-td cavities: 32x32 uniform cells, or the paper's 90-row wall-refined mesh")
    ap.add_argument("--hb-vs-td-drives", default="shear,thermal", help="--hb-vs-td drives to run")
    ap.add_argument("--hb-vs-td-abs-only", action="store_true",
                    help="--hb-vs-td: stop each run at the absolute residual (skip the relative drop)")
    ap.add_argument("--spectral-implicit", type=int, default=0,
                    help="--hb-vs-td, --ttr: HB with the spectral source at the new pseudo-time iterate (1)")
    ap.add_argument("--micro-variant", default=None,
                    help="pin every case's micro-update variant, 'tx,ty,vpl' (default: the autotuner's choice)")
    ap.add_argument("--batch-vs-single", action="store_true",
                    help="time the workload's cases together in one handle and each alone, one after another")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cases = workloads()[args.workload]()
    case = cases[0]
    W_ = max(args.warmup, 3)
    if args.ttr > 0:
        if rank == 0:
            time_to_residual(args, cases)
        return
    if args.hb_vs_td > 0:
        if rank == 0:
            hb_versus_td(args)
        return
    if args.batch_vs_single:
        if rank == 0:
            batch_versus_single(args, cases)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        procs = usable_cores()
        ups, sec, n, sample = run_oracle(case, args.steps, W_, procs=procs)
        # config names the GPU arm's workload (the metric is per update); what each step actually ran is the
        # sample, described in sample_config
        line = {"metric": METRIC, "value": ups, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": W_, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": describe(args.workload, cases, sum(c.updates_per_iteration() for c in cases), world),
                "sample": sample, "sample_config": sample_config(case, procs),
                "cpu_baseline": {"value": ups, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample,
                                 "host": host_info()},
                "e2e": {"value": ups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch
    from paper_2605_03479_gb300 import hbugks as hb

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = f"cuda:{local}"
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    s = hb.Solver(cases, device=dev, stream=stream)
    if args.micro_variant:
        mv = [int(x) for x in args.micro_variant.split(",")]
        for k in range(len(cases)):
            s.set_micro_variant(k, *mv)
    s.set_loop_mode(args.loop_mode)
    s.init_uniform(-1, 1.0, 0.0, 0.0, 1.0)
    s.enqueue_iterations(W_)
    torch.cuda.synchronize()

    clk = Clocks(torch.cuda.current_device())
    clk.start()
    time.sleep(0.25)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.enqueue_iterations(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    ms = slowest_rank_ms(e0.elapsed_time(e1) / args.steps, dist, dev)
    upd = sum(c.updates_per_iteration() for c in cases)
    value = job_updates_per_s(upd, world, ms)
    # per iteration: the iteration's kernels (and the device-side loop test); per call: the status reset (and
    # the kernel that sets the loop count)
    launches = s.launches_per_iteration() * args.steps + (2 if args.loop_mode == 0 else 1)

    # per-kernel times (CUDA events around each launch on the kernels' stream), roofline of the top kernel
    kms = s.profile_kernels(3)
    names = ("face_moments", "face_params", "macro_update", "micro_update", "residual")
    top = int(np.argmax(kms))
    bytes_per_update = 16 if case.precision == 1 else 32      # read + write of (h, b), each once
    peak, peak_kind = peaks()
    alg = {"micro_update": bytes_per_update, "face_moments": bytes_per_update // 2}
    roof = None
    if names[top] in alg:
        ach = alg[names[top]] * upd / (kms[top] * 1e-3) / 1e9
        # DRAM bytes per update of the micro update (dram__bytes_read.sum + dram__bytes_write.sum of one ncu
        # launch of k4_cells on the 64x64-cell thermal cavity with the 64x64 velocity grid and N_T = 11, per
        # micro-update variant), scaled by updates; only where the launches match that capture: the same
        # variant, the 64x64 velocity grid, N_T = 11
        traffic = None
        variants = {s.micro_variant(k) for k in range(len(cases))}
        if names[top] == "micro_update" and case.precision == 1 and len(variants) == 1 and all(
                c.nu == 64 and c.nv == 64 and c.nt == 11 for c in cases):
            per_update = K4_TRAFFIC_64.get(next(iter(variants)))
            traffic = per_update * upd if per_update else None
        roof = {"kernel": names[top], "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": peak_kind, "traffic": traffic,
                "algorithmic_bytes_per_update": alg[names[top]]}
    kernel_ms = {n: float(v) for n, v in zip(names, kms)}

    # end to end through the public API: upload the initial state from pinned host memory, iterate, read back
    # every harmonic field
    e2e = None
    if not args.no_e2e and len(cases) > 1:
        e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
               "what": "not measured for multi-case workloads (FP64 host copies of every case's state)"}
    elif not args.no_e2e:
        nt, nc, nv = case.nt, case.nc, case.nvel
        from paper_2605_03479_gb300 import inputs as I
        Wr, hr, br = I.initial_state(I.make_case("one", 1, case.nu, kn=case.kn, st=case.st,
                                                 nh=case.n_harmonics, drive="rest", half_width=case.umax))
        Wp = torch.empty((nt, nc, 4), dtype=torch.float64, pin_memory=True)
        hp = torch.empty((nt, nc, nv), dtype=torch.float64, pin_memory=True)
        bp = torch.empty((nt, nc, nv), dtype=torch.float64, pin_memory=True)
        Wp.copy_(torch.from_numpy(Wr[:, :1, :]).expand(nt, nc, 4))
        hp.copy_(torch.from_numpy(hr[:, :1, :]).expand(nt, nc, nv))
        bp.copy_(torch.from_numpy(br[:, :1, :]).expand(nt, nc, nv))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_state(0, Wp.numpy(), hp.numpy(), bp.numpy())
        rc, its, res = s.iterate(args.steps)
        outs = [s.harmonic(0, k) for k in range(case.n_harmonics + 1)]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        h2d = Wp.numel() * 8 + hp.numel() * 8 + bp.numel() * 8
        d2h = sum(o.size * 16 for o in outs) + 32 * math.ceil(args.steps / 16)
        e2e = {"value": upd * world * args.steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "what": ("set_state from pinned host FP64 arrays + iterate(steps) with residual reads + all "
                        "harmonic fields to host, host wall clock")}

    cpu = None
    if rank == 0 and not args.no_cpu:
        # the oracle on every usable host core (the baseline), and on one core
        procs = usable_cores()
        ups, sec, n, sample = run_oracle(case, 2, 0, min_seconds=10.0, procs=procs)
        ups1, sec1, n1, sample1 = run_oracle(case, 2, 0, min_seconds=8.0, procs=1)
        cpu = {"value": ups, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample,
               "sample_config": sample_config(case, procs), "host": host_info(),
               "single_core": {"value": ups1, "unit": UNIT, "cores": 1, "sample": sample1}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": W_, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32-split" if case.precision == 1 else "f64",
                "data": "synthetic",
                "config": describe(args.workload, cases, upd, world),
                "roofline": roof, "kernel_ms": kernel_ms,
                "micro_variants": sorted({s.micro_variant(k) for k in range(len(cases))}),
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "loop": "device-side (conditional while graph)" if args.loop_mode == 0 else "host-launched graphs of 16"}
        print(json.dumps(line), flush=True)
    s.destroy()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
