"""Benchmark of the fused limited-convection SSP-RK3 step (one JSON line).

Workload (default): the 256^3 periodic Taylor-Green case -- [0, 2pi]^3,
velocity from the discrete curl of an edge-sampled stream function,
sine-sum plus cube-step scalar, CFL 0.4, superbee, FP64.  A step is one
SSP-RK3 step = three fused stage launches over all cells; the metric is face
updates per second, |F| x 3 stages x steps / time.  Inputs (theta 134 MB,
u_f 403 MB in FP64) are larger than the 129 MB L2, so no flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the CPU oracle (the reference for this path) on
the host cores instead, each step a bounded sample of the same workload.
Under torchrun every rank runs an independent replica (weak scaling);
rank 0 prints the line.
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
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
# FP64 pipe: 2 lane-operations per clock per SM (1.25 TFLOP/s dense nominal,
# an FMA counting two) x 152 SMs x 2070 MHz maximum SM clock
FP64_OPS_PEAK = 2 * 152 * 2.070e9


def peaks():
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# Algorithmic HBM bytes per cell of one stage: theta in + u_f (3 faces) +
# theta out, plus theta^n for stages 2-3.
def stage_bytes_per_cell(es, stage):
    return es * (1 + 3 + 1 + (1 if stage > 0 else 0))


# FP64 operations per cell of one stage in this formulation: per face one
# difference, one fma (theta_f) and one product (flux); per cell six fmas
# (the six face fluxes) and two more for the RK combination of stages 2-3.
def stage_fp64_ops_per_cell(lim, stage):
    per_face = {"upwind": 1, "central": 3, "minmod": 3, "superbee": 3, "smart": 5,
                "vanleer": 6}[lim]
    return 3 * per_face + 6 + (2 if stage > 0 else 0)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"], f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def build_workload(n, lim):
    import workloads as W
    return W.config_taylor_green(n=n, seed=1, nsteps=100, limiter=lim)


# ------------------------------------------------------------------ ours
def run_ours(args):
    import numpy as np
    import torch

    import paper_2110_03044_gb300 as fl

    ws_, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws_ > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    fl.build()
    n, lim = args.n, args.limiter
    wl = build_workload(n, lim)
    dt64 = torch.float64 if args.dtype == "f64" else torch.float32
    es = 8 if args.dtype == "f64" else 4
    mesh = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    F = mesh.n_faces
    C = mesh.n_cells
    th_host = torch.tensor(wl.theta0, dtype=dt64)
    u_host = torch.tensor(wl.u, dtype=dt64)
    th = th_host.cuda()
    u = u_host.cuda()
    ws_t, ws_bytes = fl.workspace_for(mesh, dt64, 3)
    stream = torch.cuda.current_stream()

    def step(nsteps):
        fl.fl_step_rk(mesh.handle, lim, dt64, 3, wl.dt, nsteps, th, u, ws_t, ws_bytes, stream)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # clocks are sampled from the start of the warm-up to the end of the
    # timed region (nvidia-smi samples every 100 ms)
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step(1)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        time.sleep(0.25)
    ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    stages = 3 * args.steps
    launch_ms = ms / stages
    face_updates = F * stages * ws_
    value = face_updates / (ms * 1e-3)

    # ---- roofline of the stage kernel (all launches in the region are it)
    hbm_peak, peak_kind = peaks()
    bytes_step = sum(stage_bytes_per_cell(es, s) for s in range(3)) * C
    gbs = bytes_step * args.steps / (ms * 1e-3) / 1e9
    ops_step = sum(stage_fp64_ops_per_cell(lim, s) for s in range(3)) * C
    roof_hbm = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(gbs / hbm_peak, 4), "traffic": args.traffic,
                "peak_kind": peak_kind + " copy bandwidth"}
    if args.dtype == "f64":
        ach = ops_step * args.steps / (ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 4), "peak": round(FP64_OPS_PEAK / 1e12, 4),
                "unit": "T FP64 ops/s", "frac": round(ach * 1e12 / FP64_OPS_PEAK, 4),
                "traffic": args.traffic,
                "peak_kind": "FP64 pipe, 2 ops/clk/SM x 152 SMs x 2070 MHz (nominal)"}
    else:
        roof = roof_hbm

    # ---- end to end through the C ABI: pinned host theta and u_f copied in,
    # theta copied back, every step
    e2e = None
    if not args.no_e2e:
        th_pin = th_host.pin_memory()
        u_pin = u_host.pin_memory()
        out_pin = torch.empty_like(th_pin).pin_memory()
        for _ in range(2):
            th.copy_(th_pin, non_blocking=True)
            u.copy_(u_pin, non_blocking=True)
            step(1)
            out_pin.copy_(th, non_blocking=True)
        torch.cuda.synchronize()
        k = max(3, args.steps // 2)
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(k):
            th.copy_(th_pin, non_blocking=True)
            u.copy_(u_pin, non_blocking=True)
            step(1)
            out_pin.copy_(th, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_e = ev0.elapsed_time(ev1)
        e2e = {"value": F * 3 * k * ws_ / (ms_e * 1e-3), "unit": "face-updates/s",
               "h2d_bytes_per_step": (C + F) * es, "d2h_bytes_per_step": C * es,
               "steps": k, "ms_per_step": ms_e / k}

    variants = {}
    if not args.no_variants:
        for vd in ("f64", "f32"):
            for vl in ("minmod", "vanleer", "superbee", "smart"):
                if vd == args.dtype and vl == lim:
                    continue
                vt = torch.float64 if vd == "f64" else torch.float32
                tv = th_host.to(vt).cuda()
                uv = u_host.to(vt).cuda()
                wv, nb = fl.workspace_for(mesh, vt, 3)
                for _ in range(2):
                    fl.fl_step_rk(mesh.handle, vl, vt, 3, wl.dt, 1, tv, uv, wv, nb, stream)
                torch.cuda.synchronize()
                kk = 10
                ev0.record(stream)
                fl.fl_step_rk(mesh.handle, vl, vt, 3, wl.dt, kk, tv, uv, wv, nb, stream)
                ev1.record(stream)
                torch.cuda.synchronize()
                mv = ev0.elapsed_time(ev1)
                esv = 8 if vd == "f64" else 4
                bv = sum(stage_bytes_per_cell(esv, s) for s in range(3)) * C * kk
                variants["%s_%s" % (vd, vl)] = {
                    "face_updates_per_s": F * 3 * kk / (mv * 1e-3),
                    "ms_per_step": mv / kk,
                    "hbm_gbs": bv / (mv * 1e-3) / 1e9}
                del tv, uv, wv

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(wl, lim, args.cpu_budget)

    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": "limited-convection face-updates/s (fused SSP-RK3 step)",
        "value": value,
        "unit": "face-updates/s",
        "n_gpus": ws_,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": args.dtype,
        "data": "synthetic (seeded Taylor-Green velocity and sine+cube scalar)",
        "config": {"workload": "taylor_green_%d^3_ssprk3_cfl0.4" % n, "limiter": lim,
                   "cells": C, "faces": F, "rk_order": 3,
                   "l2": "inputs larger than L2 (theta %d MB + u_f %d MB), no flush"
                         % (C * es // 2**20, F * es // 2**20),
                   "parallelism": "replicas" if ws_ > 1 else "single"},
        "roofline": roof,
        "roofline_hbm": roof_hbm,
        "stage_launch_ms": launch_ms,
        "gpu_launches": stages,
        "clocks": clk.summary(),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "variants": variants,
    }
    print(json.dumps(line))


def cpu_baseline(wl, lim, budget_s):
    """The oracle as it stands on the host cores: one SSP-RK3 stage of the
    same mesh and fields (all cells), repeated while within budget."""
    import oracle
    threads = oracle.set_threads(os.cpu_count() or 1)
    om = oracle.OracleMesh(wl.mesh)
    t0 = time.perf_counter()
    reps = 0
    y = None
    while True:
        y = oracle.stage(om, lim, 3, 0, wl.dt, wl.theta0, wl.theta0, wl.u)
        reps += 1
        el = time.perf_counter() - t0
        if el > budget_s or reps >= 10:
            break
    del y
    return {"value": om.F * reps / el, "unit": "face-updates/s", "cores": threads,
            "kind": "oracle",
            "sample": "%d SSP-RK3 stage(s) over the full %d-cell mesh, FP64, OpenMP" % (
                reps, om.C)}


# -------------------------------------------------------------- reference
def run_reference(args):
    ws_, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = build_workload(args.n, args.limiter)
    threads = oracle.set_threads(os.cpu_count() or 1)
    om = oracle.OracleMesh(wl.mesh)
    for _ in range(args.warmup):
        oracle.stage(om, args.limiter, 3, 0, wl.dt, wl.theta0, wl.theta0, wl.u)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.stage(om, args.limiter, 3, 0, wl.dt, wl.theta0, wl.theta0, wl.u)
    el = time.perf_counter() - t0
    value = om.F * args.steps / el
    sample = "each step: one SSP-RK3 stage of the full %d-cell mesh, FP64" % om.C
    line = {
        "impl": "reference",
        "metric": "limited-convection face-updates/s (fused SSP-RK3 step)",
        "value": value, "unit": "face-updates/s", "n_gpus": ws_, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Taylor-Green velocity and sine+cube scalar)",
        "config": {"workload": "taylor_green_%d^3_ssprk3_cfl0.4" % args.n,
                   "limiter": args.limiter},
        "cpu_baseline": {"value": value, "unit": "face-updates/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "face-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--limiter", default="superbee")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu DRAM bytes per stage launch of the current kernel, if measured")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
