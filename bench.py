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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0

NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal

# The FP64 stage kernel is bound by the FP64 pipe, not by HBM: the busy
# fraction of that pipe in one ncu capture of the current kernel (the
# profile summary named beside it), reported next to the HBM roofline.
NCU_FP64_PIPE = {
    ("f64", "superbee", 256): (0.842, "sm__inst_executed_pipe_fp64, RK stage 2 launch, "
                               "profiles/k_struct_stage_traffic_tg256.md"),
    ("f64", "vanleer", 256): (0.626, "sm__inst_executed_pipe_fp64, RK stage 2 launch, "
                              "profiles/k_struct_stage_traffic_tg256.md"),
    ("f64", "smart", 256): (0.819, "sm__inst_executed_pipe_fp64, RK stage 2 launch, "
                            "profiles/k_struct_stage_traffic_tg256.md"),
}


# DRAM bytes (read + write) per launch of the dominant stage kernel at 256^3,
# from one ncu capture of the current kernels (profiles/ keeps the summaries):
# FP64 superbee, RK stages 2-3 (65 % of the step's kernel time); FP32
# superbee TMA kernel, RK stage 1.  Keyed by (dtype, limiter, n).
NCU_TRAFFIC = {
    ("f64", "superbee", 256): (808.2e6, "k_struct_stage<double, SUPERBEE, COMBINE, PRE>, "
                               "algorithmic 805.3e6 (48 B x 16.8M cells), "
                               "profiles/k_struct_stage_traffic_tg256.md"),
    ("f64", "vanleer", 256): (832.6e6, "k_struct_stage<double, VANLEER, COMBINE, PRE>, "
                              "algorithmic 805.3e6, profiles/k_struct_stage_traffic_tg256.md"),
    ("f64", "smart", 256): (829.6e6, "k_struct_stage<double, SMART, COMBINE, PRE>, "
                            "algorithmic 805.3e6, profiles/k_struct_stage_traffic_tg256.md"),
    ("f32", "superbee", 256): (330.8e6, "k_struct_stage_tma<SUPERBEE, PLAIN>, "
                               "algorithmic 335.5e6 (20 B x 16.8M cells), "
                               "profiles/k_struct_stage_traffic_tg256.md"),
}


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


# FP64 operations per cell of one stage in the kernel's formulation: per
# face one difference and the limited face value (one fma for minmod /
# superbee / central / van Leer, two for SMART);
# per cell six fmas w theta_f (the flux product folded into the update with
# the pre-scaled velocity w = dt (A/V) u) and two more for the RK blend of
# stages 2-3.  Superbee: 12 + 14 + 14 = 40 per SSP-RK3 step.
def stage_fp64_ops_per_cell(lim, stage):
    # (van Leer's quotient runs in paired FP32 off the FP64 pipe: Delta and
    # one fma per face, as for superbee)
    per_face = {"upwind": 1, "central": 2, "minmod": 2, "superbee": 2, "smart": 3,
                "vanleer": 2}[lim]
    return 3 * per_face + 6 + (2 if stage > 0 else 0)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons, every 100 ms.

    Each sample carries nvidia-smi's own timestamp, so the summary keeps the
    samples taken inside the timed region (mark() brackets it with the wall
    clock); entering waits for the first sample, so that the sampler is
    running before the region starts."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 10 and self.proc.poll() is None:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self, t0, t1):
        """The timed region's wall-clock bounds (time.time())."""
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)  # the sample that closes the region
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        import datetime
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        inside = rows
        if self.window is not None:
            # a sample stands for the 100 ms before it
            t0, t1 = self.window
            inside = [r for r in rows if t0 < r[0] <= t1 + 0.1]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                    "samples": 0}
        reasons = set()
        for r in inside:
            for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"], r[3]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median([r[1] for r in inside]), "sm_max_mhz": inside[-1][2],
                "reasons": sorted(reasons), "samples": len(inside)}


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
    from paper_2110_03044_gb300.replicas import whole_job_rate

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
    # clocks: the nvidia-smi samples taken inside the timed region
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step(1)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        w0 = time.time()
        ev0.record(stream)
        step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        clk.mark(w0, time.time())
        if dist:
            dist.barrier()
    stages = 3 * args.steps
    # units of all ranks / the slowest rank's time (replicas: no exchange)
    value, ms = whole_job_rate(F * stages, ev0.elapsed_time(ev1), device="cuda")
    launch_ms = ms / stages

    # ---- roofline of the stage kernel (all launches in the region are it):
    # algorithmic bytes of a step (3 stage launches) / the step's time, i.e.
    # the stage launches' average, against the measured copy bandwidth
    hbm_peak, peak_kind = peaks()
    traffic, traffic_note = args.traffic, None
    if traffic is None and (args.dtype, lim, n) in NCU_TRAFFIC:
        traffic, traffic_note = NCU_TRAFFIC[(args.dtype, lim, n)]
    bytes_step = sum(stage_bytes_per_cell(es, s) for s in range(3)) * C
    gbs = bytes_step * args.steps / (ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(gbs / hbm_peak, 4), "traffic": traffic,
            "traffic_kernel": traffic_note,
            "peak_kind": peak_kind + " copy bandwidth (MEASURED_PEAKS hbm_gbs)"
                         if peak_kind == "measured" else "fallback copy bandwidth",
            "bytes_per_cell_step": bytes_step // C,
            # the same achieved bandwidth against the nominal 7.9 TB/s of HBM3e
            "frac_of_nominal": round(gbs / NOMINAL_HBM_GBS, 4)}
    fp64 = None
    if args.dtype == "f64":
        ops_step = sum(stage_fp64_ops_per_cell(lim, s) for s in range(3)) * C
        pipe = NCU_FP64_PIPE.get((args.dtype, lim, n))
        fp64 = {"bound": "fp64 pipe",
                "fp64_ops_per_cell_step": ops_step // C,
                "achieved_fp64_ops_per_s": ops_step * args.steps / (ms * 1e-3),
                "pipe_busy_ncu": pipe[0] if pipe else None,
                "pipe_busy_source": pipe[1] if pipe else None}

    # ---- end to end through the C ABI: every step copies its inputs (theta
    # and u_f) in from pinned host memory and its result (theta) back out.
    # Two device input sets and two streams for the copies (host->device on
    # one, device->host on the other) let step i's copies overlap the
    # compute of its neighbours, as a streaming caller would run it.
    e2e = None
    if not args.no_e2e:
        th_pin = th_host.pin_memory()
        u_pin = u_host.pin_memory()
        out_pin = [torch.empty_like(th_pin).pin_memory() for _ in range(2)]
        th_d = [torch.empty_like(th) for _ in range(2)]
        u_d = [torch.empty_like(u) for _ in range(2)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        copied = [torch.cuda.Event() for _ in range(2)]
        computed = [torch.cuda.Event() for _ in range(2)]
        freed = [torch.cuda.Event() for _ in range(2)]

        def e2e_steps(k, with_u=True):
            for i in range(k):
                b = i % 2
                if i >= 2:
                    s_in.wait_event(freed[b])      # buffer b: step i-2 computed and read back
                with torch.cuda.stream(s_in):
                    th_d[b].copy_(th_pin, non_blocking=True)
                    if with_u:
                        u_d[b].copy_(u_pin, non_blocking=True)
                copied[b].record(s_in)
                stream.wait_event(copied[b])
                fl.fl_step_rk(mesh.handle, lim, dt64, 3, wl.dt, 1, th_d[b], u_d[b], ws_t,
                              ws_bytes, stream)
                computed[b].record(stream)
                s_out.wait_event(computed[b])
                with torch.cuda.stream(s_out):
                    out_pin[b].copy_(th_d[b], non_blocking=True)
                freed[b].record(s_out)
            stream.wait_event(freed[(k - 1) % 2])
            if k >= 2:
                stream.wait_event(freed[(k - 2) % 2])

        e2e_steps(3)
        torch.cuda.synchronize()
        k = max(4, args.steps // 2)
        ev0.record(stream)
        s_in.wait_stream(stream)
        e2e_steps(k)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_e = ev0.elapsed_time(ev1)
        # the copies alone, for the record: one step's H2D and D2H, serial
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        th_d[0].copy_(th_pin, non_blocking=True)
        u_d[0].copy_(u_pin, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        h2d_ms = c0.elapsed_time(c1)
        # for the record: the same loop with the velocity uploaded once (a
        # steady flow kept on the device), each step moving only theta in
        # and out
        for b in range(2):
            u_d[b].copy_(u_pin)
        e2e_steps(3, with_u=False)
        torch.cuda.synchronize()
        ev0.record(stream)
        s_in.wait_stream(stream)
        e2e_steps(k, with_u=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_s = ev0.elapsed_time(ev1)
        e2e = {"value": F * 3 * k * ws_ / (ms_e * 1e-3), "unit": "face-updates/s",
               "h2d_bytes_per_step": (C + F) * es, "d2h_bytes_per_step": C * es,
               "steps": k, "ms_per_step": ms_e / k,
               "h2d_gbs": (C + F) * es / (h2d_ms * 1e-3) / 1e9,
               "overlap": "copies of neighbouring steps overlap compute (2 buffers, 2 copy streams)",
               "velocity_resident": {"value": F * 3 * k * ws_ / (ms_s * 1e-3),
                                     "ms_per_step": ms_s / k, "h2d_bytes_per_step": C * es,
                                     "d2h_bytes_per_step": C * es}}

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

    # the other configurations' headline numbers, on the same GPU (one rank)
    configs = None
    if ws_ == 1 and not args.no_configs:
        del th, u, ws_t
        torch.cuda.empty_cache()
        configs = run_default_configs(args)

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
        "fp64_pipe": fp64,
        "stage_launch_ms": launch_ms,
        # the stage launches plus, in FP64, the one velocity pre-scaling
        # launch of the fl_step_rk call
        "gpu_launches": stages + (1 if args.dtype == "f64" else 0),
        "clocks": clk.summary(),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "variants": variants,
        "configs": configs,
    }
    print(json.dumps(line))


def run_default_configs(args):
    """Configurations 0, 2, 3 and 4 of the benchmark set, each in its own
    runner: the 1D rollout, the 256^3 face-based (unstructured storage) SMART
    step with its HBM fraction, batched against separate launches in FP64 and
    FP32, and the adjoint's reverse sweep against the forward rollout."""
    import argparse as ap
    import torch
    out = {}
    sub = ap.Namespace(**vars(args))
    sub.n = 256
    sub.no_cpu = True
    for name, fn in (("1d", run_config_1d), ("unstructured", run_config_unstructured),
                     ("batched", run_config_batched), ("adjoint", run_config_adjoint)):
        try:
            out[name] = fn(sub)
        except Exception as e:  # a failing runner must not hide the headline line
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_config_1d(args):
    """1D periodic advection, 1000 cells, van Leer, forward Euler, 1000 steps
    in one launch of the resident line kernel."""
    import torch

    import paper_2110_03044_gb300 as fl
    import workloads as W
    fl.build()
    wl = W.config_1d()
    m = fl.Mesh.structured(1000, 1, 1, *wl.mesh.h)
    u = torch.tensor(wl.u, device="cuda")
    th = torch.tensor(wl.theta0, device="cuda")
    for _ in range(args.warmup):
        fl.step_rk(m, "vanleer", th.clone(), u, wl.dt, 1000, rk_order=1)
    e0, e1 = _events()
    g = th.clone()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        g.copy_(th)
        fl.step_rk(m, "vanleer", g, u, wl.dt, 1000, rk_order=1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    return {"metric": "1D rollout face-updates/s (1000 Euler steps, one launch)",
            "value": 1000 * 1000 / (ms * 1e-3), "unit": "face-updates/s", "ms_per_rollout": ms,
            "dtype": "f64", "config": {"workload": "1d_n1000_vanleer_euler_1000steps"}}


def run_config_blocked(args):
    """256^3 Taylor-Green SSP-RK3 with temporal blocking (one launch per step,
    each stage's halo recomputed on chip) against the per-stage launches, on
    the same inputs, for every limiter in FP64 and FP32."""
    import torch

    import paper_2110_03044_gb300 as fl
    fl.build()
    n = args.n
    wl = build_workload(n, args.limiter)
    mesh = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    C, F = mesh.n_cells, mesh.n_faces
    stream = torch.cuda.current_stream()
    e0, e1 = _events()
    rows = {}
    for vd in ("f32", "f64"):
        vt = torch.float32 if vd == "f32" else torch.float64
        es = 4 if vd == "f32" else 8
        th = torch.tensor(wl.theta0, dtype=vt, device="cuda")
        u = torch.tensor(wl.u, dtype=vt, device="cuda")
        ws, nb = fl.workspace_for(mesh, vt, 3)
        for lim in ("minmod", "vanleer", "superbee", "smart"):
            res = {}
            for kind, fn in (("blocked", fl.fl_step_rk_blocked), ("per_stage", fl.fl_step_rk)):
                for _ in range(args.warmup):
                    fn(mesh.handle, lim, vt, 3, wl.dt, 1, th, u, ws, nb, stream)
                torch.cuda.synchronize()
                e0.record(stream)
                fn(mesh.handle, lim, vt, 3, wl.dt, args.steps, th, u, ws, nb, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                res[kind] = e0.elapsed_time(e1) / args.steps
            # algorithmic HBM bytes of a blocked step: theta^n, u_f, result
            rows["%s_%s" % (vd, lim)] = {
                "blocked_ms_per_step": res["blocked"],
                "per_stage_ms_per_step": res["per_stage"],
                "speedup": res["per_stage"] / res["blocked"],
                "blocked_face_updates_per_s": F * 3 / (res["blocked"] * 1e-3),
                "blocked_hbm_gbs": (2 * C + F) * es / (res["blocked"] * 1e-3) / 1e9}
        del th, u, ws
    main = rows["%s_%s" % (args.dtype, args.limiter)]
    return {"metric": "limited-convection face-updates/s (temporally blocked SSP-RK3 step)",
            "value": main["blocked_face_updates_per_s"], "unit": "face-updates/s",
            "ms_per_step": main["blocked_ms_per_step"], "steps": args.steps,
            "warmup": args.warmup, "dtype": args.dtype, "gpu_launches": args.steps,
            "config": {"workload": "taylor_green_%d^3_ssprk3_blocked" % n, "cells": C,
                       "faces": F, "limiter": args.limiter},
            "by_variant": rows}


def run_config_stretched(args):
    """A non-uniform n^3 hexahedral box (cell widths stretched up to 3x along
    each axis) as a face-based mesh with face distances (Algorithm 3's
    weights, the general stencil) against the same mesh without them (the
    hexahedral path); SMART, SSP-RK3, FP64, renumbered.  The face velocities
    are the 256^3 Taylor-Green values reused on the stretched geometry."""
    import torch

    import paper_2110_03044_gb300 as fl
    import workloads as W
    fl.build()
    n = args.n
    wl = W.config_taylor_green(n=n, seed=1, nsteps=50, limiter="smart")
    widths = [W.stretched_widths(n, 2 * np.pi, 3.0, s) for s in (21, 22, 23)]
    mesh = W.stretched_mesh(*widths)
    res = {}
    for kind, dist in (("weighted", mesh.distances), ("unweighted", None)):
        t0 = time.perf_counter()
        m = fl.Mesh.from_faces(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas,
                               mesh.volumes, renumber=True, distances=dist)
        t_mesh = time.perf_counter() - t0
        th = m.to_internal(torch.tensor(wl.theta0, device="cuda"), "cell")
        u = m.to_internal(torch.tensor(wl.u, device="cuda"), "face")
        dt = 0.4 * np.min(np.concatenate(widths)) / np.max(np.abs(wl.u))
        nb = fl.fl_workspace_size(m.handle, torch.float64, 3)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup):
            fl.fl_step_rk(m.handle, "smart", torch.float64, 3, dt, 1, th, u, ws, nb)
        e0, e1 = _events()
        torch.cuda.synchronize()
        e0.record()
        fl.fl_step_rk(m.handle, "smart", torch.float64, 3, dt, args.steps, th, u, ws, nb)
        e1.record()
        torch.cuda.synchronize()
        res[kind] = {"ms_per_step": e0.elapsed_time(e1) / args.steps, "mesh_create_s": t_mesh}
        m.close()
        del th, u, ws
    F = mesh.n_faces
    ms = res["weighted"]["ms_per_step"]
    return {"metric": "limited-convection face-updates/s (non-uniform face-based mesh, SSP-RK3)",
            "value": F * 3 / (ms * 1e-3), "unit": "face-updates/s", "ms_per_step": ms,
            "dtype": "f64", "steps": args.steps, "warmup": args.warmup,
            "unweighted_ms_per_step": res["unweighted"]["ms_per_step"],
            "mesh_create_s": {k: v["mesh_create_s"] for k, v in res.items()},
            "config": {"workload": "stretched_hex%d^3_ratio3_smart_ssprk3" % n,
                       "cells": mesh.n_cells, "faces": F}}


def run_config_polyhedra(args):
    """General polyhedra on the fused face-based kernel: a periodic box of
    64^3 cubes split into 6 Kuhn tetrahedra each, and one of 80^3 cubes split
    into 2 triangular prisms each (renumbered); seeded mixed-sign face
    velocities and the sine-plus-cube scalar; SMART, SSP-RK3, FP64 and FP32."""
    import torch

    import paper_2110_03044_gb300 as fl
    import workloads as W
    fl.build()
    rows = {}
    for name, make in (("tet64", lambda: W.tet_mesh(64)), ("prism80", lambda: W.prism_mesh(80))):
        mesh = make()
        t0 = time.perf_counter()
        m = fl.Mesh.from_faces(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas,
                               mesh.volumes, renumber=True)
        t_mesh = time.perf_counter() - t0
        rng = np.random.default_rng(1)
        th0 = rng.uniform(0, 1, mesh.n_cells)
        u0 = W.mixed_sign_velocity(mesh.n_faces, 2)
        dt = 0.05 * np.min(mesh.volumes) / np.max(mesh.areas) / np.max(np.abs(u0))
        for vd, vt in (("f64", torch.float64), ("f32", torch.float32)):
            th = m.to_internal(torch.tensor(th0, dtype=vt, device="cuda"), "cell")
            u = m.to_internal(torch.tensor(u0, dtype=vt, device="cuda"), "face")
            nb = fl.fl_workspace_size(m.handle, vt, 3)
            ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
            for _ in range(args.warmup):
                fl.fl_step_rk(m.handle, "smart", vt, 3, dt, 1, th, u, ws, nb)
            e0, e1 = _events()
            torch.cuda.synchronize()
            e0.record()
            fl.fl_step_rk(m.handle, "smart", vt, 3, dt, args.steps, th, u, ws, nb)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            rows["%s_%s" % (name, vd)] = {"ms_per_step": ms, "cells": mesh.n_cells,
                                          "faces": mesh.n_faces,
                                          "face_updates_per_s": mesh.n_faces * 3 / (ms * 1e-3),
                                          "mesh_create_s": t_mesh}
            del th, u, ws
        m.close()
    main = rows["tet64_f64"]
    return {"metric": "limited-convection face-updates/s (tetrahedra, SSP-RK3)",
            "value": main["face_updates_per_s"], "unit": "face-updates/s",
            "ms_per_step": main["ms_per_step"], "dtype": "f64", "steps": args.steps,
            "warmup": args.warmup,
            "config": {"workload": "kuhn_tet_64^3x6_smart_ssprk3", "cells": main["cells"],
                       "faces": main["faces"]},
            "by_mesh": rows}


def run_config_unstructured(args):
    """256^3 hex mesh in seeded random cell/face order with half of the faces
    reoriented (face-cell incidence as int32 pairs), renumbered by the
    library; SMART, SSP-RK3, FP64."""
    import torch

    import paper_2110_03044_gb300 as fl
    import workloads as W
    fl.build()
    n = args.n
    wl = W.config_taylor_green(n=n, seed=1, nsteps=50, limiter="smart")
    pm, cp, fp, flip = W.permuted_mesh(wl.mesh, seed=2)
    up = W.permute_face_field(wl.u, fp, flip)
    thp = W.permute_cell_field(wl.theta0, cp)
    t0 = time.perf_counter()
    m = fl.Mesh.from_faces(pm.n_cells, pm.face_cells, pm.normals, pm.areas, pm.volumes,
                           renumber=True)
    t_mesh = time.perf_counter() - t0
    # the fields cross into the library's numbering once, by its own kernels
    th = m.to_internal(torch.tensor(thp, device="cuda"), "cell")
    u = m.to_internal(torch.tensor(up, device="cuda"), "face")
    nb = fl.fl_workspace_size(m.handle, torch.float64, 3)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        fl.fl_step_rk(m.handle, "smart", torch.float64, 3, wl.dt, 1, th, u, ws, nb)
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record()
    fl.fl_step_rk(m.handle, "smart", torch.float64, 3, wl.dt, args.steps, th, u, ws, nb)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    C, F = pm.n_cells, pm.n_faces
    # algorithmic bytes of the face-based step: per stage theta
    # in/out, u_f, the face records (c0, c1, up0, up1) and the cell -> 6 faces
    # lists, plus theta^n in stages 2-3 (352 B per cell and SSP-RK3 step)
    hbm_peak, peak_kind = peaks()
    bpc = 352
    gbs = bpc * C / (ms * 1e-3) / 1e9
    m.close()
    return {"metric": "limited-convection face-updates/s (unstructured storage, SSP-RK3)",
            "value": F * 3 / (ms * 1e-3), "unit": "face-updates/s", "ms_per_step": ms,
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
                         "unit": "GB/s", "frac": round(gbs / hbm_peak, 4), "traffic": None,
                         "bytes_per_cell_step": bpc},
            "dtype": "f64", "mesh_create_s": t_mesh,
            "config": {"workload": "hex%d^3_permuted_flipped_smart_ssprk3" % n, "cells": C,
                       "faces": F}}


def run_config_partition(args):
    """The 256^3 hex Taylor-Green mesh as a face-based mesh, SMART, SSP-RK3,
    FP64, cut into --parts parts by the graph partitioner.  One GPU runs
    part 0's three stages (its interior and rim launches on its local mesh;
    the halo exchange, a transport between GPUs, is left out) and fl_step_rk
    on the whole face-based mesh, both in the caller's order and renumbered
    by the library; the part's time against 1/P of the whole step is the
    compute price of the partition (faces on a cut evaluated by both parts,
    two launches per stage, blocks that stop at the interior's edge)."""
    import torch

    import paper_2110_03044_gb300 as fl
    import workloads as W
    from paper_2110_03044_gb300.partition import (GraphRollout, LocalGraphTransport, build_parts,
                                                  partition_graph)
    fl.build()
    n, P = args.n, args.parts
    wl = W.config_taylor_green(n=n, seed=1, nsteps=50, limiter="smart")
    mesh = wl.mesh
    t0 = time.perf_counter()
    part = partition_graph(mesh.n_cells, mesh.face_cells, P)
    parts = build_parts(mesh.n_cells, mesh.face_cells, part)
    t_part = time.perf_counter() - t0
    gp = parts[0]
    ug = torch.tensor(wl.u, device="cuda")
    thg = torch.tensor(wl.theta0, device="cuda")
    e0, e1 = _events()

    def time_whole(renumber):
        m = fl.Mesh.from_faces(mesh.n_cells, mesh.face_cells, mesh.normals, mesh.areas,
                               mesh.volumes, renumber=renumber)
        th, u = m.to_internal(thg, "cell"), m.to_internal(ug, "face")
        nb = fl.fl_workspace_size(m.handle, torch.float64, 3)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        fl.fl_step_rk(m.handle, "smart", torch.float64, 3, wl.dt, args.warmup, th, u, ws, nb)
        torch.cuda.synchronize()
        e0.record()
        fl.fl_step_rk(m.handle, "smart", torch.float64, 3, wl.dt, args.steps, th, u, ws, nb)
        e1.record()
        torch.cuda.synchronize()
        m.close()
        return e0.elapsed_time(e1) / args.steps

    class NoExchange(LocalGraphTransport):
        """part 0 alone: its rollout loop with an exchange that moves nothing"""

        def exchange(self, gp_, x):
            return None

    def time_part(renumber, overlap=True):
        ro = GraphRollout(mesh, gp, ug, "smart", torch.float64, wl.dt, transport=NoExchange(),
                          renumber=renumber, overlap=overlap)
        tl = ro.local_field(thg)
        ro.step(tl, 3, args.warmup)
        torch.cuda.synchronize()
        e0.record()
        ro.step(tl, 3, args.steps)
        e1.record()
        torch.cuda.synchronize()
        ro.close()
        return e0.elapsed_time(e1) / args.steps

    res = {}
    for renumber in (False, True):
        key = "renumbered" if renumber else "caller_order"
        w, p_, q_ = time_whole(renumber), time_part(renumber), time_part(renumber, False)
        # with overlap: interior and rim launches per stage; without: one
        res[key] = {"whole_mesh_ms_per_step": w, "part_ms_per_step": p_,
                    "part_over_whole_per_part": p_ / (w / P),
                    "part_one_launch_ms_per_step": q_,
                    "part_one_launch_over_whole_per_part": q_ / (w / P)}
    F = mesh.n_faces
    head = res["renumbered"]
    return {"metric": "partitioned face-based SSP-RK3: one part's step time against 1/P of the "
                      "whole mesh's (both renumbered)",
            "value": head["part_over_whole_per_part"], "unit": "ratio",
            "higher_is_better": False, "dtype": "f64", "results": res,
            "whole_face_updates_per_s": F * 3 / (head["whole_mesh_ms_per_step"] * 1e-3),
            "partition_s": t_part,
            "part": {"owned": gp.n_owned, "interior": gp.n_interior,
                     "halo": int(gp.halo_ids.shape[0]),
                     "local_faces": int(gp.face_ids.shape[0]), "faces_per_part_ideal": F // P},
            "config": {"workload": "hex%d^3_faces_smart_ssprk3_%dparts" % (n, P),
                       "cells": mesh.n_cells, "faces": F, "parts": P,
                       "exchange": "not timed (no second GPU)"}}


def run_config_batched(args):
    """64 periodic boxes, sizes seeded in [32, 128]^3, each with its own
    solenoidal velocity and scalar, van Leer, SSP-RK3: one persistent launch
    per stage (graph-replayed) against 64 single-mesh launches per stage
    captured in one CUDA graph."""
    import torch

    import paper_2110_03044_gb300 as fl
    import workloads as W
    from paper_2110_03044_gb300.replicas import lpt_partition, whole_job_rate
    ws_, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws_ > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    fl.build()
    all_dims = W.batched_box_dims()
    # boxes split across ranks by cell count (no exchange between boxes)
    mine = lpt_partition([int(np.prod(d)) for d in all_dims], ws_)[rank]
    dims = [all_dims[i] for i in mine]
    boxes = [W.random_box(all_dims[i], 1000 + i) for i in mine]
    out = {}
    want = getattr(args, "batched_dtypes", "f64,f32").split(",")
    for dname, dt in (("f64", torch.float64), ("f32", torch.float32)):
        if dname not in want:
            continue
        meshes = [fl.Mesh.structured(*d, *b[0].h) for d, b in zip(dims, boxes)]
        batch = fl.fl_batch_create([mm.handle for mm in meshes])
        th = [torch.tensor(b[1], dtype=dt, device="cuda") for b in boxes]
        us = [torch.tensor(b[2], dtype=dt, device="cuda") for b in boxes]
        dts = [b[3] for b in boxes]
        nb = fl.fl_batch_workspace_size(batch, dt, 3)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        fl.fl_batch_step_rk(batch, "vanleer", dt, 3, dts, 2, th, us, ws, nb)  # tunes once
        e0, e1 = _events()
        torch.cuda.synchronize()
        if ws_ > 1:
            dist.barrier()
        e0.record()
        fl.fl_batch_step_rk(batch, "vanleer", dt, 3, dts, args.steps, th, us, ws, nb)
        e1.record()
        torch.cuda.synchronize()
        F = sum(mm.n_faces for mm in meshes)
        rate_b, ms_tot = whole_job_rate(F * 3 * args.steps, e0.elapsed_time(e1), device="cuda")
        ms_b = ms_tot / args.steps
        # separate launches: one fl_step_rk per box and step, captured in a graph
        wss = [torch.empty(fl.fl_workspace_size(mm.handle, dt, 3), dtype=torch.uint8,
                           device="cuda") for mm in meshes]
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for mm, t, u, d, w in zip(meshes, th, us, dts, wss):
                fl.fl_step_rk(mm.handle, "vanleer", dt, 3, d, 1, t, u, w, w.numel(), s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for mm, t, u, d, w in zip(meshes, th, us, dts, wss):
                fl.fl_step_rk(mm.handle, "vanleer", dt, 3, d, 1, t, u, w, w.numel(), s)
        g.replay()
        torch.cuda.synchronize()
        if ws_ > 1:
            dist.barrier()
        e0.record()
        for _ in range(args.steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        rate_s, ms_tot = whole_job_rate(F * 3 * args.steps, e0.elapsed_time(e1), device="cuda")
        ms_s = ms_tot / args.steps
        Cm = sum(mm.n_cells for mm in meshes)
        out[dname] = {"batched_ms_per_step": ms_b, "separate_ms_per_step": ms_s,
                      "batched_ps_per_cell_step": ms_b * 1e9 / Cm,
                      "batched_face_updates_per_s": rate_b,
                      "separate_face_updates_per_s": rate_s,
                      "speedup": ms_s / ms_b,
                      "tiling": dict(zip(["kind", "cells_per_thread", "warps", "z_chunk"],
                                         fl.fl_batch_tiling(batch, "vanleer", dt, 3)))}
        if getattr(args, "tiling_sweep", False):
            # every candidate of the autotuner, fixed in turn and timed alike
            sweep = {}
            cands = [(0, 1, 8, z) for z in (8, 16, 32, 64)]
            if dt == torch.float32:
                cands += [(1, c, w, z) for c in (1, 2, 4) for w in (4, 8) for z in (16, 32, 64)]
                cands += [(2, 4, w, z) for w in (1, 2, 4, 8) for z in (16, 32, 64)]
            for t in cands:
                fl.fl_batch_set_tiling(batch, "vanleer", dt, 3, *t)
                fl.fl_batch_step_rk(batch, "vanleer", dt, 3, dts, 2, th, us, ws, nb)
                torch.cuda.synchronize()
                e0.record()
                fl.fl_batch_step_rk(batch, "vanleer", dt, 3, dts, args.steps, th, us, ws, nb)
                e1.record()
                torch.cuda.synchronize()
                sweep["%d/%d/%d/%d" % t] = round(e0.elapsed_time(e1) / args.steps, 4)
            out[dname]["tiling_sweep_ms"] = sweep
        fl.fl_batch_destroy(batch)
        for mm in meshes:
            mm.close()
    C = sum(int(np.prod(d)) for d in all_dims)
    if ws_ > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return None
    head = "f64" if "f64" in out else "f32"
    return {"metric": "batched limited-convection face-updates/s (64 boxes, SSP-RK3)",
            "value": out[head]["batched_face_updates_per_s"], "unit": "face-updates/s",
            "n_gpus": ws_, "scaling": "strong", "dtype": head, "results": out,
            "config": {"workload": "64_boxes_32-128_vanleer_ssprk3", "cells": C,
                       "parallelism": "boxes split by LPT" if ws_ > 1 else "single"}}


def run_config_adjoint(args):
    """128^3 Taylor-Green, superbee, 200 SSP-RK3 steps, checkpoints every 20:
    reverse sweep time (recomputation + adjoint stages) against the forward
    rollout."""
    import torch

    import paper_2110_03044_gb300 as fl
    import workloads as W
    fl.build()
    n, nsteps, every = 128, 200, 20
    wl = W.config_taylor_green(n=n, seed=4, nsteps=nsteps, limiter="superbee")
    tgt = W.smooth_target(wl.mesh.dims, wl.mesh.h, 4)
    m = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    u = torch.tensor(wl.u, device="cuda")
    th0 = torch.tensor(wl.theta0, device="cuda")
    tg = torch.tensor(tgt, device="cuda")
    wsf = torch.empty(fl.fl_workspace_size(m.handle, torch.float64, 3), dtype=torch.uint8,
                      device="cuda")
    nb = fl.fl_adjoint_workspace_size(m.handle, torch.float64, 3, nsteps, every)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g = torch.empty_like(th0)
    e0, e1 = _events()
    fwd, ckf, rev, tot = [], [], [], []
    for rep in range(max(2, args.warmup)):
        th = th0.clone()
        torch.cuda.synchronize()
        e0.record()
        fl.fl_step_rk(m.handle, "superbee", torch.float64, 3, wl.dt, nsteps, th, u, wsf, wsf.numel())
        e1.record()
        torch.cuda.synchronize()
        fwd.append(e0.elapsed_time(e1))
        # forward rollout storing checkpoints, then the reverse sweep
        th = th0.clone()
        e0.record()
        fl.fl_step_rk_checkpointed(m.handle, "superbee", torch.float64, 3, wl.dt, nsteps, every,
                                   th, u, ws, nb)
        e1.record()
        torch.cuda.synchronize()
        ckf.append(e0.elapsed_time(e1))
        lam = th - tg
        torch.cuda.synchronize()
        e0.record()
        fl.fl_step_rk_adjoint_from_checkpoints(m.handle, "superbee", torch.float64, 3, wl.dt,
                                               nsteps, every, u, lam, g, ws, nb)
        e1.record()
        torch.cuda.synchronize()
        rev.append(e0.elapsed_time(e1))
        e0.record()
        fl.fl_step_rk_adjoint(m.handle, "superbee", torch.float64, 3, wl.dt, nsteps, every, th0,
                              u, lam, g, ws, nb)
        e1.record()
        torch.cuda.synchronize()
        tot.append(e0.elapsed_time(e1))
    f, c, r, t = min(fwd[1:]), min(ckf[1:]), min(rev[1:]), min(tot[1:])
    return {"metric": "adjoint / forward time (128^3, 200 SSP-RK3 steps, checkpoints every 20)",
            "value": r / f, "unit": "ratio", "higher_is_better": False, "forward_ms": f,
            "checkpointed_forward_ms": c, "reverse_sweep_ms": r,
            "one_call_gradient_ms": t, "gradient_over_forward": (c + r) / f, "dtype": "f64",
            "config": {"workload": "tg128_superbee_ssprk3_200steps_ckpt20"}}


def run_config_deformation(args):
    """Section 4.1: the sphere in the reversing deformation flow (eq.
    rhodonea) on n^3 hexahedra, superbee, forward Euler, the whole period
    t in [0, 3] as one fl_step_rk_modulated call.  Reports face-updates/s of
    the rollout and the benchmark's own checks: mass drift, bounds, and the
    L1 distance between theta(T) and the initial sphere."""
    import torch

    import paper_2110_03044_gb300 as fl
    import workloads as W
    fl.build()
    n = args.n
    t0 = time.perf_counter()
    # explicit face arrays only where the oracle's CPU baseline needs them
    with_cpu = not args.no_cpu and n <= 288
    wl = W.config_deformation(n, faces=with_cpu)
    t_gen = time.perf_counter() - t0
    g = wl.extra["g"]
    m = fl.Mesh.structured(n, n, n, *wl.mesh.h)
    u = torch.tensor(wl.u, device="cuda")
    th0 = torch.tensor(wl.theta0, device="cuda")
    ws, nb = fl.workspace_for(m, torch.float64, 1)
    th = th0.clone()
    warm = min(wl.nsteps, 20)
    fl.fl_step_rk_modulated(m.handle, "superbee", torch.float64, 1, wl.dt, warm, th, u, g[:warm],
                            ws, nb)
    th.copy_(th0)
    e0, e1 = _events()
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        w0 = time.time()
        e0.record()
        fl.fl_step_rk_modulated(m.handle, "superbee", torch.float64, 1, wl.dt, wl.nsteps, th, u, g,
                                ws, nb)
        e1.record()
        torch.cuda.synchronize()
        clk.mark(w0, time.time())
    ms = e0.elapsed_time(e1)
    out = th.cpu().numpy()
    F = m.n_faces
    m0 = float(wl.theta0.sum())
    ops = stage_fp64_ops_per_cell("superbee", 0) + 1  # + the velocity factor
    ach = ops * m.n_cells * wl.nsteps / (ms * 1e-3) / 1e12
    # an Euler stage moves theta in, u_f (3 faces) and theta out: 40 B per cell
    hbm_peak, _ = peaks()
    gbs = 40.0 * m.n_cells * wl.nsteps / (ms * 1e-3) / 1e9
    cpu = None
    if with_cpu:
        import oracle
        threads = oracle.set_threads(os.cpu_count() or 1)
        om = oracle.OracleMesh(wl.mesh)
        k, t1 = 0, time.perf_counter()
        y = wl.theta0
        while time.perf_counter() - t1 < args.cpu_budget / 2 and k < 50:
            y = oracle.step_modulated(om, "superbee", 1, wl.dt, 1, wl.u, g[k:k + 1], y)
            k += 1
        el = time.perf_counter() - t1
        cpu = {"value": F * k / el, "unit": "face-updates/s", "cores": threads, "kind": "oracle",
               "sample": "%d forward-Euler steps of the %d^3 mesh, FP64, OpenMP" % (k, n)}
    return {"metric": "deformation benchmark face-updates/s (Section 4.1, superbee, Euler)",
            "value": F * wl.nsteps / (ms * 1e-3), "unit": "face-updates/s",
            "ms_per_step": ms / wl.nsteps, "rollout_ms": ms, "steps": wl.nsteps, "dtype": "f64",
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
                         "unit": "GB/s", "frac": round(gbs / hbm_peak, 4), "traffic": None,
                         "bytes_per_cell_step": 40},
            "achieved_fp64_ops_per_s": ach * 1e12,
            "checks": {"mass_rel_drift": abs(float(out.sum()) - m0) / m0,
                       "min": float(out.min()), "max": float(out.max()),
                       "l1_theta_T_vs_sphere": float(np.sum(np.abs(out - wl.theta0)) / n ** 3)},
            "gpu_launches": wl.nsteps + 1, "clocks": clk.summary(), "cpu_baseline": cpu,
            "workload_gen_s": t_gen,
            "config": {"workload": "deformation_sphere_%d^3_T3_superbee_euler" % n,
                       "cells": m.n_cells, "dt": wl.dt, "courant_outflow": 0.5}}


# Algorithmic HBM bytes of one forward-Euler step of the algebraic chain
# (each kernel reads its operands and writes its result once; the gathered
# vector of an SpMV counted once, as in the paper's full-hit column).
def algebraic_step_bytes(C, F, wT, wM):
    ell = 12  # 8-byte value + 4-byte column
    b = 0
    b += 2 * ell * F + 8 * C + 8 * F            # d <- E theta
    b += 3 * 8 * F                              # d <- Q d
    b += wT * ell * F + 8 * C + 8 * F           # r <- T theta
    b += 3 * 8 * F                              # r <- Q r
    b += wT * ell * F + 8 * C + 2 * 8 * F       # r <- r + (-S) theta
    b += 3 * 8 * F                              # r <- r / d
    b += 3 * 8 * F                              # t <- F(r) d
    b += 2 * ell * F + 8 * C + 2 * 8 * F        # t <- t + Pi theta
    b += 3 * 8 * F                              # phi <- u t
    b += wM * ell * C + 8 * F + 8 * C           # R <- M phi
    b += 3 * 8 * C                              # theta <- theta + dt R
    return b


def run_config_decomp(args):
    """256^3 Taylor-Green, superbee, FP64 SSP-RK3 split into z-slabs, one
    per rank, with the halo exchanged before every stage (torch.distributed
    point-to-point, NCCL between GPUs; a single rank exchanges with itself):
    steps with the stage's interior overlapping the exchange, steps that
    exchange first, and (one rank) fl_step_rk on the whole mesh.  Strong
    scaling: the 256^3 mesh is fixed and split."""
    import torch

    import paper_2110_03044_gb300 as fl
    from paper_2110_03044_gb300.decomp import Slab, SlabRollout, TorchTransport
    from paper_2110_03044_gb300.replicas import whole_job_rate
    ws_, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws_ > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    fl.build()
    n, lim = args.n, args.limiter
    wl = build_workload(n, lim)
    dims = (n, n, n)
    slab = Slab(dims, rank, ws_)
    ug = torch.tensor(wl.u, device="cuda")
    thg = torch.tensor(wl.theta0, device="cuda")
    F = 3 * n ** 3
    e0, e1 = _events()
    out = {}
    for overlap in (True, False):
        ro = SlabRollout(slab, wl.mesh.h, ug, lim, torch.float64, wl.dt,
                         transport=TorchTransport(), overlap=overlap)
        tl = ro.local_field(thg)
        ro.step(tl, 3, args.warmup)
        torch.cuda.synchronize()
        if ws_ > 1:
            dist.barrier()
        e0.record()
        ro.step(tl, 3, args.steps)
        e1.record()
        torch.cuda.synchronize()
        rate, ms = whole_job_rate(F * 3 * args.steps / ws_, e0.elapsed_time(e1), device="cuda")
        out["overlap" if overlap else "exchange_first"] = {
            "face_updates_per_s": rate, "ms_per_step": ms / args.steps,
            "launches_per_stage": 3 if overlap and slab.nz_local > 4 else 1}
        ro.close()
    # pencils over (y, z): ranks in a near-square grid; one rank exchanges
    # with itself through the pack and unpack kernels
    from paper_2110_03044_gb300.decomp import Pencil, PencilRollout
    py = max(d for d in range(1, int(ws_ ** 0.5) + 1) if ws_ % d == 0)
    grid = (py, ws_ // py)
    pencil = Pencil(dims, rank, grid)
    for overlap in (True, False):
        ro = PencilRollout(pencil, wl.mesh.h, ug, lim, torch.float64, wl.dt, overlap=overlap)
        tl = ro.local_field(thg)
        ro.step(tl, 3, args.warmup)
        torch.cuda.synchronize()
        if ws_ > 1:
            dist.barrier()
        e0.record()
        ro.step(tl, 3, args.steps)
        e1.record()
        torch.cuda.synchronize()
        rate, ms = whole_job_rate(F * 3 * args.steps / ws_, e0.elapsed_time(e1), device="cuda")
        out["pencil_" + ("overlap" if overlap else "exchange_first")] = {
            "face_updates_per_s": rate, "ms_per_step": ms / args.steps, "grid": list(grid)}
        ro.close()
    if ws_ == 1:
        m = fl.Mesh.structured(n, n, n, *wl.mesh.h)
        ws, nb = fl.workspace_for(m, torch.float64, 3)
        th = thg.clone()
        fl.fl_step_rk(m.handle, lim, torch.float64, 3, wl.dt, args.warmup, th, ug, ws, nb)
        torch.cuda.synchronize()
        e0.record()
        fl.fl_step_rk(m.handle, lim, torch.float64, 3, wl.dt, args.steps, th, ug, ws, nb)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["whole_mesh_fl_step_rk"] = {"face_updates_per_s": F * 3 * args.steps / (ms * 1e-3),
                                        "ms_per_step": ms / args.steps}
        m.close()
    if ws_ > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return None
    return {"metric": "decomposed limited-convection face-updates/s (z-slabs, SSP-RK3)",
            "value": out["overlap"]["face_updates_per_s"], "unit": "face-updates/s",
            "n_gpus": ws_, "scaling": "strong", "dtype": "f64", "results": out,
            "config": {"workload": "taylor_green_%d^3_%s_ssprk3_zslabs" % (n, lim),
                       "halo_planes": slab.halo,
                       "halo_bytes_per_stage_per_rank": 2 * slab.halo * n * n * 8,
                       "transport": "nccl p2p" if ws_ > 1 else "local copy (one rank)",
                       "parallelism": "z-slabs over %d ranks" % ws_}}


def run_config_algebraic(args):
    """The paper's stencil-vs-algebraic comparison (Section 3's Table 2 and
    its roofline study) on GB300: one forward-Euler superbee step of the
    Taylor-Green field on n^3, as the fused stencil kernel (fl_step_rk) and
    as the algebraic chain of Algorithm 1 + Algorithm 5 (8 SpMV / kbin
    launches for theta_f, 3 for the update), both FP64."""
    import torch

    import paper_2110_03044_gb300 as fl
    import workloads as W
    fl.build()
    n = args.n
    h = 2 * np.pi / n
    wl = W.config_taylor_green(n=n, seed=1, nsteps=1, limiter="superbee")
    mesh = wl.mesh
    dt = wl.dt
    u = torch.tensor(wl.u, device="cuda")
    th0 = torch.tensor(wl.theta0, device="cuda")
    C, F = mesh.n_cells, mesh.n_faces
    reps = max(3, args.steps)
    e0, e1 = _events()
    # fused
    m = fl.Mesh.structured(n, n, n, h, h, h)
    ws, nb = fl.workspace_for(m, torch.float64, 1)
    th = th0.clone()
    fl.fl_step_rk(m.handle, "superbee", torch.float64, 1, dt, 2, th, u, ws, nb)
    torch.cuda.synchronize()
    e0.record()
    fl.fl_step_rk(m.handle, "superbee", torch.float64, 1, dt, reps, th, u, ws, nb)
    e1.record()
    torch.cuda.synchronize()
    ms_fused = e0.elapsed_time(e1) / reps
    fused_out = None
    m.close()
    del ws
    # algebraic
    t0 = time.perf_counter()
    a = fl.Algebraic(C, mesh.face_cells, mesh.normals, mesh.areas, mesh.volumes)
    t_asm = time.perf_counter() - t0
    nnz, width, mbytes = a.info()
    ta = th0.clone()
    a.step_euler("superbee", ta, u, dt, 2)
    torch.cuda.synchronize()
    e0.record()
    a.step_euler("superbee", ta, u, dt, reps)
    e1.record()
    torch.cuda.synchronize()
    ms_alg = e0.elapsed_time(e1) / reps
    # the two paths agree (one step from the same state)
    tf = th0.clone()
    m = fl.Mesh.structured(n, n, n, h, h, h)
    fl.step_rk(m, "superbee", tf, u, dt, 1, rk_order=1)
    tb = th0.clone()
    a.step_euler("superbee", tb, u, dt, 1)
    agree = float((tf - tb).abs().max() / tf.abs().max())
    m.close()
    a.close()
    hbm_peak, _ = peaks()
    b_alg = algebraic_step_bytes(C, F, width[1], width[4])
    b_fused = 5 * 8 * C  # theta + u_f (3 faces) + theta out per cell
    gbs_alg = b_alg / (ms_alg * 1e-3) / 1e9
    gbs_fused = b_fused / (ms_fused * 1e-3) / 1e9
    return {"metric": "stencil vs algebraic forward-Euler step (superbee, FP64)",
            "value": ms_alg / ms_fused, "unit": "algebraic time / fused time",
            "higher_is_better": False, "dtype": "f64",
            "fused": {"ms_per_step": ms_fused, "face_updates_per_s": F / (ms_fused * 1e-3),
                      "algorithmic_bytes_per_cell": b_fused / C, "hbm_gbs": gbs_fused,
                      "hbm_frac": gbs_fused / hbm_peak},
            "algebraic": {"ms_per_step": ms_alg, "face_updates_per_s": F / (ms_alg * 1e-3),
                          "algorithmic_bytes_per_cell": b_alg / C, "hbm_gbs": gbs_alg,
                          "hbm_frac": gbs_alg / hbm_peak, "launches_per_step": 11,
                          "matrix_bytes": mbytes, "nnz": dict(zip(["E", "T", "-S", "Pi", "M"], nnz)),
                          "assembly_s": t_asm},
            "paths_agree_rel": agree,
            "config": {"workload": "taylor_green_%d^3_euler_superbee" % n, "cells": C,
                       "faces": F}}


def _cpu_model():
    """The host CPU's model name (lscpu), for the record."""
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return None
    for line in out.splitlines():
        if line.strip().lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    return None


def cpu_baseline(wl, lim, budget_s):
    """The oracle as it stands on the host cores: whole SSP-RK3 steps of the
    same mesh and fields (all cells, three stages each), repeated while within
    budget; then one step on a single thread, for the record."""
    import oracle
    threads = oracle.set_threads(os.cpu_count() or 1)
    om = oracle.OracleMesh(wl.mesh)
    t0 = time.perf_counter()
    reps = 0
    y = wl.theta0
    while True:
        y = oracle.step(om, lim, 3, wl.dt, 1, wl.u, y)
        reps += 1
        el = time.perf_counter() - t0
        if el > budget_s or reps >= 10:
            break
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.step(om, lim, 3, wl.dt, 1, wl.u, wl.theta0)
    el1 = time.perf_counter() - t1
    oracle.set_threads(threads)
    del y
    return {"value": om.F * 3 * reps / el, "unit": "face-updates/s", "cores": threads,
            "kind": "oracle",
            "sample": "%d SSP-RK3 step(s) (3 stages each) over the full %d-cell mesh, FP64, "
                      "OpenMP" % (reps, om.C),
            "single_thread_value": om.F * 3 / el1, "nproc": os.cpu_count(),
            "cpu_model": _cpu_model()}


# -------------------------------------------------------------- reference
def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on all host cores,
    timing whole SSP-RK3 steps (three stages each) of the same 256^3 workload
    and reporting the same metric (face-updates/s = |F| x 3 x steps / time)."""
    ws_, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = build_workload(args.n, args.limiter)
    threads = oracle.set_threads(os.cpu_count() or 1)
    om = oracle.OracleMesh(wl.mesh)
    y = wl.theta0
    for _ in range(args.warmup):
        y = oracle.step(om, args.limiter, 3, wl.dt, 1, wl.u, y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y = oracle.step(om, args.limiter, 3, wl.dt, 1, wl.u, y)
    el = time.perf_counter() - t0
    value = om.F * 3 * args.steps / el
    sample = ("each step: one whole SSP-RK3 step (3 stages) of the full %d-cell mesh, FP64"
              % om.C)
    es = 8
    line = {
        "impl": "reference",
        "metric": "limited-convection face-updates/s (fused SSP-RK3 step)",
        "value": value, "unit": "face-updates/s", "n_gpus": ws_, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Taylor-Green velocity and sine+cube scalar)",
        "config": {"workload": "taylor_green_%d^3_ssprk3_cfl0.4" % args.n,
                   "limiter": args.limiter, "cells": om.C, "faces": om.F, "rk_order": 3,
                   "l2": "inputs larger than L2 (theta %d MB + u_f %d MB), no flush"
                         % (om.C * es // 2**20, om.F * es // 2**20),
                   "parallelism": "single"},
        "cpu_baseline": {"value": value, "unit": "face-updates/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "face-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--limiter", default="superbee")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations' numbers in the default line")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--batched-dtypes", default="f64,f32",
                    help="--config batched: the dtypes to run (comma-separated)")
    ap.add_argument("--tiling-sweep", action="store_true",
                    help="--config batched: also time every decomposition the autotuner tries")
    ap.add_argument("--parts", type=int, default=4,
                    help="--config partition: the number of parts")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu DRAM bytes per stage launch of the current kernel, if measured")
    ap.add_argument("--config", default="tg256",
                    choices=["tg256", "1d", "unstructured", "batched", "adjoint", "deformation",
                             "algebraic", "blocked", "stretched", "polyhedra", "decomp",
                             "partition"])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "tg256":
        run_ours(args)
    else:
        import numpy  # noqa: F401  (the config runners use np)
        fn = {"1d": run_config_1d, "unstructured": run_config_unstructured,
              "batched": run_config_batched, "adjoint": run_config_adjoint,
              "deformation": run_config_deformation,
              "algebraic": run_config_algebraic, "blocked": run_config_blocked,
              "stretched": run_config_stretched,
              "polyhedra": run_config_polyhedra, "decomp": run_config_decomp,
              "partition": run_config_partition}[args.config]
        line = fn(args)
        if line is not None:
            print(json.dumps(line))


if __name__ == "__main__":
    main()
