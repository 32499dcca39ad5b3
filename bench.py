#!/usr/bin/env python3
"""Benchmark of the ADER-DG hot path on GB300 (one JSON line on rank 0).

Workload (one bench step): ADER-DG N = 5, 1D Euler (gamma 1.4), 10^5 cells on the
periodic unit interval, seeded four-mode density (seed 12483), u = 1, p = 1,
CFL 0.4, 100 time steps, FP64 -- the whole hot path per time step: device CFL
rule, LST-DG predictor, interface flux + DG update.  Inputs are resident in HBM
when the timed region starts; L2 is flushed (a 256 MB write) before every timed
step.  value = cell-updates/s of the timed steps (10^7 cell-updates per step).

--impl reference times the CPU oracle (test infrastructure, single thread) on a
bounded sample of the same workload.
Multi-GPU (torchrun): every rank solves its own replica (no data exchange;
weak scaling); value = all ranks' cell-updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s (FP64 vs FP32-predictor); p50/p99 solve latency; % roofline"
UNIT = "cell-updates/s"
DEGREE, CELLS, TIME_STEPS, SEED = 5, 100_000, 100, 12483
WORKLOAD = ("ADER-DG N=5 (6x6 space-time GL nodes x 3 vars), 1D Euler gamma=1.4, 10^5 cells "
            "periodic [0,1], rho=1+sum_{k=1..4} a_k sin(2 pi k x+phi_k) a_k~U(0,0.05) seed 12483, "
            "u=1, p=1, CFL 0.4, 100 time steps per bench step, FP64, Rusanov flux")
# FP64 peak of a GB300 from unit counts and clocks: 152 SMs x 2 FP64 FMA lanes/clk
# x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s); a DFMA probe measured 1.20 TFLOP/s at 2.0 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
M = 3

# DRAM traffic of the predictor kernel from an ncu capture, valid only for the
# kernel sources whose hash is recorded with it (see profiles/).
TRAFFIC_RECORD = {"sha256": "a37bbf3ccba3f2d0b9a3d334289287ce81dd4eda92acf8e0b9c5b1c58362351c",
                  "bytes_per_launch": 14493525,
                  "source": "profiles/launches_dg_n5_1e5cells.md (dram read 14.489 MB + write 0.005 MB "
                            "per timed-region launch of this bench, mean of 3)"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("ader_kernels.cuh", "ader_device.cuh"):
        with open(os.path.join(ROOT, "paper_2409_12483_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def predictor_flops_per_cell(n: int, iters: float, dg: bool = True) -> float:
    """Algorithmic FLOPs of one cell's predictor launch, as the kernel runs it.

    Iteration 1 starts from q = u in every tau row, so F(u) and k~ F(u) are the
    same in every row: Euler flux at n nodes (9 flops each: 1 div, 4 for p, 2 for
    F1, 2 for F2), g = k~ F(u) (2 n^2 M), q' = u - c_p0 g (2 n^2 M) and the
    convergence difference (n^2 M).  Every later iteration: flux at n^2 nodes, k~
    along xi and kappa~ along tau (2 n^3 M each, the k_ksi_kernel and kappa_kernel
    gemms of Table lst_dg_predictor_blas) and the difference (n^2 M).  Epilogue:
    two traces (psi-conv, 2 x 2 n^2 M); for DG the flux at n^2 nodes again, the
    time average (2 n^2 M), D~ (2 n^2 M) and the addition of u (n M).
    """
    first = 9 * n + 4 * n * n * M + n * n * M
    it = 9 * n * n + 4 * n ** 3 * M + n * n * M
    epi = 4 * n * n * M
    if dg:
        epi += 9 * n * n + 4 * n * n * M + n * M
    return first + max(iters - 1.0, 0.0) * it + epi


def predictor2d_flops_per_cell(n: int, iters: float) -> float:
    """Algorithmic FLOPs of one cell's 2D predictor launch (M = 4 variables,
    n^3 space-time nodes), as the kernel runs it.  Iteration 1 starts from q = u
    in every tau row: the fluxes at the n^2 spatial nodes (25 flops each: 1
    division, 2 velocities, 5 for p, 9 for F and G, 8 scalings), k~ along xi and
    eta there (4 n^3 M), q' = u - (row sum of kappa~) s (2 n^3 M) and the
    difference (n^3 M).  Every later iteration: the fluxes at n^3 nodes, k~ along
    xi and along eta and kappa~ along tau (2 n^4 M each), q' = u - ... and the
    difference (2 n^3 M).  Epilogue: four traces (8 n^3 M), the fluxes again
    (25 n^3), the two time averages (4 n^3 M) and the two D~ contractions plus u
    (4 n^3 M + n^2 M)."""
    m = 4
    first = 25 * n ** 2 + 7 * n ** 3 * m
    it = 25 * n ** 3 + 6 * n ** 4 * m + 2 * n ** 3 * m
    epi = 8 * n ** 3 * m + 25 * n ** 3 + 4 * n ** 3 * m + 4 * n ** 3 * m + n * n * m
    return first + max(iters - 1.0, 0.0) * it + epi


def predictor3d_flops_per_cell(n: int, iters: float) -> float:
    """Algorithmic FLOPs of one cell's 3D predictor launch (M = 5, n^4 space-time
    nodes), as the kernel runs it: iteration 1 (q = u in every tau row) forms the
    three fluxes (45 flops per node) and k~ along xi, eta, zeta (6 n^4 M) at the
    n^3 spatial nodes only, then q' = u - (row sum of kappa~) s and the difference
    (3 n^4 M); every later iteration the three fluxes with their scalings at n^4
    nodes, k~ along xi, eta, zeta and kappa~ along tau (2 n^5 M each) and the
    update and difference (2 n^4 M); epilogue: six traces (12 n^4 M), the fluxes
    again, the three time averages (6 n^4 M) and the three D~ contractions
    (6 n^4 M)."""
    m = 5
    first = 45 * n ** 3 + 9 * n ** 4 * m
    it = 45 * n ** 4 + 8 * n ** 5 * m + 2 * n ** 4 * m
    epi = 12 * n ** 4 * m + 45 * n ** 4 + 6 * n ** 4 * m + 6 * n ** 4 * m
    return first + max(iters - 1.0, 0.0) * it + epi


def dg3_errors(ctx, u, t, npts=10):
    """L1, L2, Linf density errors of the 3D sine wave rho = 1 + 0.5 sin 2 pi
    (x + y + z - 3 t) (Sec. 2.1, velocity (1, 1, 1)) with an npts^3 GL rule per
    cell; measurement code, not the oracle."""
    import numpy as np
    xi = ctx.table("xi")
    n = len(xi)
    u = np.asarray(u).reshape(ctx.nz, ctx.ny, ctx.nx, n, n, n, 5)
    gx, gw = np.polynomial.legendre.leggauss(npts)
    gx, gw = 0.5 * (gx + 1), 0.5 * gw
    L = np.ones((npts, n))
    for k in range(n):
        for m in range(n):
            if m != k:
                L[:, k] *= (gx - xi[m]) / (xi[k] - xi[m])
    rho = np.einsum("ak,bl,cm,zyxklm->zyxabc", L, L, L, u[..., 0])
    X = (np.arange(ctx.nx)[None, None, :, None, None, None] + gx[None, None, None, :, None, None]) / ctx.nx
    Y = (np.arange(ctx.ny)[None, :, None, None, None, None] + gx[None, None, None, None, :, None]) / ctx.ny
    Z = (np.arange(ctx.nz)[:, None, None, None, None, None] + gx[None, None, None, None, None, :]) / ctx.nz
    err = np.abs(rho - (1 + 0.5 * np.sin(2 * np.pi * (X + Y + Z - 3 * t))))
    wts = np.einsum("a,b,c->abc", gw, gw, gw) / (ctx.nx * ctx.ny * ctx.nz)
    return float((err * wts).sum()), float(np.sqrt((err ** 2 * wts).sum())), float(err.max())


def dg2_errors(ctx, u, t, npts=25):
    """L1, L2, Linf density errors of the 2D sine wave rho = 1 + 0.5 sin 2 pi
    (x + y - 2 t) (Sec. 2.1, velocity (1, 1)) with an npts x npts GL rule per
    cell, from the library's own nodes; measurement code, not the oracle."""
    import numpy as np
    xi = ctx.table("xi")
    n = len(xi)
    u = np.asarray(u).reshape(ctx.ny, ctx.nx, n, n, 4)
    gx, gw = np.polynomial.legendre.leggauss(npts)
    gx, gw = 0.5 * (gx + 1), 0.5 * gw
    L = np.ones((npts, n))
    for k in range(n):
        for m in range(n):
            if m != k:
                L[:, k] *= (gx - xi[m]) / (xi[k] - xi[m])
    rho = np.einsum("ak,bl,yxkl->yxab", L, L, u[..., 0])
    X = (np.arange(ctx.nx)[None, :, None, None] + gx[None, None, :, None]) / ctx.nx
    Y = (np.arange(ctx.ny)[:, None, None, None] + gx[None, None, None, :]) / ctx.ny
    err = np.abs(rho - (1 + 0.5 * np.sin(2 * np.pi * (X + Y - 2 * t))))
    wts = np.outer(gw, gw) / (ctx.nx * ctx.ny)
    return float((err * wts).sum()), float(np.sqrt((err ** 2 * wts).sum())), float(err.max())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) > 8
                          for i, v in enumerate(r[5:9]) if v.strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


def measure_solve(ctx, u0, time_steps, steps, warmup, flush):
    """Time `steps` solves of `time_steps` time steps from u0 (after `warmup`),
    flushing L2 before each; returns (total ms, per-solve stats)."""
    import torch
    u = torch.empty_like(u0)
    prof, times = [], []
    for i in range(warmup + steps):
        u.copy_(u0)
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        done, t, rc = ctx.ader_solve(u, max_steps=time_steps)
        ev1.record()
        torch.cuda.synchronize()
        if done != time_steps:
            raise RuntimeError(f"solve stopped after {done} steps")
        if i >= warmup:
            times.append(ev0.elapsed_time(ev1))
            prof.append(ctx.ader_get_stats())
    return sum(times), prof, u


def variant_line(name, workload, ctx, u0, cells, degree, time_steps, steps, warmup, flush, dg=True,
                 extra=None, field=None):
    try:
        return _variant_line(name, workload, ctx, u0, cells, degree, time_steps, steps, warmup,
                             flush, dg, extra, field)
    except Exception as e:  # noqa: BLE001 -- one failing line does not hide the others
        return {"name": name, "workload": workload, "error": f"{type(e).__name__}: {e}"[:300]}


def _variant_line(name, workload, ctx, u0, cells, degree, time_steps, steps, warmup, flush, dg,
                  extra, field):
    ms, prof, u = measure_solve(ctx, u0, time_steps, steps, warmup, flush)
    n = degree + 1
    iters = sum(p["mean_iters"] for p in prof) / len(prof)
    nsteps = sum(p["profiled_steps"] for p in prof)
    pred_ms = sum(p["predict_ms"] for p in prof) / max(nsteps, 1)
    face_ms = sum(p["face_ms"] for p in prof) / max(nsteps, 1)
    weno_ms = sum(p["weno_ms"] for p in prof) / max(nsteps, 1)
    out = {"name": name, "workload": workload,
           "value": cells * time_steps * steps / (ms / 1e3), "unit": UNIT,
           "ms_per_step": ms / steps, "mean_picard_iters": iters,
           "predict_ms_per_launch": pred_ms, "face_update_ms_per_launch": face_ms}
    if not dg:
        out["weno_ms_per_launch"] = weno_ms
    if ctx.options.precision == 0:
        fl = cells * predictor_flops_per_cell(n, iters, dg)
        out["predict_fp64_tflops"] = fl / (pred_ms / 1e3) / 1e12
        out["predict_frac_of_fp64_peak"] = out["predict_fp64_tflops"] / FP64_PEAK_TFLOPS
    if extra:
        out.update(extra(u))
    if field is not None and dg:
        out["l1_density_vs_exact"] = dg_l1_error(ctx, u.cpu().numpy(), field, prof[-1]["t"])
    return out


# The headline is the LAST stdout line and carries the contract's keys only;
# every secondary study is printed on an earlier line of its own.
HEADLINE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                 "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                 "roofline", "e2e", "gpu_launches", "clocks", "errors", "cpu_baseline",
                 "fp32_predictor", "latency")
MAX_HEADLINE_BYTES = 4096

# the FP32-predictor forms of the headline workload, as named by run_variants
FP32_FORMS = (("increment", "dg5-1e5-incr"), ("fp32_ff_sweep", "dg5-1e5-fp32ff1"),
              ("fp32_fp64_sweeps", "dg5-1e5-fp32pred"))


def fp32_predictor_summary(variants, fp64_value):
    """The headline's FP32-predictor figures: each form's throughput on the
    headline workload and its distance from the FP64 path, from the
    precision_forms_and_variants study (None where the study has no such line)."""
    by_name = {v.get("name"): v for v in variants or [] if isinstance(v, dict)}
    forms = {}
    for key, name in FP32_FORMS:
        v = by_name.get(name)
        if not v or "value" not in v:
            continue
        forms[key] = {"value": v["value"], "vs_fp64": v["value"] / fp64_value,
                      "rel_linf_vs_fp64_path": v.get("rel_linf_vs_fp64_path"),
                      "l1_density_vs_exact": v.get("l1_density_vs_exact")}
    if not forms:
        return None
    return {"unit": UNIT, "workload": "the headline's (study precision_forms_and_variants)",
            "forms": forms}


def latency_summary(serving, frac=0.8):
    """p50/p99 solve latency of the continuous-batching server at `frac` of its
    saturation rate, with the plain per-solve FP64 path on the same arrivals,
    from the serving study (None where the study has no such point)."""
    if not isinstance(serving, dict):
        return None
    pts = [o for o in serving.get("open_loop", []) if o.get("arrival_rate_frac_of_saturation") == frac]
    if not pts:
        return None
    o = pts[0]
    return {"p50_s": o["server"]["p50_s"], "p99_s": o["server"]["p99_s"],
            "load": f"{frac} x saturation", "solves_per_s": o["server"]["solves_per_s"],
            "saturation_solves_per_s": serving.get("saturation", {}).get("solves_per_s"),
            "plain_fp64": {"p50_s": o["baseline_per_solve_fp64"]["p50_s"],
                           "p99_s": o["baseline_per_solve_fp64"]["p99_s"]},
            "workload": "scaled request stream (study serving)"}


def headline_line(*, world, steps, warmup, value, ms_per_step, tuning, roofline, e2e, launches,
                  clocks, errors) -> dict:
    """The headline JSON object (cpu_baseline is added once it is measured)."""
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": CELLS, "degree": DEGREE,
                   "time_steps": TIME_STEPS, "parallelism": f"replicas x{world}",
                   "tuning": {k: tuning[k] for k in ("predict_cells_per_block",
                                                     "face_cells_per_block", "graph_steps")},
                   "l2": "flushed (256 MB write) before each timed step; the 14.4 MB state "
                         "stays L2-resident across the 100 time steps of a step"},
        "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "errors": errors,
    }


def print_study(name, fn, *args, out=None):
    """Run one secondary study and print it as its own compact JSON line
    ({"study": name, ...}); a study that raises prints its error instead, so the
    headline that follows is always printed.  Returns the result (None on error)."""
    out = out or sys.stdout
    t0 = time.perf_counter()
    try:
        body = {"study": name, "result": fn(*args)}
    except Exception as e:  # noqa: BLE001 -- reported, the bench goes on
        body = {"study": name, "error": f"{type(e).__name__}: {e}"[:500]}
    body["seconds"] = round(time.perf_counter() - t0, 2)
    print(json.dumps(body, separators=(",", ":"), default=float), file=out, flush=True)
    return body.get("result")


def print_headline(head: dict, out=None) -> str:
    """Print the headline as the last line (compact, at most MAX_HEADLINE_BYTES)."""
    extra = set(head) - set(HEADLINE_KEYS)
    if extra:
        raise ValueError(f"headline keys outside the contract: {sorted(extra)}")
    line = json.dumps(head, separators=(",", ":"), default=float)
    if len(line) > MAX_HEADLINE_BYTES:
        raise ValueError(f"headline line is {len(line)} bytes (> {MAX_HEADLINE_BYTES})")
    print(line, file=out or sys.stdout, flush=True)
    return line


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Max of a per-rank time over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank in at most max_seconds."""
    return world * units_per_rank / max_seconds


def dg_l1_error(ctx, u, field, t, npts=25):
    """L1 density error of a DG state against the exact advected density (eq.
    epsilons of Sec. 2.1 in 1D: npts-point GL rule per cell), from the library's
    own nodes; measurement code, not the oracle."""
    import numpy as np
    xi = ctx.table("xi")
    n = len(xi)
    u = np.asarray(u).reshape(-1, n, 3)
    nc = u.shape[0]
    gx, gw = np.polynomial.legendre.leggauss(npts)
    gx, gw = 0.5 * (gx + 1), 0.5 * gw
    L = np.ones((npts, n))
    for k in range(n):
        for m in range(n):
            if m != k:
                L[:, k] *= (gx - xi[m]) / (xi[k] - xi[m])
    rho = u[:, :, 0] @ L.T
    xs = (np.arange(nc)[:, None] + gx[None, :]) / nc
    return float((np.abs(rho - field.rho(xs, t)) @ gw).sum() / nc)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_rate(target_s: float = 12.0):
    """Time the CPU oracle (as it stands, one thread) on whole time steps of the
    same 10^5-cell N = 5 mesh; returns (cell-updates/s, steps timed, seconds)."""
    import numpy as np

    import oracle
    import workloads as W
    o = oracle.Oracle(DEGREE)
    u = W.nodal_state(W.modes4(SEED), o.node_x(CELLS))
    t0 = time.perf_counter()
    u1, steps, _, rc = o.solve("dg", u, 1.0 / CELLS, max_steps=1)
    t1 = time.perf_counter() - t0
    more = max(0, min(TIME_STEPS - 1, int(math.ceil(target_s / max(t1, 1e-3))) - 1))
    t2 = 0.0
    if more:
        t0 = time.perf_counter()
        u1, _, _, _ = o.solve("dg", u1, 1.0 / CELLS, max_steps=more)
        t2 = time.perf_counter() - t0
    steps = 1 + more
    secs = t1 + t2
    cpu_oracle_rate.last = (u, u1, steps)
    return CELLS * steps / secs, steps, secs


def _oracle_replica(steps, barrier, out):
    """One process of the all-cores oracle timing: the oracle (one thread, as it
    stands) advances its own copy of the 10^5-cell N = 5 mesh by `steps` steps;
    every process starts its clock at the same barrier."""
    import oracle
    import workloads as W
    o = oracle.Oracle(DEGREE)
    u = W.nodal_state(W.modes4(SEED), o.node_x(CELLS))
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    _, done, _, rc = o.solve("dg", u, 1.0 / CELLS, max_steps=steps)
    out.put((done, time.perf_counter() - t0, rc))


def cpu_oracle_rate_all_cores(steps: int):
    """The same oracle on every host core at once: one spawned process per core,
    each on its own replica of the mesh (as OpenMP over independent cells would
    spread them); returns (cell-updates/s over all processes, processes, steps
    per process, slowest process's seconds)."""
    import multiprocessing as mp
    procs = (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
             else (os.cpu_count() or 1))
    ctx = mp.get_context("spawn")  # a fork after CUDA initialisation can hang
    barrier, out = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_replica, args=(steps, barrier, out)) for _ in range(procs)]
    for p in ps:
        p.start()
    res = []
    try:
        while len(res) < procs:
            try:
                res.append(out.get(timeout=2.0))
            except Exception:  # queue.Empty: give up once a process died without a result
                if any(p.exitcode not in (None, 0) for p in ps):
                    raise RuntimeError("an oracle replica process died")
    finally:
        for p in ps:
            p.join(timeout=5)
            if p.is_alive():
                p.kill()
    if any(rc != 0 or done != steps for done, _, rc in res):
        raise RuntimeError(f"oracle replica failed: {res}")
    slowest = max(t for _, t, _ in res)
    return procs * CELLS * steps / slowest, procs, steps, slowest


# CPU seconds the reference arm spends in all, warm-up included, when
# --ref-seconds is not given: each step's sample is this divided over the
# steps, between 1 and 12 s, so that a long --steps K run still ends in minutes
REF_TOTAL_SECONDS = 150.0


def ref_step_seconds(warmup: int, steps: int, given=None) -> float:
    """Seconds of oracle work per reference-arm step."""
    if given is not None:
        return float(given)
    return min(12.0, max(1.0, REF_TOTAL_SECONDS / max(1, warmup + steps)))


def run_reference(args, world, rank):
    if rank != 0:
        return
    rates = []
    target = ref_step_seconds(args.warmup, args.steps, args.ref_seconds)
    for i in range(args.warmup + args.steps):
        rate, steps, secs = cpu_oracle_rate(target_s=target)
        if i >= args.warmup:
            rates.append((rate, steps, secs))
    total_cu = sum(CELLS * s for _, s, _ in rates)
    total_s = sum(t for _, _, t in rates)
    value = total_cu / total_s
    sample = (f"{rates[0][1]} of the 100 time steps of the 10^5-cell mesh per bench step "
              f"(about {rates[0][2]:.1f} s of single-thread CPU work)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / len(rates), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": CELLS, "degree": DEGREE,
                   "time_steps": TIME_STEPS, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="oracle seconds per reference-arm step (default: 150 s over "
                         "warmup + steps, between 1 and 12 s per step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the secondary workloads (FP32 predictor, WENO5 and N=7 at 10^6 cells)")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the continuous-batching serving benchmark (scaled Poisson stream)")
    ap.add_argument("--serving-requests", type=int, default=128)
    ap.add_argument("--serving-max-cells", type=int, default=2048)
    ap.add_argument("--no-convergence", action="store_true",
                    help="skip the coarse-mesh convergence sweeps of the four precision forms")
    ap.add_argument("--no-limiter", action="store_true",
                    help="skip the subcell limiter's Riemann problems and throughput")
    ap.add_argument("--no-2d", action="store_true",
                    help="skip the 2D and 3D sine-wave tables and throughput lines")
    ap.add_argument("--no-source", action="store_true",
                    help="skip the reacting-flow (source term) throughput and ODE convergence study")
    ap.add_argument("--case", default=None,
                    help="profiling case instead of the bench line: "
                         "predict-dg5 | predict-dg5-ff | predict-dg5-incr | predict-dg7-fp32 | weno5 | "
                         "step2d-dg5 | step2d-dg3 | "
                         "step3d-dg2 | step3d-dg2-48 | step3d-dg5 | step3d-dg7 (multi-D: warmup + steps time steps of one solve) | "
                         "limiter-dg5-1e5 (the headline data, limiter on) | "
                         "paper-costs (the sine wave at the meshes of the paper's cost tables) | "
                         "serving-large (512 requests, cells up to 4096) | "
                         "sine-tables (the 2D / 3D sine-wave convergence tables against the paper's) | "
                         "sod-dg5-limiter | tracer-dg5 | reacting-dg5 (10^6 cells) | "
                         "solve-dg5 | solve-dg5-1e5 (the FP64 time loop, 10^6 / 10^5 cells)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.case:
        return run_case(args)

    import numpy as np
    import torch

    import workloads as W
    from paper_2409_12483_gb300 import Context
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    ctx = Context(CELLS, DEGREE, "dg", device=dev, profile=1)
    x = ctx.node_coords()
    u0 = torch.tensor(W.nodal_state(W.modes4(SEED), x), device=dev).reshape(-1).contiguous()
    u = torch.empty_like(u0)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    tuning = ctx.ader_autotune(u0, reps=3)  # launch shapes picked by measurement, before timing

    last = {}

    def one(prof):
        u.copy_(u0)
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        steps, t, rc = ctx.ader_solve(u, max_steps=TIME_STEPS)
        ev1.record()
        torch.cuda.synchronize()
        last["t"] = t
        st = ctx.ader_get_stats()
        if steps != TIME_STEPS:
            raise RuntimeError(f"solve stopped after {steps} steps")
        prof.append(st)
        return ev0.elapsed_time(ev1)

    warm = []
    for _ in range(args.warmup):
        one(warm)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    prof = []
    times = []
    torch.cuda.nvtx.range_push("timed")
    with ClockSampler(local) as clocks:
        for _ in range(args.steps):
            times.append(one(prof))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if pg:
        pg.barrier()
    total_ms = max_over_ranks(sum(times), pg, dev)
    u_last, t_last = u.cpu().numpy(), last["t"]
    cu_per_step = CELLS * TIME_STEPS
    value = whole_job_rate(cu_per_step * args.steps, world, total_ms / 1e3)

    # dominant kernel: the predictor (FP64 ALU bound)
    pred_ms = sum(p["predict_ms"] for p in prof)
    face_ms = sum(p["face_ms"] for p in prof)
    nsteps = sum(p["profiled_steps"] for p in prof)
    iters = sum(p["mean_iters"] for p in prof) / len(prof)
    n = DEGREE + 1
    flops_launch = CELLS * predictor_flops_per_cell(n, iters)
    avg_pred_s = pred_ms / nsteps / 1e3
    achieved = flops_launch / avg_pred_s / 1e12
    traffic = None
    if TRAFFIC_RECORD["sha256"] == kernel_source_hash():
        traffic = TRAFFIC_RECORD["bytes_per_launch"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "kernel": "predict_kernel<5, fp64>", "mean_picard_iters": iters,
                "predict_ms_per_launch": 1e3 * avg_pred_s,
                "face_update_ms_per_launch": face_ms / nsteps,
                "peak_note": "FP64 from unit counts and max clock (152 SM x 2 DFMA/clk x 2.07 GHz)"}

    # end to end through the C ABI with host buffers (H2D + solve + D2H in the region)
    uh = torch.empty(u0.numel(), dtype=torch.float64, pin_memory=True)
    u0_host = u0.cpu()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        uh.copy_(u0_host)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.ader_solve_host(uh, max_steps=TIME_STEPS)
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_times), pg, dev)
    state_bytes = u0.numel() * 8
    e2e = {"value": whole_job_rate(cu_per_step * args.steps, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes}
    launches = sum(p["kernel_launches"] for p in prof)

    if rank == 0:
        head = headline_line(
            world=world, steps=args.steps, warmup=args.warmup, value=value,
            ms_per_step=total_ms / args.steps, tuning=tuning, roofline=roofline, e2e=e2e,
            launches=launches, clocks=clocks.summary(),
            errors={"l1_density_vs_exact": dg_l1_error(ctx, u_last, W.modes4(SEED), t_last)})
        studies = []
        if not args.no_variants:
            studies.append(("precision_forms_and_variants", run_variants, (args, dev, flush)))
            studies.append(("small_meshes_graphs_vs_plain", run_small_meshes, (dev,)))
        if not args.no_serving:
            studies.append(("serving", run_serving, (dev, args.serving_requests,
                                                     args.serving_max_cells)))
        if not args.no_convergence:
            studies.append(("convergence", run_convergence, (dev,)))
        if not args.no_source:
            studies.append(("source_terms", run_source, (args, dev, flush)))
        if not args.no_limiter:
            studies.append(("limiter", run_limiter, (args, dev, flush)))
        if not args.no_source:
            studies.append(("non_conservative", run_tracer, (args, dev, flush)))
        if not args.no_2d:
            studies.append(("two_d", run_2d, (args, dev, flush)))
            studies.append(("three_d", run_3d, (args, dev, flush)))
        results = {name: print_study(name, fn, *fargs) for name, fn, fargs in studies}
        fp32 = fp32_predictor_summary(results.get("precision_forms_and_variants"), value)
        if fp32:
            head["fp32_predictor"] = fp32
        lat = latency_summary(results.get("serving"))
        if lat:
            head["latency"] = lat
        if not args.no_cpu_baseline:
            rate, steps, secs = cpu_oracle_rate()
            u_in, u_or, k = cpu_oracle_rate.last
            ug = torch.tensor(u_in, device=dev).reshape(-1)
            ctx.ader_solve(ug, max_steps=k)
            torch.cuda.synchronize()
            par = float(np.abs(ug.cpu().numpy() - u_or.ravel()).max() / np.abs(u_or).max())
            head["errors"]["rel_linf_vs_fp64_oracle_after_oracle_steps"] = par
            head["cpu_baseline"] = {
                "value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"{steps} time steps of the same 10^5-cell N=5 mesh ({secs:.1f} s, 1 thread)"}
            # the same oracle on all host cores: steps per process sized like the
            # single-thread sample (about 12 s)
            k_all = max(1, min(TIME_STEPS, int(round(steps * 12.0 / max(secs, 1e-3)))))
            r_all, procs, k_all, s_all = cpu_oracle_rate_all_cores(k_all)
            head["cpu_baseline"]["all_cores"] = {
                "value": r_all, "unit": UNIT, "cores": procs, "kind": "oracle",
                "sample": f"{procs} processes, each {k_all} time steps of its own copy of the "
                          f"10^5-cell N=5 mesh (slowest {s_all:.1f} s)"}
        print_headline(head)
    if pg:
        pg.destroy_process_group()


def run_convergence(dev):
    """Convergence sweeps on coarse meshes to t_end = 1, where the discretisation
    error is above FP32 round-off: the L1 density error against the exact advected
    solution of the FP64, FP32-predictor (1 and 2 FP64 sweeps) and float-float
    forms, each form's ratio to FP64, and the FP64 order between meshes.  N = 2 on
    the sine wave (rho = 1 + 0.2 sin 2 pi x), N = 5 on the four-mode data."""
    import math

    import torch

    import workloads as W
    from paper_2409_12483_gb300 import Context
    forms = {"fp64": dict(precision="fp64"),
             "fp32_1sweep": dict(precision="fp32", fp64_sweeps=1),
             "fp32_2sweeps": dict(precision="fp32", fp64_sweeps=2),
             "fp32ff_1sweep": dict(precision="fp32ff", fp64_sweeps=1),
             "fp32ff_2sweeps": dict(precision="fp32ff", fp64_sweeps=2),
             "incr": dict(precision="incr"),
             "ff": dict(precision="ff")}
    out = []
    for N, data, field, meshes in ((2, "sine", W.sine(), (50, 100, 200, 400)),
                                   (5, "modes4", W.modes4(SEED), (20, 40, 80, 160))):
        rows = []
        for nc in meshes:
            row = {"cells": nc, "l1": {}}
            for name, kw in forms.items():
                ctx = Context(nc, N, "dg", device=dev, **kw)
                u = torch.tensor(W.nodal_state(field, ctx.node_coords()), device=dev).reshape(-1)
                steps, t, _ = ctx.ader_solve(u, t_end=1.0)
                torch.cuda.synchronize()
                row["l1"][name] = dg_l1_error(ctx, u.cpu().numpy(), field, t)
                row["steps"] = steps
                del ctx
            row["ratio_to_fp64"] = {k: v / row["l1"]["fp64"] for k, v in row["l1"].items() if k != "fp64"}
            rows.append(row)
        orders = [math.log(a["l1"]["fp64"] / b["l1"]["fp64"]) / math.log(b["cells"] / a["cells"])
                  for a, b in zip(rows, rows[1:])]
        out.append({"degree": N, "data": data, "t_end": 1.0, "meshes": rows, "order_fp64": orders,
                    "within_2x_of_fp64": {k: all(r["ratio_to_fp64"][k] <= 2.0 for r in rows)
                                          for k in forms if k != "fp64"}})
    return out


def lagrange_matrix(x, nodes):
    """L[i, k] = phi_k(x_i) for the Lagrange basis on the given nodes."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    L = np.ones((x.size, len(nodes)))
    for k in range(len(nodes)):
        for m in range(len(nodes)):
            if m != k:
                L[:, k] *= (x - nodes[m]) / (nodes[k] - nodes[m])
    return L


def ode_errors(xi, dt, nodes, locs, omega=1.0, npts=25):
    """Errors of the ODE problem of Sec. 2.1 (eq. harm_osc; norms of eq.
    epsilons_q, vector norms summed over the two components): at the time nodes
    t_n = n dt (the corrector's u^n) and of the local predictor solution over
    each step (npts-point GL rule in time); measurement code, not the oracle."""
    import numpy as np
    nodes = np.asarray(nodes)
    K = len(nodes)
    t = dt * np.arange(1, K + 1)
    e = np.abs(nodes - np.stack([np.cos(omega * t), -omega * np.sin(omega * t)], 1)).sum(1)
    glob = [float(dt * e.sum()), float(np.sqrt(dt * (e ** 2).sum())), float(e.max())]
    gx, gw = np.polynomial.legendre.leggauss(npts)
    gx, gw = 0.5 * (gx + 1.0), 0.5 * gw
    L = lagrange_matrix(gx, xi)
    l1 = l2 = linf = 0.0
    for k in range(K):
        ts = dt * (k + gx)
        ek = np.abs(L @ np.asarray(locs[k]) -
                    np.stack([np.cos(omega * ts), -omega * np.sin(omega * ts)], 1)).sum(1)
        l1 += dt * float(gw @ ek)
        l2 += dt * float(gw @ ek ** 2)
        linf = max(linf, float(ek.max()))
    return glob, [l1, float(np.sqrt(l2)), linf]


def run_source(args, dev, flush):
    """The system with algebraic sources (Sec. 2 eq. pdes_2_comps in 1D: Euler plus
    two reacting species, nested Picard predictor): throughput at the headline's
    size for a mild (omega = 1) and a fast (omega dt ~ 0.2) reaction, and the
    ODE convergence study of Sec. 2.1 (one uniform cell, K uniform steps to 2 pi,
    errors at the time nodes and of the local predictor solution)."""
    import math

    import numpy as np
    import torch

    import workloads as W
    from paper_2409_12483_gb300 import Context
    out = {"throughput": [], "ode": []}
    st = max(2, min(args.steps, 3))
    for omega in (1.0, 1.0e6):
        ctx = Context(CELLS, DEGREE, "dg", device=dev, profile=1, system="reacting", omega=omega)
        u0 = torch.tensor(W.reacting_state(ctx.node_coords(), seed=SEED), device=dev).reshape(-1)
        dt = ctx.ader_compute_dt(u0)
        line = variant_line(f"reacting-dg5-1e5-omega{omega:g}",
                            "1D two-component reacting flow, DG N=5, 10^5 cells, 100 steps, FP64, "
                            "nested Picard (outer: fluxes, inner: sources)",
                            ctx, u0, CELLS, DEGREE, TIME_STEPS, st, 2, flush)
        for k in ("predict_fp64_tflops", "predict_frac_of_fp64_peak"):
            line.pop(k, None)  # the Euler FLOP model does not cover the inner source loop
        line["omega_dt"] = omega * dt
        out["throughput"].append(line)
        del ctx
    ode_dx = 1.0e3  # uniform data: a wide cell keeps the inactive spatial operator stable
    for N, Ks in ((1, (10, 20, 40)), (2, (10, 20, 40)), (3, (10, 20)), (4, (10, 20)), (5, (4, 8))):
        rows = []
        for K in Ks:
            dt = 2 * math.pi / K
            ctx = Context(1, N, "dg", device=dev, system="reacting", omega=1.0, picard_tol=1e-14,
                          picard_max_iter=200, x1=ode_dx)
            n = N + 1
            u = torch.tensor(W.ode_state(n), device=dev).reshape(-1)
            q = torch.empty(ctx.predictor_count, dtype=torch.float64, device=dev)
            nodes, locs = [], []
            for _ in range(K):
                ctx.ader_predict(u, dt, q)
                nxt = torch.empty_like(u)
                ctx.ader_step(u, nxt, dt)
                u = nxt
                locs.append(q.view(n, n, 5)[:, 0, 3:5].cpu().numpy())
                nodes.append(u.view(n, 5)[0, 3:5].cpu().numpy())
            g, l = ode_errors(ctx.table("xi"), dt, nodes, locs)
            rows.append({"steps": K, "global": g, "local": l})
            del ctx
        for a, b in zip(rows, rows[1:]):
            r = math.log(b["steps"] / a["steps"])
            b["order_global"] = [math.log(x / y) / r for x, y in zip(a["global"], b["global"])]
            b["order_local"] = [math.log(x / y) / r for x, y in zip(a["local"], b["local"])]
        out["ode"].append({"degree": N, "theory_global": 2 * N + 1, "theory_local": N + 1,
                           "rows": rows})
    return out


def riemann_density_l1(ctx, u, test, t, npts=25):
    """L1 density error of a DG state against the exact Riemann solution (the
    library's own nodes, npts-point GL rule per cell); measurement code."""
    import numpy as np

    import workloads as W
    xi = ctx.table("xi")
    n = len(xi)
    u = np.asarray(u).reshape(-1, n, 3)
    nc = u.shape[0]
    gx, gw = np.polynomial.legendre.leggauss(npts)
    gx, gw = 0.5 * (gx + 1), 0.5 * gw
    rho = u[:, :, 0] @ lagrange_matrix(gx, xi).T
    xs = (np.arange(nc)[:, None] + gx[None, :]) / nc
    L, R = W.RIEMANN_TESTS[test]
    exact, _, _ = W.riemann_solution(L, R, xs, t)
    return float((np.abs(rho - exact) @ gw).sum() / nc)


# Table conv_orders_pde_2d (Sec. 2.1), eps_L1 per (N, cells per direction),
# printed beside this library's errors for comparison only
PAPER_2D_L1 = {(1, 10): 5.48e-3, (1, 15): 2.44e-3, (1, 20): 1.37e-3, (1, 25): 8.78e-4,
               (2, 10): 2.87e-4, (2, 15): 8.44e-5, (2, 20): 3.55e-5, (2, 25): 1.81e-5,
               (3, 10): 1.13e-5, (3, 15): 2.22e-6, (3, 20): 7.02e-7, (3, 25): 2.87e-7,
               (4, 10): 3.58e-7, (4, 15): 4.67e-8, (4, 20): 1.10e-8, (4, 25): 3.61e-9,
               (5, 5): 6.09e-7, (5, 10): 9.33e-9, (5, 15): 8.18e-10, (5, 20): 1.45e-10,
               (6, 5): 2.75e-8, (6, 10): 2.12e-10, (6, 15): 1.23e-11, (6, 20): 1.63e-12,
               (7, 5): 1.08e-9, (7, 10): 4.13e-12, (7, 15): 1.61e-13, (7, 20): 1.60e-14}


# Table conv_orders_pde_3d (Sec. 2.1), eps_L1 per (N, cells per direction)
PAPER_3D_L1 = {(1, 10): 5.24e-2, (1, 15): 1.08e-2, (1, 20): 4.62e-3, (1, 25): 2.82e-3,
               (2, 10): 7.69e-4, (2, 15): 2.22e-4, (2, 20): 9.29e-5, (2, 25): 4.74e-5,
               (3, 10): 2.17e-5, (3, 15): 4.28e-6, (3, 20): 1.35e-6, (3, 25): 5.54e-7,
               (4, 10): 7.69e-7, (4, 15): 1.03e-7, (4, 20): 2.48e-8, (4, 25): 8.16e-9,
               (5, 5): 1.11e-6, (5, 10): 1.67e-8, (5, 15): 1.46e-9, (5, 20): 2.60e-10,
               (6, 5): 5.24e-8, (6, 10): 4.36e-10, (6, 15): 2.59e-11, (6, 20): 3.49e-12,
               (7, 5): 1.90e-9, (7, 10): 7.14e-12, (7, 15): 2.78e-13, (7, 20): 2.74e-14}


# Tables comp_costs_dg_2d / comp_costs_dg_3d (Sec. 3): T_JIT, whole-run CPU
# seconds of the paper's fastest implementation (i9-10980XE, 4 OpenMP threads,
# limiter admissibility checks every step) for the sine wave to t = 1 on 16^2 and
# 7^3 cells, printed beside this library's GPU solve time for context only
PAPER_2D_TJIT_16 = {1: 0.931, 2: 2.10, 3: 3.72, 4: 6.30, 5: 29.5, 6: 78.3, 7: 168.0}
PAPER_3D_TJIT_7 = {1: 5.20, 2: 12.3, 3: 46.5, 4: 87.4, 5: 170.0, 6: 333.0, 7: 638.0}


def paper_cost_rows(make_ctx, state_fn, table, cells_label, dev):
    """The sine wave to t = 1 at the mesh of the paper's cost table, per degree:
    the GPU solve time (state resident, CUDA events; after one untimed solve) and
    the same solve through the host-buffer call (copies in and out included)."""
    import numpy as np
    import torch
    rows = []
    for N, t_paper in table.items():
        ctx = make_ctx(N)
        u_init = np.ascontiguousarray(state_fn(ctx).ravel())
        u = torch.tensor(u_init, device=dev)
        ctx.ader_solve(u, t_end=1.0)  # untimed: first-use setup
        u = torch.tensor(u_init, device=dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        steps, t, rc = ctx.ader_solve(u, t_end=1.0)
        e1.record()
        torch.cuda.synchronize()
        host = u_init.copy()
        h0 = time.perf_counter()
        ctx.ader_solve_host(host, t_end=1.0)
        h_s = time.perf_counter() - h0
        s = e0.elapsed_time(e1) / 1e3
        rows.append({"degree": N, "cells": cells_label, "steps": steps, "status": rc,
                     "gpu_solve_s": s, "host_call_s": h_s, "paper_t_jit_s": t_paper,
                     "paper_over_gpu": t_paper / s})
        del ctx
    return rows

def sine3d_state(ctx):
    import numpy as np
    X, Y, Z = ctx.node_coords()
    rho = 1 + 0.5 * np.sin(2 * np.pi * (X + Y + Z))
    return np.stack([rho, rho, rho, rho, 1 / 0.4 + 1.5 * rho], -1)  # velocity (1, 1, 1), p = 1


def run_3d(args, dev, flush, tables=False):
    """3D Euler (ader_init_3d, degrees 1..7): throughput of the 3D solve and,
    with tables, the sine-wave advection problem of Sec. 2.1 at the meshes of
    Table conv_orders_pde_3d to t = 1 through the GPU path."""
    import numpy as np
    import torch

    from paper_2409_12483_gb300 import Context3D
    out = {"sine_wave": [], "throughput": []}
    # the paper's meshes, the finest ones for N <= 2 only (N = 4 on 25^3 alone
    # takes about two minutes)
    meshes = {1: (10, 15, 20, 25), 2: (10, 15, 20), 3: (10, 15), 4: (10, 15), 5: (5, 10),
              6: (5, 10), 7: (5, 10)}
    for N in (range(1, 8) if tables else ()):
        prev = None
        for nc in meshes[N]:
            ctx = Context3D(nc, nc, nc, N, device=dev)
            u = torch.tensor(sine3d_state(ctx).ravel(), device=dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            steps, t, rc = ctx.ader_solve(u, t_end=1.0)
            e1.record()
            torch.cuda.synchronize()
            err = dg3_errors(ctx, u.cpu().numpy(), t)
            row = {"degree": N, "cells": f"{nc}^3", "steps": steps, "status": rc,
                   "eps_l1": err[0], "eps_l2": err[1], "eps_linf": err[2],
                   "paper_eps_l1": PAPER_3D_L1[(N, nc)], "ms": e0.elapsed_time(e1)}
            if prev is not None:
                row["order_l1"] = float(np.log(prev[1] / err[0]) / np.log(nc / prev[0]))
            prev = (nc, err[0])
            out["sine_wave"].append(row)
            del ctx
    st_ = max(2, min(args.steps, 3))
    for N, nc, ts in ((2, 96, 10), (3, 64, 10), (4, 40, 10), (5, 24, 10), (6, 16, 10), (7, 12, 10)):
        ctx = Context3D(nc, nc, nc, N, device=dev, profile=1)
        u0 = torch.tensor(sine3d_state(ctx).ravel(), device=dev)
        cells = nc ** 3
        ms, prof, u = measure_solve(ctx, u0, ts, st_, 2, flush)
        iters = sum(p["mean_iters"] for p in prof) / len(prof)
        nsteps = sum(p["profiled_steps"] for p in prof)
        pred_ms = sum(p["predict_ms"] for p in prof) / max(nsteps, 1)
        face_ms = sum(p["face_ms"] for p in prof) / max(nsteps, 1)
        fl = cells * predictor3d_flops_per_cell(N + 1, iters)
        out["throughput"].append({
            "name": f"dg{N}-3d-{nc}^3", "workload": f"3D sine wave (Sec. 2.1), DG N={N}, "
            f"{nc}^3 cells periodic, {ts} steps, FP64", "value": cells * ts * st_ / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms / st_, "mean_picard_iters": iters,
            "predict_ms_per_launch": pred_ms, "face_update_cfl_ms_per_launch": face_ms,
            "predict_fp64_tflops": fl / (pred_ms / 1e3) / 1e12,
            "predict_frac_of_fp64_peak": fl / (pred_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS})
        del ctx
    return out


def sine2d_state(ctx):
    import numpy as np
    X, Y = ctx.node_coords()
    rho = 1 + 0.5 * np.sin(2 * np.pi * (X + Y))
    g = 1.4
    return np.stack([rho, rho, rho, 1 / (g - 1) + rho], -1)  # u = v = 1, p = 1


def run_2d(args, dev, flush, tables=False):
    """2D Euler (ader_init_2d): throughput of the 2D solve and, with tables, the
    sine-wave advection problem of Sec. 2.1 at the meshes of Table
    conv_orders_pde_2d to t = 1 through the GPU path (errors, orders, the
    paper's eps_L1 beside them)."""
    import numpy as np
    import torch

    from paper_2409_12483_gb300 import Context2D
    out = {"sine_wave": [], "throughput": []}
    for N in (range(1, 8) if tables else ()):
        meshes = (10, 15, 20, 25) if N <= 4 else (5, 10, 15, 20)
        prev = None
        for nc in meshes:
            ctx = Context2D(nc, nc, N, device=dev)
            u = torch.tensor(sine2d_state(ctx).ravel(), device=dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            steps, t, rc = ctx.ader_solve(u, t_end=1.0)
            e1.record()
            torch.cuda.synchronize()
            err = dg2_errors(ctx, u.cpu().numpy(), t)
            row = {"degree": N, "cells": f"{nc}x{nc}", "steps": steps, "status": rc,
                   "eps_l1": err[0], "eps_l2": err[1], "eps_linf": err[2],
                   "paper_eps_l1": PAPER_2D_L1[(N, nc)], "ms": e0.elapsed_time(e1)}
            if prev is not None:
                row["order_l1"] = float(np.log(prev[1] / err[0]) / np.log(nc / prev[0]))
            prev = (nc, err[0])
            out["sine_wave"].append(row)
            del ctx
    st_ = max(2, min(args.steps, 3))
    for N, nc, ts in ((3, 512, 20), (5, 320, 20), (7, 160, 10)):
        ctx = Context2D(nc, nc, N, device=dev, profile=1)
        u0 = torch.tensor(sine2d_state(ctx).ravel(), device=dev)
        cells = nc * nc
        ms, prof, u = measure_solve(ctx, u0, ts, st_, 2, flush)
        iters = sum(p["mean_iters"] for p in prof) / len(prof)
        nsteps = sum(p["profiled_steps"] for p in prof)
        pred_ms = sum(p["predict_ms"] for p in prof) / max(nsteps, 1)
        face_ms = sum(p["face_ms"] for p in prof) / max(nsteps, 1)
        fl = cells * predictor2d_flops_per_cell(N + 1, iters)
        out["throughput"].append({
            "name": f"dg{N}-2d-{nc}x{nc}", "workload": f"2D sine wave (Sec. 2.1), DG N={N}, "
            f"{nc}x{nc} cells periodic, {ts} steps, FP64", "value": cells * ts * st_ / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms / st_, "mean_picard_iters": iters,
            "predict_ms_per_launch": pred_ms, "face_update_cfl_ms_per_launch": face_ms,
            "predict_fp64_tflops": fl / (pred_ms / 1e3) / 1e12,
            "predict_frac_of_fp64_peak": fl / (pred_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS})
        del ctx
    return out


def run_tracer(args, dev, flush):
    """The non-conservative product (Euler + passive tracer in non-conservative
    form): throughput at the headline's size, and the tracer's deviation from
    rho in uniform flow (u = p = 1, tracer started equal to rho), where the
    non-conservative scheme must reproduce the conservative one."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2409_12483_gb300 import Context
    st_ = max(2, min(args.steps, 3))
    ctx = Context(CELLS, DEGREE, "dg", device=dev, profile=1, system="tracer")
    x = ctx.node_coords()
    e = W.nodal_state(W.modes4(SEED), x)  # rho, m, E of the headline data
    u0 = torch.tensor(np.concatenate([e, 0.5 + 0.3 * np.cos(2 * np.pi * x)[..., None]], -1),
                      device=dev).reshape(-1)
    line = variant_line("tracer-dg5-1e5", "Euler + non-conservative tracer (B dU/dx = u dphi/dx), "
                        "DG N=5, 10^5 cells, 100 steps, FP64", ctx, u0, CELLS, DEGREE, TIME_STEPS,
                        st_, 2, flush)
    for k in ("predict_fp64_tflops", "predict_frac_of_fp64_peak"):
        line.pop(k, None)
    del ctx
    nc = 64
    ctx = Context(nc, DEGREE, "dg", device=dev, system="tracer")
    x = ctx.node_coords()
    rho = 1 + 0.2 * np.sin(2 * np.pi * x)
    u = torch.tensor(np.stack([rho, rho, 1 / 0.4 + 0.5 * rho, rho], -1), device=dev).reshape(-1)
    steps, t, rc = ctx.ader_solve(u, t_end=1.0)
    torch.cuda.synchronize()
    v = u.cpu().numpy().reshape(nc, DEGREE + 1, 4)
    line["uniform_flow_check"] = {"cells": nc, "t": t, "steps": steps,
                                  "max_abs_tracer_minus_rho": float(np.abs(v[..., 3] - v[..., 0]).max())}
    return line


def run_limiter(args, dev, flush):
    """The a posteriori subcell limiter with outflow boundaries: the four
    classical Riemann problems of Sec. 2 (Table classical_tests_1d) to t = 0.15
    (L1 density error against the exact solution, troubled cells per step), and
    throughput at the headline's size: Sod data, the smooth headline data with
    every cell recomputed by the subcell ADER-WENO2 scheme (limiter mode 2), and
    with the limiter on against off (the limiter's cost where it never acts)."""
    import torch

    import workloads as W
    from paper_2409_12483_gb300 import Context
    out = {"riemann": [], "throughput": []}
    cases = [(N, nc) for N in (3, 5) for nc in (200, 1000)]
    cases.append((7, 50))  # nearest to the paper's DG-P9 on 50 cells (N <= 7 here)
    for test in (1, 2, 3, 4):
        for N, nc in cases:
            ctx = Context(nc, N, "dg", device=dev, bc="outflow", limiter=1)
            u = torch.tensor(W.riemann_initial(ctx.node_coords(), test), device=dev).reshape(-1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            steps, t, rc = ctx.ader_solve(u, t_end=0.15)
            e1.record()
            torch.cuda.synchronize()
            st = ctx.ader_get_stats()
            out["riemann"].append({
                "test": test, "degree": N, "cells": nc, "steps": steps, "status": rc,
                "l1_density_vs_exact": riemann_density_l1(ctx, u.cpu().numpy(), test, t),
                "troubled_per_step": st["troubled_cells"] / max(steps, 1),
                "ms": e0.elapsed_time(e1)})
            del ctx
    st_ = max(2, min(args.steps, 3))
    ctx = Context(CELLS, DEGREE, "dg", device=dev, profile=1, bc="outflow", limiter=1)
    u0 = torch.tensor(W.riemann_initial(ctx.node_coords(), 1), device=dev).reshape(-1)
    line = variant_line("sod-dg5-1e5-limiter", "Sod data (Table classical_tests_1d test 1), DG N=5, "
                        "10^5 cells, outflow, subcell limiter, 100 steps, FP64",
                        ctx, u0, CELLS, DEGREE, TIME_STEPS, st_, 2, flush)
    line["troubled_per_step"] = ctx.ader_get_stats()["troubled_cells"] / TIME_STEPS
    for k in ("predict_fp64_tflops", "predict_frac_of_fp64_peak"):
        line.pop(k, None)
    out["throughput"].append(line)
    del ctx
    ctx = Context(CELLS, DEGREE, "dg", device=dev, profile=1, limiter=2)
    u0 = torch.tensor(W.nodal_state(W.modes4(SEED), ctx.node_coords()), device=dev).reshape(-1)
    line = variant_line("dg5-1e5-modes4-limiter2", "the headline workload, every cell recomputed "
                        "on its 11 subcells by ADER-WENO2 (limiter mode 2)",
                        ctx, u0, CELLS, DEGREE, TIME_STEPS, st_, 2, flush)
    line["troubled_cells"] = ctx.ader_get_stats()["troubled_cells"]
    for k in ("predict_fp64_tflops", "predict_frac_of_fp64_peak"):
        line.pop(k, None)
    out["throughput"].append(line)
    del ctx
    for lim in (1, 0):
        ctx = Context(CELLS, DEGREE, "dg", device=dev, profile=1, limiter=lim)
        u0 = torch.tensor(W.nodal_state(W.modes4(SEED), ctx.node_coords()), device=dev).reshape(-1)
        line = variant_line(f"dg5-1e5-modes4-limiter{lim}", "the headline workload, limiter "
                            + ("on (never triggered on smooth data)" if lim else "off"),
                            ctx, u0, CELLS, DEGREE, TIME_STEPS, st_, 2, flush)
        line["troubled_cells"] = ctx.ader_get_stats()["troubled_cells"]
        out["throughput"].append(line)
        del ctx
    return out


def run_variants(args, dev, flush):
    """Secondary workloads measured on rank 0 after the headline."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2409_12483_gb300 import Context
    out = []
    st = max(2, min(args.steps, 3))
    # the headline workload in the other precision forms of the predictor; each
    # states its distance from the FP64 path after one step and after the
    # bench's 100 steps (the FP64 path matches the FP64 oracle to ~1e-15 per step)
    ref = Context(CELLS, DEGREE, "dg", device=dev)
    u0 = torch.tensor(W.nodal_state(W.modes4(SEED), ref.node_coords()), device=dev).reshape(-1)
    uref = u0.clone()
    ref.ader_solve(uref, max_steps=TIME_STEPS)
    one_ref = torch.empty_like(u0)
    ref.ader_step(u0, one_ref, 0.0)

    def err_vs_fp64(ctx_):
        def f(u):
            one = torch.empty_like(u0)
            ctx_.ader_step(u0, one, 0.0)
            return {"rel_linf_vs_fp64_path": (u - uref).abs().max().item() / uref.abs().max().item(),
                    "rel_linf_vs_fp64_path_one_step":
                        (one - one_ref).abs().max().item() / one_ref.abs().max().item()}
        return f
    forms5 = (("dg5-1e5-incr", "as the headline, increment form: float-float first iteration "
               "and terms of u, FP32 Picard on the correction with exact flux differences",
               dict(precision="incr")),
              ("dg5-1e5-fp32ff1", "as the headline, FP32 Picard + 1 float-float sweep and "
               "float-float epilogue", dict(precision="fp32ff", fp64_sweeps=1)),
              ("dg5-1e5-fp32ff2", "as the headline, FP32 Picard + 2 float-float sweeps and "
               "float-float epilogue", dict(precision="fp32ff", fp64_sweeps=2)),
              ("dg5-1e5-fp32pred", "as the headline, FP32 Picard + 2 FP64 sweeps",
               dict(precision="fp32", fp64_sweeps=2)),
              ("dg5-1e5-ffpred", "as the headline, float-float Picard (FP64-accurate)",
               dict(precision="ff")))
    for name, desc, kw in forms5:
        ctx = Context(CELLS, DEGREE, "dg", device=dev, profile=1, **kw)
        ctx.ader_autotune(u0, reps=2)
        out.append(variant_line(name, desc, ctx, u0, CELLS, DEGREE, TIME_STEPS, st, 2, flush,
                                extra=err_vs_fp64(ctx), field=W.modes4(SEED)))
        del ctx
    del ref, uref, one_ref
    # ADER-WENO5 (WENO N=4 + LST-DG N=4), 10^6 cells, 100 steps, FP64
    nc = 1_000_000
    ctx = Context(nc, 4, "fv", device=dev, profile=1)
    v0 = torch.tensor(W.cell_average_state(W.modes4(SEED), nc), device=dev).reshape(-1)
    ctx.ader_autotune(v0, reps=2)
    wl = variant_line("weno5-1e6-fp64", "ADER-WENO5 FV, 10^6 cells, modes4, 100 steps, FP64, "
                      "autotuned shapes, time loop as device-resident CUDA graphs",
                      ctx, v0, nc, 4, TIME_STEPS, st, 1, flush, dg=False)
    # the same 100 steps launched plainly: one host call per step (CFL, WENO,
    # predictor, update launched from the host; default launch shapes)
    plain = Context(nc, 4, "fv", device=dev)
    a = v0.clone()
    b = torch.empty_like(a)
    plain.ader_step(a, b, 0.0)
    torch.cuda.synchronize()
    a.copy_(v0)
    flush.zero_()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(TIME_STEPS):
        plain.ader_step(a, b, 0.0)
        a, b = b, a
    ev1.record()
    torch.cuda.synchronize()
    wl["plain_host_launched"] = {"value": nc * TIME_STEPS / (ev0.elapsed_time(ev1) / 1e3),
                                 "unit": UNIT, "ms_per_step": ev0.elapsed_time(ev1)}
    out.append(wl)
    w64 = torch.empty_like(v0)
    w64.copy_(v0)
    ctx.ader_solve(w64, max_steps=TIME_STEPS)
    del ctx, plain, a, b
    # the same workload with the faster predictor forms (WENO, interface and CFL in FP64)
    for name, kw in (("weno5-1e6-incr", dict(precision="incr")),
                     ("weno5-1e6-ffpred", dict(precision="ff"))):
        c = Context(nc, 4, "fv", device=dev, profile=1, **kw)
        c.ader_autotune(v0, reps=2)

        def errw(u):
            return {"rel_linf_vs_fp64_path": (u - w64).abs().max().item() / w64.abs().max().item()}
        out.append(variant_line(name, f"ADER-WENO5 FV, 10^6 cells, modes4, 100 steps, predictor "
                                f"{kw['precision']}", c, v0, nc, 4, TIME_STEPS, st, 1, flush,
                                dg=False, extra=errw))
        del c
    del v0, w64
    # ADER-DG N=7, 10^6 cells: FP64 and FP32-predictor (2 FP64 sweeps), 20 steps
    ts = 20
    c64 = Context(nc, 7, "dg", device=dev, profile=1)
    x = c64.node_coords()
    u0 = torch.tensor(W.nodal_state(W.modes4(SEED), x), device=dev).reshape(-1)
    keep = {}

    def grab(u):
        keep["u64"] = u.clone()
        return {}
    out.append(variant_line("dg7-1e6-fp64", "ADER-DG N=7, 10^6 cells, modes4, 20 steps, FP64",
                            c64, u0, nc, 7, ts, st, 1, flush, extra=grab))
    del c64
    for name, desc, kw in (
            ("dg7-1e6-incr", "ADER-DG N=7, 10^6 cells, increment form (FP32 Picard on the "
             "correction)", dict(precision="incr")),
            ("dg7-1e6-ffpred", "ADER-DG N=7, 10^6 cells, float-float Picard", dict(precision="ff")),
            ("dg7-1e6-fp32ff2", "ADER-DG N=7, 10^6 cells, FP32 Picard + 2 float-float sweeps",
             dict(precision="fp32ff", fp64_sweeps=2)),
            ("dg7-1e6-fp32pred", "ADER-DG N=7, 10^6 cells, FP32 Picard + 2 FP64 sweeps",
             dict(precision="fp32", fp64_sweeps=2))):
        c = Context(nc, 7, "dg", device=dev, profile=1, **kw)

        def err7(u):
            u64 = keep["u64"]
            return {"rel_linf_vs_fp64_path": (u - u64).abs().max().item() / u64.abs().max().item()}
        out.append(variant_line(name, desc, c, u0, nc, 7, ts, st, 1, flush, extra=err7))
        del c
    return out


def run_small_meshes(dev, steps_n=2000):
    """Batching pattern on small meshes, where one step is short: the same
    ader_solve time loop as device-resident CUDA graphs (autotuned tile shapes
    and graph length) against one host-launched ader_step per step (device CFL
    step, default shapes), FP64 and the float-float predictor.  Time per step
    from the host clock around whole solves (synchronised)."""
    import torch

    import workloads as W
    from paper_2409_12483_gb300 import Context
    out = []
    for N, nc in ((2, 100), (2, 1000), (5, 1000), (2, 10000), (5, 10000)):
        for prec in ("fp64", "ff"):
            ctx = Context(nc, N, "dg", device=dev, precision=prec)
            u0 = torch.tensor(W.nodal_state(W.sine(), ctx.node_coords()), device=dev).reshape(-1)
            plain = Context(nc, N, "dg", device=dev, precision=prec)
            tune = ctx.ader_autotune(u0, reps=3)
            g = p = 0.0
            for _ in range(2):  # the second pass is timed
                u = u0.clone()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ctx.ader_solve(u, max_steps=steps_n)
                torch.cuda.synchronize()
                g = (time.perf_counter() - t0) / steps_n
                a, b = u0.clone(), torch.empty_like(u0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(steps_n):
                    plain.ader_step(a, b, 0.0)
                    a, b = b, a
                torch.cuda.synchronize()
                p = (time.perf_counter() - t0) / steps_n
            out.append({"degree": N, "cells": nc, "precision": prec,
                        "graph_us_per_step": 1e6 * g, "plain_us_per_step": 1e6 * p,
                        "graph_speedup": p / g, "graph_cell_updates_per_s": nc / g,
                        "tuning": {k: tune[k] for k in ("predict_cells_per_block",
                                                         "face_cells_per_block", "graph_steps")}})
            del ctx, plain
    return out


SERVING_NOTE = ("scaled stand-in for the 4096-request stream (cells log-uniform in [64, 65536], "
                "t_end 0.5: ~2.5e13 cell-updates, days of GPU time): {n} requests, cells "
                "log-uniform in [64, {cmax}], N ~ U{{1..7}}, rho and p = 1 + 3 modes (amplitudes "
                "<= 0.1/3), u = 0.5, t_end = {tend}, seed 12483; FP32 predictor (increment form: "
                "FP32 Picard on the correction, float-float terms of u) + FP64 corrector/CFL")


def serving_stream(n, cmax, tend, seed=SEED):
    import workloads as W
    reqs = W.serving_requests(count=n, seed=seed, rate=1.0, max_cells=cmax, t_end=tend)
    return reqs


def run_serving(dev, n=128, cmax=2048, tend=0.05, rates=(0.5, 0.8, 1.0), ticks=16,
                tick_sweep=(4, 64), precision="incr", sweeps=1):
    """Continuous-batching server vs the plain per-solve FP64 path on one GPU.

    Saturation: every request queued at t = 0.  Open loop: Poisson arrivals at
    fractions of the server's saturation rate, server clock = wall clock.
    Baseline: each request solved alone with ader_solve (FP64) in arrival order;
    its latencies replay the same arrival times on a FIFO single server with the
    measured per-request service times.

    Latency breakdown per request: queue wait (admitted - arrival), run time
    (finished - admitted) and the request's own time steps.  Every admitted
    solve advances one step per tick, so run time ~ steps x tick time: the
    spread of latencies follows the spread of step counts (cells x (2N+1)),
    which the p50/p99 of run time per step isolates.  The open loop at 0.8 x
    saturation is repeated with shorter and longer graph rounds
    (ticks_per_round in tick_sweep)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2409_12483_gb300 import Context
    from paper_2409_12483_gb300.capi import REQ_DONE, Server
    reqs = serving_stream(n, cmax, tend)
    states = []
    for r in reqs:
        ctx = Context(r.cells, r.degree, "dg", device=dev)
        states.append(W.nodal_state(r.field, ctx.node_coords()).ravel())
        del ctx
    pool = sum(Server.request_bytes(r.degree, r.cells) for r in reqs) + (64 << 20)

    def run_server(arrivals, tpr=ticks):
        srv = Server(pool_bytes=pool, max_slots=len(reqs), ticks_per_round=tpr,
                     precision=precision, fp64_sweeps=sweeps, device=dev)
        ids = [srv.submit(r.degree, st, r.t_end, arrival=a) for r, st, a in zip(reqs, states, arrivals)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while True:
            run, que = srv.progress(time.perf_counter() - t0)
            if run == 0 and que == 0:
                break
            if run == 0:
                time.sleep(1e-4)
        wall = time.perf_counter() - t0
        res = [srv.poll(i) for i in ids]
        assert all(x["state"] == REQ_DONE for x in res)
        lat = np.array([x["finished"] - x["arrival"] for x in res])
        wait = np.array([x["admitted"] - x["arrival"] for x in res])
        steps = np.array([x["steps"] for x in res], dtype=float)
        tot = srv.totals()
        srv.close()
        run_per_step = (lat - wait) / steps
        pct = lambda a: {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99))}
        tot["breakdown"] = {"queue_wait_s": pct(wait), "run_s": pct(lat - wait),
                            "steps": pct(steps), "run_s_per_step": pct(run_per_step),
                            "corr_latency_steps": float(np.corrcoef(lat, steps)[0, 1])}
        return wall, lat, tot

    wall0, lat0, tot0 = run_server([0.0] * len(reqs))
    sat = len(reqs) / wall0
    out = {"workload": SERVING_NOTE.format(n=n, cmax=cmax, tend=tend),
           "cell_updates": tot0["cell_updates"],
           "ticks_per_round": ticks,
           "saturation": {"solves_per_s": sat, "cell_updates_per_s": tot0["cell_updates"] / wall0,
                          "makespan_s": wall0, "rounds": tot0["rounds"], "ticks": tot0["ticks"],
                          "kernel_launches": tot0["kernel_launches"]},
           "open_loop": [], "tick_sweep_at_0.8": []}
    # plain per-solve FP64 baseline: service time of every request alone
    service = []
    for r, st in zip(reqs, states):
        ctx = Context(r.cells, r.degree, "dg", device=dev)
        u = torch.tensor(st, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.ader_solve(u, t_end=r.t_end)
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t0)
        del ctx, u
    service = np.array(service)
    base_sat = len(reqs) / service.sum()
    out["baseline_per_solve_fp64"] = {"solves_per_s": base_sat,
                                      "cell_updates_per_s": tot0["cell_updates"] / service.sum()}
    rng = np.random.default_rng(SEED + 1)
    for frac in rates:
        rate = frac * sat
        gaps = rng.exponential(1.0 / rate, size=len(reqs))
        arr = np.cumsum(gaps) - gaps[0]
        wall, lat, tot = run_server(list(arr))
        # FIFO replay of the baseline on the same arrivals
        end, blat = 0.0, []
        for a, sv in zip(arr, service):
            start = max(a, end)
            end = start + sv
            blat.append(end - a)
        blat = np.array(blat)
        out["open_loop"].append({
            "arrival_rate_frac_of_saturation": frac, "arrival_rate_solves_per_s": rate,
            "server": {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                       "solves_per_s": len(reqs) / wall, "breakdown": tot["breakdown"]},
            "baseline_per_solve_fp64": {"p50_s": float(np.percentile(blat, 50)),
                                        "p99_s": float(np.percentile(blat, 99)),
                                        "solves_per_s": len(reqs) / max(end, 1e-9)}})
        if frac == 0.8:
            for tpr in tick_sweep:
                wall, lat, tot = run_server(list(arr), tpr)
                out["tick_sweep_at_0.8"].append({
                    "ticks_per_round": tpr, "p50_s": float(np.percentile(lat, 50)),
                    "p99_s": float(np.percentile(lat, 99)), "solves_per_s": len(reqs) / wall,
                    "queue_wait_p99_s": tot["breakdown"]["queue_wait_s"]["p99"]})
    return out


def run_case(args):
    """Small fixed cases for ncu captures (inputs larger than L2, a few GB at most)."""
    import torch

    import workloads as W
    from paper_2409_12483_gb300 import Context
    dev = torch.device("cuda", 0)
    nc = 1_000_000
    if args.case == "predict-dg5":
        ctx = Context(nc, 5, "dg", device=dev)
        u = torch.tensor(W.nodal_state(W.modes4(SEED), ctx.node_coords()), device=dev).reshape(-1)
    elif args.case == "predict-dg5-ff":
        ctx = Context(nc, 5, "dg", device=dev, precision="ff")
        u = torch.tensor(W.nodal_state(W.modes4(SEED), ctx.node_coords()), device=dev).reshape(-1)
    elif args.case == "predict-dg5-incr":
        ctx = Context(nc, 5, "dg", device=dev, precision="incr")
        u = torch.tensor(W.nodal_state(W.modes4(SEED), ctx.node_coords()), device=dev).reshape(-1)
    elif args.case == "predict-dg7-fp32":
        ctx = Context(nc, 7, "dg", device=dev, precision="fp32", fp64_sweeps=2)
        u = torch.tensor(W.nodal_state(W.modes4(SEED), ctx.node_coords()), device=dev).reshape(-1)
    elif args.case == "weno5":
        ctx = Context(nc, 4, "fv", device=dev)
        u = torch.tensor(W.cell_average_state(W.modes4(SEED), nc), device=dev).reshape(-1)
    elif args.case in ("step2d-dg5", "step2d-dg3", "step3d-dg2", "step3d-dg2-48", "step3d-dg5",
                       "step3d-dg7"):
        from paper_2409_12483_gb300 import Context2D, Context3D
        if args.case == "step2d-dg5":  # 96^2 cells: 35 MB state
            ctx = Context2D(96, 96, 5, device=dev)
            u = torch.tensor(sine2d_state(ctx).ravel(), device=dev)
        elif args.case == "step2d-dg3":  # 512^2 cells: 134 MB state, 0.67 GB traces
            ctx = Context2D(512, 512, 3, device=dev)
            u = torch.tensor(sine2d_state(ctx).ravel(), device=dev)
        elif args.case == "step3d-dg5":  # 24^3 cells: 119 MB state, 0.84 GB traces
            ctx = Context3D(24, 24, 24, 5, device=dev)
            u = torch.tensor(sine3d_state(ctx).ravel(), device=dev)
        elif args.case == "step3d-dg7":  # 12^3 cells: 35 MB state, 248 MB traces
            ctx = Context3D(12, 12, 12, 7, device=dev)
            u = torch.tensor(sine3d_state(ctx).ravel(), device=dev)
        elif args.case == "step3d-dg2-48":  # 48^3 cells: 119 MB state, 0.84 GB traces
            ctx = Context3D(48, 48, 48, 2, device=dev)
            u = torch.tensor(sine3d_state(ctx).ravel(), device=dev)
        else:  # 96^3 cells: 0.96 GB state
            ctx = Context3D(96, 96, 96, 2, device=dev)
            u = torch.tensor(sine3d_state(ctx).ravel(), device=dev)
        steps, t, rc = ctx.ader_solve(u, max_steps=args.warmup + args.steps)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "cells": ctx.n_cells, "steps": steps, "status": rc}))
        return
    elif args.case in ("sod-dg5-limiter", "tracer-dg5", "reacting-dg5", "solve-dg5", "solve-dg5-1e5",
                       "limiter-dg5-1e5"):
        # 10^6 cells (144-192 MB of state, above L2): warmup + steps time steps
        import numpy as np
        if args.case in ("solve-dg5", "solve-dg5-1e5"):  # the interface kernel with lambda_max
            ctx = Context(nc if args.case == "solve-dg5" else CELLS, 5, "dg")
            u = torch.tensor(W.nodal_state(W.modes4(SEED), ctx.node_coords()), device=dev).reshape(-1)
        elif args.case == "limiter-dg5-1e5":  # the headline data with the limiter on (never acting)
            ctx = Context(CELLS, 5, "dg", device=dev, limiter=1)
            u = torch.tensor(W.nodal_state(W.modes4(SEED), ctx.node_coords()), device=dev).reshape(-1)
        elif args.case == "sod-dg5-limiter":
            ctx = Context(nc, 5, "dg", device=dev, bc="outflow", limiter=1)
            u = torch.tensor(W.riemann_initial(ctx.node_coords(), 1), device=dev).reshape(-1)
        elif args.case == "tracer-dg5":
            ctx = Context(nc, 5, "dg", device=dev, system="tracer")
            x = ctx.node_coords()
            e = W.nodal_state(W.modes4(SEED), x)
            u = torch.tensor(np.concatenate([e, 0.5 + 0.3 * np.cos(2 * np.pi * x)[..., None]], -1),
                             device=dev).reshape(-1)
        else:
            ctx = Context(nc, 5, "dg", device=dev, system="reacting", omega=1.0)
            u = torch.tensor(W.reacting_state(ctx.node_coords(), seed=SEED), device=dev).reshape(-1)
        steps, t, rc = ctx.ader_solve(u, max_steps=args.warmup + args.steps)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "cells": ctx.n_cells, "steps": steps, "status": rc}))
        return
    elif args.case == "sine-tables":  # the 2D and 3D convergence tables of Sec. 2.1
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
        print_study("two_d_sine_wave_table", lambda: run_2d(args, dev, flush, True)["sine_wave"])
        print_study("three_d_sine_wave_table", lambda: run_3d(args, dev, flush, True)["sine_wave"])
        return
    elif args.case == "serving-large":  # a larger slice of the serving stream
        print_study("serving_512_requests_cells_to_4096", run_serving, dev, 512, 4096)
        return
    elif args.case == "paper-costs":  # the cost-table comparison alone
        from paper_2409_12483_gb300 import Context2D, Context3D
        print(json.dumps({
            "two_d": paper_cost_rows(lambda N: Context2D(16, 16, N, device=dev), sine2d_state,
                                     PAPER_2D_TJIT_16, "16x16", dev),
            "three_d": paper_cost_rows(lambda N: Context3D(7, 7, 7, N, device=dev), sine3d_state,
                                       PAPER_3D_TJIT_7, "7^3", dev)}))
        return
    else:
        raise SystemExit(f"unknown case {args.case}")
    out = torch.empty_like(u)
    tuning = ctx.ader_autotune(u, reps=3)  # the launch shapes the bench would time
    times = []
    for i in range(args.warmup + args.steps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        if i == args.warmup:
            torch.cuda.nvtx.range_push("timed")  # ncu --nvtx-include "timed/" captures these steps
        ev0.record()
        ctx.ader_step(u, out, 0.0)
        ev1.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(ev0.elapsed_time(ev1))
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"case": args.case, "cells": nc, "ms_per_step": sum(times) / len(times),
                      "tuning": tuning, "stats": ctx.ader_get_stats()}))


if __name__ == "__main__":
    main()
