#!/usr/bin/env python3
"""Throughput of the cut-cell multi-material update on GB300.

Headline workload: the 3D Mach-1.22 shock on a heavy sphere, 256 x 128 x 128
cells, two stiffened gases (the largest single-GPU configuration; synthetic
initial data). One step is one full TVD-RK3 step (three stages of every step
of the method) over the whole grid; the metric is cell-stage updates per
second (cells x 3 per step). The headline value is the FP32-bulk form; the
plain FP64 path runs beside it on the same workload, and the difference of the
two after the same steps is reported for every output (density, velocity,
pressure, volume fractions, level set, totals).

Side keys: the 2D triple point (896 x 384: first steps and a window from
t = 0.3), the two-bubble shock (2048 x 512), the batched 1D problems, Case II's
shell study and the adjoint step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl msf|reference]

--impl reference times the CPU oracle (the plain FP64 C implementation under
oracle/) on the host cores for the same workload and metric.
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="shock_sphere_256x128x128", n=(256, 128, 128))
METRIC = "cell-stage updates/s: FP32/batched/adjoint vs plain FP64 on GB300 at stated L1"
UNIT = "cell-stage updates/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="msf", choices=["msf", "reference"])
    ap.add_argument("--only", default=None, choices=["fp32", "fp64"],
                    help="profiling aid: run warm-up and timed steps of one precision only, print nothing else")
    ap.add_argument("--case", default="sphere", choices=["sphere", "triple", "bubbles"],
                    help="workload of --only (default: the headline sphere)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_case(which="sphere"):
    import paper_1704_00519_gb300.cases as cs
    if which == "triple":
        return cs.triple_point(896, 384)
    if which == "bubbles":
        return cs.shock_bubbles(2048, 512)
    return cs.shock_sphere(WORKLOAD["n"])


# ------------------------------------------------------------ reference arm
def oracle_rate(case, steps, warmup, openmp=True, budget_s=None):
    """Time the CPU oracle as it stands on full steps of the workload (the
    OpenMP build on every host core, or the plain build on one); with a time
    budget, fewer steps are timed when one step is slow. Returns
    (cell-stages/s, seconds, steps timed, threads)."""
    from oracle.oracle import Oracle, threads
    o = Oracle(case, openmp=openmp)
    t0 = time.perf_counter()
    if warmup:
        o.step(warmup, case.t_end)
    per_step = (time.perf_counter() - t0) / warmup if warmup else None
    if budget_s and per_step:
        steps = max(1, min(steps, int(budget_s / per_step)))
    t0 = time.perf_counter()
    o.step(steps, case.t_end)
    dt = time.perf_counter() - t0
    return case.cells * 3 * steps / dt, dt, steps, threads(openmp)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as orc
    orc.build(openmp=True)
    case = make_case()
    # one OpenMP oracle step of the workload takes seconds: bound the run to a few minutes
    warm = max(1, min(args.warmup, 1))
    val, secs, steps, nthr = oracle_rate(case, args.steps, warm, openmp=True, budget_s=150.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
        "n_gpus": 0, "steps": steps, "warmup": warm, "ms_per_step": 1e3 * secs / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "cells": case.cells, "materials": case.nmat},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": nthr, "kind": "oracle",
                         "sample": f"{steps} full TVD-RK3 steps of the {WORKLOAD['name']} workload after {warm} "
                                   f"warm-up step(s), OpenMP oracle on {nthr} threads (capped at 150 s of timed steps)"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def flux_kernel_hash():
    h = hashlib.sha256()
    for f in ("msf_kernels.cuh", "msf_device.cuh", "msf_types.cuh", "msf_prec.inc"):
        with open(os.path.join(ROOT, "paper_1704_00519_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(precision):
    """DRAM bytes per flux-update launch from the committed ncu summary, when
    it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "flux_update_shock_sphere_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_hash") != flux_kernel_hash():
        return None
    return d.get(precision, {}).get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def icf_rates(msf, torch, stream, K):
    """Case II's shell-thickness study (Sec. 3.2) as one batched launch: 256
    cylindrical implosions of 1280 cells (r2 - r1 in [0.05, 0.3]) driven by the
    free-surface pressure p(t), FP64 and FP32-bulk, device-timed over K steps
    after 5 warm-up steps."""
    import paper_1704_00519_gb300.cases as cs
    cases = cs.icf_shell_study(1280, 256)
    out = {"workload": "icf_shell_study_256x1280", "cells": int(sum(c.cells for c in cases)),
           "instances": len(cases), "steps": K}
    for key, prec in (("fp32", msf.MSF_FP32_BULK), ("fp64", msf.MSF_FP64)):
        b = msf.Batch(cases, precision=prec, stream=stream)
        b.step(5, 1.0, sync=False)
        before = [b.info(i)[1] for i in range(len(cases))]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        b.step(K, 1.0, sync=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        info = [b.info(i) for i in range(len(cases))]
        work = sum(c.cells * 3 * (info[i][1] - before[i]) for i, c in enumerate(cases))
        out[key] = {"value": work / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K,
                    "instances_with_device_error": sum(1 for x in info if x[2] != 0)}
        b.close()
    return out


def batched_rates(msf, torch, stream, K_persistent, K_sequence):
    """256 seeded 1D multi-material Riemann problems (FP32-bulk): one
    persistent launch per call (one CTA per instance, autotuned CTA size)
    against the per-instance kernel sequences, both device-timed."""
    import paper_1704_00519_gb300.cases as cs
    cases = cs.batched_1d(256, 20170403)
    cells = [c.cells for c in cases]

    def run(mode, K, warm):
        b = msf.Batch(cases, precision=msf.MSF_FP32_BULK, batch_mode=mode, stream=stream)
        b.step(warm, 0.1, sync=False)
        before = [b.info(i)[1] for i in range(len(cases))]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        b.step(K, 0.1, sync=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        info = [b.info(i) for i in range(len(cases))]
        work = sum(cells[i] * 3 * (info[i][1] - before[i]) for i in range(len(cases)))
        bad = sum(1 for x in info if x[2] != 0)
        bs = b.block_size()
        b.close()
        return work / (ms / 1e3), ms / K, bad, bs

    v1, ms1, bad1, bs = run(0, K_persistent, 5)
    v2, ms2, bad2, _ = run(1, K_sequence, 1)
    return {"workload": "256 seeded 1D Riemann problems (seed 20170403), 200-20000 cells, 2-4 stiffened gases",
            "cells": int(sum(cells)), "instances": len(cases), "precision": "fp32_bulk",
            "value": v1, "unit": UNIT, "ms_per_step": ms1, "cta_threads": bs, "steps": K_persistent,
            "per_instance_launches": {"value": v2, "unit": UNIT, "ms_per_step": ms2, "steps": K_sequence},
            "speedup_vs_per_instance": v1 / v2, "instances_with_device_error": max(bad1, bad2)}


def workload_rates(msf, torch, stream, K):
    """Forward throughput of the two-bubble (2D, 2048 x 512) and triple-point
    (2D, 896 x 384) workloads from their first steps, FP32-bulk and FP64, device-timed, with
    the L1 density difference of the two after the same steps."""
    import paper_1704_00519_gb300.cases as cs
    out = {}
    for name, maker in (("shock_bubbles_2048x512", lambda: cs.shock_bubbles(2048, 512)),
                        ("triple_point_896x384", lambda: cs.triple_point(896, 384))):
        case = maker()
        r = {"cells": case.cells, "steps": K}
        rho = {}
        for key, prec in (("fp32", msf.MSF_FP32_BULK), ("fp64", msf.MSF_FP64)):
            s = msf.Solver(case, precision=prec, stream=stream)
            s.step(2, case.t_end)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            s.step(K, case.t_end, sync=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / K
            r[key] = {"value": case.cells * 3 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms}
            rho[key] = s.state()["Q"][:, 0].sum(0)
            s.close()
        r["fp32_over_fp64"] = r["fp32"]["value"] / r["fp64"]["value"]
        r["l1_rho_fp32_vs_fp64"] = float(np.abs(rho["fp32"] - rho["fp64"]).sum() / np.abs(rho["fp64"]).sum())
        out[name] = r
    return out


def adjoint_rates(msf, torch, stream, K):
    """Adjoint form on the 3D shock-sphere workload (256 x 128 x 128), FP32-bulk
    context: K taped steps (forward with stage checkpoints), then K adjoint
    steps of a unit seed, each timed on the context stream; cell-stage/s of
    the reverse sweep."""
    import paper_1704_00519_gb300.cases as cs
    case = cs.shock_sphere((256, 128, 128))
    s = msf.Solver(case, precision=msf.MSF_FP32_BULK, stream=stream)
    s.step(2, case.t_end)
    tapes = [s.new_tape() for _ in range(K)]
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record()
    for tp in tapes:
        s.step_taped(tp, case.t_end)
    e[1].record()
    lam = torch.ones((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
    lam1, _, _ = s.adjoint_step(tapes[-1], lam)   # allocates the adjoint workspace
    torch.cuda.synchronize()
    e[1].synchronize()
    fwd_ms = e[0].elapsed_time(e[1]) / K
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record()
    d_eos = np.zeros((case.nmat, 2))
    for tp in reversed(tapes):
        lam, de, _ = s.adjoint_step(tp, lam)
        d_eos += de
    b1.record()
    torch.cuda.synchronize()
    bwd_ms = b0.elapsed_time(b1) / K
    finite = bool(torch.isfinite(lam).all()) and bool(np.all(np.isfinite(d_eos)))
    tb = s.tape_bytes()
    s.close()
    return {"workload": "shock_sphere_256x128x128", "cells": case.cells, "steps": K, "precision": "fp32_bulk",
            "value": case.cells * 3 / (bwd_ms / 1e3), "unit": UNIT, "adjoint_ms_per_step": bwd_ms,
            "taped_forward_ms_per_step": fwd_ms, "tape_bytes_per_step": tb, "finite": finite,
            "how": "msf_adjoint_step per step (recomputes the stages from the tape); events on the context stream"}


def adjoint_gradient(msf, torch, stream, steps=200):
    """The adjoint form at the configured scale: d(J1, J2)/d(rho_bubble,
    gamma_bubble, Mach) of the 3D shock-sphere workload (256 x 128 x 128,
    FP32-bulk context) over `steps` TVD-RK3 steps, through the autograd
    function MsfStep (taped forward steps, msf_adjoint_step in the backward
    pass). Only the tapes (the stage checkpoints) stay resident between the
    passes, with the wall rows J2 needs; the step count is reduced when the
    device has no room for the tapes."""
    from paper_1704_00519_gb300 import adjoint as adj
    import paper_1704_00519_gb300.cases as cs
    prob = adj.ShockBubble((256, 128, 128))
    th0 = prob.theta0()
    case0 = prob.case(th0)
    solver = msf.Solver(case0, precision=msf.MSF_FP32_BULK, stream=stream)
    free, _ = torch.cuda.mem_get_info()
    tb = solver.tape_bytes()
    fit = int(0.8 * free / (tb + 4 * 1024 * 1024))
    K = max(1, min(steps, fit))
    st0 = solver.state()
    alpha0 = torch.tensor(st0["alpha"], device="cuda")
    xs = torch.tensor(cs.centres(prob.n, case0.lo, case0.hi)[0].ravel(), device="cuda")
    wall = torch.tensor(np.nonzero(cs.centres(prob.n, case0.lo, case0.hi)[1].ravel() < 1.0 / prob.n[1])[0],
                        device="cuda")
    h = [(case0.hi[d] - case0.lo[d]) / prob.n[d] for d in range(3)]
    farea = h[0] * h[2]
    torch.cuda.reset_peak_memory_stats()
    theta = th0.clone().cuda().requires_grad_(True)
    eos = prob.eos(theta)
    inflow = prob.inflow(theta)
    Q0 = prob.conserved(prob.prim(theta, "cuda"), eos, alpha0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Q, tapes, J2 = Q0, [], 0.0
    alpha = torch.empty_like(alpha0)
    for _ in range(K):
        Q = adj.MsfStep.apply(Q, eos, inflow, solver, case0.t_end, tapes)
        solver.get_alpha_device(alpha)
        J2 = J2 + adj.tape_dt(tapes[-1]) * adj.wall_pressure_rows(Q, eos, alpha[:, wall].clone(), wall, farea)
    J1 = adj.mass_centroid_x(Q, 1, xs) - adj.mass_centroid_x(Q0, 1, xs)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    g1 = torch.autograd.grad(J1, theta, retain_graph=True)[0]
    g2 = torch.autograd.grad(J2, theta)[0]
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    out = {"workload": "shock_sphere_256x128x128", "precision": "fp32_bulk", "steps": K,
           "theta": ["rho_bubble", "gamma_bubble", "mach"], "theta0": th0.tolist(),
           "J1": float(J1), "J2": float(J2), "dJ1_dtheta": g1.cpu().tolist(), "dJ2_dtheta": g2.cpu().tolist(),
           "forward_ms_per_step": 1e3 * (t1 - t0) / K, "backward_ms_per_step": 1e3 * (t2 - t1) / (2 * K),
           "tape_bytes_per_step": tb, "peak_device_bytes": int(torch.cuda.max_memory_allocated()),
           "how": "taped forward steps through MsfStep (tapes are torch allocations), two autograd.grad calls "
                  "(each runs the K adjoint steps); wall clock with synchronisation, Python included"}
    del tapes, Q, Q0, J1, J2
    solver.close()
    torch.cuda.empty_cache()
    return out


def later_window(msf, torch, stream, flush, K, t_start=0.3):
    """Triple point advanced to t = t_start (the waves have spread over much of
    the domain, so fewer tiles are idle), then K device-timed steps per
    precision. A device-detected error is reported, not raised."""
    case = make_case("triple")
    out = {"t_start": t_start, "steps": K}
    for key, prec in (("fp32", msf.MSF_FP32_BULK), ("fp64", msf.MSF_FP64)):
        s = msf.Solver(case, precision=prec, stream=stream)
        try:
            s.step(100000, t_start)
        except msf.MsfError as e:
            out[key] = {"error": str(e)[:120]}
            s.close()
            continue
        ms = []
        for k in range(K):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.step(1, case.t_end, sync=False)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = sum(ms) / K
        out[key] = {"value": case.cells * 3 / (t / 1e3), "unit": UNIT, "ms_per_step": t}
        s.close()
    if "value" in out["fp32"] and "value" in out["fp64"]:
        out["fp32_over_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    return out


def pairs_per_cell(s):
    """(cell, material) pairs the flux update processes: popcount of the step mask."""
    vals, counts = np.unique(s.debug(5).astype(np.int64), return_counts=True)
    return int(sum(bin(int(v)).count("1") * int(c) for v, c in zip(vals, counts)))


def flux_flops_per_pair_stage(dim):
    """Floating-point operations of the flux update per (cell, material) pair
    and stage, counted from the operations the kernels execute (a division or
    square root counts as one): one WENO5 value 67 (three candidate values 16,
    smoothness indicators 34, weights and normalisation 17), the split fluxes
    of one variable over the 6-cell stencil 39, so one face and variable
    2 * 67 + 39 + 1 = 174, one face nv * 174 + 6 (wave-speed maximum); per
    pair dim faces, plus 17 for the primitive quantities and 19 * nv for the
    aperture-weighted difference, the exchange and the RK combination."""
    nv = dim + 2
    return dim * (nv * 174 + 6) + 17 + 19 * nv


def flux_bytes_per_step(case, npairs):
    """Algorithmic DRAM bytes of the three flux-update launches of one step:
    per (cell, material) pair the stage state is read and the new state written
    (FP64, nv values each), stages 2 and 3 also read Q^n; per cell one indicator
    byte and one mask byte."""
    nv = case.nv
    per_pair = nv * 8 * (2 + 3 + 3)
    return npairs * per_pair + case.cells * 2 * 3


def max_over_ranks(vals, device=None):
    """Largest value of each entry over all ranks (the slowest rank sets the
    job's time); the values themselves on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: every rank processes the same units (weak scaling),
    in the time of the slowest rank."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------------ GPU arm
def output_errors(case, a, b):
    """Difference of state a (FP32-bulk form) from state b (plain FP64 path)
    for every output: L1 relative of the density summed over materials, of
    each material's velocity and pressure where both give it a volume, of the
    volume fractions; the largest level-set difference in cells h; the largest
    relative difference of the per-material totals is taken separately."""
    N, D = case.nmat, case.dim
    Qa, Qb, aa, ab = a["Q"], b["Q"], a["alpha"], b["alpha"]
    out = {}
    ra, rb = Qa[:, 0].sum(0), Qb[:, 0].sum(0)
    out["rho_l1"] = float(np.abs(ra - rb).sum() / np.abs(rb).sum())
    du = dun = dp = dpn = 0.0
    for m in range(N):
        on = (aa[m] > 0) & (ab[m] > 0) & (Qa[m, 0] > 0) & (Qb[m, 0] > 0)
        if not on.any():
            continue
        Ua, Ub = Qa[m][:, on] / aa[m, on], Qb[m][:, on] / ab[m, on]
        va, vb = Ua[1:1 + D] / Ua[0], Ub[1:1 + D] / Ub[0]
        g, pi = case.gamma[m], case.pinf[m]
        pa = (g - 1) * (Ua[D + 1] - 0.5 * Ua[0] * (va ** 2).sum(0)) - g * pi
        pb = (g - 1) * (Ub[D + 1] - 0.5 * Ub[0] * (vb ** 2).sum(0)) - g * pi
        w = ab[m, on]
        du += float((w * np.abs(va - vb).sum(0)).sum())
        dun += float((w * np.sqrt((vb ** 2).sum(0))).sum())
        dp += float((w * np.abs(pa - pb)).sum())
        dpn += float((w * np.abs(pb)).sum())
    out["u_l1"] = du / max(dun, 1e-300)
    out["p_l1"] = dp / max(dpn, 1e-300)
    out["alpha_l1"] = float(np.abs(aa - ab).sum() / np.abs(ab).sum())
    h = min((case.hi[d] - case.lo[d]) / case.n[d] for d in range(D))
    out["phi_max_over_h"] = float(np.abs(a["phi"] - b["phi"]).max() / h)
    out["chi_cells_differ"] = int((a["chi"] != b["chi"]).sum())
    return out


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        from paper_1704_00519_gb300 import build
        build.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_1704_00519_gb300.msf as msf
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    case = make_case(args.case if args.only else "sphere")
    cells, stages = case.cells, 3
    K, W = args.steps, max(3, args.warmup)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def timed(precision, k_steps):
        s = msf.Solver(case, precision=precision, stream=sptr, profile=1)
        s.step(W, case.t_end)
        flux_ms = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k_steps)]
        clocks = ClockSampler(local)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks.start()
        for k in range(k_steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            s.step(1, case.t_end, sync=False)
            ev[k][1].record(stream)
            flux_ms.append(s.flux_ms())   # synchronises after the step
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = clocks.stop()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        return s, step_ms, flux_ms, clk

    if args.only:
        s, ms, fl, _ = timed(msf.MSF_FP32_BULK if args.only == "fp32" else msf.MSF_FP64, K)
        if rank == 0:
            print(json.dumps({"only": args.only, "case": args.case, "ms_per_step": sum(ms) / K,
                              "flux_ms_per_step": sum(map(sum, fl)) / K}))
        return 0
    K64 = min(K, 20)
    s32, ms32, fl32, clk = timed(msf.MSF_FP32_BULK, K)
    s64, ms64, fl64, _ = timed(msf.MSF_FP64, K64)
    total32 = sum(ms32) / 1e3
    total64 = sum(ms64) / 1e3
    total32, total64 = max_over_ranks([total32, total64], dev)
    value = job_rate(cells * stages * K, world, total32)
    value64 = job_rate(cells * stages * K64, world, total64)

    # roofline of the dominant kernel (flux update), FP32-bulk form
    npairs = pairs_per_cell(s32)
    bytes_step = flux_bytes_per_step(case, npairs)
    flux_s = sum(sum(x) for x in fl32) / 1e3 / K
    achieved = bytes_step / flux_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = profiled_traffic("fp32_bulk")
    flux64_s = sum(sum(x) for x in fl64) / 1e3 / K64
    npairs64 = pairs_per_cell(s64)
    s32.close()
    s64.close()
    fma64 = msf.fma_peak(msf.MSF_FP64, sptr)
    fma32 = msf.fma_peak(msf.MSF_FP32_BULK, sptr)
    flops64 = npairs64 * 3 * flux_flops_per_pair_stage(case.dim)
    achieved64 = flops64 / flux64_s
    achieved32_flops = npairs * 3 * flux_flops_per_pair_stage(case.dim) / flux_s

    # every output of the FP32-bulk form against the plain FP64 path after the
    # same steps from the same start
    errs = {}
    pair = []
    for prec in (msf.MSF_FP32_BULK, msf.MSF_FP64):
        s = msf.Solver(case, precision=prec, stream=sptr)
        s.step(W + K64, case.t_end)
        pair.append((s.state(), s.totals()[0]))
        s.close()
    errs = output_errors(case, pair[0][0], pair[1][0])
    t32, t64 = pair[0][1], pair[1][1]
    errs["totals_max_rel"] = float(np.abs(t32 - t64).max() / np.abs(t64).sum())
    errs["steps"] = W + K64
    del pair

    # end to end through the public API with host buffers: initial data in,
    # K steps, final state out (wall clock)
    torch.cuda.synchronize()
    phi = np.ascontiguousarray(case.phi.ravel(), np.float64)
    chi = np.ascontiguousarray(case.chi.ravel(), np.int32)
    prim = np.ascontiguousarray(case.prim, np.float64)
    se = msf.Solver(case, precision=msf.MSF_FP32_BULK, stream=sptr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    se.set_levelset(phi, chi, prim)
    se.step(K, case.t_end)
    st = se.state()
    t1 = time.perf_counter()
    (e2e_s,) = max_over_ranks([t1 - t0], dev)
    e2e_val = job_rate(cells * stages * K, world, e2e_s)
    h2d = phi.nbytes + chi.nbytes + prim.nbytes
    d2h = st["Q"].nbytes + st["alpha"].nbytes + st["phi"].nbytes + st["chi"].nbytes
    launches = se.launches_per_step() * K
    se.close()
    del st

    batched = batched_rates(msf, torch, sptr, max(K, 10), 3)
    icf = icf_rates(msf, torch, sptr, 50)
    workloads = workload_rates(msf, torch, sptr, 10)
    later = later_window(msf, torch, sptr, flush, 10)
    adjoint = adjoint_rates(msf, torch, sptr, 4)
    adjoint["vs_fp64_forward"] = adjoint["value"] / value64
    adjoint["gradient_200_steps"] = adjoint_gradient(msf, torch, sptr, 200)
    if rank != 0:
        return 0

    # CPU oracle on a bounded sample of the same workload: one full step on
    # every host core (OpenMP build; the plain build gives the same bits)
    from oracle import oracle as orc
    orc.build(openmp=True)
    cpu_val, cpu_secs, cpu_steps, cpu_thr = oracle_rate(case, 1, 0, openmp=True)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * total32 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "cells": cells, "materials": case.nmat,
                   "precision": "fp32_bulk (FP32 fluxes, FP64 storage/geometry/correction/totals)",
                   "l2": "flushed between timed steps (256 MiB write outside the timed events); the state (1.1 GB) exceeds L2",
                   "parallelism": f"replicas{world}"},
        "fp64": {"value": value64, "unit": UNIT, "ms_per_step": 1e3 * total64 / K64, "steps": K64,
                 "flux_ms_per_step": 1e3 * flux64_s},
        "fp32_over_fp64": value / value64,
        "roofline_fp64": {"kernel": "k_flux_update<3,double>", "bound": "alu", "achieved": achieved64 / 1e12,
                          "peak": fma64 / 1e12, "unit": "TFLOP/s", "frac": achieved64 / fma64,
                          "peak_source": "measured here: msf_fma_peak FP64 (independent FMA chains on every SM)",
                          "flops_per_pair_stage": flux_flops_per_pair_stage(case.dim),
                          "flux_ms_per_step": 1e3 * flux64_s},
        "roofline_alu_fp32": {"kernel": "k_flux_update<3,float>", "bound": "alu",
                              "achieved": achieved32_flops / 1e12, "peak": fma32 / 1e12, "unit": "TFLOP/s",
                              "frac": achieved32_flops / fma32,
                              "peak_source": "measured here: msf_fma_peak FP32 (independent FMA chains on every SM)",
                              "flops_per_pair_stage": flux_flops_per_pair_stage(case.dim)},
        "fma_peak_tflops": {"fp64": fma64 / 1e12, "fp32": fma32 / 1e12},
        "fp32_error_vs_fp64": errs,
        "roofline": {"kernel": "k_flux_update<3,float>", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                     "algorithmic_bytes_per_step": bytes_step, "flux_ms_per_step": 1e3 * flux_s,
                     "flux_share_of_step": flux_s / (total32 / K)},
        "cpu_baseline": {"value": cpu_val, "unit": UNIT, "cores": cpu_thr, "kind": "oracle",
                         "sample": f"{cpu_steps} full TVD-RK3 step of {WORKLOAD['name']} from its initial state "
                                   f"({cpu_secs:.1f} s), OpenMP oracle on {cpu_thr} threads"},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
                "how": "wall clock: msf_set_levelset from host arrays, K steps, msf_get_state to host"},
        "gpu_launches": launches,
        "clocks": clk,
        "workloads": workloads,
        "triple_point_from_t_0.3": later,
        "batched_1d": batched,
        "icf_shell_study": icf,
        "adjoint": adjoint,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
