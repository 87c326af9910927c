"""Benchmark: batched FP64 cell-steps/s of the explicit-implicit splitting scheme on GB300.

Workload (one bench step = one whole run): 4096 independent liquid|vapour Riemann instances with
N uniform in [200, 2000] background cells, cut fractions alpha log-uniform in [1e-6, 1e-1] and kinetic
coefficients c log-uniform in [1e-4, 1e-2] (tau = c * tau_paper), all advanced to t_end = 2e-4 s
(every instance takes 0.6 N .. 0.7 N time steps). Synthetic seeded data (no dataset exists).
cell-steps = sum over instances of (cells at the end of the run x time steps taken).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own full batch (weak scaling, no collective on the data
path); value = cell-steps of all ranks / max-over-ranks time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "batched FP64 cell-steps/s (fwd, adjoint) vs plain GPU step at ≤1e-9 rel err; %HBM"
UNIT = "cell-steps/s"
# algorithmic FP64 flops of one explicit cell-step (a multiply and an add count separately, so a fused
# multiply-add counts two, a division one), in the smallest arrangement of the scheme's arithmetic: per cell u,
# p, the momentum flux m u + p, |u| + a and the max (7); per face the two Davis speeds (4), S_R - S_L (1), the
# weight w = S_R / (S_R - S_L) (1), the differences of rho and m (2), the HLL average of each component as
# F_r + w ((F_l - F_r) + S_L (U_r - U_l)) (4 for mass, 5 for momentum); the update of rho and m (6)
SWEEP_FLOP_PER_CELL = 30
FP64_PEAK_TFLOPS = 1.25   # GB300 dense FP64 (nominal; no FP64 figure in MEASURED_PEAKS.json)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture each; profiles/) of the kernels as
# committed, for the traffic entry of the roofline objects: the per-step sweep per lattice cell it updates (a
# launch with every instance active: 198.1 MB for 4.48 M cells), the resident group kernel per explicit
# cell-step of a whole run of this workload (dual time, 96 threads: 187.5 GB for 3.69e9; Newton, 256 threads:
# 173.6 GB). Scaled by the cells or cell-steps of the launch being reported.
SWEEP_TRAFFIC_BYTES_PER_CELL = 44.25
GROUP_TRAFFIC_BYTES_PER_CELL_STEP = {0: 50.85, 1: 47.06}
# FP64 issue of the same captures (sm__inst_executed_pipe_fp64.sum, sm__pipe_fp64_cycles_active): the sweep issues
# one warp instruction for the 30 cells of a tile; the group kernel's count is per explicit cell-step of the run
# (sweep warps and block solves together).
SWEEP_FP64_ISSUE = {"warp_instructions_per_30_cell_tile": 27.8, "fp64_pipe_busy_pct": 87.2}
GROUP_FP64_ISSUE = {0: {"warp_instructions_per_cell_step": 1.98, "fp64_pipe_busy_pct": 54.4},
                    1: {"warp_instructions_per_cell_step": 1.14, "fp64_pipe_busy_pct": 62.6}}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, ws: int, device) -> float:
    """Maximum of a per-rank value over all ranks (the timed region's slowest rank); x itself for one rank."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cell_steps_per_rank: float, steps: int, ws: int, t_max: float) -> float:
    """Whole-job throughput: the cell-steps every rank processed (one replica of the batch per GPU, weak
    scaling) over the slowest rank's time."""
    return cell_steps_per_rank * steps * ws / t_max


def workload(scale=1.0):
    from paper_2211_00705_gb300 import inputs as I
    return I.workload(1, scale=scale)


def cell_steps(stats, counts):
    return float(np.sum(stats["steps"].astype(np.float64) * counts.astype(np.float64)))


def measure_adjoint(dev, steps, warmup, scale=1.0, n_steps=2000, block_solver=0, checkpoint_every=None):
    """The adjoint on its workload (Riemann instances, N=500, 2000 steps): forward run (also a target run with
    tau x 1.1 for the misfit), then imexds_adjoint timed. Checkpoints every `checkpoint_every` steps (default:
    the whole run, i.e. one taped replay and one reverse sweep, its tape ~34 GB of HBM at full size; with 64,
    a replay writing checkpoints, a taped recompute of every segment but the last, and the reverse sweep).
    Cell-steps of the adjoint = initial cells x steps of every instance (replay, recompute and reverse sweep
    together count as one reverse cell-step). Returns the JSON object of the adjoint line."""
    import dataclasses
    import torch
    from paper_2211_00705_gb300 import inputs as I
    from paper_2211_00705_gb300.imexds import Imexds
    n = max(1, int(round(1024 * scale)))
    b = I.adjoint_batch(n_inst=n, n_steps=n_steps)
    if block_solver:
        b = with_block_solver(b, block_solver)
    prog_steps = b.n_steps
    tctx = Imexds.from_batch(dataclasses.replace(b, tau=b.tau * 1.1))
    tctx.step(prog_steps)
    ts = tctx.get_states()
    tctx.close()
    rs_t, _ = I.sample_density(ts, ts["offsets"], b.n_lattice, b.x_left, b.x_right)
    ctx = Imexds.from_batch(b)
    k = int(checkpoint_every or prog_steps)
    ctx.set_adjoint_checkpoint(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.step(prog_steps)
    e1.record()
    torch.cuda.synchronize()
    fwd_s = e0.elapsed_time(e1) / 1e3
    s = ctx.get_states()
    rs, idx = I.sample_density(s, s["offsets"], b.n_lattice, b.x_left, b.x_right)
    h = np.repeat((b.x_right - b.x_left) / b.n_lattice, b.n_lattice)
    g_rho = np.zeros(int(s["offsets"][-1]))
    np.add.at(g_rho, idx, h * (rs - rs_t))
    g_m = np.zeros_like(g_rho)
    free0 = torch.cuda.mem_get_info(dev)[0]
    for _ in range(max(1, warmup)):
        g = ctx.adjoint(g_rho, g_m)
    adj_bytes = max(0, free0 - torch.cuda.mem_get_info(dev)[0])
    kern, wall = [], []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = ctx.adjoint(g_rho, g_m)
        wall.append(time.perf_counter() - t0)
        kern.append(ctx.adjoint_info()["kernel_ms"] / 1e3)
    info = ctx.adjoint_info()
    st = ctx.stats()
    fwd_cs = float(np.sum(st["steps"] * np.diff(b.cell_offsets)))
    ctx.close()
    cs = float(info["cell_steps"])
    return {"value": cs / float(np.mean(kern)), "unit": UNIT, "workload": b.name, "checkpoint_every": k,
            "adjoint_device_gb": round(adj_bytes / 1e9, 2),
            "seconds_per_call": float(np.mean(kern)), "calls": steps,
            "e2e": {"value": cs / float(np.mean(wall)), "unit": UNIT,
                    "note": "imexds_adjoint call with host seed/gradient arrays, layout and copies included"},
            "replay_err": info["replay_err"], "instances_without_gradient": int(np.count_nonzero(g["status"])),
            "forward_value": fwd_cs / fwd_s, "forward_note": "imexds_step over the same workload (tight tolerances)",
            "block_solver": "newton" if block_solver else "dual time stepping (Alg. 2)",
            "dts_iters_per_step": float(st["dts_iters"].sum() / max(1, st["steps"].sum()))}


def measure_cavitation(dev, scale=1.0, n_steps=5000, adj_inst=1024, fd_inst=4):
    """The phase-creation workload (16384 cavitation instances, N in [64, 4096], 5000 steps): the forward run at
    full size with dual time stepping and with Newton's method on the blocks (autotuned schedule, one timed run
    each after a 64-step warm-up), then dJ/dV of the mean final pressure (V enters the initial momentum) by the
    adjoint on the first adj_inst instances (Newton forward run and replay), with central differences of the
    forward run on fd_inst of them. Returns the JSON object of the cavitation line."""
    import dataclasses
    import torch
    from paper_2211_00705_gb300 import autotune
    from paper_2211_00705_gb300 import inputs as I
    from paper_2211_00705_gb300.imexds import Imexds
    b = I.workload(4, scale=scale)
    b.n_steps = n_steps
    out = {"workload": b.name, "instances": b.n_inst, "cells": int(b.rho.shape[0]), "steps": n_steps}
    for solver in (0, 1):
        bb = with_block_solver(b, solver)
        tuned = autotune.tune(bb, steps=64)
        ctx = Imexds.from_batch(bb, schedule=tuned["schedule"], group_threads=tuned.get("group_threads", 0),
                                group_cells=tuned.get("group_cells", 0))
        ctx.step(64)
        ctx.reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.step(n_steps)
        e1.record()
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        st = ctx.stats()
        cs = float(np.sum(st["steps"] * ctx.cell_counts()))
        status = ctx.get_states()["status"]
        ctx.close()
        out["newton" if solver else "dual_time"] = {
            "value": cs / secs, "unit": UNIT, "seconds": secs, "cell_steps": cs,
            "schedule": {k: tuned[k] for k in ("schedule", "group_threads", "group_cells") if k in tuned},
            "block_iters_per_step": float(st["dts_iters"].sum() / max(1, st["steps"].sum())),
            "creations_per_instance": float(st["creations"].mean()),
            "instance_status_nonzero": int(np.count_nonzero(status))}
    # dJ/dV by the adjoint on a sample, Newton forward run, block tolerances x 1e-4 (the adjoint differentiates
    # the converged block systems; near the production tolerance a stop decision taken one iteration apart moves
    # a state by up to the tolerance, which central differences would see)
    sb = with_block_solver(b.subset(list(range(min(adj_inst, b.n_inst)))), 1)
    sb = dataclasses.replace(sb, options=dataclasses.replace(sb.options, tol_nb=sb.options.tol_nb * 1e-4,
                                                             tol_k=sb.options.tol_k * 1e-4))
    sb.n_steps = n_steps

    def mean_pressure(st, bb):
        f = bb.fluid
        off = st["offsets"]
        J = np.zeros(bb.n_inst)
        gr = np.zeros(int(off[-1]))
        gw = np.zeros(int(off[-1]))
        for i in range(bb.n_inst):
            sl = slice(off[i], off[i + 1])
            ph, r, w = st["phase"][sl], st["rho"][sl], st["widths"][sl]
            a2 = np.where(ph == 0, f.a2_vap, f.a2_liq)
            p = np.where(ph == 0, f.a2_vap * r, f.p_sat + f.a2_liq * (r - f.rho0_liq))
            W = w.sum()
            J[i] = float((w * p).sum() / W)
            gr[sl] = w * a2 / W
            gw[sl] = (p - J[i]) / W
        return J, gr, gw

    ctx = Imexds.from_batch(sb)
    ctx.set_adjoint_checkpoint(64)
    ctx.step(n_steps)
    s = ctx.get_states()
    J, gr, gw = mean_pressure(s, sb)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = ctx.adjoint(gr, np.zeros_like(gr), gw)
    wall = time.perf_counter() - t0
    info = ctx.adjoint_info()
    ctx.close()
    V = np.array([abs(sb.m[sb.cell_offsets[i]] / sb.rho[sb.cell_offsets[i]]) for i in range(sb.n_inst)])
    dmdV = np.sign(sb.m / sb.rho) * sb.rho
    off0 = sb.cell_offsets
    adj = np.array([np.dot(g["m"][off0[i]:off0[i + 1]], dmdV[off0[i]:off0[i + 1]]) for i in range(sb.n_inst)])
    fb = sb.subset(list(range(min(fd_inst, sb.n_inst))))
    fb.n_steps = n_steps
    eps = 1e-6
    vals = []
    Vf = V[:fb.n_inst]
    for sgn in (1.0, -1.0):
        bb = dataclasses.replace(fb, m=fb.m + sgn * eps * np.repeat(Vf, np.diff(fb.cell_offsets))
                                 * (np.sign(fb.m / fb.rho) * fb.rho))
        c = Imexds.from_batch(bb)
        c.step(n_steps)
        vals.append(mean_pressure(c.get_states(), bb)[0])
        c.close()
    fd = (vals[0] - vals[1]) / (2 * eps * Vf)
    out["adjoint"] = {"value": info["cell_steps"] / (info["kernel_ms"] / 1e3), "unit": UNIT,
                      "instances": sb.n_inst, "seconds": info["kernel_ms"] / 1e3, "wall_seconds": wall,
                      "replay_err": info["replay_err"], "instances_without_gradient": int(np.count_nonzero(g["status"])),
                      "dJ_dV_sample": adj[:fb.n_inst].tolist(), "fd_sample": fd.tolist(),
                      "fd_rel_err_max": float(np.max(np.abs(adj[:fb.n_inst] - fd) / np.abs(adj[:fb.n_inst]))),
                      "note": "Newton forward run and replay; checkpoints every 64 steps; central differences of "
                              "the forward run at step 1e-6 V on the first instances"}
    return out


def measure_large_domain_sweep(n_steps=100, full_steps=1000):
    """The large single domain (2^24 cells, 1024 vapour bubbles, 2048 boundaries), per-step schedule. (1) The
    explicit sweep: n_steps steps with CUDA events around every kernel; its algorithmic traffic is 32 B per
    lattice cell (rho, m read and written) against the measured HBM copy bandwidth (state arrays 2 x 268 MB,
    far above L2, so every launch streams from HBM). (2) The workload's configured 1000 steps timed whole, with
    dual time stepping and with Newton's method on the blocks (cell-steps per second)."""
    import torch
    from paper_2211_00705_gb300 import inputs as I
    from paper_2211_00705_gb300.imexds import Imexds
    b = I.workload(2)
    ctx = Imexds.from_batch(b, schedule=1)
    ctx.step(8)                                  # warm-up: graph build, first steps
    ctx.set_kernel_timing(True)
    ctx.step(n_steps)
    kt = ctx.kernel_times()
    ctx.set_kernel_timing(False)
    st = ctx.get_states()
    ctx.close()
    ms, n = kt["k_sweep"]
    per = ms / 1e3 / max(n, 1)
    cells = int(b.n_lattice[0])
    gbs = 32.0 * cells / per / 1e9
    peak = load_peak("hbm_gbs")
    tot = sum(v[0] for v in kt.values())
    out = {"workload": b.name, "steps_timed": n_steps, "k_sweep_ms_per_launch": per * 1e3,
           "algorithmic_bytes_per_launch": 32.0 * cells, "achieved_gbs": gbs, "peak_gbs": peak,
           "frac": (gbs / peak) if peak else None, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
           "cell_steps_per_s_sweep": cells / per, "status": int(st["status"][0]),
           "per_step_share": {k: round(v[0] / tot, 4) if tot else None for k, v in kt.items()}}
    for solver in (0, 1):
        bb = with_block_solver(b, solver)
        ctx = Imexds.from_batch(bb, schedule=1)
        ctx.step(8)
        ctx.reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.step(full_steps)
        e1.record()
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        stt = ctx.stats()
        cs = float(np.sum(stt["steps"] * ctx.cell_counts()))
        out["newton" if solver else "dual_time"] = {
            "steps": full_steps, "seconds": secs, "ms_per_step": 1e3 * secs / full_steps, "value": cs / secs,
            "unit": UNIT, "block_iters_per_step_per_block": float(stt["dts_iters"].sum() / max(1, stt["steps"].sum()) / 2048),
            "status": int(ctx.get_states()["status"][0])}
        ctx.close()
    return out


def measure_plain(batch, n_sample=16):
    """The plain single-instance GPU step: the same kernels, one instance per context, per-step schedule
    (one launch per kernel and step), on a sample of the workload's instances run one after another."""
    import torch
    from paper_2211_00705_gb300.imexds import Imexds
    idx = np.linspace(0, batch.n_inst - 1, n_sample).astype(int)
    sub = batch.subset(list(idx))
    cs, secs = 0.0, 0.0
    for i in range(sub.n_inst):
        one = sub.subset([i])
        ctx = Imexds.from_batch(one, schedule=1)
        ctx.run_to(one.t_end)   # warm-up (graph build)
        ctx.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.run_to(one.t_end)
        torch.cuda.synchronize()
        secs += time.perf_counter() - t0
        cs += cell_steps(ctx.stats(), ctx.cell_counts())
        ctx.close()
    return {"value": cs / secs, "unit": UNIT, "sample": f"{sub.n_inst} of {batch.n_inst} instances, one context each, "
            "per-step schedule, run one after another", "seconds": secs}


def oracle_rate(batch, n_steps=None, max_inst=None, threads=None):
    """Oracle cell-steps/s on a bounded sample of a batch (all host cores over instances)."""
    from oracle import pyoracle as P
    cores = threads or os.cpu_count() or 1
    b = batch if max_inst is None or batch.n_inst <= max_inst else batch.subset(
        list(np.linspace(0, batch.n_inst - 1, max_inst).astype(int)))
    o = P.Oracle(b)
    t0 = time.perf_counter()
    if n_steps is None and b.t_end > 0:
        o.run_to(b.t_end, cores)
    else:
        o.step(n_steps or b.n_steps, cores)
    secs = time.perf_counter() - t0
    st = o.stats()
    cs = float(np.sum(st["steps"] * np.diff(b.cell_offsets)))
    return cs / secs, cores, f"{b.n_inst} of {batch.n_inst} instances, {int(st['steps'].max())} steps, {secs:.1f} s"


def gpu_rate(batch, n_steps=None, **kw):
    """Batched GPU cell-steps/s of one run (after a warm-up run) and the run's statistics."""
    import torch
    from paper_2211_00705_gb300.imexds import Imexds
    ctx = Imexds.from_batch(batch, **kw)
    run = (lambda: ctx.run_to(batch.t_end)) if (n_steps is None and batch.t_end > 0) else \
        (lambda: ctx.step(n_steps or batch.n_steps))
    run()
    ctx.reset()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run()
    e1.record()
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    st = ctx.stats()
    cs = float(np.sum(st["steps"] * np.diff(batch.cell_offsets)))
    ctx.close()
    return cs / secs, st


def table(args):
    """One row per workload: GPU batched, the plain single-instance GPU step, the oracle on the host cores
    (bounded samples, stated), printed as one JSON object."""
    from paper_2211_00705_gb300 import inputs as I
    rows = {}
    b0 = I.workload(0)
    g0, _ = gpu_rate(b0)
    o0 = oracle_rate(b0)
    rows["0"] = {"workload": b0.name, "gpu_batched": g0, "gpu_plain": g0, "oracle": o0[0], "cores": o0[1],
                 "oracle_sample": o0[2]}
    print(json.dumps({"0": rows["0"]}), flush=True)
    b1 = I.workload(1)
    g1, _ = gpu_rate(b1)
    p1 = measure_plain(b1)
    o1 = oracle_rate(b1, max_inst=512)
    rows["1"] = {"workload": b1.name, "gpu_batched": g1, "gpu_plain": p1["value"], "oracle": o1[0],
                 "cores": o1[1], "oracle_sample": o1[2]}
    print(json.dumps({"1": rows["1"]}), flush=True)
    b2 = I.workload(2)
    g2, _ = gpu_rate(b2, n_steps=100, schedule=1)
    # the oracle copies the cell list inside its dual-time loop (plain, O(cells) per iteration): it is timed
    # on a 2^16-cell domain with the same bubble density
    b2s = I.bubbles_domain(2, n_cells=1 << 16, n_bubbles=4, n_steps=20)
    o2 = oracle_rate(b2s, n_steps=20)
    rows["2"] = {"workload": b2.name, "gpu_batched": g2, "gpu_note": "100 steps (per-step schedule)",
                 "oracle": o2[0], "cores": o2[1], "oracle_sample": "2^16-cell domain, 4 bubbles: " + o2[2]}
    print(json.dumps({"2": rows["2"]}), flush=True)
    b3 = I.adjoint_batch()
    g3, _ = gpu_rate(b3)
    o3 = oracle_rate(b3, max_inst=64)
    rows["3"] = {"workload": b3.name, "gpu_batched": g3, "oracle": o3[0], "cores": o3[1], "oracle_sample": o3[2]}
    print(json.dumps({"3": rows["3"]}), flush=True)
    b4 = I.workload(4, scale=1024 / 16384)
    g4, _ = gpu_rate(b4)
    o4 = oracle_rate(b4, max_inst=64, n_steps=500)
    rows["4"] = {"workload": b4.name, "gpu_batched": g4, "gpu_note": "1024 of the 16384 instances, 5000 steps",
                 "oracle": o4[0], "cores": o4[1], "oracle_sample": o4[2]}
    import platform
    rows["host"] = {"machine": platform.machine(), "cores": os.cpu_count(), "python": platform.python_version()}
    print(json.dumps(rows))
    return 0


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

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
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(batch, target_s=15.0):
    """The oracle on the host cores on a bounded sample of the workload: instances taken in a fixed
    stride until their estimated work (0.62 N^2 cell-steps each) fills about target_s seconds."""
    from oracle import pyoracle as P
    cores = os.cpu_count() or 1
    # calibrate on one mid-size instance
    order = np.argsort(batch.n_lattice)
    probe = batch.subset([order[len(order) // 2]])
    o = P.Oracle(probe)
    t0 = time.perf_counter()
    o.run_to(probe.t_end, 1)
    dt1 = time.perf_counter() - t0
    st = o.stats()
    rate1 = cell_steps(st, np.array([len(o.states()["rho"])])) / max(dt1, 1e-9)
    budget = target_s * rate1 * cores
    est = 0.62 * batch.n_lattice.astype(np.float64) ** 2
    stride = max(1, int(round(len(est) * 1.0 / max(1.0, budget / est.mean()))))
    idx = np.arange(0, batch.n_inst, stride)
    sample = batch.subset(idx)
    o = P.Oracle(sample)
    t0 = time.perf_counter()
    o.run_to(sample.t_end, cores)
    wall = time.perf_counter() - t0
    s = o.states()
    counts = np.diff(s["offsets"])
    cs = cell_steps(o.stats(), counts)
    return {"value": cs / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(idx)} of {batch.n_inst} instances (every {stride}th), run to t_end on {cores} "
                      f"threads: {cs:.3e} cell-steps in {wall:.1f} s"}


def run_reference(args, ws, rank):
    """The oracle as the reference arm: each step is a bounded sample of the workload on host cores."""
    if rank != 0:
        return 0
    batch = workload()
    from oracle import pyoracle as P
    cores = os.cpu_count() or 1
    idx = np.arange(0, batch.n_inst, 64)
    sample = batch.subset(idx)
    times, css = [], []
    for k in range(args.warmup + args.steps):
        o = P.Oracle(sample)
        t0 = time.perf_counter()
        o.run_to(sample.t_end, cores)
        wall = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(wall)
            css.append(cell_steps(o.stats(), np.diff(o.states()["offsets"])))
    value = sum(css) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": batch.name, "sample": f"{len(idx)} of {batch.n_inst} instances per step",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(idx)} of {batch.n_inst} instances (every 64th) per step, {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def with_block_solver(batch, block_solver):
    import dataclasses
    return dataclasses.replace(batch, options=dataclasses.replace(batch.options, block_solver=block_solver))


def load_peak(key):
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key]
    except (OSError, ValueError, KeyError):
        return None


def measure_run(batch, steps, warmup, schedule, flush, barrier, sampler=None, ws=1, dev=None, group_threads=0,
                group_cells=0):
    """The headline measurement of one batch: the autotuned schedule (schedule 0) or the given one, warm-up runs,
    then `steps` whole runs to t_end timed with CUDA events (L2 flushed between them, outside the events), max
    over ranks. With a group schedule the library's own events around the resident kernel (on its stream) run
    inside the same timed region and give that kernel's duration and its per-phase SM cycles; otherwise one
    extra instrumented run gives the per-kernel durations. Returns the context (still open) and the figures."""
    import torch
    from paper_2211_00705_gb300.imexds import Imexds
    tuned = None
    if schedule == 0:
        from paper_2211_00705_gb300 import autotune
        tuned = autotune.tune(batch, steps=64)
        ctx = Imexds.from_batch(batch, schedule=tuned["schedule"], group_threads=tuned.get("group_threads", 0),
                                group_cells=tuned.get("group_cells", 0))
        schedule_used = tuned["schedule"]
    else:
        ctx = Imexds.from_batch(batch, schedule=schedule, group_threads=group_threads, group_cells=group_cells)
        schedule_used = schedule
    group = schedule_used in (2, 3)
    if group:
        ctx.set_kernel_timing(True)   # events around the resident kernel; the launch itself is unchanged
    for _ in range(max(warmup, 3)):
        ctx.reset()
        ctx.run_to(batch.t_end)
    torch.cuda.synchronize()
    counts = ctx.cell_counts()
    st = ctx.stats()
    cs_run = cell_steps(st, counts)
    status = ctx.get_states()["status"]
    if group:
        ctx.set_kernel_timing(True)   # zero the durations and phase counters of the warm-up runs
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    launches = 0
    barrier()
    if sampler:
        sampler.start()
    for k in range(steps):
        flush.fill_(float(k))
        ctx.reset()
        barrier()
        ev0[k].record()
        ctx.run_to(batch.t_end)
        ev1[k].record()
        barrier()
        launches += int(ctx.stats()["launches"][0])
    clocks = sampler.stop() if sampler else None
    ms = sum(e0.elapsed_time(e1) for e0, e1 in zip(ev0, ev1))
    t_max = reduce_max(ms / 1e3, ws, dev)
    if group:
        kt = ctx.kernel_times()
        phase = ctx.group_phase_cycles()
        ctx.set_kernel_timing(False)
    else:
        phase = None
        ctx.set_kernel_timing(True)
        ctx.reset()
        ctx.run_to(batch.t_end)
        kt = ctx.kernel_times()
        ctx.set_kernel_timing(False)
    dominant = max(kt, key=lambda k: kt[k][0])
    kms, kn = kt[dominant]
    per_launch_s = kms / 1e3 / max(kn, 1)
    launches_per_run = kn / (steps if group else 1)
    # algorithmic work per launch of the dominant kernel: 30 FP64 flops and 32 bytes per explicit cell-step
    cs_launch = cs_run / max(launches_per_run, 1)
    ach = SWEEP_FLOP_PER_CELL * cs_launch / per_launch_s / 1e12 if per_launch_s > 0 else None
    hbm_peak = load_peak("hbm_gbs")
    gbs = 32.0 * cs_launch / per_launch_s / 1e9 if per_launch_s > 0 else None
    roof = {"bound": "alu", "kernel": dominant, "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": (ach / FP64_PEAK_TFLOPS) if ach else None,
            "traffic": (GROUP_TRAFFIC_BYTES_PER_CELL_STEP[batch.options.block_solver] * cs_launch
                        if dominant == "k_group" else None),
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one full launch (profiles/"
                              "k_group_riemann4096.md), per explicit cell-step, times this launch's cell-steps",
            "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (recipe table; no FP64 entry in MEASURED_PEAKS.json)",
            "ms_per_launch": per_launch_s * 1e3, "launches_per_run": launches_per_run,
            "algorithmic_flops_per_launch": SWEEP_FLOP_PER_CELL * cs_launch,
            "algorithmic_bytes_per_launch": 32.0 * cs_launch,
            "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": (gbs / hbm_peak) if (gbs and hbm_peak) else None,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
            "timed_in": "the timed region (library events around the resident kernel)" if group else
                        "one instrumented run after the timed region",
            "phase_cycles": phase}
    if dominant == "k_group":
        roof["fp64_issue"] = dict(GROUP_FP64_ISSUE[batch.options.block_solver],
                                  source="ncu, one full launch (profiles/k_group_riemann4096.md)")
    return {"ctx": ctx, "tuned": tuned, "stats": st, "value": job_value(cs_run, steps, ws, t_max),
            "ms_per_step": 1e3 * t_max / steps, "cell_steps_run": cs_run, "launches": launches, "clocks": clocks,
            "block_iters_per_step": float(st["dts_iters"].sum() / max(1, st["steps"].sum())),
            "pb_newton_per_step": float(st["newton"].sum() / max(1, st["steps"].sum())),
            "status_nonzero": int(np.count_nonzero(status)), "roofline": roof}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", type=int, default=0, help="0 autotuned, 1 per-step kernels, 2 instance groups in lockstep, "
                                                            "3 instance groups advancing independently")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="fraction of the 4096 instances (smaller cases for profiling only)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    ap.add_argument("--no-plain", action="store_true", help="skip the single-instance comparison")
    ap.add_argument("--no-hbm", action="store_true", help="skip the large-domain sweep (HBM) measurement")
    ap.add_argument("--no-newton", action="store_true", help="skip the Newton block-solver leg")
    ap.add_argument("--only", choices=["adjoint", "hbm", "cavitation"], default=None,
                    help="run one auxiliary measurement alone and print its JSON (profiling)")
    ap.add_argument("--adjoint-steps", type=int, default=2000, help="steps of the adjoint workload")
    ap.add_argument("--adjoint-checkpoint", type=int, default=0,
                    help="checkpoint interval of the adjoint (0: the whole run taped at once)")
    ap.add_argument("--adjoint-solver", type=int, default=0, choices=[0, 1],
                    help="block solver of the --only adjoint run: 0 dual time stepping, 1 Newton")
    ap.add_argument("--table", action="store_true", help="per-workload rates (GPU, plain GPU, oracle) as JSON")
    ap.add_argument("--group-threads", type=int, default=0,
                    help="CTA width of the group schedules when --schedule is 2 or 3 (0: the library's default)")
    ap.add_argument("--group-cells", type=int, default=0,
                    help="lattice cells per instance group when --schedule is 2 or 3 (0: the library's default)")
    ap.add_argument("--block-solver", type=int, default=0, choices=[0, 1],
                    help="solver of the implicit blocks for the headline run: 0 dual time stepping (Alg. 2), 1 Newton")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import torch.distributed as dist
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2211_00705_gb300.imexds import Imexds
    if args.table:
        return table(args)
    if args.only == "adjoint":
        print(json.dumps(measure_adjoint(dev, args.steps, args.warmup, scale=args.scale, n_steps=args.adjoint_steps,
                                         block_solver=args.adjoint_solver,
                                         checkpoint_every=args.adjoint_checkpoint or None)))
        return 0
    if args.only == "hbm":
        print(json.dumps(measure_large_domain_sweep()))
        return 0
    if args.only == "cavitation":
        print(json.dumps(measure_cavitation(dev, scale=args.scale)))
        return 0

    batch = workload(args.scale)
    if args.block_solver:
        batch = with_block_solver(batch, args.block_solver)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(dev.index) if rank == 0 else None
    head = measure_run(batch, args.steps, args.warmup, args.schedule, flush, barrier, sampler=sampler, ws=ws, dev=dev,
                       group_threads=args.group_threads, group_cells=args.group_cells)
    ctx, tuned, st = head["ctx"], head["tuned"], head["stats"]
    value = head["value"]

    # per-kernel durations of the per-step kernel schedule (one instrumented run), which separates the sweep
    # from the block solves
    kt_steps = {}
    try:
        ctx.set_schedule(1)
        ctx.set_kernel_timing(True)
        ctx.reset()
        ctx.run_to(batch.t_end)
        kt_steps = ctx.kernel_times()
        ctx.set_kernel_timing(False)
        ctx.set_schedule(tuned["schedule"] if tuned else args.schedule)
    except Exception as e:  # keep the measured line even if the instrumented pass fails
        print(f"kernel timing failed: {e}", file=sys.stderr)
        kt_steps = {k: (0.0, 0) for k in Imexds.KERNELS}
    tot = sum(v[0] for v in kt_steps.values())

    # end to end through the public API with host buffers: upload, run, download every step
    h2d = int(batch.widths.nbytes + batch.rho.nbytes + batch.m.nbytes + batch.phase.nbytes
              + batch.cell_offsets.nbytes)
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    d2h = 0
    barrier()
    for k in range(args.steps):
        flush.fill_(float(k))
        barrier()
        e0[k].record()
        ctx.set_states(batch.cell_offsets, batch.widths, batch.rho, batch.m, batch.phase)
        ctx.run_to(batch.t_end)
        out = ctx.get_states()
        e1[k].record()
        barrier()
        d2h = int(out["widths"].nbytes + out["rho"].nbytes + out["m"].nbytes + out["phase"].nbytes
                  + out["offsets"].nbytes + out["t"].nbytes + out["status"].nbytes)
    e2e_s = reduce_max(sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / 1e3, ws, dev)
    e2e = {"value": job_value(head["cell_steps_run"], args.steps, ws, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # roofline of the timed kernel (the resident group kernel, or the sweep of the per-step schedule)
    roof = head["roofline"]
    # the explicit sweep alone (FP64 ALU bound), in the per-step schedule: algorithmic flops of the cells it
    # updated over its measured time
    sweep_cells = float(np.sum(st["steps"] * batch.n_lattice))   # lattice cells swept per run (upper bound)
    n_sw = max(kt_steps["k_sweep"][1], 1)
    per_launch_s = kt_steps["k_sweep"][0] / 1e3 / n_sw
    sw_ach = SWEEP_FLOP_PER_CELL * sweep_cells / n_sw / per_launch_s / 1e12 if per_launch_s > 0 else None
    roof["sweep_per_step_schedule"] = {
        "kernel": "k_sweep", "bound": "alu", "achieved": sw_ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": (sw_ach / FP64_PEAK_TFLOPS) if sw_ach else None,
        "traffic": SWEEP_TRAFFIC_BYTES_PER_CELL * sweep_cells / n_sw,
        "traffic_source": "ncu DRAM bytes of one launch with every instance active (profiles/k_sweep_riemann4096.md) "
                          "per lattice cell, times this run's average cells per launch",
        "algorithmic_bytes": 32.0 * sweep_cells / n_sw, "ms_per_launch": per_launch_s * 1e3,
        "fp64_issue": dict(SWEEP_FP64_ISSUE, source="ncu, one launch at step 101 (profiles/k_sweep_riemann4096.md)"),
        "share": {k: round(v[0] / tot, 4) if tot else None for k, v in kt_steps.items()},
        "ms_per_launch_by_kernel": {k: (v[0] / v[1] if v[1] else None) for k, v in kt_steps.items()}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
                "config": {"workload": batch.name, "instances": batch.n_inst, "cells": int(batch.rho.shape[0]),
                           "block_solver": "newton" if args.block_solver else "dual time stepping (Alg. 2)",
                           "schedule": tuned if tuned else {"schedule": args.schedule},
                           "cell_steps_per_step": head["cell_steps_run"],
                           "l2": "flushed (256 MB write) between timed runs",
                           "dts_iters_per_step": head["block_iters_per_step"],
                           "newton_iters_per_step": head["pb_newton_per_step"],
                           "instance_status_nonzero": head["status_nonzero"]},
                "roofline": roof, "e2e": e2e, "gpu_launches": head["launches"], "clocks": head["clocks"]}
        if not args.block_solver and not args.no_newton:
            # the same workload with Newton's method on every implicit block (the paper's outlook, Sec. 5)
            nb = with_block_solver(batch, 1)
            nw = measure_run(nb, args.steps, args.warmup, args.schedule, flush, barrier, sampler=None, ws=ws, dev=dev)
            nw["ctx"].close()
            line["newton"] = {"value": nw["value"], "unit": UNIT, "ms_per_step": nw["ms_per_step"],
                              "over_dual_time": nw["value"] / value,
                              "schedule": nw["tuned"] if nw["tuned"] else {"schedule": args.schedule},
                              "newton_steps_per_step": nw["block_iters_per_step"],
                              "pb_newton_iters_per_step": nw["pb_newton_per_step"],
                              "instance_status_nonzero": nw["status_nonzero"], "roofline": nw["roofline"],
                              "note": "options.block_solver = 1: Newton on each implicit block's system with the "
                                      "Sec. 4 stop test; parity against the oracle's Newton option"}
        if not args.no_plain:
            plain = measure_plain(batch)
            plain["batched_over_plain"] = value / plain["value"]
            line["plain_single_instance"] = plain
        if not args.no_adjoint:
            # at most two timed calls (~13 s each at full size): the adjoint is reported beside the headline
            line["adjoint"] = measure_adjoint(dev, max(1, min(2, args.steps // 2)), 1, scale=args.scale,
                                              n_steps=args.adjoint_steps,
                                              checkpoint_every=args.adjoint_checkpoint or None)
            # the same adjoint of a Newton run (forward and replay with Newton on the blocks; the reverse step
            # differentiates the converged block systems either way)
            line["adjoint"]["newton"] = measure_adjoint(dev, 1, 1, scale=args.scale, n_steps=args.adjoint_steps,
                                                        block_solver=1,
                                                        checkpoint_every=args.adjoint_checkpoint or None)
        if not args.no_hbm:
            line["large_domain_sweep"] = measure_large_domain_sweep()
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(batch)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
