"""Throughput of the five-equation RHS / SSP-RK3 step on GB300.

Headline workload: the 256^3 two-fluid water/air shock-bubble in FP64 (a step =
one CFL reduction + three RHS evaluations + three RK stage updates).  The metric
is the grind time t_RHS / (cells * equations) in ns/(cell*eqn*RHS) (lower is
better), with cell-updates/s beside it.  The other forms (mixed precision,
learned weights, WENO3, Kapila, stretched grid, characteristic boundaries,
six-equation model) are timed on the same workload under "forms", and every
form on the configuration it is defined on (the 384^3 bubble cloud in FP64,
mixed and learned; the 512^3 three-fluid workload in FP64 and mixed) under
"configs".  Every timed run starts from the initial state developed by
--develop steps (so shock and interfaces are present), then --warmup untimed
steps, then the timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU FP64 oracle (plain C, OpenMP over the host
cores) on a bounded slab of the same workload.  With torchrun (N > 1) every rank
runs an independent replica (the path needs no exchange on one GPU); the
reference arm runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "grind time ns/(cell·eqn·RHS) & cell-updates/s, FP64 vs mixed vs learned"
UNIT = "ns/(cell*eqn*RHS)"
CFL = 0.3

# Algorithmic floating-point work of one directional sweep per cell (3D), as
# the oracle's plain formulation spends it: + - * / and sqrt one each, counted
# by the oracle's counting build (oracle.rhs_flop_breakdown; recounted by
# tests/test_oracle_flops.py): WENO edges of every variable on both sides of a
# face plus HLLC per face, the flux difference and volume-fraction source per
# cell, primitive recovery once per cell (a third per sweep).  Keyed by
# (reconstruction or model, fluids).
ORACLE_FLOP_PER_CELL_SWEEP = {
    ("weno5", 2): 3860 / 3, ("weno5", 3): 4941 / 3, ("weno3", 2): 1970 / 3, ("weno3", 3): 2511 / 3,
    ("kapila", 2): 4016 / 3, ("kapila", 3): 5151 / 3,
}
# SSP-RK3 update per conserved variable, by its definition: stage 1
# q + dt R (2), stages 2 and 3 a q + b (q_s + dt R) (5): 4 per stage on average.
RK_FLOP_PER_VAR_STAGE = 4.0
# Forms the bench can time on the 256^3 shock-bubble: name -> (precision, extra
# solver parameters, workload variant, work variant for the FLOP count).
FORMS = {
    "fp64": ("fp64", {}, "uniform", "weno5"),
    "mixed": ("mixed", {}, "uniform", "weno5"),
    "learned": ("learned", {}, "uniform", "weno5"),
    "fp64_weno3": ("fp64", {"weno_order": 3}, "uniform", "weno3"),
    "mixed_weno3": ("mixed", {"weno_order": 3}, "uniform", "weno3"),
    "fp64_kapila": ("fp64", {"model": 1}, "uniform", "kapila"),
    "fp64_stretched": ("fp64", {}, "stretched", "weno5"),
    "mixed_stretched": ("mixed", {}, "stretched", "weno5"),
    "fp64_cbc": ("fp64", {}, "cbc", "weno5"),
    "fp64_six": ("fp64", {"model": 2}, "six", "weno5"),
    "mixed_six": ("mixed", {"model": 2}, "six", "weno5"),
}
# Every form on the configuration it is defined on: name -> (workload, precision).
CONFIG_RUNS = {
    "bubble_cloud_384_fp64": ("bubble_cloud", "fp64"),
    "bubble_cloud_384_mixed": ("bubble_cloud", "mixed"),
    "bubble_cloud_384_learned": ("bubble_cloud", "learned"),
    "three_fluid_512_fp64": ("three_fluid", "fp64"),
    "three_fluid_512_mixed": ("three_fluid", "mixed"),
}
# Issue-slot peak: 152 SMs x 4 schedulers x one warp instruction per clock.
SCHEDULERS = 152 * 4
# Warp instructions per cell of the FP64 WENO5 sweeps (x, y, z; 3D, two
# fluids, smsp__inst_executed.sum / cells of one ncu capture).  Re-measured
# whenever the FP64 sweeps change: NCU_FP64_SWEEPS says which capture.
FP64_SWEEP_WARP_INST_PER_CELL = (173.4, 176.9, 187.1)
# From the same capture: FP64-pipe and FP32 (fma) pipe activity of the sweeps
# (mean over x, y, z) and DRAM bytes per cell per launch (the z sweep of an RK
# stage also writes the next stage's primitives).
FP64_SWEEP_PIPE_FP64 = 0.404
FP64_SWEEP_PIPE_FMA = 0.588
FP64_SWEEP_DRAM_BYTES_PER_CELL = (101.7 + 158.1 + 334.9) / 3.0
NCU_FP64_SWEEPS = "profiles/sweep_fp64_shock_bubble_160.md"
# The same count for the other FP64 forms (x, y, z; 160^3 shock-bubble, RK
# stage 2; profiles/sweep_fp64_forms_shock_bubble_160.md).
FP64_SWEEP_WARP_INST_PER_CELL_FORM = {
    "fp64_weno3": (114.7, 117.0, 127.6),
    "fp64_kapila": (187.2, 189.8, 200.1),
    "fp64_stretched": (221.4, 206.6, 217.6),
    "fp64_cbc": (174.1, 177.2, 187.5),
    "fp64_six": (188.6, 191.7, 261.2),
}
NCU_FP64_FORMS = "profiles/sweep_fp64_forms_shock_bubble_160.md"
# Nominal FP32 peak: 152 SMs x 128 FMA/clk x 2 FLOP x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Algorithmic DRAM bytes per cell of the three mixed-form sweeps of one stage
# (FP32 primitives and accumulator, FP64 state), for ns state rows and nw
# reconstructed rows (nw = ns except in the six-equation model): x reads w and
# writes R, y reads w and updates R, z reads w and R and the FP64 stage states
# and writes the new state (stage 1 has no q^n term).
def bytes_mixed_sweeps_stage(ns, nw):
    x = 4 * nw + 4 * ns
    y = 4 * nw + 8 * ns
    z1 = 4 * nw + 4 * ns + 8 * ns + 8 * ns
    z23 = z1 + 8 * ns
    return x + y + (z1 + 2 * z23) / 3.0


# Useful tensor-core FLOPs of the learned network per stencil
# (5x32 + 32x32 + 32x3 multiply-adds) and stencils per cell and sweep (2 edges x 7 variables).
FLOP_MLP_STENCIL = 2 * (5 * 32 + 32 * 32 + 32 * 3)
STENCILS_PER_CELL_SWEEP = 14


def max_over_ranks(x: float, ws: int, device="cpu") -> float:
    """Maximum of a per-rank scalar over all ranks (the step time of the
    slowest replica); a no-op on one rank."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def grind_ns(ms_per_step, ws, cells, ns, rhs_per_step=3):
    """Whole-job grind time: the slowest rank's step time over every cell,
    equation and RHS evaluation that all ws replicas processed in it."""
    return ms_per_step * 1e-3 / (ws * cells * ns * rhs_per_step) * 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        return False

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(self.out or "")) if len(r) >= 9]
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# Training data of the learned weights: runs of the plain method (mixed form)
# on the 256^3 shock-bubble and the 384^3 bubble cloud, harvested at five
# snapshots each (the coarse stencils are the runs restricted by 2 per axis,
# 128^3 and 192^3, with the fine face values as targets), 1e6 stencils per
# snapshot: 1e7 in all.
TRAIN_RUNS = (("shock_bubble", 256, 200, (0, 50, 100, 150, 200), 1_000_000, 1),
              ("bubble_cloud", 384, 200, (0, 50, 100, 150, 200), 1_000_000, 2))


# Useful FLOPs of one sample's loss gradient: the forward layers (5x32, 32x32,
# 32x3 multiply-adds), the backward data products (3x32, 32x32) and the
# weight-gradient products (32x5, 32x32, 3x32), two FLOPs per multiply-add.
FLOP_MLP_GRAD_SAMPLE = 2 * ((5 * 32 + 32 * 32 + 32 * 3) + (3 * 32 + 32 * 32) + (32 * 5 + 32 * 32 + 3 * 32))


def time_mlp_grad(m, torch, P, samples, batch=65536, passes=3):
    """Milliseconds per pass over the training samples of the loss gradient on
    the tcgen05 tensor cores (mfc_mlp_grad) and on warp-level mma.sync
    (mfc_mlp_grad_mma), timed with CUDA events on the current stream."""
    n = len(samples) - len(samples) % batch
    G = torch.empty_like(P)
    L = torch.empty(1, dtype=torch.float32, device=P.device)
    work = torch.empty(m.MLP_WORK_FLOATS, dtype=torch.float32, device=P.device)
    out = {"samples_per_pass": n, "batch": batch}
    peaks = _measured_peaks()
    bf = float(peaks.get("bf16_tflops", 1900.0))
    for name, fn in (("tcgen05", m.mfc_mlp_grad), ("mma_sync", m.mfc_mlp_grad_mma)):
        def one_pass():
            for a in range(0, n, batch):
                sb = samples.slice(a, a + batch)
                fn(P, sb.x, sb.phat, sb.target, sb.smooth, 1.0, G, L, work)
        one_pass()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(passes):
            one_pass()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / passes
        tf = FLOP_MLP_GRAD_SAMPLE * n / (ms * 1e-3) / 1e12
        out[name] = {"ms_per_pass": ms, "samples_per_s": n / (ms * 1e-3), "tensor_tflops": tf,
                     "tensor_frac": tf / bf}
    if m.mfc_mlp_tc_status():
        out["tcgen05"]["error"] = "a bounded tensor-core wait gave up"
    out["note"] = ("useful FLOPs %d per sample; tensor_frac against the measured bf16 burst peak: the 5-32-32-3 "
                   "network is far too small to load the tensor cores (one 128-sample tile per CTA and MMA "
                   "round trip)" % FLOP_MLP_GRAD_SAMPLE)
    return out


def train_learned(m, torch, log=None, runs=TRAIN_RUNS, time_grad=False):
    """Train the learned weights on stencils harvested from runs of the
    shock-bubble and bubble-cloud workloads (done before, and outside, every
    timed region); with time_grad also time the two gradient kernels."""
    from paper_2305_09163_gb300 import learned
    t0 = time.perf_counter()
    parts = []
    for name, n, steps, snaps, per, seed in runs:
        wl = getattr(workloads, name)(n)
        parts.append(learned.harvest_run(wl, steps, set(snaps), per, seed))
        torch.cuda.empty_cache()
    th = time.perf_counter()
    samples = learned.Samples.cat(parts)
    del parts
    P, hist = learned.train(samples)
    torch.cuda.synchronize()
    info = {"samples": len(samples),
            "runs": ["%s %d^3, steps %s, %d per snapshot" % (name, n, list(snaps), per)
                     for name, n, _, snaps, per, _ in runs],
            "final_loss": hist[-1], "harvest_seconds": th - t0, "train_seconds": time.perf_counter() - th}
    if time_grad:
        info["grad_kernels"] = time_mlp_grad(m, torch, P, learned.smooth_part(samples))
    del samples
    torch.cuda.empty_cache()
    return P.cpu().numpy(), info


def _sweep_profile(prof):
    ms = sum(prof[k][0] for k in ("sweep_x", "sweep_y", "sweep_z"))
    n = sum(prof[k][1] for k in ("sweep_x", "sweep_y", "sweep_z"))
    return ms, n


def time_form(m, torch, wl, w_dev, precision, params, steps, warmup, develop, dist_barrier, sampler_gpu=None,
              mlp=None):
    """Develop the initial state by `develop` steps, warm up by `warmup` more,
    then time `steps` steps (CFL + SSP-RK3) with CUDA events on the solver's
    stream.  Returns a dict of measurements."""
    stream = torch.cuda.current_stream()
    s = m.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision=precision, fallback=1, **params)
    if wl.faces is not None:
        for d in range(3):
            s.set_grid(d, wl.faces[d])
    if mlp is not None:
        s.set_mlp(mlp)
    s.set_state_prim(w_dev)
    for _ in range(develop + warmup):
        s.step(s.cfl_dt(CFL))
    torch.cuda.synchronize()
    dist_barrier()
    torch.cuda.synchronize()
    s.set_param("profile", 1)
    s.profile()  # clear anything pending
    prof0 = s.profile()
    l0 = s.launch_count()
    r0 = s.network_rows()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(sampler_gpu) if sampler_gpu is not None else None
    if sampler:
        sampler.__enter__()
    e0.record(stream)
    for _ in range(steps):
        s.step(s.cfl_dt(CFL))
    e1.record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__(None, None, None)
    dist_barrier()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof1 = s.profile()
    s.set_param("profile", 0)
    launches = s.launch_count() - l0
    rows = s.network_rows() - r0
    sweep_ms = _sweep_profile(prof1)[0] - _sweep_profile(prof0)[0]
    sweep_n = _sweep_profile(prof1)[1] - _sweep_profile(prof0)[1]
    kern = {k: (prof1[k][0] - prof0[k][0], prof1[k][1] - prof0[k][1]) for k in prof1}
    fb = s.fallback_count()
    s.close()
    return {"ms_per_step": ms, "launches": launches, "sweep_ms": sweep_ms, "sweep_launches": sweep_n,
            "kernels": kern, "clocks": sampler.summary() if sampler else None, "fallback_faces": fb,
            "network_rows": rows, "steps": steps, "warmup": warmup, "develop": develop}


def e2e_form(m, torch, wl, w_host, precision, steps, warmup):
    """Same metric through the C ABI with HOST buffers: every step copies the
    state in from pinned host memory, steps, and reads the state back."""
    s = m.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision=precision, fallback=1)
    s.set_state_prim(w_host)
    q_host = torch.empty(s.shape, dtype=torch.float64, pin_memory=True)
    m.mfc_get_state(s.ctx, q_host)
    for _ in range(warmup):
        m.mfc_set_state(s.ctx, q_host)
        s.step(s.cfl_dt(CFL))
        m.mfc_get_state(s.ctx, q_host)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        m.mfc_set_state(s.ctx, q_host)
        s.step(s.cfl_dt(CFL))
        m.mfc_get_state(s.ctx, q_host)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    nbytes = q_host.numel() * 8
    s.close()
    return dt, nbytes


def cpu_baseline_sample(wl, w_host, min_seconds=10.0, min_calls=2):
    """The oracle as it stands (C, OpenMP over all host cores) on a 32-plane slab
    through the bubble centre of the same workload; returns grind time."""
    import oracle
    nz = 32
    z0 = wl.n[2] // 2 - nz // 2
    sub = np.ascontiguousarray(w_host[:, z0:z0 + nz])
    h = (wl.hi[2] - wl.lo[2]) / wl.n[2]
    pb = oracle.Problem((wl.n[0], wl.n[1], nz), wl.lo, (wl.hi[0], wl.hi[1], wl.lo[2] + nz * h), wl.bc,
                        wl.gamma, wl.pi_inf, fallback=True)
    q = oracle.cons_from_prims(pb, sub)
    oracle.rhs(pb, q)  # warm (page-in, thread pool)
    calls = 0
    t0 = time.perf_counter()
    while calls < min_calls or time.perf_counter() - t0 < min_seconds:
        oracle.rhs(pb, q)
        calls += 1
    el = time.perf_counter() - t0
    grind = el / calls / (pb.ncell * pb.sys_size) * 1e9
    cores = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    return {"value": grind, "unit": UNIT, "cores": int(cores), "kind": "oracle",
            "sample": "%d oracle RHS calls on a %dx%dx%d slab (z planes %d..%d) of the %s initial state, %.1f s"
                      % (calls, wl.n[0], wl.n[1], nz, z0, z0 + nz - 1, wl.name, el),
            "one_core": cpu_one_core_sample(wl.n[0])}


# The same oracle RHS on one host core: a child process with OMP_NUM_THREADS=1
# (OpenMP fixes its team size at first use, so the parent cannot shrink it).
_ONE_CORE_CHILD = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle, workloads
n, nz, min_seconds = int(sys.argv[2]), 4, float(sys.argv[3])
wl = workloads.shock_bubble(n)
w = wl.prims()
z0 = n // 2 - nz // 2
sub = np.ascontiguousarray(w[:, z0:z0 + nz])
h = (wl.hi[2] - wl.lo[2]) / n
pb = oracle.Problem((n, n, nz), wl.lo, (wl.hi[0], wl.hi[1], wl.lo[2] + nz * h), wl.bc, wl.gamma, wl.pi_inf,
                    fallback=True)
q = oracle.cons_from_prims(pb, sub)
oracle.rhs(pb, q)
calls, t0 = 0, time.perf_counter()
while calls < 2 or time.perf_counter() - t0 < min_seconds:
    oracle.rhs(pb, q)
    calls += 1
el = time.perf_counter() - t0
print(json.dumps({"value": el / calls / (pb.ncell * pb.sys_size) * 1e9, "cores": 1,
                  "sample": "%d oracle RHS calls on a %dx%dx%d slab (z planes %d..%d), one thread, %.1f s"
                            % (calls, n, n, nz, z0, z0 + nz - 1, el)}))
"""


def cpu_one_core_sample(n, min_seconds=5.0):
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        res = subprocess.run([sys.executable, "-c", _ONE_CORE_CHILD, ROOT, str(n), str(min_seconds)], env=env,
                             capture_output=True, text=True, timeout=300)
        if res.returncode != 0:
            return {"error": (res.stderr.strip().splitlines() or ["exit %d" % res.returncode])[-1]}
        out = json.loads(res.stdout.strip().splitlines()[-1])
        out["unit"] = UNIT
        return out
    except (OSError, ValueError, IndexError, subprocess.SubprocessError) as e:
        return {"error": str(e) or type(e).__name__}


def run_reference(args, wl):
    import oracle as orc  # test infrastructure: the reference arm is the CPU oracle
    w_host = wl.prims()
    nz = 32
    z0 = wl.n[2] // 2 - nz // 2
    sub = np.ascontiguousarray(w_host[:, z0:z0 + nz])
    h = (wl.hi[2] - wl.lo[2]) / wl.n[2]
    pb = orc.Problem((wl.n[0], wl.n[1], nz), wl.lo, (wl.hi[0], wl.hi[1], wl.lo[2] + nz * h), wl.bc,
                     wl.gamma, wl.pi_inf, fallback=True)
    q = orc.cons_from_prims(pb, sub)
    for _ in range(max(args.warmup, 0)):
        orc.rk3_step(pb, q, orc.cfl_dt(pb, q, CFL))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q = orc.rk3_step(pb, q, orc.cfl_dt(pb, q, CFL))
    el = time.perf_counter() - t0
    ms = el / args.steps * 1e3
    grind = el / args.steps / (3 * pb.ncell * pb.sys_size) * 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count())
    sample = ("%d oracle SSP-RK3 steps (CFL + 3 RHS) on a %dx%dx%d slab (z planes %d..%d) of the %s initial state"
              % (args.steps, wl.n[0], wl.n[1], nz, z0, z0 + nz - 1, wl.name))
    line = {"impl": "reference", "metric": METRIC, "value": grind, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "cells": pb.ncell, "sys_size": pb.sys_size, "form": "fp64",
                       "sample": sample},
            "cell_updates_per_s": pb.ncell / (el / args.steps),
            "cpu_baseline": {"value": grind, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": grind, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _l1_fields(w, ref, nf):
    """L1 differences of density (relative), pressure (relative) and the first
    volume fraction (absolute mean) between two primitive states."""
    rho = lambda a: a[:nf].sum(axis=0)
    ip = nf + 3  # 3D: pressure follows the three velocities, volume fractions follow
    ia = ip + 1
    return {"rho": float(np.abs(rho(w) - rho(ref)).mean() / np.abs(rho(ref)).mean()),
            "p": float(np.abs(w[ip] - ref[ip]).mean() / np.abs(ref[ip]).mean()),
            "alpha": float(np.abs(w[ia] - ref[ia]).mean())}


def _run_schedule(m, torch, wl, precision, dts=None, steps=None, mlp=None, init=None):
    """Run a workload; returns (final primitives on the host, dt list).  With
    dts given the same time steps are replayed."""
    s = m.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision=precision, fallback=1)
    if mlp is not None:
        s.set_mlp(mlp)
    s.set_state_prim(torch.from_numpy(init if init is not None else wl.prims()).cuda())
    out = []
    n = len(dts) if dts is not None else steps
    for k in range(n):
        dt = dts[k] if dts is not None else s.cfl_dt(CFL)
        s.step(dt)
        out.append(dt)
    w = s.get_prims().cpu().numpy()
    s.close()
    torch.cuda.empty_cache()
    return w, out


def run_accuracy(args):
    """Accuracy of the mixed and learned forms against the FP64 GPU path (itself
    parity-gated against the oracle per RHS call) on the full-size workloads,
    replaying the FP64 run's time steps; and of the learned form against a
    2x-resolution FP64 run on a reduced bubble-cloud box."""
    import torch
    import paper_2305_09163_gb300 as m
    m.build()
    m.load()
    mlp, training = train_learned(m, torch)
    cases = {"1": workloads.shock_bubble(256), "2": workloads.bubble_cloud(384), "4": workloads.three_fluid(512)}
    for key in [c.strip() for c in args.configs.split(",") if c.strip() and c.strip() in cases]:
        wl = cases[key]
        t0 = time.perf_counter()
        try:
            _accuracy_case(m, torch, wl, key, mlp, t0)
        except Exception as exc:  # report and go on with the next workload
            print(json.dumps({"config": key, "workload": wl.name, "error": repr(exc)}), flush=True)
    if "3" in args.configs:
        _accuracy_learned_2x(m, torch, mlp, training)


def _accuracy_case(m, torch, wl, key, mlp, t0):
    init = wl.prims()
    ref, dts = _run_schedule(m, torch, wl, "fp64", steps=wl.steps, init=init)
    res = {"config": key, "workload": wl.name, "steps": wl.steps, "t_end": float(sum(dts))}
    res["mixed_vs_fp64"] = _l1_fields(_run_schedule(m, torch, wl, "mixed", dts=dts, init=init)[0], ref, wl.nf)
    if wl.nf == 2:
        res["learned_vs_fp64"] = _l1_fields(
            _run_schedule(m, torch, wl, "learned", dts=dts, mlp=mlp, init=init)[0], ref, wl.nf)
    res["seconds"] = time.perf_counter() - t0
    print(json.dumps(res), flush=True)


def _accuracy_learned_2x(m, torch, mlp, training, n=192, t_end=1.0e-4, taus=(10.0, 30.0)):
    """Learned weights against WENO5-JS at the bubble cloud's own cell size
    (1/384): a 192^3 box of the cloud ([0, 0.5] x [0.25, 0.75]^2, the shock and
    the first bubbles), judged against the FP64 run of the same box at 2x
    resolution (384^3) restricted to the coarse grid, same physical time; the
    coarse runs start from the restricted fine initial state."""
    fine = workloads.bubble_cloud_box(2 * n)
    coarse = workloads.bubble_cloud_box(n)
    fw = fine.prims()
    init = np.ascontiguousarray(fw.reshape(fw.shape[0], n, 2, n, 2, n, 2).mean(axis=(2, 4, 6)))
    del fw

    def run_to(wl, precision, mlp=None, init=None, **params):
        s = m.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision=precision, fallback=1, **params)
        if mlp is not None:
            s.set_mlp(mlp)
        s.set_state_prim(torch.from_numpy(init if init is not None else wl.prims()).cuda())
        t, k = 0.0, 0
        try:
            while t < t_end:
                dt = min(s.cfl_dt(CFL), t_end - t)
                s.step(dt)
                t += dt
                k += 1
            w = s.get_prims().cpu().numpy()
        except m.MFCError as exc:   # a non-physical state: reported, not timed
            w = "failed at step %d (t = %.3g s): %s" % (k, t, exc)
        s.close()
        torch.cuda.empty_cache()
        return w, k
    t0 = time.perf_counter()
    ref, kf = run_to(fine, "fp64")
    ref = ref.reshape(ref.shape[0], n, 2, n, 2, n, 2).mean(axis=(2, 4, 6))
    js = _l1_fields(run_to(coarse, "mixed", None, init)[0], ref, 2)
    res = {"config": "3", "workload": "bubble-cloud box %d^3 (cell 1/384) vs restricted FP64 %d^3" % (n, 2 * n),
           "t_end": t_end, "steps_fine": kf, "mixed_js_vs_2x": js,
           "fp64_js_vs_2x": _l1_fields(run_to(coarse, "fp64", None, init)[0], ref, 2),
           "training": training}
    for tau in taus:
        wl_, kc = run_to(coarse, "learned", mlp, init, sensor_tau=tau)
        key = "learned_tau%g" % tau
        if isinstance(wl_, str):
            res[key] = {"error": wl_}
            continue
        e = _l1_fields(wl_, ref, 2)
        res[key] = {"vs_2x": e, "steps": kc, "gain_vs_js": {k: 1.0 - e[k] / js[k] for k in ("rho", "p", "alpha")}}
    res["seconds"] = time.perf_counter() - t0
    print(json.dumps(res), flush=True)


def _sweep_roofline_fp64(r, cells, ns, variant, nf, clocks, inst_per_cell=FP64_SWEEP_WARP_INST_PER_CELL,
                         ncu=NCU_FP64_SWEEPS):
    """Roofline of the FP64 sweeps.  Their work runs mostly on the FP32 pipes
    (the WENO weights and HLLC in float-float, the weights in packed FP32x2
    instructions: one issue slot, two FMA-pipe cycles each), and neither the
    FP64 pipe nor DRAM is saturated: the binding resources are issue slots and
    the FMA pipe, with latency-bound dependency chains at 16 warps per SM.
    frac = warp instructions issued per second (the stored per-cell count x
    cells x launches / the library's own launch times) over 152 SMs x 4
    schedulers x the SM clock sampled during the run; the FMA- and FP64-pipe
    activity of the same capture and the FP64-accurate algorithmic FLOP rate
    (oracle-counted work) are reported beside it."""
    sweep_s = r["sweep_ms"] * 1e-3
    launches = r["sweep_launches"]
    stages = launches / 3.0
    flop = ORACLE_FLOP_PER_CELL_SWEEP[(variant, nf)] * cells * launches + RK_FLOP_PER_VAR_STAGE * ns * cells * stages
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    inst = sum(inst_per_cell) / 3.0 * cells * launches
    achieved = inst / sweep_s / 1e9
    peak = SCHEDULERS * mhz * 1e6 / 1e9
    return {"bound": "alu", "resource": "issue slots (and FMA pipe)", "kernel": "sweep (x, y, z)", "achieved": achieved,
            "peak": peak, "unit": "Gwarp-inst/s", "frac": achieved / peak, "issue_frac": achieved / peak,
            "peak_note": "152 SMs x 4 schedulers x 1 warp instruction per clock x the sampled SM clock (%.0f MHz)"
                         % mhz,
            "warp_inst_per_cell_per_sweep": sum(inst_per_cell) / 3.0,
            "flop_tflops": flop / sweep_s / 1e12,
            "flop_per_cell_per_sweep": ORACLE_FLOP_PER_CELL_SWEEP[(variant, nf)],
            "flop_note": "FP64-accurate work of the oracle's plain formulation (counted), + RK update",
            "fp64_pipe_frac_ncu": FP64_SWEEP_PIPE_FP64, "fma_pipe_frac_ncu": FP64_SWEEP_PIPE_FMA,
            "traffic": FP64_SWEEP_DRAM_BYTES_PER_CELL * cells if FP64_SWEEP_DRAM_BYTES_PER_CELL else None,
            "traffic_note": "DRAM bytes per sweep launch, per-cell counts of one ncu capture scaled by cells",
            "ncu": ncu}


def _sweep_roofline_hbm(r, cells, ns, nw, variant, nf, peaks, learned=False):
    """Mixed and learned forms: algorithmic DRAM bytes of the three sweeps of a
    stage over the measured copy bandwidth, and the oracle-counted FLOPs (run in
    FP32) over the nominal FP32 peak."""
    sweep_s = r["sweep_ms"] * 1e-3
    stages = r["sweep_launches"] / 3.0
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbs = bytes_mixed_sweeps_stage(ns, nw) * cells * stages / sweep_s / 1e9
    tf = ORACLE_FLOP_PER_CELL_SWEEP[(variant, nf)] * cells * r["sweep_launches"] / sweep_s / 1e12
    out = {"bound": "hbm", "kernel": "sweep (x, y, z)", "achieved": gbs, "peak": hbm, "unit": "GB/s",
           "frac": gbs / hbm, "hbm_gbs": gbs, "hbm_frac": gbs / hbm,
           "bytes_per_cell_stage": bytes_mixed_sweeps_stage(ns, nw),
           "fp32_tflops": tf, "fp32_peak": FP32_PEAK_TFLOPS, "fp32_frac": tf / FP32_PEAK_TFLOPS,
           "note": "peaks: HBM of measured copy, FP32 nominal; FLOPs: the oracle's count, run in FP32"}
    if learned:
        edges = STENCILS_PER_CELL_SWEEP * cells * r["sweep_launches"]
        tfl = FLOP_MLP_STENCIL * r["network_rows"] / sweep_s / 1e12
        bf = float(peaks.get("bf16_tflops_sustained", 1700.0))
        out.update({"kernel": "sweep (x, y, z) with the network", "network_edges": r["network_rows"],
                    "network_fraction": r["network_rows"] / edges, "tensor_tflops": tfl, "tensor_peak": bf,
                    "tensor_frac": tfl / bf})
    return out


def _form_entry(r, ws, cells, neq, head_ms=None):
    g = grind_ns(r["ms_max"], ws, cells, neq)
    e = {"grind": g, "unit": UNIT, "ms_per_step": r["ms_max"], "cell_updates_per_s": ws * cells / (r["ms_max"] * 1e-3),
         "gpu_launches": r["launches"], "steps": r["steps"], "warmup": r["warmup"], "develop": r["develop"],
         "kernels_ms": {k: v[0] for k, v in r["kernels"].items() if v[1]}, "workload": r["workload"],
         "equations": neq, "fallback_faces": r["fallback_faces"]}
    if head_ms is not None:
        e["speedup_vs_fp64"] = head_ms / r["ms_max"]
    if r.get("clocks"):
        e["clocks"] = r["clocks"]
    return e


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--develop", type=int, default=20,
                    help="steps from the initial state before the warm-up (shock and interfaces developed)")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=256, help="cells per direction of the shock-bubble cube")
    ap.add_argument("--forms", default="fp64,mixed,learned,fp64_weno3,mixed_weno3,fp64_kapila,fp64_stretched,"
                                       "mixed_stretched,fp64_cbc,fp64_six,mixed_six",
                    help="comma list of " + ",".join(FORMS))
    ap.add_argument("--config-runs", default=",".join(CONFIG_RUNS),
                    help="comma list of " + ",".join(CONFIG_RUNS) + " (or 'none'); each times at least 20 steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--accuracy", action="store_true",
                    help="accuracy study of the mixed and learned forms instead of timing")
    ap.add_argument("--configs", default="1,2,3,4", help="accuracy study: which workloads")
    args = ap.parse_args()
    if args.accuracy:
        run_accuracy(args)
        return
    ws, rank, local = _dist()
    wl = workloads.shock_bubble(args.n)

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return

    import torch
    import paper_2305_09163_gb300 as m
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        barrier = lambda: dist.barrier()
    else:
        barrier = lambda: None
    m.build() if rank == 0 else None
    if ws > 1:
        barrier()
    m.load()

    w_host = wl.prims()
    w_dev = torch.from_numpy(w_host).cuda()
    cells = wl.ncell
    ns = wl.sys_size
    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    for f in forms:
        if f not in FORMS:
            raise SystemExit("unknown form %r (known: %s)" % (f, ", ".join(FORMS)))
    runs = [c.strip() for c in args.config_runs.split(",") if c.strip() and c.strip() != "none"]
    for c in runs:
        if c not in CONFIG_RUNS:
            raise SystemExit("unknown config run %r (known: %s)" % (c, ", ".join(CONFIG_RUNS)))
    results = {}
    training = None
    mlp = None
    if "learned" in forms or any(CONFIG_RUNS[c][1] == "learned" for c in runs):
        mlp, training = train_learned(m, torch, time_grad=True)
    head = "fp64" if "fp64" in forms else forms[0]
    stretched = None
    six_w = None
    for form in forms:
        precision, params, variant, _ = FORMS[form]
        fwl, fw = wl, w_dev
        if variant == "cbc":   # same cells and state, non-reflecting faces
            fwl = workloads.shock_bubble_cbc(args.n)
        if variant == "six":   # same cells and state, phases in pressure equilibrium
            if six_w is None:
                six_w = torch.from_numpy(workloads.six_equation_prims(w_host, wl.nf)).cuda()
            fw = six_w
        if variant == "stretched":
            if stretched is None:
                swl = workloads.shock_bubble_stretched(args.n)
                stretched = (swl, torch.from_numpy(swl.prims()).cuda())
            fwl, fw = stretched
        r = time_form(m, torch, fwl, fw, precision, params, args.steps, args.warmup, args.develop, barrier,
                      sampler_gpu=local if form == head else None, mlp=mlp if precision == "learned" else None)
        r["workload"] = fwl.name
        r["ms_max"] = max_over_ranks(r["ms_per_step"], ws, "cuda")
        results[form] = r
    del six_w, stretched
    torch.cuda.empty_cache()

    fp = results[head]
    ms = fp["ms_max"]
    grind = grind_ns(ms, ws, cells, ns)
    peaks = _measured_peaks()
    line = {
        "metric": METRIC, "value": grind, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name + " (FP64, 2 fluids, 7 equations)", "cells": cells, "sys_size": ns,
                   "rhs_per_step": 3, "cfl": CFL, "develop_steps": args.develop,
                   "parallelism": "replicas" if ws > 1 else "single-gpu",
                   "l2": "inputs larger than L2 (state %.2f GB per array)" % (cells * ns * 8 / 1e9),
                   "arithmetic": "FP64 state, primitives, differences, fluxes, RK; WENO weights and HLLC in "
                                 "float-float (~48 bits, FP32 exponent range); parity <= 1e-11 vs the FP64 oracle"},
        "cell_updates_per_s": ws * cells / (ms * 1e-3),
        "roofline": _sweep_roofline_fp64(fp, cells, ns, "weno5", wl.nf, fp["clocks"]) if head == "fp64" else None,
        "gpu_launches": fp["launches"],
        "kernels_ms": {k: v[0] for k, v in fp["kernels"].items() if v[1]},
        "fallback_faces": fp["fallback_faces"],
        "clocks": fp["clocks"],
        "forms": {},
        "configs": {},
    }
    for form, r in results.items():
        if form == head:
            continue
        precision, params, variant, work = FORMS[form]
        six = variant == "six"
        # equations per cell: the six-equation model adds the N phase energies
        neq = ns + wl.nf if six else ns
        entry = _form_entry(r, ws, cells, neq, ms)
        if precision == "fp64":
            entry["roofline"] = _sweep_roofline_fp64(r, cells, neq, work, wl.nf, fp["clocks"],
                                                     FP64_SWEEP_WARP_INST_PER_CELL_FORM[form], NCU_FP64_FORMS)
            entry["roofline"]["note"] = ("instruction count per cell of this form's sweeps (ncu); FLOPs of the "
                                         "oracle's %s formulation%s"
                                         % (work, "; the per-cell tables of the stretched grid and the "
                                            "six-equation rows and relaxation add work" if variant in
                                            ("stretched", "six") else ""))
        else:
            entry["roofline"] = _sweep_roofline_hbm(r, cells, neq, ns, work, wl.nf, peaks,
                                                    learned=precision == "learned")
            if precision == "learned":
                entry["training"] = training
        line["forms"][form] = entry
    for name in runs:
        wname, precision = CONFIG_RUNS[name]
        cwl = getattr(workloads, wname)()
        cw = torch.from_numpy(cwl.prims()).cuda()
        r = time_form(m, torch, cwl, cw, precision, {}, max(args.steps, 20), args.warmup, args.develop, barrier,
                      sampler_gpu=local, mlp=mlp if precision == "learned" else None)
        del cw
        torch.cuda.empty_cache()
        r["workload"] = cwl.name
        r["ms_max"] = max_over_ranks(r["ms_per_step"], ws, "cuda")
        entry = _form_entry(r, ws, cwl.ncell, cwl.sys_size)
        entry["config"] = {"workload": cwl.name, "cells": cwl.ncell, "fluids": cwl.nf, "form": precision,
                           "notes": cwl.notes}
        if precision == "fp64":
            entry["roofline"] = _sweep_roofline_fp64(r, cwl.ncell, cwl.sys_size, "weno5", cwl.nf, r["clocks"])
            if cwl.nf != 2:
                entry["roofline"]["note"] = "instruction count per cell of the two-fluid FP64 sweeps"
        else:
            entry["roofline"] = _sweep_roofline_hbm(r, cwl.ncell, cwl.sys_size, cwl.sys_size, "weno5", cwl.nf, peaks,
                                                    learned=precision == "learned")
        line["configs"][name] = entry
    if not args.no_e2e:
        k = max(5, min(args.steps, 10))
        dt, nbytes = e2e_form(m, torch, wl, w_host, "fp64", k, max(3, args.warmup))
        dt = max_over_ranks(dt, ws, "cuda")
        line["e2e"] = {"value": grind_ns(dt * 1e3, ws, cells, ns), "unit": UNIT,
                       "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": k,
                       "note": "C ABI with pinned host buffers: set_state + CFL + step + get_state per step"}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(wl, w_host)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
