"""Throughput of the five-equation RHS / SSP-RK3 step on GB300.

Default workload: the 256^3 two-fluid water/air shock-bubble in FP64 (a step =
one CFL reduction + three RHS evaluations + three RK stage updates).  The metric
is the grind time t_RHS / (cells * equations) in ns/(cell*eqn*RHS) (lower is
better), with cell-updates/s beside it; the mixed-precision (and, when built,
learned-weight) forms are timed on the same workload and reported under "forms".

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

# Algorithmic FP64 operations of one directional sweep per cell (3D, two fluids,
# seven equations), counted from the formulation the kernels evaluate with
# FMA = 2 and every add, multiply, divide, square root, min and max = 1:
#   WENO5 edges (both sides of a cell) 70 per variable x 7, HLLC 87 per face,
#   flux difference + alpha div(u) source 18 per cell.
FLOP_SWEEP_CELL_3D_2F = 70 * 7 + 87 + 18
# The same with the third-order reconstruction: WENO3 edges (both sides) 31 per
# variable (two differences, t = eps + d^2, t^2, the two weight denominators
# and their product, one reciprocal, the two numerators and the two edges).
FLOP_SWEEP_CELL_3D_2F_W3 = 31 * 7 + 87 + 18
# The Kapila model adds K (two Z_k = gamma_k (p + pinf_k), the weighted sum,
# one reciprocal, K = alpha (Z_2/D - 1)) and its source term: 13 per cell and sweep.
FLOP_SWEEP_CELL_3D_2F_KAPILA = FLOP_SWEEP_CELL_3D_2F + 13
# Forms the bench can time: name -> (precision, extra solver parameters,
# workload: the shock-bubble, or the same on the tanh-stretched grid).
FORMS = {
    "fp64": ("fp64", {}, "uniform"),
    "mixed": ("mixed", {}, "uniform"),
    "learned": ("learned", {}, "uniform"),
    "fp64_weno3": ("fp64", {"weno_order": 3}, "uniform"),
    "mixed_weno3": ("mixed", {"weno_order": 3}, "uniform"),
    "fp64_kapila": ("fp64", {"model": 1}, "uniform"),
    "fp64_stretched": ("fp64", {}, "stretched"),
    "mixed_stretched": ("mixed", {}, "stretched"),
    "fp64_cbc": ("fp64", {}, "cbc"),
    "fp64_six": ("fp64", {"model": 2}, "six"),
    "mixed_six": ("mixed", {"model": 2}, "six"),
}
# RK3 stage epilogue in the last sweep: 6 per variable (stages 2, 3), 4 in stage 1
FLOP_RK_CELL_2F = 7 * (6 + 6 + 4) / 3.0
# Nominal FP64 peak: 152 SMs x 4 FP64 FLOP/clk/SM (2 DFMA) x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
# Nominal FP32 peak: 152 SMs x 128 FMA/clk x 2 FLOP x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Algorithmic DRAM bytes per cell of the three mixed-form sweeps of one stage
# (FP32 primitives and accumulator, FP64 state): x reads w and writes R (56 B),
# y reads w and updates R (84 B), z reads w and R and the FP64 stage states and
# writes the new state (224 B; 168 B in stage 1, which has no q^n term).
BYTES_MIXED_SWEEPS_STAGE = (56 + 84 + (168 + 224 + 224) / 3.0)
# DRAM bytes per cell of one FP64 sweep launch, averaged over the x, y and z
# sweeps of a stage: dram__bytes_read.sum + dram__bytes_write.sum of one ncu
# capture of the 160^3 shock-bubble (x 102.7, y 158.7, z 279.0 B/cell; the
# algorithmic w + R (+ RK states) bytes are 112, 168 and 280), scaled to the
# bench size by the cell count.  Must be re-measured when the FP64 sweeps change.
FP64_SWEEP_DRAM_BYTES_PER_CELL = (102.7 + 158.7 + 279.0) / 3.0
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


def train_learned(m, torch, log=None):
    """Train the learned weights on stencils of 128^3 shock-bubble and
    bubble-cloud runs (done before, and outside, the timed region)."""
    from paper_2305_09163_gb300 import learned
    t0 = time.perf_counter()
    parts = [learned.harvest_run(workloads.shock_bubble(128, steps=80), 80, {20, 40, 60, 80}, 1_000_000, 1),
             learned.harvest_run(workloads.bubble_cloud(128, steps=80, seed=230509163), 80, {20, 40, 60, 80},
                                 1_000_000, 2)]
    P, hist = learned.train(learned.Samples.cat(parts))
    torch.cuda.synchronize()
    return P.cpu().numpy(), {"samples": sum(len(p) for p in parts), "final_loss": hist[-1],
                             "seconds": time.perf_counter() - t0}


def _sweep_profile(prof):
    ms = sum(prof[k][0] for k in ("sweep_x", "sweep_y", "sweep_z"))
    n = sum(prof[k][1] for k in ("sweep_x", "sweep_y", "sweep_z"))
    return ms, n


def time_form(m, torch, wl, w_dev, form, steps, warmup, dist_barrier, sampler_gpu=None, mlp=None):
    """Warm up, then time `steps` steps (CFL + SSP-RK3) of one form (FORMS) with
    CUDA events on the solver's stream.  Returns a dict of measurements."""
    stream = torch.cuda.current_stream()
    precision, params, _ = FORMS[form]
    s = m.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision=precision, fallback=1, **params)
    if wl.faces is not None:
        for d in range(3):
            s.set_grid(d, wl.faces[d])
    if mlp is not None:
        s.set_mlp(mlp)
    s.set_state_prim(w_dev)
    for _ in range(warmup):
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
            "network_rows": rows}


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


def _accuracy_learned_2x(m, torch, mlp, training):
    # learned vs WENO5-JS at 128^3 against FP64 at 256^3 (the 768^3 reference of the
    # 384^3 cloud is out of reach of a bench run), same physical time
    n = 128
    fine = workloads.bubble_cloud(2 * n)
    coarse = workloads.bubble_cloud(n)
    fw = fine.prims()
    init = fw.reshape(fw.shape[0], n, 2, n, 2, n, 2).mean(axis=(2, 4, 6))
    del fw
    t_end = 1.0e-4
    def run_to(wl, precision, mlp=None, init=None):
        s = m.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision=precision, fallback=1)
        if mlp is not None:
            s.set_mlp(mlp)
        s.set_state_prim(torch.from_numpy(init if init is not None else wl.prims()).cuda())
        t = 0.0
        while t < t_end:
            dt = min(s.cfl_dt(CFL), t_end - t)
            s.step(dt)
            t += dt
        w = s.get_prims().cpu().numpy()
        s.close()
        return w
    ref = run_to(fine, "fp64")
    ref = ref.reshape(ref.shape[0], n, 2, n, 2, n, 2).mean(axis=(2, 4, 6))
    res = {"config": "3", "workload": "bubble_cloud 128^3 vs restricted FP64 256^3", "t_end": t_end,
           "learned_vs_2x": _l1_fields(run_to(coarse, "learned", mlp, init), ref, 2),
           "mixed_js_vs_2x": _l1_fields(run_to(coarse, "mixed", None, init), ref, 2),
           "fp64_js_vs_2x": _l1_fields(run_to(coarse, "fp64", None, init), ref, 2),
           "training": training}
    print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=256, help="cells per direction of the shock-bubble cube")
    ap.add_argument("--forms", default="fp64,mixed,learned,fp64_weno3,mixed_weno3,fp64_kapila,fp64_stretched,"
                                       "mixed_stretched,fp64_cbc,fp64_six,mixed_six",
                    help="comma list of " + ",".join(FORMS))
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
    results = {}
    training = None
    head = "fp64" if "fp64" in forms else forms[0]
    stretched = None
    six_w = None
    for form in forms:
        mlp = None
        if form == "learned":
            mlp, training = train_learned(m, torch)
        fwl, fw = wl, w_dev
        if FORMS[form][2] == "cbc":   # same cells and state, non-reflecting faces
            fwl = workloads.shock_bubble_cbc(args.n)
        if FORMS[form][2] == "six":   # same cells and state, phases in pressure equilibrium
            if six_w is None:
                six_w = torch.from_numpy(workloads.six_equation_prims(w_host, wl.nf)).cuda()
            fw = six_w
        if FORMS[form][2] == "stretched":
            if stretched is None:
                swl = workloads.shock_bubble_stretched(args.n)
                stretched = (swl, torch.from_numpy(swl.prims()).cuda())
            fwl, fw = stretched
        r = time_form(m, torch, fwl, fw, form, args.steps, args.warmup, barrier,
                      sampler_gpu=local if form == head else None, mlp=mlp)
        r["workload"] = fwl.name
        r["ms_max"] = max_over_ranks(r["ms_per_step"], ws, "cuda")
        results[form] = r

    fp = results[head]
    ms = fp["ms_max"]
    grind = grind_ns(ms, ws, cells, ns)
    flops_per_sweep_launch = (FLOP_SWEEP_CELL_3D_2F + FLOP_RK_CELL_2F / 3.0) * cells
    achieved = flops_per_sweep_launch * fp["sweep_launches"] / (fp["sweep_ms"] * 1e-3) / 1e12

    line = {
        "metric": METRIC, "value": grind, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name + " (FP64, 2 fluids, 7 equations)", "cells": cells, "sys_size": ns,
                   "rhs_per_step": 3, "cfl": CFL, "parallelism": "replicas" if ws > 1 else "single-gpu",
                   "l2": "inputs larger than L2 (state %.2f GB per array)" % (cells * ns * 8 / 1e9)},
        "cell_updates_per_s": ws * cells / (ms * 1e-3),
        "roofline": {"bound": "alu", "kernel": "sweep (x, y, z)", "achieved": achieved,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "peak_note": "nominal FP64: 152 SMs x 4 FLOP/clk x 2.07 GHz",
                     "flop_per_cell_per_sweep": FLOP_SWEEP_CELL_3D_2F,
                     "traffic": FP64_SWEEP_DRAM_BYTES_PER_CELL * cells if head == "fp64" else None,
                     "traffic_note": "DRAM bytes per sweep launch (ncu at 160^3, scaled by cells)",
                     "ncu_issue_active": 0.48,
                     "note": "FLOPs at FP64 accuracy; the WENO weights and HLLC run in float-float on the FP32 "
                             "pipes, so the rate can pass the FP64 pipe's nominal peak.  ncu (160^3): FP64 pipe "
                             "44-51% busy, issue 48-49% active (ncu_issue_active: their mean), ~12 warps per SM: "
                             "latency-bound"},
        "gpu_launches": fp["launches"],
        "kernels_ms": {k: v[0] for k, v in fp["kernels"].items() if v[1]},
        "fallback_faces": fp["fallback_faces"],
        "clocks": fp["clocks"],
        "forms": {},
    }
    for form, r in results.items():
        if form == head:
            continue
        if r is None:
            line["forms"][form] = None
            continue
        # equations per cell: the six-equation model adds the N phase energies
        neq = ns + wl.nf if FORMS[form][2] == "six" else ns
        g = grind_ns(r["ms_max"], ws, cells, neq)
        entry = {"grind": g, "unit": UNIT, "ms_per_step": r["ms_max"],
                 "cell_updates_per_s": ws * cells / (r["ms_max"] * 1e-3),
                 "speedup_vs_fp64": ms / r["ms_max"], "gpu_launches": r["launches"],
                 "kernels_ms": {k: v[0] for k, v in r["kernels"].items() if v[1]}}
        sweep_s = r["sweep_ms"] * 1e-3
        stages = r["sweep_launches"] / 3.0
        peaks = _measured_peaks()
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        entry["workload"] = r["workload"]
        entry["equations"] = neq
        if form in ("fp64_weno3", "fp64_kapila", "fp64_stretched", "fp64_cbc", "fp64_six"):
            fl = {"fp64_weno3": FLOP_SWEEP_CELL_3D_2F_W3, "fp64_kapila": FLOP_SWEEP_CELL_3D_2F_KAPILA,
                  "fp64_stretched": FLOP_SWEEP_CELL_3D_2F, "fp64_cbc": FLOP_SWEEP_CELL_3D_2F,
                  "fp64_six": FLOP_SWEEP_CELL_3D_2F}[form]
            tf = (fl + FLOP_RK_CELL_2F / 3.0) * cells * r["sweep_launches"] / sweep_s / 1e12
            entry["roofline"] = {"kernel": "sweep (x, y, z), " + {"fp64_weno3": "WENO3", "fp64_kapila": "Kapila",
                                                                  "fp64_stretched": "non-uniform grid",
                                                                  "fp64_cbc": "characteristic boundaries",
                                                                  "fp64_six": "six-equation model"}[form],
                                 "bound": "alu", "achieved": tf,
                                 "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS,
                                 "flop_per_cell_per_sweep": fl,
                                 "note": "nominal FP64 peak as for the WENO5 form" + (
                                     "; FLOPs counted as on a uniform grid (the per-cell coefficients add work)"
                                     if form == "fp64_stretched" else
                                     "; FLOPs counted as the five-equation sweep (the phase-energy rows and the "
                                     "relaxation add work)" if form == "fp64_six" else "")}
        elif form in ("mixed", "mixed_weno3", "mixed_stretched", "mixed_six"):
            gbs = BYTES_MIXED_SWEEPS_STAGE * cells * stages / sweep_s / 1e9
            fl = FLOP_SWEEP_CELL_3D_2F_W3 if form == "mixed_weno3" else FLOP_SWEEP_CELL_3D_2F
            tf = fl * cells * r["sweep_launches"] / sweep_s / 1e12
            entry["roofline"] = {"kernel": "sweep (x, y, z)", "hbm_gbs": gbs, "hbm_peak": hbm,
                                 "hbm_frac": gbs / hbm, "fp32_tflops": tf, "fp32_peak": FP32_PEAK_TFLOPS,
                                 "fp32_frac": tf / FP32_PEAK_TFLOPS,
                                 "note": "peaks: HBM of measured copy, FP32 nominal"}
        elif form == "learned":
            # the sweeps do the mixed form's work plus the sensor and, on the
            # edges it does not trip, the network (counted on the device)
            gbs = BYTES_MIXED_SWEEPS_STAGE * cells * stages / sweep_s / 1e9
            tf = FLOP_SWEEP_CELL_3D_2F * cells * r["sweep_launches"] / sweep_s / 1e12
            edges = STENCILS_PER_CELL_SWEEP * cells * r["sweep_launches"]
            tfl = FLOP_MLP_STENCIL * r["network_rows"] / sweep_s / 1e12
            bf = float(peaks.get("bf16_tflops_sustained", 1700.0))
            entry["roofline"] = {"kernel": "sweep (x, y, z) with the network", "hbm_gbs": gbs, "hbm_peak": hbm,
                                 "hbm_frac": gbs / hbm, "fp32_tflops": tf, "fp32_peak": FP32_PEAK_TFLOPS,
                                 "fp32_frac": tf / FP32_PEAK_TFLOPS,
                                 "network_edges": r["network_rows"], "network_fraction": r["network_rows"] / edges,
                                 "tensor_tflops": tfl, "tensor_peak": bf, "tensor_frac": tfl / bf,
                                 "note": "HBM/FP32 as the mixed form (its algorithmic bytes and FLOPs); network "
                                         "FLOPs of the edges evaluated, averaged over the sweep time; peaks: HBM "
                                         "of measured copy, FP32 nominal, BF16 measured sustained"}
            entry["training"] = training
        line["forms"][form] = entry
    if not args.no_e2e:
        k = max(2, min(args.steps, 5))
        dt, nbytes = e2e_form(m, torch, wl, w_host, "fp64", k, 1)
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
