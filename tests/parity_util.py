"""Relative L-infinity error of a right-hand side against the oracle's.

For each conserved component v (the metric of the per-RHS parity gate):

    S_v     = max( max_cells |R_oracle_v|,  max_faces |F_v| / dx_min )
    floor_v = 64 * u * max_cells |q_v| * lam
    err_v   = max(0, max_cells |R_gpu - R_oracle| - floor_v) / S_v

with lam = max_cells max_d (|u_d| + c)/dx_d (the CFL rate) and u the unit
round-off of the arithmetic under test (2^-53 for the FP64 path, 2^-24 for the
FP32 reconstruction and fluxes of the mixed and learned forms).  S_v is the scale of
the semi-discrete operator of Eq. "fvmdis" (Sec. 3.1): the larger of the
component's right-hand side and its largest face flux over the finest cell.
floor_v is an absolute round-off allowance, not a scale: a face flux is a sum of
terms of size |q_v| (|u| + c) (the HLLC upwinding), so the rounding of one RHS
evaluation is a few dozen units u of |q_v| lam.  It matters only where a
component's flux vanishes while its density does not, e.g. air at rest inside a
bubble at t = 0: there both sides' FP64 rounding of a uniform 1e5 Pa pressure
moves the O(1) air density at ~1e-14 m/s, which the first two terms alone would
read as an error far above 1e-11.  Where a component's flux scale is of the
order of |q_v| lam the floor is ~1e-14 of S_v and the gate is the plain relative
error; only for a partial density whose flux is small against |q_v| lam (the air
of a resting bubble beside shocked water) is floor_v / S_v larger, which the
table shows.

``rhs_table`` formats, per component, the error under S_v without the floor,
floor_v / S_v and the gated error, for test output; ``rhs_error_raw`` is the
error under S_v alone (used to check that a reduced-precision form really
differs from FP64).
"""
import numpy as np

import oracle

ROUNDOFF_ULPS = 64.0
FP64_UNIT = 2.0 ** -53
FP32_UNIT = 2.0 ** -24


def _components(pb, q, dR, Rc, fmax, unit=FP64_UNIT):
    """dR, Rc: [ns][cells] arrays (difference and oracle); returns (raw, floor_rel, gated)."""
    lam, _ = oracle.max_rate(pb, q)
    dxmin = min(pb.dx[:pb.ndim])
    ns = pb.sys_size
    qf = np.asarray(q).reshape(ns, -1)
    raw = np.zeros(ns)
    flo = np.zeros(ns)
    gated = np.zeros(ns)
    for v in range(ns):
        scale = max(np.abs(Rc[v]).max(initial=0.0), fmax[v] / dxmin, 1e-300)
        floor = ROUNDOFF_ULPS * unit * np.abs(qf[v]).max() * lam
        d = np.abs(dR[v]).max(initial=0.0)
        raw[v] = d / scale
        flo[v] = floor / scale
        gated[v] = max(0.0, d - floor) / scale
    return raw, flo, gated


def _diff(pb, R_gpu, R_cpu, cells):
    ns = pb.sys_size
    if cells is None:
        Rc = np.asarray(R_cpu).reshape(ns, -1)
        return np.asarray(R_gpu).reshape(ns, -1) - Rc, Rc
    Rc = np.asarray(R_cpu).T
    return np.asarray(R_gpu).reshape(ns, -1)[:, cells] - Rc, Rc


def rhs_error(pb, q, R_gpu, R_cpu, fmax, unit=FP64_UNIT):
    dR, Rc = _diff(pb, R_gpu, R_cpu, None)
    return _components(pb, q, dR, Rc, fmax, unit)[2]


def rhs_error_raw(pb, q, R_gpu, R_cpu, fmax):
    dR, Rc = _diff(pb, R_gpu, R_cpu, None)
    return _components(pb, q, dR, Rc, fmax)[0]


def sampled_rhs_error(pb, q, R_gpu_flat, cells, Rc, fmax, unit=FP64_UNIT):
    """Same metric on sampled cells: R_gpu_flat is [ns][ncell], Rc is [ncells][ns]."""
    dR, Rc = _diff(pb, R_gpu_flat, Rc, cells)
    return _components(pb, q, dR, Rc, fmax, unit)[2]


def rhs_table(pb, q, R_gpu, R_cpu, fmax, cells=None, unit=FP64_UNIT):
    """Per-component table: error under S_v alone, floor_v / S_v, gated error."""
    ns = pb.sys_size
    dR, Rc = _diff(pb, R_gpu, R_cpu, cells)
    raw, flo, gated = _components(pb, q, dR, Rc, fmax, unit)
    lines = ["  v   err/S_v    floor/S_v  gated"]
    for v in range(ns):
        lines.append("%3d  %9.2e  %9.2e  %9.2e" % (v, raw[v], flo[v], gated[v]))
    return "\n".join(lines)


def state_error(pb, qa, qb):
    """Per-component max difference of two conserved states, relative to the
    component's magnitude (momentum components share the momentum magnitude,
    volume fractions use 1; the six-equation model's phase energies their own
    magnitude)."""
    ns = pb.sys_size
    nf, nd = pb.nf, pb.ndim
    qa = np.asarray(qa).reshape(ns, -1)
    qb = np.asarray(qb).reshape(ns, -1)
    mom = np.abs(qb[nf:nf + nd]).max()
    err = np.zeros(ns)
    for v in range(ns):
        if nf <= v < nf + nd:
            scale = mom
        elif nf + nd < v < 2 * nf + nd:
            scale = 1.0
        else:
            scale = np.abs(qb[v]).max()
        err[v] = np.abs(qa[v] - qb[v]).max() / max(scale, 1e-300)
    return err
