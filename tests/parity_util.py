"""Relative L-infinity error of a right-hand side against the oracle's.

For each conserved component v:
    err_v = max_cells |R_gpu - R_oracle| / S_v
    S_v   = max( max_cells |R_oracle_v|,  max_faces |F_v| / dx_min,  max_cells |q_v| * lam )
with lam = max_cells max_d (|u_d| + c)/dx_d (the CFL rate).  The last term is the
natural rate scale of component v; without it a component whose flux happens to
vanish (air at rest inside a bubble) would be compared at the level of FP64
round-off of the pressure reconstruction.
"""
import numpy as np

import oracle


def rhs_error(pb, q, R_gpu, R_cpu, fmax):
    lam, _ = oracle.max_rate(pb, q)
    dxmin = min(pb.dx[:pb.ndim])
    ns = pb.sys_size
    qf = np.asarray(q).reshape(ns, -1)
    Rg = np.asarray(R_gpu).reshape(ns, -1)
    Rc = np.asarray(R_cpu).reshape(ns, -1)
    err = np.zeros(ns)
    for v in range(ns):
        scale = max(np.abs(Rc[v]).max(), fmax[v] / dxmin, np.abs(qf[v]).max() * lam, 1e-300)
        err[v] = np.abs(Rg[v] - Rc[v]).max() / scale
    return err


def sampled_rhs_error(pb, q, R_gpu_flat, cells, Rc, fmax):
    """Same metric on sampled cells: R_gpu_flat is [ns][ncell], Rc is [ncells][ns]."""
    lam, _ = oracle.max_rate(pb, q)
    dxmin = min(pb.dx[:pb.ndim])
    ns = pb.sys_size
    qf = np.asarray(q).reshape(ns, -1)
    err = np.zeros(ns)
    for v in range(ns):
        scale = max(np.abs(Rc[:, v]).max(), fmax[v] / dxmin, np.abs(qf[v]).max() * lam, 1e-300)
        err[v] = np.abs(R_gpu_flat[v, cells] - Rc[:, v]).max() / scale
    return err


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
