"""Parity of characteristic (non-reflecting) boundaries (bc 3; Sec. 3.3,
characteristic-based conditions after Thompson) with the CPU FP64 oracle,
through the C ABI: the boundary cells' normal rates in every kernel form that
finishes cells (x stream, y/z stream, pencil marching), on uniform and
stretched grids, in the allocation-free entry point, and over SSP-RK3 steps.
The same error metric and FP64 gate as everywhere else."""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import FP32_UNIT, rhs_error, rhs_error_raw, state_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CBC = oracle.BC_CHARACTERISTIC
TOL_FP64 = 1e-11
TOL_MIXED_RHS = 2e-4


@pytest.fixture(scope="module")
def mfc():
    import paper_2305_09163_gb300 as m
    m.build()
    m.load()
    return m


def _boundary_mask(n, bc):
    nd = len(n)
    shape = tuple(n[::-1])
    m = np.zeros(shape, dtype=bool)
    for d in range(nd):
        ax = nd - 1 - d
        for side, idx in ((0, 0), (1, n[d] - 1)):
            if bc[2 * d + side] == CBC:
                sl = [slice(None)] * nd
                sl[ax] = idx
                m[tuple(sl)] = True
    return m


CASES = [
    # (n, nf, bc[:2*ndim], yz_kernel)
    ((45,), 2, (CBC, CBC), 1),
    ((37,), 3, (CBC, 1), 1),
    ((31, 19), 2, (CBC, CBC, 2, 2), 1),
    ((23, 29), 1, (1, CBC, CBC, CBC), 1),
    ((37, 23, 19), 2, (CBC,) * 6, 1),
    ((21, 14, 35), 3, (CBC, 1, 2, CBC, CBC, 2), 1),
    ((33, 20, 18), 2, (CBC,) * 6, 0),
    ((19, 26, 22), 3, (2, CBC, CBC, 1, 1, CBC), 0),
]


def _id(c):
    return "n%s_nf%d_bc%s_yz%d" % ("x".join(map(str, c[0])), c[1], "".join(map(str, c[2])), c[3])


@pytest.mark.parametrize("case", CASES, ids=_id)
def test_cbc_rhs_parity_fp64(mfc, case):
    n, nf, bc, yz = case
    gam, pin = workloads.fluids(nf)
    bc6 = tuple(bc) + (1,) * (6 - len(bc))
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, bc6, gam, pin, fallback=True)
    s = mfc.Solver(pb.n, (0,) * 3, (1,) * 3, pb.bc, gam, pin, precision="fp64", fallback=1, yz_kernel=yz)
    w = workloads.random_prims(n, nf, seed=90 + nf + len(n))
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy()
    assert rhs_error(pb, q, R, R_cpu, fmax).max() <= TOL_FP64
    # the boundary rates are in use: transmissive ghosts alone differ there
    pt = oracle.Problem(n, (0,) * 3, (1,) * 3, tuple(1 if b == CBC else b for b in bc6), gam, pin, fallback=True)
    Rt = oracle.rhs(pt, q)
    mask = _boundary_mask(n, bc6)
    ns = pb.sys_size
    assert rhs_error(pb, q, R.reshape(ns, -1)[:, mask.ravel()], Rt.reshape(ns, -1)[:, mask.ravel()],
                     fmax).max() > 1e3 * TOL_FP64


def test_cbc_on_stretched_grid_fp64(mfc):
    """The boundary cell's width from the grid enters the one-sided derivative."""
    n, nf = (29, 17, 13), 2
    gam, pin = workloads.fluids(nf)
    faces = [workloads.stretched_faces(m, 0.0, 1.0, 3.0, 0.3, 0.7) for m in n]
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (CBC,) * 6, gam, pin, fallback=True, faces=faces)
    s = mfc.Solver(pb.n, (0,) * 3, (1,) * 3, pb.bc, gam, pin, precision="fp64", fallback=1)
    for d in range(3):
        s.set_grid(d, faces[d])
    w = workloads.random_prims(n, nf, seed=97)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s.set_state_prim(torch.from_numpy(w).cuda())
    assert rhs_error(pb, q, s.rhs().cpu().numpy(), R_cpu, fmax).max() <= TOL_FP64


def test_cbc_mixed_rhs_close_to_oracle(mfc):
    n, nf = (37, 23, 19), 2
    gam, pin = workloads.fluids(nf)
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (CBC,) * 6, gam, pin, fallback=True)
    s = mfc.Solver(pb.n, (0,) * 3, (1,) * 3, pb.bc, gam, pin, precision="mixed", fallback=1)
    w = workloads.random_prims(n, nf, seed=98)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy()
    err = rhs_error(pb, q, R, R_cpu, fmax, unit=FP32_UNIT)
    assert err.max() <= TOL_MIXED_RHS, err
    assert rhs_error_raw(pb, q, R, R_cpu, fmax).max() > 1e-12  # FP32 arithmetic in use


def test_cbc_noalloc_matches_oracle(mfc):
    n, nf = (24, 18, 16), 2
    gam, pin = workloads.fluids(nf)
    bc = (CBC, CBC, 1, CBC, CBC, 2)
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, bc, gam, pin, fallback=True)
    w = workloads.random_prims(n, nf, seed=99)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    Rd = torch.empty_like(qd)
    mfc.mfc_rhs_noalloc(qd, Rd, n, (0,) * 3, (1,) * 3, bc, gam, pin, 1e-6, 1)
    torch.cuda.synchronize()
    assert rhs_error(pb, q, Rd.cpu().numpy(), R_cpu, fmax).max() <= TOL_FP64


def test_cbc_shock_bubble_steps_match_oracle(mfc):
    """The small shock-bubble with non-reflecting faces on every side: CFL dt
    and five SSP-RK3 steps, as the shocked water reaches the low-x face."""
    wl = workloads.shock_bubble(24)
    bc = (CBC,) * 6
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, bc, wl.gamma, wl.pi_inf, fallback=True)
    w = wl.prims()
    q = oracle.cons_from_prims(pb, w)
    s = mfc.Solver(wl.n, wl.lo, wl.hi, bc, wl.gamma, wl.pi_inf, precision="fp64", fallback=1)
    s.set_state_prim(torch.from_numpy(w).cuda())
    for _ in range(5):
        dt = oracle.cfl_dt(pb, q, 0.3)
        assert s.cfl_dt(0.3) == pytest.approx(dt, rel=1e-13)
        q = oracle.rk3_step(pb, q, dt)
        s.step(dt)
    assert state_error(pb, s.get_state().cpu().numpy(), q).max() <= 1e-10


def test_cbc_rejected_forms(mfc):
    gam, pin = workloads.fluids(2)
    with pytest.raises(mfc.MFCError):
        mfc.Solver((8, 8), (0, 0), (1, 1), (CBC, 1, 1, 1, 1, 1), gam, pin, precision="learned")
    s = mfc.Solver((8, 8), (0, 0), (1, 1), (1, 1, CBC, 1, 1, 1), gam, pin, precision="fp64")
    with pytest.raises(mfc.MFCError):
        s.set_param("model", 1)
    with pytest.raises(mfc.MFCError):
        mfc.Solver((8, 8), (0, 0), (1, 1), (4, 1, 1, 1, 1, 1), gam, pin, precision="fp64")
    # an inactive direction's entry is not a boundary of the problem
    mfc.Solver((8, 8), (0, 0), (1, 1), (1, 1, 1, 1, CBC, CBC), gam, pin, precision="learned")
