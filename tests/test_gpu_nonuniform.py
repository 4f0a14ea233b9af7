"""Parity of the non-uniform-grid sweeps (mfc_set_grid; Sec. 4.1 and Listing 1's
per-cell coefficients; Sec. 6.3's tanh stretching) with the CPU FP64 oracle,
through the C ABI; the same metric and FP64 gate as on uniform grids."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import nonuniform as nu
from parity_util import FP32_UNIT, rhs_error, rhs_error_raw, state_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11
TOL_MIXED_RHS = 2e-4


@pytest.fixture(scope="module")
def mfc():
    import paper_2305_09163_gb300 as m
    m.build()
    m.load()
    return m


def _faces(n, d, kind):
    if kind == "tanh":
        return workloads.stretched_faces(n, 0.0, 1.0, 3.0, 0.35 + 0.05 * d, 0.65 - 0.05 * d)
    xi = np.linspace(0.0, 1.0, n + 1)
    return xi + 0.5 * np.sin(2 * np.pi * xi) / (2 * np.pi)


def _setup(mfc, n, nf, bc, kind, precision="fp64", **params):
    gam, pin = workloads.fluids(nf)
    nd = len(n)
    faces = [_faces(n[d], d, kind) for d in range(nd)]
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (bc,) * 6, gam, pin, fallback=True, faces=faces, **params)
    s = mfc.Solver(pb.n, (0,) * 3, (1,) * 3, pb.bc, gam, pin, precision=precision, fallback=1)
    for d in range(nd):
        s.set_grid(d, faces[d])
    return pb, s


CASES = [
    # (n, nf, bc, kind)
    ((41,), 2, 1, "tanh"),
    ((37,), 1, 0, "sine"),
    ((29, 17), 2, 2, "tanh"),
    ((23, 19), 3, 0, "sine"),
    ((37, 23, 19), 2, 1, "tanh"),
    ((21, 13, 11), 3, 2, "tanh"),
    ((33, 20, 18), 2, 0, "sine"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%s_nf%d_bc%d_%s" % ("x".join(map(str, c[0])), *c[1:]))
def test_nonuniform_rhs_parity_fp64(mfc, case):
    n, nf, bc, kind = case
    pb, s = _setup(mfc, n, nf, bc, kind)
    w = workloads.random_prims(n, nf, seed=70 + nf)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy()
    assert rhs_error(pb, q, R, R_cpu, fmax).max() <= TOL_FP64
    # the grid matters: the uniform-grid oracle differs
    gam, pin = workloads.fluids(nf)
    pu = oracle.Problem(n, (0,) * 3, (1,) * 3, (bc,) * 6, gam, pin, fallback=True)
    assert rhs_error(pb, q, R, oracle.rhs(pu, q), fmax).max() > 1e3 * TOL_FP64


def test_nonuniform_mixed_rhs_close_to_oracle(mfc):
    n, nf = (37, 23, 19), 2
    pb, s = _setup(mfc, n, nf, 1, "tanh", precision="mixed")
    w = workloads.random_prims(n, nf, seed=75)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy()
    err = rhs_error(pb, q, R, R_cpu, fmax, unit=FP32_UNIT)
    assert err.max() <= TOL_MIXED_RHS, err
    assert rhs_error_raw(pb, q, R, R_cpu, fmax).max() > 1e-12  # FP32 arithmetic in use


def test_nonuniform_cfl_and_steps_match_oracle(mfc):
    """The paper's stretching on the small shock-bubble: CFL dt from the smallest
    cells and five SSP-RK3 steps."""
    wl = workloads.shock_bubble(24)
    faces = [workloads.stretched_faces(24, 0.0, 1.0, 4.0, 0.35, 0.65) for _ in range(3)]
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True, faces=faces)
    w = wl.prims()
    q = oracle.cons_from_prims(pb, w)
    s = mfc.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision="fp64", fallback=1)
    for d in range(3):
        s.set_grid(d, faces[d])
    s.set_state_prim(torch.from_numpy(w).cuda())
    for _ in range(5):
        dt = oracle.cfl_dt(pb, q, 0.3)
        assert s.cfl_dt(0.3) == pytest.approx(dt, rel=1e-13)
        q = oracle.rk3_step(pb, q, dt)
        s.step(dt)
    assert state_error(pb, s.get_state().cpu().numpy(), q).max() <= 1e-10


def test_nonuniform_bad_grids_are_rejected(mfc):
    gam, pin = workloads.fluids(2)
    s = mfc.Solver((8, 8), (0, 0), (1, 1), (0,) * 6, gam, pin, precision="fp64")
    with pytest.raises(mfc.MFCError):
        s.set_grid(0, np.linspace(0, 1, 8))            # wrong count
    with pytest.raises(mfc.MFCError):
        s.set_grid(2, np.linspace(0, 1, 2))            # inactive direction
    with pytest.raises(mfc.MFCError):
        s.set_grid(0, np.array([0, 1, 2, 1.5, 3, 4, 5, 6, 7.0]))   # not increasing
    s.set_grid(0, np.linspace(0, 1, 9) ** 1.2)
    with pytest.raises(mfc.MFCError):
        s.set_param("weno_order", 3)
    learned = mfc.Solver((8, 8), (0, 0), (1, 1), (0,) * 6, gam, pin, precision="learned")
    with pytest.raises(mfc.MFCError):
        learned.set_grid(0, np.linspace(0, 1, 9))
