"""Parity of the third-order reconstruction (weno_order 3, Sec. 3.2) and of the
SSP-RK1/RK2 options of mfc_step (Sec. 3.4) with the CPU FP64 oracle, through
the C ABI.  Same metric and FP64 gate as the WENO5 parity tests."""
import numpy as np
import pytest

import oracle
import workloads
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


def _solver(mfc, pb, precision="fp64", **params):
    return mfc.Solver(pb.n, pb.lo, pb.hi, pb.bc, pb.gamma, pb.pi_inf, precision=precision, weno_eps=pb.eps,
                      fallback=1 if pb.fallback else 0, weno_order=3, **params)


CASES = [
    # (n, nf, bc, fallback, yz_kernel)
    ((37,), 2, 0, False, -1),
    ((41,), 1, 2, True, -1),
    ((29, 17), 2, 1, False, -1),
    ((23, 19), 3, 0, True, -1),
    ((37, 23, 19), 2, 1, False, -1),
    ((37, 23, 19), 2, 0, True, 1),
    ((21, 13, 11), 3, 2, False, -1),
    ((70, 33, 21), 2, 1, True, 1),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%s_nf%d_bc%d_fb%d_yz%d" % ("x".join(map(str, c[0])), *c[1:3], c[3], c[4]))
def test_weno3_rhs_parity_fp64(mfc, case):
    n, nf, bc, fb, yz = case
    gam, pin = workloads.fluids(nf)
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (bc,) * 6, gam, pin, fallback=fb, weno_order=3)
    w = workloads.random_prims(n, nf, seed=40 + nf)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = _solver(mfc, pb, yz_kernel=yz, segment=16 if n[-1] > 16 else 0)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy()
    err = rhs_error(pb, q, R, R_cpu, fmax)
    assert err.max() <= TOL_FP64, err
    # and it is the third-order scheme, not the fifth-order one
    R5 = oracle.rhs(oracle.Problem(n, (0,) * 3, (1,) * 3, (bc,) * 6, gam, pin, fallback=fb), q)
    assert rhs_error(pb, q, R, R5, fmax).max() > 1e3 * TOL_FP64


def test_weno3_shock_bubble_parity_fp64(mfc):
    wl = workloads.shock_bubble(40)
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True, weno_order=3)
    w = wl.prims()
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = _solver(mfc, pb)
    s.set_state_prim(torch.from_numpy(w).cuda())
    assert rhs_error(pb, q, s.rhs().cpu().numpy(), R_cpu, fmax).max() <= TOL_FP64


@pytest.mark.parametrize("n,nf", [((37, 23, 19), 2), ((21, 13, 11), 3), ((41,), 2)])
def test_weno3_mixed_rhs_close_to_fp64_oracle(mfc, n, nf):
    gam, pin = workloads.fluids(nf)
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (1,) * 6, gam, pin, fallback=True, weno_order=3)
    w = workloads.random_prims(n, nf, seed=23)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = _solver(mfc, pb, precision="mixed")
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy()
    err = rhs_error(pb, q, R, R_cpu, fmax, unit=FP32_UNIT)
    assert err.max() <= TOL_MIXED_RHS, err
    assert rhs_error_raw(pb, q, R, R_cpu, fmax).max() > 1e-12  # FP32 arithmetic in use


@pytest.mark.parametrize("rk_order,weno_order", [(1, 5), (2, 5), (2, 3), (3, 3)])
def test_rk_orders_and_weno3_steps_match_oracle(mfc, rk_order, weno_order):
    """Five steps of the chosen SSP-RK order on the small shock-bubble, with CFL
    time steps, against the oracle's rk_step."""
    wl = workloads.shock_bubble(24)
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True, weno_order=weno_order)
    w = wl.prims()
    q = oracle.cons_from_prims(pb, w)
    s = mfc.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision="fp64", fallback=1,
                   weno_order=weno_order, rk_order=rk_order)
    s.set_state_prim(torch.from_numpy(w).cuda())
    cfl = 0.3 if rk_order > 1 else 0.1
    for _ in range(5):
        dt = oracle.cfl_dt(pb, q, cfl)
        assert s.cfl_dt(cfl) == pytest.approx(dt, rel=1e-13)
        q = oracle.rk_step(pb, q, dt, rk_order)
        s.step(dt)
    err = state_error(pb, s.get_state().cpu().numpy(), q)
    assert err.max() <= 1e-10, err


def test_bad_orders_are_rejected(mfc):
    gam, pin = workloads.fluids(2)
    s = mfc.Solver((8, 8), (0, 0), (1, 1), (0,) * 6, gam, pin, precision="fp64")
    for name, value in (("weno_order", 4), ("weno_order", 1), ("rk_order", 4), ("rk_order", 0)):
        with pytest.raises(mfc.MFCError):
            s.set_param(name, value)
    learned = mfc.Solver((8, 8), (0, 0), (1, 1), (0,) * 6, gam, pin, precision="learned")
    with pytest.raises(mfc.MFCError):
        learned.set_param("weno_order", 3)
