"""Parity of the Kapila model (model 1: K div(u) in the volume-fraction rows,
Sec. 2.1) with the CPU FP64 oracle, through the C ABI; same metric and gates
as the Allaire-model tests."""
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


CASES = [
    # (n, nf, bc, weno_order)
    ((41,), 2, 1, 5),
    ((29, 17), 3, 0, 5),
    ((37, 23, 19), 2, 1, 5),
    ((21, 13, 11), 3, 2, 5),
    ((33, 18, 12), 2, 0, 3),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%s_nf%d_bc%d_w%d" % ("x".join(map(str, c[0])), *c[1:]))
def test_kapila_rhs_parity_fp64(mfc, case):
    n, nf, bc, order = case
    gam, pin = workloads.fluids(nf)
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (bc,) * 6, gam, pin, fallback=True, weno_order=order,
                        model="kapila")
    w = workloads.random_prims(n, nf, seed=60 + nf)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = mfc.Solver(pb.n, pb.lo, pb.hi, pb.bc, gam, pin, precision="fp64", fallback=1, weno_order=order, model=1)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy()
    assert rhs_error(pb, q, R, R_cpu, fmax).max() <= TOL_FP64
    # the K term is really there: the Allaire oracle differs in the alpha rows
    pa = oracle.Problem(n, (0,) * 3, (1,) * 3, (bc,) * 6, gam, pin, fallback=True, weno_order=order)
    assert rhs_error(pb, q, R, oracle.rhs(pa, q), fmax).max() > 1e3 * TOL_FP64


def test_kapila_mixed_rhs_close_to_oracle(mfc):
    n, nf = (37, 23, 19), 2
    gam, pin = workloads.fluids(nf)
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (1,) * 6, gam, pin, fallback=True, model="kapila")
    w = workloads.random_prims(n, nf, seed=64)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = mfc.Solver(pb.n, pb.lo, pb.hi, pb.bc, gam, pin, precision="mixed", fallback=1, model=1)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy()
    err = rhs_error(pb, q, R, R_cpu, fmax, unit=FP32_UNIT)
    assert err.max() <= TOL_MIXED_RHS, err
    assert rhs_error_raw(pb, q, R, R_cpu, fmax).max() > 1e-12  # FP32 arithmetic in use


def test_kapila_steps_match_oracle_on_shock_bubble(mfc):
    wl = workloads.shock_bubble(24)
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True, model="kapila")
    w = wl.prims()
    q = oracle.cons_from_prims(pb, w)
    s = mfc.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision="fp64", fallback=1, model=1)
    s.set_state_prim(torch.from_numpy(w).cuda())
    for _ in range(5):
        dt = oracle.cfl_dt(pb, q, 0.3)
        assert s.cfl_dt(0.3) == pytest.approx(dt, rel=1e-13)
        q = oracle.rk3_step(pb, q, dt)
        s.step(dt)
    assert state_error(pb, s.get_state().cpu().numpy(), q).max() <= 1e-10
    with pytest.raises(mfc.MFCError):
        s.set_param("model", 2)
