"""The mixed form (FP32 reconstruction and HLLC; FP64 pressure recovery and RK
accumulation) against the FP64 oracle.  Its accuracy is measured, not a parity
claim: the gates bound the FP32 round-off the form is allowed to add."""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import FP32_UNIT, rhs_error, rhs_error_raw, state_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED_RHS = 2e-4


@pytest.fixture(scope="module")
def mfc():
    import paper_2305_09163_gb300 as m
    m.build()
    m.load()
    return m


@pytest.mark.parametrize("n,nf", [((37, 23, 19), 2), ((21, 13, 11), 3), ((41,), 2), ((29, 17), 2)])
def test_mixed_rhs_close_to_fp64_oracle(mfc, n, nf):
    gam, pin = workloads.fluids(nf)
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (1,) * 6, gam, pin, fallback=True)
    w = workloads.random_prims(n, nf, seed=21)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    s = mfc.Solver(pb.n, pb.lo, pb.hi, pb.bc, gam, pin, precision="mixed", fallback=1)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy()
    err = rhs_error(pb, q, R, R_cpu, fmax, unit=FP32_UNIT)
    print("mixed rhs err", n, nf, err)
    assert err.max() <= TOL_MIXED_RHS, err
    assert rhs_error_raw(pb, q, R, R_cpu, fmax).max() > 1e-12  # really computed in FP32


def test_mixed_steps_track_fp64_on_shock_bubble(mfc):
    wl = workloads.shock_bubble(32)
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True)
    w = wl.prims()
    q = oracle.cons_from_prims(pb, w)
    s = mfc.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision="mixed", fallback=1)
    s.set_state_prim(torch.from_numpy(w).cuda())
    for _ in range(10):
        dt = oracle.cfl_dt(pb, q, 0.3)
        q = oracle.rk3_step(pb, q, dt)
        s.step(dt)
    err = state_error(pb, s.get_state().cpu().numpy(), q)
    print("mixed state err after 10 steps", err)
    assert err.max() <= 1e-4, err
