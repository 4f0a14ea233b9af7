"""The algorithmic work per cell and sweep, counted on the oracle.

The oracle's source is compiled a second time with every double replaced by a
counting type (oracle/flop_count.h): the count is that of the plain textbook
formulation of Sec. 3.1-3.2 (WENO5-JS or WENO3-JS on every primitive variable
at both sides of a face, HLLC, the flux difference and the volume-fraction
source, primitive recovery once per cell), independent of how the CUDA kernels
fold it.  bench.py's roofline uses the stored counts; these tests recount them.
"""
import numpy as np
import pytest

import bench
import oracle
import workloads


def _problem(n, nf, bc=0, **kw):
    gam, pin = workloads.fluids(nf)
    return oracle.Problem(n, (0, 0, 0), (1, 1, 1), (bc,) * 6, gam, pin, fallback=False, **kw)


def test_counting_build_computes_the_same_rhs():
    """Only the arithmetic type changes: the right-hand side is bit for bit the
    plain build's."""
    pb = _problem((12, 10, 9), 2, bc=1)
    q = oracle.cons_from_prims(pb, workloads.random_prims(pb.n, 2, seed=5))
    count, R = oracle.rhs_flops(pb, q)
    assert count > 0
    assert np.array_equal(R, oracle.rhs(pb, q))


@pytest.mark.parametrize("variant,nf,kw", [("weno5", 2, {}), ("weno5", 3, {}), ("weno3", 2, {"weno_order": 3}),
                                           ("kapila", 2, {"model": "kapila"})])
def test_stored_counts_match_the_oracle(variant, nf, kw):
    pb = _problem((16, 16, 16), nf, **kw)
    q = oracle.cons_from_prims(pb, workloads.random_prims(pb.n, nf, seed=3))
    b = oracle.rhs_flop_breakdown(pb, q)
    assert b["per_cell_sweep"] == pytest.approx(bench.ORACLE_FLOP_PER_CELL_SWEEP[(variant, nf)], rel=1e-5)


def test_count_is_independent_of_grid_size_and_data():
    """Per unit the count does not depend on the number of cells, the boundary
    type or the state (the shock-bubble's faces are subsonic like the random
    state's, so HLLC takes star-region branches everywhere).  A handful of
    operations per direction (1/dx) add O(1/cells)."""
    a = oracle.rhs_flop_breakdown(_problem((16, 16, 16), 2),
                                  oracle.cons_from_prims(_problem((16, 16, 16), 2),
                                                         workloads.random_prims((16, 16, 16), 2, seed=3)))
    pb = _problem((20, 18, 16), 2, bc=1)
    b = oracle.rhs_flop_breakdown(pb, oracle.cons_from_prims(pb, workloads.random_prims(pb.n, 2, seed=4)))
    wl = workloads.shock_bubble(24)
    ps = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=False)
    c = oracle.rhs_flop_breakdown(ps, oracle.cons_from_prims(ps, wl.prims()))
    for k in ("prims", "face", "div", "per_cell_sweep"):
        assert a[k] == pytest.approx(b[k], rel=1e-4) == pytest.approx(c[k], rel=1e-4)


def test_count_decomposition_adds_up():
    """The parts: per face the WENO edges of all variables on both sides plus
    HLLC; WENO3 replaces only the reconstruction, so the per-face difference
    between WENO5 and WENO3 is 2 x sys_size times the per-edge difference, and
    the other parts are unchanged."""
    p5 = _problem((12, 12, 12), 2)
    p3 = _problem((12, 12, 12), 2, weno_order=3)
    q = oracle.cons_from_prims(p5, workloads.random_prims(p5.n, 2, seed=8))
    b5, b3 = oracle.rhs_flop_breakdown(p5, q), oracle.rhs_flop_breakdown(p3, q)
    assert b5["prims"] == b3["prims"] and b5["div"] == pytest.approx(b3["div"])
    per_edge = (b5["face"] - b3["face"]) / (2 * p5.sys_size)
    assert per_edge == pytest.approx(round(per_edge), abs=1e-6) and per_edge > 0
