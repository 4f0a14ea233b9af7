"""Parity at full size: every FP64 form the bench times besides the headline
(which test_gpu_parity covers) on the 256^3 shock-bubble workloads in the
bench's launch configuration, and the FP64 and mixed forms on the 384^3 bubble
cloud and the 512^3 three-fluid workload.  The whole right-hand side runs on
the GPU; the oracle evaluates sampled cells (random cells, domain faces and
edges, the shock front, the interfaces).  The FP64 gate, and the mixed gate for
the mixed form."""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import FP32_UNIT, FP64_UNIT, rhs_table, sampled_rhs_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11
N = 256

# form: (workload builder, solver parameters, oracle options, six-equation state)
FORMS = {
    "fp64_weno3": (workloads.shock_bubble, {"weno_order": 3}, {"weno_order": 3}, False),
    "fp64_kapila": (workloads.shock_bubble, {"model": 1}, {"model": "kapila"}, False),
    "fp64_stretched": (workloads.shock_bubble_stretched, {}, {}, False),
    "fp64_cbc": (workloads.shock_bubble_cbc, {}, {}, False),
    "fp64_six": (workloads.shock_bubble, {"model": 2}, {"model": "six"}, True),
}


@pytest.fixture(scope="module")
def mfc():
    import paper_2305_09163_gb300 as m
    m.build()
    m.load()
    return m


def _cells(pb, shock_x):
    rng = np.random.default_rng(13)
    n = N
    pick = [rng.integers(0, pb.ncell, 1200)]
    for (x, y, z) in [(0, 0, 0), (n - 1, n - 1, n - 1), (0, 128, 128), (n - 1, 128, 128), (128, 0, 128),
                      (128, n - 1, 128), (128, 128, 0), (128, 128, n - 1), (128, 128, 128 + 25),
                      (128 + 26, 128, 128), (128, 102, 128)]:
        pick.append(np.array([(z * n + y) * n + x]))
    xs = rng.integers(max(0, shock_x - 5), shock_x + 6, 300)
    ys = rng.integers(0, n, 300)
    zs = rng.integers(0, n, 300)
    pick.append((zs * n + ys) * n + xs)
    return np.unique(np.concatenate(pick))


@pytest.mark.parametrize("form", list(FORMS))
def test_full_size_sampled_parity_of_each_form(mfc, form, capsys):
    build, params, opts, six = FORMS[form]
    wl = build(N)
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True, faces=wl.faces, **opts)
    w = wl.prims()
    if six:
        w = workloads.six_equation_prims(w, wl.nf)
    q = oracle.cons_from_prims(pb, w)
    s = mfc.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision="fp64", fallback=1, **params)
    if wl.faces is not None:
        for d in range(3):
            s.set_grid(d, wl.faces[d])
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy().reshape(pb.sys_size, -1)
    # the shock front: the first x cell whose centre lies beyond 0.05
    centers = 0.5 * (wl.faces[0][1:] + wl.faces[0][:-1]) if wl.faces is not None else (np.arange(N) + 0.5) / N
    cells = _cells(pb, int(np.searchsorted(centers, 0.05)))
    Rc, fmax = oracle.rhs_cells(pb, q, cells, return_fmax=True)
    err = sampled_rhs_error(pb, q, R, cells, Rc, fmax)
    with capsys.disabled():
        print("\n%s 256^3 FP64 RHS at %d sampled cells:\n" % (form, cells.size)
              + rhs_table(pb, q, R, Rc, fmax, cells=cells))
    assert err.max() <= TOL_FP64, (form, err)


def _sampled_check(mfc, wl, precision, tol, seed, capsys=None):
    pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, fallback=True)
    w = wl.prims()
    q = oracle.cons_from_prims(pb, w)
    s = mfc.Solver(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, precision=precision, fallback=1)
    s.set_state_prim(torch.from_numpy(w).cuda())
    R = s.rhs().cpu().numpy().reshape(pb.sys_size, -1)
    del s
    torch.cuda.empty_cache()
    n = wl.n[0]
    rng = np.random.default_rng(seed)
    # random cells, the domain's corners, and cells near the shock front (x < 0.05)
    pick = [rng.integers(0, pb.ncell, 1500), np.array([0, pb.ncell - 1, n - 1, pb.ncell - n])]
    xs = rng.integers(0, int(0.05 * n) + 6, 400)
    ys = rng.integers(0, n, 400)
    zs = rng.integers(0, n, 400)
    pick.append((zs * n + ys) * n + xs)
    # cells where the volume fractions vary (bubble interfaces, the solid slab's faces)
    a = w[pb.nf + pb.ndim + 1].reshape(-1)
    inter = np.flatnonzero((a > 0.01) & (a < 0.99))
    if inter.size:
        pick.append(rng.choice(inter, min(400, inter.size), replace=False))
    cells = np.unique(np.concatenate(pick))
    Rc, fmax = oracle.rhs_cells(pb, q, cells, return_fmax=True)
    unit = FP64_UNIT if precision == "fp64" else FP32_UNIT
    err = sampled_rhs_error(pb, q, R, cells, Rc, fmax, unit=unit)
    if capsys is not None:
        with capsys.disabled():
            print("\n%s %s RHS at %d sampled cells:\n" % (wl.name, precision, cells.size)
                  + rhs_table(pb, q, R, Rc, fmax, cells=cells, unit=unit))
    assert err.max() <= tol, (wl.name, precision, err)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("mixed", 2e-4)])
def test_full_size_bubble_cloud(mfc, precision, tol, capsys):
    """The 384^3 shock-bubble-cloud workload (64 air bubbles with lognormal
    radii in water, planar shock)."""
    _sampled_check(mfc, workloads.bubble_cloud(384), precision, tol, 17, capsys)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("mixed", 2e-4)])
def test_full_size_three_fluid(mfc, precision, tol, capsys):
    """The 512^3 three-fluid workload (water, an air bubble cloud and a stiff
    solid slab; ~10 GB per state array)."""
    _sampled_check(mfc, workloads.three_fluid(512), precision, tol, 19, capsys)
