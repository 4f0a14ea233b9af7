"""CPU pins of the oracle's non-uniform-grid WENO5 (Sec. 4.1; Listing 1's
per-index coefficient tables; Sec. 6.3's tanh stretching).  Each pin comes from
outside the generator: closed forms on a uniform grid, exactness for
polynomials on random non-uniform cells, the smoothness indicators against
Gauss quadrature of an independently built interpolant, symmetries, and the
order of accuracy of the whole scheme on a smoothly stretched grid."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import nonuniform as nu


def _avg(F, faces):
    """Cell averages of the function with antiderivative F over the cells of `faces`."""
    return (F(faces[1:]) - F(faces[:-1])) / np.diff(faces)


def test_uniform_tables_are_the_jiang_shu_constants():
    t = nu.cell_tables(np.full(5, 0.37))
    assert np.allclose(t["cL"] * 6, [[2, -7, 11, 0, 0], [0, -1, 5, 2, 0], [0, 0, 2, 5, -1]], atol=1e-12)
    assert np.allclose(t["cR"] * 6, [[-1, 5, 2, 0, 0], [0, 2, 5, -1, 0], [0, 0, 11, -7, 2]], atol=1e-12)
    assert np.allclose(t["dL"], [0.1, 0.6, 0.3], atol=1e-13) and np.allclose(t["dR"], [0.3, 0.6, 0.1], atol=1e-13)
    v = np.random.default_rng(0).standard_normal(5)
    b = [13 / 12 * (v[0] - 2 * v[1] + v[2]) ** 2 + 0.25 * (v[0] - 4 * v[1] + 3 * v[2]) ** 2,
         13 / 12 * (v[1] - 2 * v[2] + v[3]) ** 2 + 0.25 * (v[1] - v[3]) ** 2,
         13 / 12 * (v[2] - 2 * v[3] + v[4]) ** 2 + 0.25 * (3 * v[2] - 4 * v[3] + v[4]) ** 2]
    assert np.allclose([v @ t["B"][r] @ v for r in range(3)], b, rtol=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_non_uniform_exactness_for_polynomials(seed):
    """Each candidate reconstructs cell averages of quadratics exactly at both
    edges, the ideal-weight combination those of quartics, on random widths."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.3, 2.0, 5)
    faces = np.concatenate([[0.0], np.cumsum(h)])
    t = nu.cell_tables(h)
    xL, xR = faces[3], faces[2]
    for deg, check in ((2, "candidates"), (4, "ideal")):
        c = rng.standard_normal(deg + 1)
        F = lambda x, c=c: sum(c[k] * x ** (k + 1) / (k + 1) for k in range(len(c)))
        f = lambda x, c=c: sum(c[k] * x ** k for k in range(len(c)))
        v = _avg(F, faces)
        for side, xe in (("L", xL), ("R", xR)):
            cand = t["c" + side] @ v
            if check == "candidates":
                assert np.allclose(cand, f(xe), rtol=1e-10, atol=1e-10)
            else:
                assert t["d" + side] @ cand == pytest.approx(f(xe), rel=1e-10, abs=1e-10)


@pytest.mark.parametrize("seed", range(3))
def test_smoothness_indicators_match_quadrature(seed):
    """beta_r = sum_l dx_i^(2l-1) int_cell (p_r^(l))^2 from numpy's least-squares
    fit of the primitive function (exact: four points, a cubic) and
    Gauss-Legendre quadrature."""
    rng = np.random.default_rng(10 + seed)
    h = rng.uniform(0.5, 1.8, 5)
    faces = np.concatenate([[0.0], np.cumsum(h)])
    v = rng.standard_normal(5)
    t = nu.cell_tables(h)
    xg, wg = np.polynomial.legendre.leggauss(8)
    a, b = faces[2], faces[3]
    x = 0.5 * (b - a) * xg + 0.5 * (a + b)
    for r in range(3):
        fr = faces[r:r + 4]
        V = np.concatenate([[0.0], np.cumsum(v[r:r + 3] * h[r:r + 3])])
        P = np.polynomial.Polynomial.fit(fr, V, 3)
        beta = 0.0
        for l in (1, 2):
            dl = P.deriv(l + 1)
            beta += h[2] ** (2 * l - 1) * 0.5 * (b - a) * np.sum(wg * dl(x) ** 2)
        assert v @ t["B"][r] @ v == pytest.approx(beta, rel=1e-9)


def test_tables_scale_free_and_mirror_symmetric():
    rng = np.random.default_rng(4)
    h = rng.uniform(0.4, 1.6, 5)
    t, ts = nu.cell_tables(h), nu.cell_tables(7.5 * h)
    for k in ("cL", "cR", "dL", "dR", "B"):
        assert np.allclose(t[k], ts[k], rtol=1e-11, atol=1e-12)
    tm = nu.cell_tables(h[::-1])   # mirrored stencil: the left edge becomes the right one
    assert np.allclose(tm["cL"], t["cR"][::-1, ::-1], atol=1e-12)
    assert np.allclose(tm["dL"], t["dR"][::-1], atol=1e-12)


def test_paper_stretching_refines_near_the_droplet():
    """Sec. 6.3's mapping with a = 4, x_a = -1.2 D, x_b = 1.2 D on [-10 D, 10 D]:
    monotone, finer between x_a and x_b than near the ends."""
    f = workloads.stretched_faces(400, -10.0, 10.0, 4.0, -1.2, 1.2)
    h = np.diff(f)
    assert np.all(h > 0)
    mid = h[(f[:-1] > -1.0) & (f[1:] < 1.0)]
    assert mid.max() < 0.5 * h[:20].min()


def _wave_problem(n, amp):
    xi = np.linspace(0.0, 1.0, n + 1)
    faces = xi + amp * np.sin(2 * np.pi * xi) / (2 * np.pi)
    pb = oracle.Problem((n,), (0,), (1,), (0,) * 6, (1.4,), (0.0,), eps=1e-40, faces=[faces])
    return pb, faces


def test_stretched_grid_uniform_state_and_conservation():
    pb, faces = _wave_problem(24, 0.6)
    h = np.diff(faces)
    w = np.zeros(pb.shape())
    w[0], w[1], w[2] = 1.3, 20.0, 1e5
    # the table candidates sum to one only to rounding: R vanishes to rounding
    # of the flux scale (p + rho u^2)/dx_min
    R = oracle.rhs(pb, oracle.cons_from_prims(pb, w))
    assert np.abs(R).max() <= 1e-12 * (1e5 + 1.3 * 400.0) / h.min()
    gam, pin = workloads.fluids(2)
    f3 = [workloads.stretched_faces(n, 0.0, 1.0, 3.0, 0.4, 0.6) for n in (10, 9, 8)]
    pb3 = oracle.Problem((10, 9, 8), (0,) * 3, (1,) * 3, (0,) * 6, gam, pin, faces=f3)
    q = oracle.cons_from_prims(pb3, workloads.random_prims((10, 9, 8), 2, 11))
    R = oracle.rhs(pb3, q)
    vol = np.einsum("k,j,i->kji", np.diff(f3[2]), np.diff(f3[1]), np.diff(f3[0]))
    for v in range(5):
        assert abs((R[v] * vol).sum()) <= 1e-13 * np.abs(R[v] * vol).sum()


def test_stretched_grid_fifth_order_convergence():
    """Smooth periodic density wave (air) on x = xi + 0.6 sin(2 pi xi)/(2 pi)
    (cell widths vary by a factor 4): L1 order >= 4.5 with dt ~ dx^(5/3)."""
    errs = []
    for n in (16, 32, 64):
        pb, faces = _wave_problem(n, 0.6)
        u0, p0, t_end = 1.0, 1.0, 0.1
        F = lambda x, t: x - 0.2 * np.cos(2 * np.pi * (x - u0 * t)) / (2 * np.pi)
        rho = _avg(lambda x: F(x, 0.0), faces)
        q = np.stack([rho, rho * u0, np.full(n, p0 / 0.4) + 0.5 * rho * u0 * u0]).reshape(3, 1, 1, n)
        hmin = np.diff(faces).min()
        steps = int(math.ceil(t_end / (0.2 * hmin ** (5.0 / 3.0))))
        for _ in range(steps):
            q = oracle.rk3_step(pb, q, t_end / steps)
        errs.append((np.abs(q[0].ravel() - _avg(lambda x: F(x, t_end), faces)) * np.diff(faces)).sum())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] >= 4.5, (errs, orders)
