"""CPU pins of the oracle's third-order variant (Sec. 3.2: the method also runs
with WENO3; (2k-1)th order from k = 2 candidates) and of the SSP Runge-Kutta
options of order 1 and 2 (Sec. 3.4).  Each pin is a closed form or an order of
accuracy, chosen so that a wrong candidate, ideal weight, smoothness indicator
or stencil orientation fails one of them."""
import math

import numpy as np
import pytest

import oracle
import workloads


def _cell_averages(F, N, shift=0.0):
    """Cell averages over [j h, (j+1) h] of the function with antiderivative F."""
    h = 1.0 / N
    x = np.arange(N) * h + shift
    return (F(x + h) - F(x)) / h, x + h


# ---------------------------------------------------------------- reconstruction
def test_weno3_candidates_and_value_exact_for_linear_data():
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = rng.normal(size=2)
        v = a + b * np.arange(3)           # cells i-1, i, i+1 at unit spacing
        edge = a + b * 1.5                 # the face between cells i and i+1
        om, cand = oracle.weno3_weights(v, 1e-6)
        assert np.allclose(cand, edge, rtol=0, atol=1e-14 * (abs(a) + abs(b)))
        assert oracle.weno3(v) == pytest.approx(edge, abs=1e-14 * (abs(a) + abs(b)))
        # linear data: equal smoothness indicators, so the ideal weights
        assert np.allclose(om, [1.0 / 3.0, 2.0 / 3.0], rtol=1e-12)


def test_weno3_linear_limit_exact_for_quadratics_not_cubics():
    """eps -> infinity gives the ideal-weight combination (-v0 + 5 v1 + 2 v2)/6:
    exact on cell averages of quadratics (third order), not on cubics."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        c = rng.normal(size=3)
        F = lambda x: c[0] * x + c[1] * x ** 2 / 2 + c[2] * x ** 3 / 3    # antiderivative of a quadratic
        f = lambda x: c[0] + c[1] * x + c[2] * x ** 2
        v = np.array([F(j + 1) - F(j) for j in range(3)])
        assert oracle.weno3(v, 1e30) == pytest.approx(f(2.0), rel=1e-12, abs=1e-12)
    v = np.array([((j + 1) ** 4 - j ** 4) / 4 for j in range(3)])            # cubic x^3
    assert abs(oracle.weno3(v, 1e30) - 8.0) > 1e-3


def test_weno3_eno_property_at_a_step():
    """A jump inside one candidate's stencil: the weight moves to the smooth one."""
    val = oracle.weno3([0.0, 0.0, 1.0])   # smooth candidate (i-1, i) -> 0
    assert abs(val) < 1e-10
    val = oracle.weno3([0.0, 1.0, 1.0])   # smooth candidate (i, i+1) -> 1
    assert val == pytest.approx(1.0, abs=1e-10)
    om, _ = oracle.weno3_weights([0.0, 1.0, 1.0], 1e-6)
    assert om[1] > 1 - 1e-10


@pytest.mark.parametrize("eps,order_max,order_l1", [(1e30, 2.95, 2.95), (1e-40, 1.95, 2.5)])
def test_weno3_face_value_order_on_smooth_data(eps, order_max, order_l1):
    """Face values from cell averages of sin(2 pi x): third order in the linear
    limit; WENO3-JS with a vanishing epsilon drops to second order at the
    extrema (the max norm) and stays above 2.5 in L1."""
    em, e1 = [], []
    for N in (64, 128, 256, 512):
        avg, xr = _cell_averages(lambda x: -np.cos(2 * np.pi * x) / (2 * np.pi), N)
        exact = np.sin(2 * np.pi * xr)
        vals = np.array([oracle.weno3(avg[[(i - 1) % N, i, (i + 1) % N]], eps) for i in range(N)])
        em.append(np.abs(vals - exact).max())
        e1.append(np.abs(vals - exact).mean())
    om = [math.log2(em[i] / em[i + 1]) for i in range(3)]
    o1 = [math.log2(e1[i] / e1[i + 1]) for i in range(3)]
    assert min(om) >= order_max, om
    assert min(o1) >= order_l1, o1


# ---------------------------------------------------------------- full RHS with WENO3
def _problem(n, nf=2, bc=0, seed=0, **kw):
    gam, pin = workloads.fluids(nf)
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (bc,) * 6, gam, pin, weno_order=3, **kw)
    return pb, oracle.cons_from_prims(pb, workloads.random_prims(n, nf, seed))


def test_weno3_uniform_state_has_zero_rhs():
    for bc in (0, 1, 2):
        gam, pin = workloads.fluids(2)
        pb = oracle.Problem((6, 5, 7), (0,) * 3, (1,) * 3, (bc,) * 6, gam, pin, weno_order=3)
        w = np.zeros(pb.shape())
        w[0], w[1], w[2:5], w[5], w[6] = 600.0, 0.4, 0.0 if bc == 2 else 13.0, 2e5, 0.6
        assert np.all(oracle.rhs(pb, oracle.cons_from_prims(pb, w)) == 0.0)


def test_weno3_periodic_conservation_and_mirror_symmetry():
    pb, q = _problem((10, 9, 8), seed=11)
    R = oracle.rhs(pb, q)
    for v in range(5):
        assert abs(R[v].sum()) <= 1e-13 * np.abs(R[v]).sum() + 1e-300
    pb, q = _problem((11, 6, 5), bc=1, seed=12)
    R = oracle.rhs(pb, q)
    qm = q[:, :, :, ::-1].copy()
    qm[2] *= -1
    Rm = oracle.rhs(pb, qm)[:, :, :, ::-1]
    Rm[2] *= -1
    scale = np.abs(R).reshape(7, -1).max(axis=1)[:, None, None, None]
    assert np.all(np.abs(Rm - R) <= 1e-12 * scale)


def test_weno3_volume_fraction_rhs_is_upwind_weno3_advection():
    """Uniform u > 0 and p: the alpha row is -u (alpha^L_{i+1/2} - alpha^L_{i-1/2})/dx
    with alpha^L the WENO3 value from cells i-1, i, i+1 (the left state)."""
    gam, pin = workloads.fluids(2)
    n = 16
    pb = oracle.Problem((n,), (0,), (1,), (0,) * 6, gam, pin, weno_order=3)
    x = (np.arange(n) + 0.5) / n
    a = 0.5 + 0.4 * np.sin(2 * np.pi * x) ** 3
    w = np.stack([a * 1000.0, (1 - a) * 1.0, np.full(n, 40.0), np.full(n, 1e5), a]).reshape(5, 1, 1, n)
    R = oracle.rhs(pb, oracle.cons_from_prims(pb, w))
    aL = np.array([oracle.weno3(a[[(i + k) % n for k in (-1, 0, 1)]], pb.eps) for i in range(n)])
    expect = -40.0 * (aL - np.roll(aL, 1)) * n
    assert np.allclose(R[4].ravel(), expect, rtol=1e-9, atol=1e-9 * np.abs(expect).max())
    # and it differs from the fifth-order scheme's
    R5 = oracle.rhs(oracle.Problem((n,), (0,), (1,), (0,) * 6, gam, pin), oracle.cons_from_prims(pb, w))
    assert np.abs(R5[4] - R[4]).max() > 1e-3 * np.abs(expect).max()


def test_weno3_single_fluid_third_order_where_eps_dominates():
    """Smooth periodic density wave (air), eps = 1e-6: once the smoothness
    indicators fall below eps the weights are the ideal ones and the scheme is
    third order (finest pair >= 2.9); an error in the ideal weights would leave
    it at first or second order."""
    errs = []
    for n in (32, 64, 128):
        pb = oracle.Problem((n,), (0,), (1,), (0,) * 6, (1.4,), (0.0,), eps=1e-6, weno_order=3)
        x = (np.arange(n) + 0.5) / n
        u0, p0, t_end, h = 1.0, 1.0, 0.1, 1.0 / n
        avg = lambda t: 1.0 + 0.2 * (np.cos(2 * np.pi * (x - h / 2 - u0 * t)) -
                                     np.cos(2 * np.pi * (x + h / 2 - u0 * t))) / (2 * np.pi * h)
        rho = avg(0.0)
        q = np.stack([rho, rho * u0, np.full(n, p0 / 0.4) + 0.5 * rho * u0 * u0]).reshape(3, 1, 1, n)
        steps = int(math.ceil(t_end / (0.2 * h)))
        for _ in range(steps):
            q = oracle.rk3_step(pb, q, t_end / steps)
        errs.append(np.abs(q[0].ravel() - avg(t_end)).mean())
    assert math.log2(errs[-2] / errs[-1]) >= 2.9, errs


# ---------------------------------------------------------------- SSP-RK options
@pytest.mark.parametrize("order", [1, 2, 3])
def test_ssp_rk_stability_polynomials(order):
    for z in (-0.3, 0.1, -1.7, 0.5):
        q1 = oracle.rk_step(None, np.array([1.0]), 1.0, order, rhs_fn=lambda s: z * s)
        expect = sum(z ** k / math.factorial(k) for k in range(order + 1))
        assert q1[0] == pytest.approx(expect, rel=1e-15)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_ssp_rk_order_on_nonlinear_ode(order):
    f = lambda s: -s * s  # y' = -y^2, y(0) = 1 -> y(1) = 1/2
    errs = []
    for m in (20, 40, 80, 160):
        y = np.array([1.0])
        for _ in range(m):
            y = oracle.rk_step(None, y, 1.0 / m, order, rhs_fn=f)
        errs.append(abs(y[0] - 0.5))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert min(orders) > order - 0.1, orders
