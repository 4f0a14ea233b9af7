"""Pins of the CPU FP64 oracle against facts fixed outside it.

Every check here compares the oracle with mathematics or published values it
does not itself compute: integral definitions, polynomial exactness, exact
Riemann solutions (Toro's printed tables), Rankine-Hugoniot conditions,
symmetries, conservation, pressure-velocity equilibrium and convergence orders.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads
from oracle.exact_riemann import Side, sample, shocked_state, star_densities, star_state, wave_speeds

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def ideal_problem(n=(8,), gamma=1.4, bc=None, **kw):
    nd = len([m for m in n if m > 1]) or 1
    bc = bc or (oracle.BC_PERIODIC,) * 6
    return oracle.Problem(n, (0, 0, 0), (1, 1, 1), bc, (gamma,), (0.0,), **kw)


# ---------------------------------------------------------------- EOS (Sec. 2.1)
def test_eos_single_stiffened_gas_matches_soe():
    """One fluid: rho E = (p + gamma pinf)/(gamma-1) + rho|u|^2/2 (Eq. soe with kinetic energy)."""
    g, pi = 4.4, 6.0e8
    pb = oracle.Problem((4, 4, 4), (0,) * 3, (1,) * 3, (0,) * 6, (g,), (pi,))
    w = np.array([1000.0, 3.0, -2.0, 5.0, 2.0e5])
    q = oracle.cons_from_prim_cell(pb, w)
    ke = 0.5 * 1000.0 * (9 + 4 + 25)
    assert q[4] == pytest.approx((2.0e5 + g * pi) / (g - 1.0) + ke, rel=1e-15)
    assert np.allclose(q[1:4], 1000.0 * w[1:4], rtol=1e-15)


def test_eos_mixture_is_sum_of_phase_energies_at_common_pressure():
    """Allaire mixture: rho e = sum_k alpha_k rho_k e_k(p) with each phase at the
    common pressure; each phase obeys its own stiffened-gas law."""
    rng = np.random.default_rng(1)
    gam, pin = (4.4, 1.4, 3.0), (6.0e8, 0.0, 1.0e10)
    pb = oracle.Problem((4, 4, 4), (0,) * 3, (1,) * 3, (0,) * 6, gam, pin)
    for _ in range(20):
        a = rng.dirichlet([2, 2, 2])
        rk = rng.uniform(1, 2000, 3)
        u = rng.uniform(-300, 300, 3)
        p = rng.uniform(1e4, 1e9)
        w = np.concatenate([a * rk, u, [p], a[:2]])
        q = oracle.cons_from_prim_cell(pb, w)
        rho = (a * rk).sum()
        e_phase = sum(a[k] * (p + gam[k] * pin[k]) / (gam[k] - 1.0) for k in range(3))
        assert q[6] == pytest.approx(e_phase + 0.5 * rho * (u ** 2).sum(), rel=1e-13)
        # and the inverse recovers p and u
        w2 = oracle.prim_from_cons_cell(pb, q)
        assert w2[6] == pytest.approx(p, rel=1e-6, abs=1e-6 * 7.8e8)
        assert np.allclose(w2[3:6], u, rtol=1e-12, atol=1e-9)


def test_sound_speed_is_isentropic_derivative_of_mixture_eos():
    """c^2 = dp/drho at fixed volume fractions and entropy, by finite differences:
    dp = (dp/drho)_e drho + (dp/de)_rho de with de = p/rho^2 drho."""
    gam, pin = (4.4, 1.4), (6.0e8, 0.0)
    pb = oracle.Problem((1, 1, 1), (0,) * 3, (1,) * 3, (1,) * 6, gam, pin)
    for a1 in (0.3, 0.9, 1e-6):
        rk = np.array([1000.0, 1.2])
        p = 3.0e5
        w = np.array([a1 * rk[0], (1 - a1) * rk[1], 0.0, p, a1])
        q = oracle.cons_from_prim_cell(pb, w)
        rho = q[0] + q[1]
        e = q[3] / rho
        def p_of(r, ee):
            qq = q.copy()
            qq[0:2] = q[0:2] * (r / rho)
            qq[3] = r * ee
            return oracle.prim_from_cons_cell(pb, qq)[3]
        h = 1e-4 * rho
        dpdr = (p_of(rho + h, e) - p_of(rho - h, e)) / (2 * h)
        he = 1e-4 * e
        dpde = (p_of(rho, e + he) - p_of(rho, e - he)) / (2 * he)
        c2_fd = dpdr + p / rho ** 2 * dpde
        qa = q.reshape(5, 1, 1, 1)
        rate, bad = oracle.max_rate(pb, qa)
        assert bad == 0
        assert rate ** 2 == pytest.approx(c2_fd, rel=1e-6)


# ---------------------------------------------------------------- WENO5 (Sec. 3.2)
def _cell_averages(coefs, centers, h):
    """Cell averages of the polynomial sum c_k x^k over [x-h/2, x+h/2]."""
    P = np.polynomial.polynomial.Polynomial(coefs).integ()
    return (P(centers + h / 2) - P(centers - h / 2)) / h


def test_weno5_exact_for_quadratics():
    rng = np.random.default_rng(2)
    h = 0.1
    xc = np.arange(-2, 3) * h
    for _ in range(50):
        c = rng.normal(size=3)
        v = _cell_averages(c, xc, h)
        exact = np.polynomial.polynomial.polyval(h / 2, c)
        for eps in (1e-6, 1e-30, 1e3):
            assert oracle.weno5(v, eps) == pytest.approx(exact, abs=1e-13)
            om, cand = oracle.weno5_weights(v, eps)
            assert np.allclose(cand, exact, atol=1e-13)
            assert om.sum() == pytest.approx(1.0, abs=1e-15)


def test_weno5_linear_limit_exact_for_quartics():
    """With epsilon dominant the weights become the ideal ones and WENO5 is the
    fifth-order linear interpolant: exact on cell averages of degree-4 data."""
    rng = np.random.default_rng(3)
    h = 0.05
    xc = np.arange(-2, 3) * h
    for _ in range(30):
        c = rng.normal(size=5)
        v = _cell_averages(c, xc, h)
        exact = np.polynomial.polynomial.polyval(h / 2, c)
        om, _ = oracle.weno5_weights(v, 1e30)
        assert np.allclose(om, [0.1, 0.6, 0.3], atol=1e-14)
        assert oracle.weno5(v, 1e30) == pytest.approx(exact, abs=1e-12)


def test_weno5_beta_matches_integral_definition():
    """beta_r = sum_{l=1,2} h^(2l-1) int_cell (d^l p_r/dx^l)^2 dx with p_r the
    quadratic whose cell averages match stencil r (Jiang & Shu 1996)."""
    rng = np.random.default_rng(4)
    h = 1.0
    for _ in range(30):
        v = rng.normal(size=5)
        beta = oracle.weno5_beta(v)
        for r, cells in enumerate(([-2, -1, 0], [-1, 0, 1], [0, 1, 2])):
            A = np.zeros((3, 3))
            for i, j in enumerate(cells):
                for k in range(3):
                    A[i, k] = ((j + 0.5) ** (k + 1) - (j - 0.5) ** (k + 1)) / (k + 1)
            coef = np.linalg.solve(A, v[np.array(cells) + 2])
            poly = np.polynomial.polynomial.Polynomial(coef)
            tot = 0.0
            for l in (1, 2):
                d = poly.deriv(l)
                I = (d * d).integ()
                tot += h ** (2 * l - 1) * (I(0.5) - I(-0.5))
            assert beta[r] == pytest.approx(tot, rel=1e-12, abs=1e-12)


def test_weno5_eno_property_at_a_step():
    """A stencil crossing a jump gets a vanishing weight; the value stays between
    the neighbouring cell values (no new extremum at a step)."""
    v = np.array([1.0, 1.0, 1.0, 0.0, 0.0])
    om, _ = oracle.weno5_weights(v, 1e-6)
    assert om[1] < 1e-10 and om[2] < 1e-10
    assert oracle.weno5(v, 1e-6) == pytest.approx(1.0, abs=1e-10)
    v = np.array([0.0, 0.0, 1.0, 1.0, 1.0])
    assert -1e-10 <= oracle.weno5(v, 1e-6) <= 1.0 + 1e-10


def test_weno5_fifth_order_on_smooth_data():
    errs = []
    ns = [16, 32, 64, 128, 256]
    for n in ns:
        h = 1.0 / n
        xc = (np.arange(n) + 0.5) * h
        avg = (np.cos(2 * np.pi * (xc - h / 2)) - np.cos(2 * np.pi * (xc + h / 2))) / (2 * np.pi * h)
        e = 0.0
        for i in range(n):
            v = avg[[(i + k) % n for k in range(-2, 3)]]
            e = max(e, abs(oracle.weno5(v, 1e-40) - math.sin(2 * np.pi * (xc[i] + h / 2))))
        errs.append(e)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    assert orders[-1] >= 4.8 and orders[-2] >= 4.5, orders


# ---------------------------------------------------------------- HLLC (Sec. 3.2.1)
def _euler_flux(rho, u, p, g):
    E = p / (g - 1) + 0.5 * rho * u * u
    return np.array([rho * u, rho * u * u + p, (E + p) * u])


def test_hllc_consistency():
    pb = ideal_problem()
    rng = np.random.default_rng(5)
    for _ in range(20):
        rho, u, p = rng.uniform(0.1, 3), rng.uniform(-2, 2), rng.uniform(0.1, 3)
        w = np.array([rho, u, p])
        F, ut = oracle.hllc(pb, 0, w, w)
        assert np.allclose(F, _euler_flux(rho, u, p, 1.4), rtol=1e-14, atol=1e-14)
        assert ut == pytest.approx(u, rel=1e-14, abs=1e-15)


def test_hllc_star_states_satisfy_rankine_hugoniot():
    """HLLC star states (Toro Sec. 10.4): across each outer wave s_K the star state
    has velocity s* and a common pressure p* = p_K + rho_K (s_K-u_K)(s*-u_K), and
    the interface flux equals the Euler flux of that star state."""
    g = 1.4
    pb = ideal_problem(gamma=g)
    rng = np.random.default_rng(6)
    checked = 0
    for _ in range(200):
        wL = np.array([rng.uniform(0.2, 2), rng.uniform(-1, 1), rng.uniform(0.2, 2)])
        wR = np.array([rng.uniform(0.2, 2), rng.uniform(-1, 1), rng.uniform(0.2, 2)])
        F, ut = oracle.hllc(pb, 0, wL, wR)
        cL, cR = math.sqrt(g * wL[2] / wL[0]), math.sqrt(g * wR[2] / wR[0])
        sL = min(wL[1] - cL, wR[1] - cR)
        sR = max(wL[1] + cL, wR[1] + cR)
        if not (sL < 0 < sR):
            continue
        # The interface lies in one star region.  Recover the star state of each
        # side from F; the pressure p* of the Rankine-Hugoniot relations follows
        # from the momentum flux (it is not the EOS pressure of the star state).
        ok = []
        for (w, s) in ((wL, sL), (wR, sR)):
            qK = np.array([w[0], w[0] * w[1], w[2] / (g - 1) + 0.5 * w[0] * w[1] ** 2])
            qs = qK + (F - _euler_flux(w[0], w[1], w[2], g)) / s
            rs, us = qs[0], qs[1] / qs[0]
            ps = F[1] - rs * us * us
            good = (abs(F[0] - rs * us) <= 1e-11 * (1 + abs(F[0]))
                    and abs(F[2] - (qs[2] + ps) * us) <= 1e-10 * (1 + abs(F[2]))
                    and abs(ps - (w[2] + w[0] * (s - w[1]) * (us - w[1]))) <= 1e-10 * (1 + abs(ps))
                    and abs(rs - w[0] * (s - w[1]) / (s - us)) <= 1e-10 * rs
                    and ((us >= 0) == (s < 0)))
            ok.append((good, us, ps))
        assert ok[0][0] != ok[1][0], ok
        _, us, ps = ok[0] if ok[0][0] else ok[1]
        # both outer waves see the same star pressure and velocity
        for (w, s) in ((wL, sL), (wR, sR)):
            assert ps == pytest.approx(w[2] + w[0] * (s - w[1]) * (us - w[1]), rel=1e-9)
        checked += 1
    assert checked > 50


def test_hllc_resolves_isolated_contacts_exactly():
    """A material interface with equal p and u is an exact HLLC solution: the
    flux is the upwind physical flux and the face velocity is u."""
    gam, pin = (4.4, 1.4), (6.0e8, 0.0)
    pb = oracle.Problem((4, 1, 1), (0,) * 3, (1,) * 3, (1,) * 6, gam, pin)
    for u in (0.0, 37.5, -12.25):
        p = 1.0e5
        wL = np.array([999.0, 1e-3 * 1.0, u, p, 0.999])
        wR = np.array([1e-3, 0.999, u, p, 1e-6])
        F, ut = oracle.hllc(pb, 0, wL, wR)
        up = wL if u >= 0 else wR
        Fup, _ = oracle.hllc(pb, 0, up, up)
        assert ut == u
        assert np.allclose(F, Fup, rtol=1e-13, atol=1e-9)
        if u == 0.0:
            assert F[0] == 0 and F[1] == 0 and F[3] == 0 and F[4] == 0
            assert F[2] == pytest.approx(p, rel=1e-15)


def test_hllc_mirror_symmetry_and_rotation():
    gam, pin = (4.4, 1.4), (6.0e8, 0.0)
    pb = oracle.Problem((4, 4, 4), (0,) * 3, (1,) * 3, (0,) * 6, gam, pin)
    rng = np.random.default_rng(7)
    for _ in range(20):
        def rnd():
            a = rng.uniform(0.05, 0.95)
            return np.array([a * rng.uniform(500, 1500), (1 - a) * rng.uniform(0.5, 2),
                             *rng.uniform(-200, 200, 3), rng.uniform(1e5, 1e8), a])
        wL, wR = rnd(), rnd()
        F, ut = oracle.hllc(pb, 0, wL, wR)
        mL, mR = wR.copy(), wL.copy()
        mL[2] *= -1
        mR[2] *= -1
        Fm, um = oracle.hllc(pb, 0, mL, mR)
        sign = np.array([-1, -1, 1, -1, -1, -1, -1])
        assert np.allclose(Fm, sign * F, rtol=1e-12, atol=1e-12 * np.abs(F).max())
        assert um == pytest.approx(-ut, rel=1e-12, abs=1e-12)
        # rotation: normal y with (u, v, w) -> (w, u, v) equals normal x
        perm = np.array([0, 1, 4, 2, 3, 5, 6])  # y-state whose v equals the x-state's u
        Fy, uy = oracle.hllc(pb, 1, wL[perm], wR[perm])
        assert np.allclose(Fy, F[perm], rtol=1e-13, atol=1e-13 * np.abs(F).max())
        assert uy == pytest.approx(ut, rel=1e-13)


def test_two_identical_fluids_reduce_to_one():
    """Two fluids with the same EOS reproduce the single-fluid flux (sum of partial
    mass fluxes = mass flux; momentum and energy identical)."""
    g, pi = 1.4, 0.0
    pb2 = oracle.Problem((4, 1, 1), (0,) * 3, (1,) * 3, (1,) * 6, (g, g), (pi, pi))
    pb1 = oracle.Problem((4, 1, 1), (0,) * 3, (1,) * 3, (1,) * 6, (g,), (pi,))
    rng = np.random.default_rng(8)
    for _ in range(20):
        aL, aR = rng.uniform(0.1, 0.9, 2)
        rL, rR = rng.uniform(0.2, 2, 2)
        wL2 = np.array([aL * rL, (1 - aL) * rL, rng.uniform(-1, 1), rng.uniform(0.2, 2), aL])
        wR2 = np.array([aR * rR, (1 - aR) * rR, rng.uniform(-1, 1), rng.uniform(0.2, 2), aR])
        F2, _ = oracle.hllc(pb2, 0, wL2, wR2)
        F1, _ = oracle.hllc(pb1, 0, np.array([rL, wL2[2], wL2[3]]), np.array([rR, wR2[2], wR2[3]]))
        assert F2[0] + F2[1] == pytest.approx(F1[0], rel=1e-12, abs=1e-14)
        assert np.allclose(F2[2:4], F1[1:3], rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- exact Riemann solver
def _golden_toro():
    rows = []
    with open(os.path.join(GOLDEN, "toro_exact_riemann.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            left, right = line.split("|")
            a = [float(x) for x in left.split()]
            b = [float(x) for x in right.split()]
            rows.append((a, b))
    return rows


@pytest.mark.parametrize("row", _golden_toro(), ids=lambda r: "toro%d" % int(r[0][0]))
def test_exact_riemann_matches_toro_tables(row):
    a, b = row
    L = Side(a[1], a[2], a[3], 1.4)
    R = Side(a[4], a[5], a[6], 1.4)
    p, u = star_state(L, R)
    rl, rr = star_densities(L, R, p)
    for got, want in ((p, b[0]), (u, b[1]), (rl, b[2]), (rr, b[3])):
        assert got == pytest.approx(want, rel=2e-5, abs=1e-5)


def test_exact_riemann_two_materials_satisfies_jump_conditions():
    """Water (4.4, 6e8) at 1e9 Pa against air at 1e5 Pa: the right shock obeys
    Rankine-Hugoniot, the left rarefaction keeps (p+pinf)/rho^g and
    u + 2c/(g-1) constant, and p, u are continuous at the contact."""
    L = Side(1000.0, 0.0, 1e9, 4.4, 6e8)
    R = Side(1.0, 0.0, 1e5, 1.4, 0.0)
    p, u = star_state(L, R)
    rl, rr = star_densities(L, R, p)
    hL, tL, tR, hR = wave_speeds(L, R, p, u)
    # shock into air, speed S
    S = hR
    m = R.rho * (R.u - S)
    assert rr * (u - S) == pytest.approx(m, rel=1e-12)
    assert rr * (u - S) ** 2 + p == pytest.approx(R.rho * (R.u - S) ** 2 + R.p, rel=1e-12)
    eR = (R.p + R.gamma * R.pinf) / ((R.gamma - 1) * R.rho)
    es = (p + R.gamma * R.pinf) / ((R.gamma - 1) * rr)
    # energy flux in the shock frame: m (e + v^2/2) + p v with v = u - S
    lhs = rr * (u - S) * (es + 0.5 * (u - S) ** 2) + p * (u - S)
    rhs = R.rho * (R.u - S) * (eR + 0.5 * (R.u - S) ** 2) + R.p * (R.u - S)
    assert lhs == pytest.approx(rhs, rel=1e-10)
    # rarefaction in water
    g = L.gamma
    assert (p + L.pinf) / rl ** g == pytest.approx(L.P / L.rho ** g, rel=1e-12)
    cs = math.sqrt(g * (p + L.pinf) / rl)
    assert u + 2 * cs / (g - 1) == pytest.approx(L.u + 2 * L.c / (g - 1), rel=1e-12)
    # fan samples lie on the same invariants
    rho, uu, pp, _ = sample(L, R, np.linspace(hL, tL, 7)[1:-1])
    for r_, u_, p_ in zip(rho, uu, pp):
        assert (p_ + L.pinf) / r_ ** g == pytest.approx(L.P / L.rho ** g, rel=1e-10)
        c_ = math.sqrt(g * (p_ + L.pinf) / r_)
        assert u_ + 2 * c_ / (g - 1) == pytest.approx(L.u + 2 * L.c / (g - 1), rel=1e-10)


def test_workload_shock_constants_match_oracle():
    from oracle.shock_constants import post_shock_water
    rho, u, s = post_shock_water()
    assert workloads.SHOCK_RHO == pytest.approx(rho, rel=1e-14)
    assert workloads.SHOCK_U == pytest.approx(u, rel=1e-14)
    assert workloads.SHOCK_SPEED == pytest.approx(s, rel=1e-14)


# ---------------------------------------------------------------- full RHS (Sec. 3.1)
def _random_problem(n, nf=2, bc=0, seed=0, water_air=True, **kw):
    gam, pin = workloads.fluids(nf, water_air)
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (bc,) * 6, gam, pin, **kw)
    w = workloads.random_prims(n, nf, seed, water_air=water_air)
    return pb, oracle.cons_from_prims(pb, w)


def test_uniform_state_has_zero_rhs():
    for bc in (0, 1, 2):
        gam, pin = workloads.fluids(2)
        pb = oracle.Problem((6, 5, 7), (0,) * 3, (1,) * 3, (bc,) * 6, gam, pin)
        w = np.zeros(pb.shape())
        w[0], w[1], w[2:5], w[5], w[6] = 600.0, 0.4, 0.0 if bc == 2 else 13.0, 2e5, 0.6
        q = oracle.cons_from_prims(pb, w)
        R = oracle.rhs(pb, q)
        assert np.all(R == 0.0)


def test_axis_permutation_gives_identical_rhs():
    """A 1D profile laid along x, y or z gives the same R (bitwise)."""
    n = 12
    gam, pin = workloads.fluids(2)
    w1 = workloads.random_prims((n,), 2, 9)  # 1D: [5][1][1][n]
    Rs = []
    for d in range(3):
        nn = [3, 3, 3]
        nn[d] = n
        pb = oracle.Problem(nn, (0,) * 3, (1,) * 3, (0,) * 6, gam, pin)
        w = np.zeros(pb.shape())
        prof = w1[:, 0, 0, :]
        shape = [1, 1, 1]
        shape[2 - d] = n
        for v_src, v_dst in ((0, 0), (1, 1), (3, 5), (4, 6)):
            w[v_dst] = prof[v_src].reshape(shape)
        w[2 + d] = prof[2].reshape(shape)
        R = oracle.rhs(pb, oracle.cons_from_prims(pb, w))
        sl = [0, 0, 0]
        sl[2 - d] = slice(None)
        Rd = np.stack([R[v][tuple(sl)] for v in (0, 1, 2 + d, 5, 6)])
        others = [2 + e for e in range(3) if e != d]
        assert np.all(R[others] == 0.0)
        Rs.append(Rd)
    assert np.array_equal(Rs[0], Rs[1]) and np.array_equal(Rs[0], Rs[2])


def test_rhs_cells_matches_full_rhs():
    pb, q = _random_problem((9, 7, 8), nf=3, bc=1, seed=10)
    R = oracle.rhs(pb, q)
    cells = np.array([0, 5, 77, 200, pb.ncell - 1])
    Rc = oracle.rhs_cells(pb, q, cells)
    assert np.array_equal(Rc, R.reshape(pb.sys_size, -1)[:, cells].T)


def test_periodic_conservation():
    pb, q = _random_problem((10, 9, 8), nf=2, bc=0, seed=11)
    R, fmax, _ = oracle.rhs(pb, q, return_info=True)
    for v in range(5):  # partial masses, momentum, energy
        s = R[v].sum()
        assert abs(s) <= 1e-13 * np.abs(R[v]).sum() + 1e-300, (v, s)


def test_mirror_symmetry_of_rhs():
    pb, q = _random_problem((11, 6, 5), nf=2, bc=1, seed=12)
    R = oracle.rhs(pb, q)
    qm = q[:, :, :, ::-1].copy()
    qm[2] *= -1
    Rm = oracle.rhs(pb, qm)
    Rm = Rm[:, :, :, ::-1]
    Rm[2] *= -1
    scale = np.abs(R).reshape(7, -1).max(axis=1)[:, None, None, None]
    assert np.all(np.abs(Rm - R) <= 1e-12 * scale)


def test_reflective_walls_equal_mirrored_periodic_domain():
    """Reflective walls at both ends = the middle of a periodic domain built from the
    state and its mirror image (u_x negated)."""
    gam, pin = workloads.fluids(2)
    n = 10
    w = workloads.random_prims((n, 4, 3), 2, 13)
    pbr = oracle.Problem((n, 4, 3), (0,) * 3, (1,) * 3, (2, 2, 0, 0, 0, 0), gam, pin)
    R = oracle.rhs(pbr, oracle.cons_from_prims(pbr, w))
    wm = w[:, :, :, ::-1].copy()
    wm[2] *= -1
    wp = np.concatenate([wm, w], axis=3)
    pbp = oracle.Problem((2 * n, 4, 3), (-1, 0, 0), (1, 1, 1), (0,) * 6, gam, pin)
    Rp = oracle.rhs(pbp, oracle.cons_from_prims(pbp, wp))[:, :, :, n:]
    scale = np.abs(R).reshape(7, -1).max(axis=1)[:, None, None, None]
    assert np.all(np.abs(Rp - R) <= 1e-13 * scale)


def test_transmissive_ghosts_equal_padded_domain():
    gam, pin = workloads.fluids(2)
    n = 9
    w = workloads.random_prims((n, 3, 3), 2, 14)
    pbt = oracle.Problem((n, 3, 3), (0,) * 3, (1,) * 3, (1, 1, 0, 0, 0, 0), gam, pin)
    R = oracle.rhs(pbt, oracle.cons_from_prims(pbt, w))
    pad = 6
    wpad = np.concatenate([np.repeat(w[:, :, :, :1], pad, axis=3), w,
                           np.repeat(w[:, :, :, -1:], pad, axis=3)], axis=3)
    h = 1.0 / n
    pbp = oracle.Problem((n + 2 * pad, 3, 3), (-pad * h, 0, 0), (1 + pad * h, 1, 1), (0,) * 6, gam, pin)
    Rp = oracle.rhs(pbp, oracle.cons_from_prims(pbp, wpad))[:, :, :, pad:pad + n]
    scale = np.abs(R).reshape(7, -1).max(axis=1)[:, None, None, None]
    assert np.all(np.abs(Rp - R) <= 1e-12 * scale)


def test_volume_fraction_rhs_is_upwind_weno_advection():
    """Uniform u > 0 and p: every face is an upwind contact, so the alpha row is
    -u (alpha^L_{i+1/2} - alpha^L_{i-1/2})/dx with alpha^L from WENO5."""
    gam, pin = workloads.fluids(2)
    n = 16
    pb = oracle.Problem((n,), (0,), (1,), (0,) * 6, gam, pin)
    x = (np.arange(n) + 0.5) / n
    a = 0.5 + 0.4 * np.sin(2 * np.pi * x) ** 3
    w = np.stack([a * 1000.0, (1 - a) * 1.0, np.full(n, 40.0), np.full(n, 1e5), a]).reshape(5, 1, 1, n)
    R = oracle.rhs(pb, oracle.cons_from_prims(pb, w))
    aL = np.array([oracle.weno5(a[[(i + k) % n for k in range(-2, 3)]], pb.eps) for i in range(n)])
    expect = -40.0 * (aL - np.roll(aL, 1)) * n
    assert np.allclose(R[4].ravel(), expect, rtol=1e-9, atol=1e-9 * np.abs(expect).max())


@pytest.mark.parametrize("width,fallback", [(2.0, False), (1.0, True)])
def test_pressure_velocity_equilibrium_across_advected_interface(width, fallback):
    """Water/air interface advected at u = (100, 50, 25) m/s in uniform p = 1e5 Pa,
    periodic: p and u stay uniform (to round-off) over 200 SSP-RK3 steps.  A
    one-cell tanh interface needs the first-order fallback to keep the partial
    densities positive; the fallback keeps the equilibrium too."""
    gam, pin = workloads.fluids(2)
    n = 12
    pb = oracle.Problem((n, n, n), (0,) * 3, (1,) * 3, (0,) * 6, gam, pin, fallback=fallback)
    g = np.meshgrid(*[(np.arange(n) + 0.5) / n] * 3, indexing="ij")
    r = np.sqrt((g[2] - 0.5) ** 2 + (g[1] - 0.5) ** 2 + (g[0] - 0.5) ** 2)
    a_air = 1e-6 + (1 - 2e-6) * 0.5 * (1 - np.tanh((r - 0.25) * n / width))
    a_w = 1 - a_air
    u0 = (100.0, 50.0, 25.0)
    w = np.stack([a_w * 1000.0, a_air * 1.0, np.full_like(r, u0[0]), np.full_like(r, u0[1]),
                  np.full_like(r, u0[2]), np.full_like(r, 1e5), a_w])
    q = oracle.cons_from_prims(pb, w)
    for _ in range(200):
        dt = oracle.cfl_dt(pb, q, 0.3)
        q = oracle.rk3_step(pb, q, dt)
    wp = oracle.prims_from_cons(pb, q)
    assert np.abs(wp[5] / 1e5 - 1).max() <= 1e-8
    for d in range(3):
        assert np.abs(wp[2 + d] - u0[d]).max() / abs(u0[d]) <= 1e-8
    # the interface really moved and stayed bounded
    assert np.abs(wp[6] - w[6]).max() > 0.1
    assert wp[6].min() > -1e-3 and wp[6].max() < 1 + 1e-3


# ---------------------------------------------------------------- RK3 and CFL (Sec. 3.4)
def test_ssp_rk3_stability_polynomial():
    for z in (-0.3, 0.1, -1.7, 0.5):
        lam, dt = z, 1.0
        q1 = oracle.rk3_step(None, np.array([1.0]), dt, rhs_fn=lambda s: lam * s)
        assert q1[0] == pytest.approx(1 + z + z * z / 2 + z ** 3 / 6, rel=1e-15)


def test_ssp_rk3_third_order_on_nonlinear_ode():
    f = lambda s: -s * s  # y' = -y^2, y(0)=1 -> y = 1/(1+t)
    errs = []
    for m in (10, 20, 40, 80):
        y = np.array([1.0])
        for _ in range(m):
            y = oracle.rk3_step(None, y, 1.0 / m, rhs_fn=f)
        errs.append(abs(y[0] - 0.5))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert min(orders) > 2.9, orders


def test_cfl_time_step():
    g, pi = 4.4, 6.0e8
    pb = oracle.Problem((2, 3, 1), (0, 0, 0), (1, 2, 1), (1,) * 6, (g,), (pi,))
    w = np.zeros(pb.shape())
    w[0] = 1000.0
    w[1] = 10.0
    w[2] = -300.0
    w[3] = 1e5
    w[1, 0, 1, 1] = 50.0
    q = oracle.cons_from_prims(pb, w)
    c = math.sqrt(g * (1e5 + pi) / 1000.0)
    expect = max((50.0 + c) / 0.5, (300.0 + c) / (2 / 3))
    assert oracle.cfl_dt(pb, q, 0.3) == pytest.approx(0.3 / expect, rel=1e-14)


# ---------------------------------------------------------------- whole method
def test_single_fluid_smooth_convergence_order():
    """Smooth periodic density wave (air): L1 order >= 4.5 with dt ~ dx^(5/3)."""
    errs = []
    ns = (16, 32, 64)
    for n in ns:
        pb = oracle.Problem((n,), (0,), (1,), (0,) * 6, (1.4,), (0.0,), eps=1e-40)
        x = (np.arange(n) + 0.5) / n
        u0, p0, t_end = 1.0, 1.0, 0.1
        h = 1.0 / n
        avg = lambda t: 1.0 + 0.2 * (np.cos(2 * np.pi * (x - h / 2 - u0 * t)) -
                                     np.cos(2 * np.pi * (x + h / 2 - u0 * t))) / (2 * np.pi * h)
        # conserved cell averages of the exact solution (linear in rho at constant u, p)
        rho = avg(0.0)
        q = np.stack([rho, rho * u0, np.full(n, p0 / 0.4) + 0.5 * rho * u0 * u0]).reshape(3, 1, 1, n)
        steps = int(math.ceil(t_end / (0.2 * h ** (5.0 / 3.0))))
        dt = t_end / steps
        for _ in range(steps):
            q = oracle.rk3_step(pb, q, dt)
        errs.append(np.abs(q[0].ravel() - avg(t_end)).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    assert orders[-1] >= 4.5, (errs, orders)


def _l1(a, b):
    return np.abs(a - b).mean() / np.abs(b).mean()


def test_sod_converges_to_exact_solution():
    errs = []
    for n in (100, 400):
        pb = oracle.Problem((n,), (0,), (1,), (1,) * 6, (1.4,), (0.0,))
        x = (np.arange(n) + 0.5) / n
        left = x < 0.5
        w = np.stack([np.where(left, 1.0, 0.125), np.zeros(n), np.where(left, 1.0, 0.1)]).reshape(3, 1, 1, n)
        q, t, _ = oracle.run(pb, oracle.cons_from_prims(pb, w), 0.2, 0.5)
        wp = oracle.prims_from_cons(pb, q)
        rho_e, u_e, p_e, _ = sample(Side(1, 0, 1, 1.4), Side(0.125, 0, 0.1, 1.4), (x - 0.5) / t)
        errs.append(_l1(wp[0].ravel(), rho_e))
    assert errs[0] < 2e-2 and errs[1] < 0.5 * errs[0]


@pytest.mark.slow
def test_water_air_shock_tube_matches_exact_solution():
    """The 1000-cell water/air shock tube (left water at 1e9 Pa, right air at 1e5 Pa,
    interface x = 0.7, t = 240 us) against the exact two-material solution;
    errors fall under refinement."""
    L = Side(1000.0, 0.0, 1e9, 4.4, 6e8)
    R = Side(1.0, 0.0, 1e5, 1.4, 0.0)
    errs = {}
    for n in (250, 1000):
        wl = workloads.shock_tube(n)
        pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf)
        q, t, _ = oracle.run(pb, oracle.cons_from_prims(pb, wl.prims()), wl.t_end, wl.cfl)
        assert t == pytest.approx(240e-6, rel=1e-14)
        wp = oracle.prims_from_cons(pb, q)
        x = (np.arange(n) + 0.5) / n
        rho_e, u_e, p_e, _ = sample(L, R, (x - 0.7) / t)
        errs[n] = (_l1((wp[0] + wp[1]).ravel(), rho_e), _l1(wp[2].ravel(), u_e), _l1(wp[3].ravel(), p_e))
    assert errs[1000][0] < 5e-3 and errs[1000][1] < 1.2e-2 and errs[1000][2] < 5e-3, errs
    assert all(errs[1000][i] < 0.6 * errs[250][i] for i in range(3)), errs
