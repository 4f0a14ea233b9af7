"""CPU pins of the oracle's six-equation model with pressure relaxation
(Sec. 2.3: the pressure-disequilibrium model, evolved without its relaxation
source and then relaxed with infinite stiffness).  Each pin comes from outside
the code it checks: uniform states, conservation, the single-fluid reduction
to the five-equation oracle, the closed-form right-hand side of a uniform
compression, the defining equations of the relaxation (each phase's energy
balance at the relaxed pressure, unit total volume, conserved mass, momentum
and total energy, one pressure afterwards), its limit, the Kapila model's
K div(u) of Sec. 2.1 (itself pinned to the paper's formula), and the exact
two-material shock-tube solution."""
import numpy as np
import pytest

import oracle
import workloads
from oracle.exact_riemann import Side, sample


def _six(n, bc, nf=2, **kw):
    gam, pin = workloads.fluids(nf)
    return oracle.Problem(n, (0,) * 3, (1,) * 3, bc, gam, pin, model="six", **kw)


def _idx(pb):
    nf, nd = pb.nf, pb.ndim
    return {"mom": nf, "E": nf + nd, "alpha": nf + nd + 1, "int": 2 * nf + nd}


def test_layout_and_round_trip():
    pb = _six((6, 5, 4), (1,) * 6, nf=3)
    assert pb.sys_size == 3 * 3 + 3
    w = workloads.six_equation_prims(workloads.random_prims((6, 5, 4), 3, seed=1), 3, spread=0.2, seed=2)
    q = oracle.cons_from_prims(pb, w)
    w2 = oracle.prims_from_cons(pb, q)
    i = _idx(pb)
    keep = [v for v in range(pb.sys_size) if v != i["E"]]
    assert np.allclose(w2[keep], w[keep], rtol=1e-12, atol=1e-12 * np.abs(w).max())
    # the primitive pressure slot is the pressure of the mixture law for the
    # total energy: the phase pressures averaged with weights a_k/(g_k - 1)
    # (water's p_k = (g-1) E/a - g pinf cancels g pinf ~ 2.6e9 against
    # p ~ 1e6: ~3.4 digits lost)
    a = np.concatenate([w[i["alpha"]:i["alpha"] + 2], 1 - w[i["alpha"]:i["alpha"] + 2].sum(0, keepdims=True)])
    g = np.array(pb.gamma)[:, None, None, None] - 1.0
    assert np.allclose(w2[i["E"]], (a / g * w[i["int"]:]).sum(0) / (a / g).sum(0), rtol=1e-10)


def test_uniform_disequilibrium_state_has_zero_rhs():
    pb = _six((9, 7, 6), (0,) * 6)
    w = np.zeros(pb.shape())
    w[0], w[1], w[2], w[3], w[4], w[5], w[6] = 700.0, 0.3, 25.0, -12.0, 8.0, 2e5, 0.55
    w[7], w[8] = 3e5, 1.2e5                        # phase pressures differ
    q = oracle.cons_from_prims(pb, w)
    R = oracle.rhs(pb, q)
    assert np.abs(R).max() <= 1e-9 * np.abs(q).max()


def test_mass_momentum_and_total_energy_are_conserved():
    n = (10, 9, 8)
    pb = _six(n, (0,) * 6)
    w = workloads.six_equation_prims(workloads.random_prims(n, 2, seed=4), 2, spread=0.1, seed=5)
    R = oracle.rhs(pb, oracle.cons_from_prims(pb, w))
    i = _idx(pb)
    for v in range(i["E"] + 1):
        assert abs(R[v].sum()) <= 1e-13 * np.abs(R[v]).sum(), v
    # the internal energies are not conserved (their work term)
    assert abs(R[i["int"]].sum()) > 1e-6 * np.abs(R[i["int"]]).sum()


@pytest.mark.parametrize("n", [(40,), (14, 11), (10, 9, 7)])
def test_single_fluid_reduces_to_the_five_equation_model(n):
    """N = 1: the frozen sound speed is the stiffened-gas one and the phase
    pressure is the mixture pressure, so the mass, momentum and energy rows of
    the five-equation oracle come out."""
    w5 = workloads.random_prims(n, 1, seed=6)
    p5 = oracle.Problem(n, (0,) * 3, (1,) * 3, (1,) * 6, (4.4,), (6e8,), fallback=True)
    p6 = oracle.Problem(n, (0,) * 3, (1,) * 3, (1,) * 6, (4.4,), (6e8,), fallback=True, model="six")
    R5 = oracle.rhs(p5, oracle.cons_from_prims(p5, w5))
    R6 = oracle.rhs(p6, oracle.cons_from_prims(p6, workloads.six_equation_prims(w5, 1)))
    for v in range(p5.sys_size):
        assert np.abs(R6[v] - R5[v]).max() <= 1e-11 * np.abs(R5[v]).max(), v


def _compression(a_rate=100.0, n=40, nf=2):
    """Uniform mixture at rest in pressure with the linear velocity u = -a (x - 1/2)."""
    pb = _six((n,), (1,) * 6, nf=nf)
    x = (np.arange(n) + 0.5) / n
    w5 = np.zeros((2 * nf + 1, 1, 1, n))
    if nf == 2:
        w5[0], w5[1], w5[3], w5[4] = 0.4 * 1000.0, 0.6 * 1.2, 3e5, 0.4
    else:
        w5[0], w5[1], w5[2], w5[4], w5[5], w5[6] = 0.3 * 1000.0, 0.5 * 1.2, 0.2 * 2000.0, 3e5, 0.3, 0.5
    w5[nf] = -a_rate * (x - 0.5)
    w = workloads.six_equation_prims(w5, nf)
    return pb, w


@pytest.mark.parametrize("nf", [2, 3])
def test_uniform_compression_rates_in_closed_form(nf):
    """u_x = -a: at interior cells the mass rows are a a_k r_k, the volume
    fractions stay, and the internal energies gain a (a_k r_k e_k + a_k p)
    (advection plus the compression work a_k p div(u))."""
    a_rate = 100.0
    pb, w = _compression(a_rate, nf=nf)
    q = oracle.cons_from_prims(pb, w)
    R = oracle.rhs(pb, q)[:, 0, 0, 4:-4]
    qi = q[:, 0, 0, 4:-4]
    i = _idx(pb)
    p = w[i["E"], 0, 0, 4:-4]
    alphas = list(w[i["alpha"]:i["alpha"] + nf - 1, 0, 0, 4:-4])
    alphas.append(1.0 - sum(alphas))
    for k in range(nf):
        assert np.allclose(R[k], a_rate * qi[k], rtol=1e-10)
        assert np.allclose(R[i["int"] + k], a_rate * (qi[i["int"] + k] + alphas[k] * p), rtol=1e-10)
    assert np.abs(R[i["alpha"]:i["alpha"] + nf - 1]).max() <= 1e-12


def _phase_parts(pb, q):
    i = _idx(pb)
    m = q[:pb.nf]
    a = list(q[i["alpha"]:i["alpha"] + pb.nf - 1])
    a.append(1.0 - sum(a))
    return m, np.array(a), q[i["int"]:i["int"] + pb.nf]


@pytest.mark.parametrize("nf", [2, 3])
def test_relaxation_satisfies_its_defining_equations(nf):
    """Per cell, with v_k = a_k / m_k the phase specific volume: each phase's
    energy obeys e_k(p^, v_k) - e_k0 = -p^ (v_k - v_k0) with the stiffened-gas
    e(p, v) = (p + g pinf) v/(g - 1); the fractions sum to one; mass, momentum
    and total energy are unchanged; afterwards every phase is at the pressure
    the mixture law gives for the total energy."""
    n = (7, 6, 5)
    pb = _six(n, (1,) * 6, nf=nf)
    w = workloads.six_equation_prims(workloads.random_prims(n, nf, seed=8), nf, spread=0.3, seed=9)
    q0 = oracle.cons_from_prims(pb, w).reshape(pb.sys_size, -1)
    gam, pin = np.array(pb.gamma), np.array(pb.pi_inf)
    i = _idx(pb)
    for c in range(0, q0.shape[1], 7):
        qc0 = q0[:, c]
        qc, ph = oracle.relax_cell(pb, qc0)
        m, a0, E0 = _phase_parts(pb, qc0)
        _, a1, E1 = _phase_parts(pb, qc)
        v0, v1 = a0 / m, a1 / m
        e0 = E0 / m
        lhs = (ph + gam * pin) * v1 / (gam - 1) - e0
        assert np.allclose(lhs, -ph * (v1 - v0), rtol=1e-9, atol=1e-9 * np.abs(e0).max())
        assert np.all(a1 > 0) and np.all(a1 < 1)
        assert np.array_equal(qc[:i["E"] + 1], qc0[:i["E"] + 1])
        # one pressure, from the total energy and the mixture law of the new fractions
        pk = (gam - 1) * E1 / a1 - gam * pin
        ke = 0.5 * (qc[i["mom"]:i["E"]] ** 2).sum() / m.sum()
        G = (a1 / (gam - 1)).sum()
        Pi = (a1 * gam * pin / (gam - 1)).sum()
        p_mix = (qc[i["E"]] - ke - Pi) / G
        assert np.allclose(pk, p_mix, rtol=1e-9, atol=1e-3)
        assert E1.sum() + ke == pytest.approx(qc[i["E"]], rel=1e-13)


def test_relaxation_of_an_equilibrium_state_is_the_identity():
    n = (6, 5, 4)
    pb = _six(n, (1,) * 6, nf=3)
    w = workloads.six_equation_prims(workloads.random_prims(n, 3, seed=10), 3)
    q = oracle.cons_from_prims(pb, w)
    assert np.allclose(oracle.relax(pb, q), q, rtol=1e-12, atol=1e-12 * np.abs(q).max())


def test_two_phase_relaxed_pressure_is_the_quadratic_root():
    """N = 2: unit total volume of the relaxed phases is a quadratic in p^;
    its root above -min pinf (numpy.roots) is the oracle's p^."""
    pb = _six((1,), (1,) * 6)
    g1, g2 = pb.gamma
    q1, q2 = pb.pi_inf
    w = workloads.six_equation_prims(np.array([400.0, 0.72, 3.0, 2e5, 0.4]).reshape(5, 1, 1, 1), 2)
    w[5], w[6] = 2.5e6, 4e4
    q = oracle.cons_from_prims(pb, w).ravel()
    _, ph = oracle.relax_cell(pb, q)
    a1, a2, p1, p2 = 0.4, 0.6, 2.5e6, 4e4
    A1, A2 = p1 + g1 * q1, p2 + g2 * q2
    # a1 (A1 + (g1-1) p) g2 (p + q2) + a2 (A2 + (g2-1) p) g1 (p + q1) = g1 g2 (p + q1)(p + q2)
    P = np.polynomial.Polynomial
    poly = (a1 * g2 * P([A1, g1 - 1]) * P([q2, 1]) + a2 * g1 * P([A2, g2 - 1]) * P([q1, 1])
            - g1 * g2 * P([q1, 1]) * P([q2, 1]))
    roots = [r.real for r in poly.roots() if abs(r.imag) < 1e-6 * abs(r) and r.real > -min(q1, q2)]
    assert len(roots) == 1
    # the root (~4e4) sits far below the coefficients' scale pinf = 6e8: both
    # evaluations lose ~log10(6e8/4e4) digits
    assert ph == pytest.approx(roots[0], rel=1e-10)


@pytest.mark.parametrize("nf", [2, 3])
def test_relaxed_compression_approaches_the_kapila_rate(nf):
    """Infinite relaxation drives the six-equation model to the Kapila model
    (Sec. 2.1): one forward-Euler step of the uniform compression followed by
    the relaxation moves the volume fractions at the rate K div(u), with
    K from the oracle's Kapila coefficients."""
    a_rate = 100.0
    pb, w = _compression(a_rate, nf=nf)
    q = oracle.cons_from_prims(pb, w)
    i = _idx(pb)
    dt = 1e-9
    q1 = oracle.rk_step(pb, q, dt, order=1)
    rate = (q1[i["alpha"]:i["alpha"] + nf - 1, 0, 0, 20] - q[i["alpha"]:i["alpha"] + nf - 1, 0, 0, 20]) / dt
    gam, pin = workloads.fluids(nf)
    p5 = oracle.Problem((40,), (0,), (1,), (1,) * 6, gam, pin, model="kapila")
    K = oracle.kapila_K(p5, w[:p5.sys_size, 0, 0, 20])
    expect = K * (-a_rate)
    assert np.allclose(rate, expect, rtol=1e-5), (rate, expect)
    assert np.abs(expect).min() > 1e-4


def test_water_air_shock_tube_matches_exact_solution():
    """The water/air shock tube run with the six-equation model and relaxation
    after every stage: the same exact two-material solution as the
    five-equation model (pure phases on both sides), errors falling under
    refinement."""
    L = Side(1000.0, 0.0, 1e9, 4.4, 6e8)
    R = Side(1.0, 0.0, 1e5, 1.4, 0.0)
    errs = {}
    for n in (250, 1000):
        wl = workloads.shock_tube(n)
        pb = oracle.Problem(wl.n, wl.lo, wl.hi, wl.bc, wl.gamma, wl.pi_inf, model="six")
        q0 = oracle.cons_from_prims(pb, workloads.six_equation_prims(wl.prims(), 2))
        q, t, _ = oracle.run(pb, q0, wl.t_end, wl.cfl)
        wp = oracle.prims_from_cons(pb, q)
        x = (np.arange(n) + 0.5) / n
        rho_e, u_e, p_e, _ = sample(L, R, (x - 0.7) / t)
        l1 = lambda a, b: np.abs(a - b).mean() / np.abs(b).mean()
        errs[n] = (l1((wp[0] + wp[1]).ravel(), rho_e), l1(wp[2].ravel(), u_e), l1(wp[3].ravel(), p_e))
    assert errs[1000][0] < 5e-3 and errs[1000][1] < 1.2e-2 and errs[1000][2] < 5e-3, errs
    assert all(errs[1000][i] < 0.6 * errs[250][i] for i in range(3)), errs


def test_wave_speed_is_the_models_frozen_sound_speed():
    """The CFL rate of a uniform mixture is |u| + c with c the largest
    eigenvalue offset of the model's quasi-linear 1D system in the variables
    (a_1, a_k r_k, u, p_k): a advected, a_k r_k and u as in the equations,
    and each phase pressure following its own isentrope, p_k,t + u p_k,x +
    r_k c_k^2 u_x = 0 (r_k c_k^2 = g_k (p + pinf_k)).  The eigenvalues come
    from numpy; the oracle's closed form is not used."""
    gam, pin = workloads.fluids(2)
    pb = oracle.Problem((8,), (0,), (1,), (0,) * 6, gam, pin, model="six")
    a1, r1, r2, u, p = 0.3, 1000.0, 1.2, 40.0, 2e5
    m1, m2 = a1 * r1, (1 - a1) * r2
    rho = m1 + m2
    # variables: a1, m1, m2, u, p1, p2 (p = a1 p1 + (1-a1) p2, p1 = p2 = p)
    A = np.diag([u] * 6)
    A[1, 3], A[2, 3] = m1, m2
    A[3, 0] = (p - p) / rho                             # d p / d a1 = p1 - p2 = 0 at equilibrium
    A[3, 4], A[3, 5] = a1 / rho, (1 - a1) / rho
    A[4, 3], A[5, 3] = gam[0] * (p + pin[0]), gam[1] * (p + pin[1])
    lam = np.linalg.eigvals(A).real
    w = np.zeros(pb.shape())
    w[0], w[1], w[2], w[3], w[4] = m1, m2, u, p, a1
    w[5], w[6] = p, p
    rate, bad = oracle.max_rate(pb, oracle.cons_from_prims(pb, w))
    assert bad == 0
    assert rate * pb.dx[0] == pytest.approx(lam.max(), rel=1e-12)
    # far above the five-equation (Allaire) mixture's sound speed
    p5 = oracle.Problem((8,), (0,), (1,), (0,) * 6, gam, pin)
    rate5, _ = oracle.max_rate(p5, oracle.cons_from_prims(p5, w[:5]))
    assert rate > 1.5 * rate5


def test_hllc_carries_every_energy_at_the_face_velocity():
    """HLLC moves every quantity that is transported with the mass by the
    same star factor, so each phase energy's flux is its upwind face value
    times the face velocity F(a_1)/a_1,upwind, on random face pairs whose
    Riemann fans cover all four branches."""
    gam, pin = workloads.fluids(2)
    pb = oracle.Problem((8,), (0,), (1,), (0,) * 6, gam, pin, model="six")
    rng = np.random.default_rng(12)
    seen = set()
    for _ in range(200):
        wl, wr = [], []
        for side in range(2):
            a = rng.uniform(0.05, 0.95)
            p = 10 ** rng.uniform(5, 8.5)
            s = np.array([a * 1000 * rng.uniform(0.9, 1.1), (1 - a) * 1.2 * rng.uniform(0.5, 2),
                          rng.normal(0, 800), p, a, p, p])
            (wl if side == 0 else wr).append(s)
        wl, wr = wl[0], wr[0]
        F, ut = oracle.hllc(pb, 0, wl, wr)
        up = wl if abs(F[4] - wl[4] * ut) <= 1e-12 * abs(F[4]) + 1e-300 else wr
        assert F[4] == pytest.approx(up[4] * ut, rel=1e-12, abs=1e-300)
        E = oracle.cons_from_prim_cell(pb, up)[5:7]
        assert np.allclose(F[5:7], E * ut, rtol=1e-11)
        seen.add("L" if up is wl else "R")
    assert seen == {"L", "R"}


def test_rhs_acts_on_relaxed_states():
    """Stages end relaxed, so the right-hand side takes the phases at the
    mixture pressure: changing the phase energies (not the total energy)
    leaves it unchanged."""
    n = (9, 8, 7)
    pb = _six(n, (2,) * 6)
    w = workloads.six_equation_prims(workloads.random_prims(n, 2, seed=13), 2)
    q = oracle.cons_from_prims(pb, w)
    i = _idx(pb)
    q2 = q.copy()
    q2[i["int"]] *= 1 + 0.1 * np.random.default_rng(14).standard_normal(q2[i["int"]].shape)
    assert np.array_equal(oracle.rhs(pb, q), oracle.rhs(pb, q2))


def test_selected_cells_agree_with_the_full_rhs():
    """rhs_cells (the sampled check of large grids) follows the same
    definitions as rhs, internal-energy work term included."""
    n = (11, 9, 8)
    pb = _six(n, (0, 0, 1, 1, 2, 2), fallback=True)
    w = workloads.six_equation_prims(workloads.random_prims(n, 2, seed=15), 2)
    q = oracle.cons_from_prims(pb, w)
    R = oracle.rhs(pb, q).reshape(pb.sys_size, -1)
    cells = np.array([0, 7, 100, 431, pb.ncell - 1])
    Rc = oracle.rhs_cells(pb, q, cells)
    assert np.allclose(Rc, R[:, cells].T, rtol=1e-13, atol=1e-13 * np.abs(R).max())
