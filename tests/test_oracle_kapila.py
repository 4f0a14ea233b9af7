"""CPU pins of the oracle's Kapila five-equation model (Sec. 2.1): the
volume-fraction equations carry K div(u).  Pins: the two-component K as printed
(phase densities and sound speeds formed the textbook way), reductions (a
missing phase, identical phases), a closed form of the whole right-hand side
under uniform compression, agreement with the Allaire model where div(u) = 0
(bitwise outside the volume-fraction rows), and the property the section gives K for: every phase follows its
own isentrope, d(rho_k) = dp / c_k^2."""
import numpy as np
import pytest

import oracle
import workloads


def _pb(nf, n=(8,), bc=1, model="kapila", water_air=True):
    gam, pin = workloads.fluids(nf, water_air)
    return oracle.Problem(n, (-0.5,) * 3, (0.5,) * 3, (bc,) * 6, gam, pin, model=model)


def _phase_rho_c2(pb, w):
    """rho_k and c_k^2 of every phase from a primitive cell state."""
    nf, nd = pb.nf, pb.ndim
    a = list(w[nf + nd + 1:]) + [1.0 - sum(w[nf + nd + 1:])]
    p = w[nf + nd]
    rho = [w[k] / a[k] for k in range(nf)]
    c2 = [pb.gamma[k] * (p + pb.pi_inf[k]) / rho[k] for k in range(nf)]
    return a, rho, c2, p


def _random_cell(pb, rng):
    nf, nd = pb.nf, pb.ndim
    a = rng.dirichlet(np.ones(nf) * 2.0) * 0.98 + 0.02 / nf
    rho_pure = [1000.0, 1.2, 2000.0][:nf]
    w = np.zeros(pb.sys_size)
    w[:nf] = a * np.array(rho_pure) * rng.uniform(0.8, 1.2, nf)
    w[nf:nf + nd] = rng.normal(0, 50, nd)
    w[nf + nd] = rng.uniform(1e5, 1e8)
    w[nf + nd + 1:] = a[:-1]
    return w


def test_two_component_K_is_the_printed_formula():
    pb = _pb(2)
    rng = np.random.default_rng(3)
    for _ in range(20):
        w = _random_cell(pb, rng)
        a, rho, c2, _ = _phase_rho_c2(pb, w)
        K = (rho[1] * c2[1] - rho[0] * c2[0]) / (rho[1] * c2[1] / a[1] + rho[0] * c2[0] / a[0])
        assert oracle.kapila_K(pb, w)[0] == pytest.approx(K, rel=1e-13)


def test_three_components_reduce_to_two_and_identical_phases_give_zero():
    pb3, pb2 = _pb(3), _pb(2)
    rng = np.random.default_rng(4)
    for _ in range(10):
        w2 = _random_cell(pb2, rng)
        # the same state with a third phase of zero volume fraction
        w3 = np.concatenate([w2[:2], [0.0], w2[2:4], [w2[4], 1.0 - w2[4]]])
        K3 = oracle.kapila_K(pb3, w3)
        assert K3[0] == pytest.approx(oracle.kapila_K(pb2, w2)[0], rel=1e-12)
        assert K3[1] == pytest.approx(-K3[0], rel=1e-12)  # K over all phases sums to zero; K_3 = 0
    same = oracle.Problem((8,), (0,), (1,), (1,) * 6, (4.4, 4.4, 4.4), (6e8, 6e8, 6e8), model="kapila")
    w = np.array([300.0, 300.0, 400.0, 1.0, 1e6, 0.3, 0.3])
    assert np.all(np.abs(oracle.kapila_K(same, w)) <= 1e-15)


@pytest.mark.parametrize("nf", [2, 3])
def test_uniform_compression_closed_form(nf):
    """u = -eps x, uniform pressure, densities and fractions: in the interior the
    face velocities are exact, so R_alpha = -eps K and the partial densities
    compress as rho_k alpha_k eps (and the Allaire model gives R_alpha = 0)."""
    n, eps = 32, 100.0
    pb = _pb(nf, (n,))
    rng = np.random.default_rng(5)
    c0 = _random_cell(pb, rng)
    x = -0.5 + (np.arange(n) + 0.5) / n
    w = np.repeat(c0[:, None], n, axis=1)
    w[nf] = -eps * x
    w = w.reshape(pb.sys_size, 1, 1, n)
    q = oracle.cons_from_prims(pb, w)
    R = oracle.rhs(pb, q)[:, 0, 0, :]
    Ra = oracle.rhs(_pb(nf, (n,), model="allaire"), q)[:, 0, 0, :]
    inner = slice(4, n - 4)
    ia = nf + 2
    for k in range(nf - 1):
        K = np.array([oracle.kapila_K(pb, w[:, 0, 0, i])[k] for i in range(n)])
        assert np.allclose(R[ia + k, inner], -eps * K[inner], rtol=1e-9, atol=0)
        assert np.all(np.abs(Ra[ia + k, inner]) <= 1e-9 * eps)
    for k in range(nf):
        assert np.allclose(R[k, inner], eps * w[k, 0, 0, inner], rtol=1e-9)


def test_kapila_equals_allaire_where_velocity_is_uniform():
    """K multiplies div(u): with one uniform velocity and pressure (contacts
    only) div(u) vanishes up to the rounding of the HLLC contact speed, so the
    two models agree: bitwise outside the volume-fraction rows, to 1e-12 of
    the row's scale in them."""
    n = (14, 9, 7)
    gam, pin = workloads.fluids(2)
    w = workloads.random_prims(n, 2, seed=6)
    w[2:5] = np.array([30.0, -20.0, 10.0])[:, None, None, None]
    w[5] = 2e5
    pk = oracle.Problem(n, (0,) * 3, (1,) * 3, (0,) * 6, gam, pin, model="kapila")
    pa = oracle.Problem(n, (0,) * 3, (1,) * 3, (0,) * 6, gam, pin)
    q = oracle.cons_from_prims(pk, w)
    Rk, Ra = oracle.rhs(pk, q), oracle.rhs(pa, q)
    assert np.array_equal(Rk[:6], Ra[:6])
    assert np.abs(Rk[6] - Ra[6]).max() <= 1e-12 * np.abs(Ra[6]).max()


def test_only_the_volume_fraction_rows_change():
    n = (12, 10, 6)
    gam, pin = workloads.fluids(3)
    w = workloads.random_prims(n, 3, seed=7)
    pk = oracle.Problem(n, (0,) * 3, (1,) * 3, (1,) * 6, gam, pin, model="kapila")
    pa = oracle.Problem(n, (0,) * 3, (1,) * 3, (1,) * 6, gam, pin)
    q = oracle.cons_from_prims(pk, w)
    Rk, Ra = oracle.rhs(pk, q), oracle.rhs(pa, q)
    assert np.array_equal(Rk[:7], Ra[:7])
    assert np.abs(Rk[7:] - Ra[7:]).max() > 1e-3 * np.abs(Ra[7:]).max()


@pytest.mark.parametrize("nf", [2, 3])
def test_phases_compress_along_their_own_isentropes(nf):
    """Under the uniform compression above, the rates of the interior cells
    satisfy d(rho_k)/dt = (dp/dt) / c_k^2 for every phase (phase entropy
    conserved), with rho_k = (alpha_k rho_k)/alpha_k and p from the mixture EOS,
    both differentiated along R by a small finite step.  The Allaire model
    violates it for the gas phase."""
    n, eps = 32, 100.0
    rng = np.random.default_rng(8)
    for model, holds in (("kapila", True), ("allaire", False)):
        pb = _pb(nf, (n,), model=model)
        c0 = _random_cell(pb, rng)
        x = -0.5 + (np.arange(n) + 0.5) / n
        w = np.repeat(c0[:, None], n, axis=1)
        w[nf] = -eps * x
        q = oracle.cons_from_prims(pb, w.reshape(pb.sys_size, 1, 1, n))
        R = oracle.rhs(pb, q)
        h = 1e-7 / eps
        wp = oracle.prims_from_cons(pb, q + h * R)[:, 0, 0, :]
        wm = oracle.prims_from_cons(pb, q - h * R)[:, 0, 0, :]
        i = n // 2
        a0, rho0, c20, p0 = _phase_rho_c2(pb, w[:, i])
        ap, rhop, _, pp = _phase_rho_c2(pb, wp[:, i])
        am, rhom, _, pm = _phase_rho_c2(pb, wm[:, i])
        dp = (pp - pm) / (2 * h)
        ok = []
        for k in range(nf):
            drho = (rhop[k] - rhom[k]) / (2 * h)
            ok.append(abs(drho - dp / c20[k]) <= 1e-5 * abs(dp / c20[k]))
        assert all(ok) == holds, (model, ok)
