"""CPU pins of the oracle's characteristic (non-reflecting) boundaries (Sec. 3.3:
characteristic-based conditions after Thompson; bc 3).  The pins: a uniform
moving state stays uniform; only the boundary cells differ from transmissive
ghosts; with every wave outgoing the boundary rate equals the quasi-linear
equations of the model evaluated directly and mapped to conserved variables
by a finite-difference Jacobian; a purely incoming acoustic wave gives no
boundary rate; and an acoustic pulse leaves the domain with little
reflection."""
import numpy as np
import pytest

import oracle
import workloads

CBC = oracle.BC_CHARACTERISTIC


def _gas(n, bc):
    return oracle.Problem(n, (0,) * 3, (1,) * 3, bc, (1.4,), (0.0,))


def test_uniform_moving_state_has_zero_rhs():
    gam, pin = workloads.fluids(2)
    pb = oracle.Problem((9, 7, 6), (0,) * 3, (1,) * 3, (CBC,) * 6, gam, pin)
    w = np.zeros(pb.shape())
    w[0], w[1], w[2], w[3], w[4], w[5], w[6] = 600.0, 0.4, 30.0, -20.0, 10.0, 2e5, 0.6
    R = oracle.rhs(pb, oracle.cons_from_prims(pb, w))
    assert np.abs(R).max() <= 1e-9 * np.abs(oracle.cons_from_prims(pb, w)).max()


def test_only_boundary_cells_differ_from_transmissive():
    n = (12, 9, 8)
    gam, pin = workloads.fluids(2)
    w = workloads.random_prims(n, 2, seed=3)
    pc = oracle.Problem(n, (0,) * 3, (1,) * 3, (CBC, CBC, 1, 1, CBC, 1), gam, pin)
    pt = oracle.Problem(n, (0,) * 3, (1,) * 3, (1,) * 6, gam, pin)
    q = oracle.cons_from_prims(pc, w)
    Rc, Rt = oracle.rhs(pc, q), oracle.rhs(pt, q)
    boundary = np.zeros(n[::-1], dtype=bool)
    boundary[:, :, 0] = boundary[:, :, -1] = True      # x low and high
    boundary[0, :, :] = True                            # z low
    assert np.array_equal(Rc[:, ~boundary], Rt[:, ~boundary])
    assert np.abs(Rc[:, boundary] - Rt[:, boundary]).max() > 0
    cells = np.array([0, 5, 11, 12 * 9 * 8 - 1, 40])
    assert np.allclose(oracle.rhs_cells(pc, q, cells), Rc.reshape(7, -1)[:, cells].T, rtol=1e-13, atol=1e-300)


def _quasi_linear_rate(pb, wb, wx, d):
    """dw/dt of the primitive equations along d, evaluated directly."""
    nf, nd = pb.nf, pb.ndim
    ie, ia = nf + nd, nf + nd + 1
    rho = wb[:nf].sum()
    a = list(wb[ia:]) + [1 - sum(wb[ia:])]
    G = sum(a[k] / (pb.gamma[k] - 1) for k in range(nf))
    P = sum(a[k] * pb.gamma[k] * pb.pi_inf[k] / (pb.gamma[k] - 1) for k in range(nf))
    c2 = ((G + 1) * wb[ie] + P) / (G * rho)
    u = wb[nf + d]
    wt = -u * wx
    wt[:nf] -= wb[:nf] * wx[nf + d]
    wt[nf + d] -= wx[ie] / rho
    wt[ie] -= rho * c2 * wx[nf + d]
    return wt


def _jacobian(pb, w, h=1e-7):
    J = np.zeros((pb.sys_size, pb.sys_size))
    for j in range(pb.sys_size):
        dw = np.zeros(pb.sys_size)
        dw[j] = h * max(1.0, abs(w[j]))
        J[:, j] = (oracle.cons_from_prim_cell(pb, w + dw) - oracle.cons_from_prim_cell(pb, w - dw)) / (2 * dw[j])
    return J


@pytest.mark.parametrize("high", [False, True])
def test_all_outgoing_boundary_rate_is_the_quasi_linear_form(high):
    """Supersonic outflow (|u| > c, pointing out of the domain): nothing is set
    to zero, so the characteristic rate must equal the model's own equations."""
    gam, pin = workloads.fluids(2)
    n = 8
    pb = oracle.Problem((n,), (0,), (1,), (CBC,) * 6, gam, pin)
    rng = np.random.default_rng(7 + high)
    x = (np.arange(n) + 0.5) / n
    w = np.zeros(pb.shape())
    u0 = 2500.0 if high else -2500.0                   # faster than water's ~1600 m/s sound speed
    w[0, 0, 0] = 800 * (1 + 0.05 * np.sin(3 * x + rng.uniform()))
    w[1, 0, 0] = 0.5 * (1 + 0.05 * np.cos(2 * x))
    w[2, 0, 0] = u0 * (1 + 0.02 * np.sin(5 * x))
    w[3, 0, 0] = 3e5 * (1 + 0.1 * np.sin(4 * x))
    w[4, 0, 0] = 0.8 + 0.05 * np.sin(6 * x)
    q = oracle.cons_from_prims(pb, w)
    R = oracle.rhs(pb, q)
    b, nb = (n - 1, n - 2) if high else (0, 1)
    wb, wn = w[:, 0, 0, b], w[:, 0, 0, nb]
    wx = (wb - wn) * n if high else (wn - wb) * n
    expect = _jacobian(pb, wb) @ _quasi_linear_rate(pb, wb, wx, 0)
    scale = np.abs(expect).max()
    assert np.allclose(R[:, 0, 0, b], expect, rtol=1e-6, atol=1e-6 * scale)


def test_incoming_acoustic_wave_gives_no_boundary_rate():
    """Fluid at rest, a small left-running simple wave (dp = -rho c du,
    isentropic density) touching the high boundary: its amplitude enters the
    domain and is dropped, so the boundary cell's normal rate is of second
    order in the amplitude, against the first-order rate of the same wave
    without the boundary condition (the quasi-linear form)."""
    n = 16
    pb = _gas((n,), (CBC,) * 6)
    rho0, p0 = 1.2, 1e5
    c0 = np.sqrt(1.4 * p0 / rho0)
    x = (np.arange(n) + 0.5) / n
    dp = 1e-4 * p0 * np.exp(-((x - 0.95) / 0.1) ** 2)
    w = np.zeros(pb.shape())
    w[0, 0, 0] = rho0 + dp / c0 ** 2
    w[1, 0, 0] = -dp / (rho0 * c0)
    w[2, 0, 0] = p0 + dp
    R = oracle.rhs(pb, oracle.cons_from_prims(pb, w))
    wb, wn = w[:, 0, 0, -1], w[:, 0, 0, -2]
    full = _jacobian(pb, wb) @ _quasi_linear_rate(pb, wb, (wb - wn) * n, 0)
    assert np.abs(full).max() > 0
    for v in range(3):
        assert abs(R[v, 0, 0, -1]) <= 1e-3 * np.abs(full[v]).max() + 1e-12, (v, R[v, 0, 0, -1], full[v])


def _pulse_residual(bc, n=200, t_factor=1.6):
    pb = _gas((n,), bc)
    rho0, p0 = 1.2, 1e5
    c0 = np.sqrt(1.4 * p0 / rho0)
    x = (np.arange(n) + 0.5) / n
    dp = 0.01 * p0 * np.exp(-((x - 0.6) / 0.05) ** 2)
    w = np.zeros(pb.shape())
    w[0, 0, 0] = rho0 + dp / c0 ** 2
    w[1, 0, 0] = dp / (rho0 * c0)                       # right-running
    w[2, 0, 0] = p0 + dp
    q = oracle.cons_from_prims(pb, w)
    t_end = t_factor * 0.4 / c0                         # the pulse has left through x = 1
    q, t, steps = oracle.run(pb, q, t_end, 0.4)
    wp = oracle.prims_from_cons(pb, q)
    return np.abs(wp[2] - p0).max() / (0.01 * p0)


def test_acoustic_pulse_leaves_with_little_reflection():
    cbc = _pulse_residual((CBC,) * 6)
    reflective = _pulse_residual((2,) * 6)
    transmissive = _pulse_residual((1,) * 6)
    assert reflective > 0.5
    assert cbc < 0.05 and cbc < 0.1 * reflective
    assert cbc <= 1.5 * transmissive + 0.01
