"""Pins of the FP64 reference of the learned WENO weights (oracle/mlp.py)."""
import numpy as np
import pytest

import oracle
from oracle import mlp


def _batch(rng, B=64):
    v = rng.normal(size=(B, 5)).cumsum(axis=1)
    x, phat, s = mlp.stencil_features(v)
    t = rng.normal(scale=0.3, size=B)
    mask = (rng.uniform(size=B) < 0.5).astype(float)
    return v, x, phat, t, mask


def test_gradient_matches_central_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(1) + rng.normal(scale=0.05, size=mlp.N_PARAMS)
    _, x, phat, t, mask = _batch(rng)
    L, g = mlp.loss_and_grad(theta, x, phat, t, mask, 0.3)
    assert L == pytest.approx(mlp.loss(theta, x, phat, t, mask, 0.3), rel=1e-14)
    fd = np.zeros_like(g)
    for i in range(mlp.N_PARAMS):
        h = 1e-6 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (mlp.loss(tp, x, phat, t, mask, 0.3) - mlp.loss(tm, x, phat, t, mask, 0.3)) / (2 * h)
    err = np.abs(fd - g).max() / np.abs(g).max()
    assert err < 1e-6, err


def test_zero_output_layer_gives_uniform_weights():
    theta = mlp.unpack(mlp.init_params(2))
    theta["W3"][:] = 0
    theta["b3"][:] = 0
    om, _ = mlp.forward(mlp.pack(theta), np.random.default_rng(3).normal(size=(10, 5)))
    assert np.all(om == 1.0 / 3.0)


def test_ideal_weights_reproduce_linear_fifth_order_interpolation():
    """omega = d makes the learned edge the fifth-order linear WENO5 value:
    exact on cell averages of quartic polynomials."""
    p = mlp.unpack(mlp.init_params(4))
    p["W3"][:] = 0
    p["b3"][:] = np.log(mlp.D_IDEAL)
    theta = mlp.pack(p)
    rng = np.random.default_rng(5)
    h = 0.1
    xc = np.arange(-2, 3) * h
    for _ in range(20):
        c = rng.normal(size=5)
        P = np.polynomial.polynomial.Polynomial(c).integ()
        v = ((P(xc + h / 2) - P(xc - h / 2)) / h)[None, :]
        exact = np.polynomial.polynomial.polyval(h / 2, c)
        assert mlp.edge_value(theta, v)[0] == pytest.approx(exact, abs=1e-12)


def test_one_hot_weights_select_candidates_exact_on_quadratics():
    rng = np.random.default_rng(6)
    h = 0.2
    xc = np.arange(-2, 3) * h
    for r in range(3):
        p = mlp.unpack(mlp.init_params(7))
        p["W3"][:] = 0
        p["b3"][:] = -200.0
        p["b3"][r] = 200.0
        theta = mlp.pack(p)
        c = rng.normal(size=3)
        P = np.polynomial.polynomial.Polynomial(c).integ()
        v = ((P(xc + h / 2) - P(xc - h / 2)) / h)[None, :]
        assert mlp.edge_value(theta, v)[0] == pytest.approx(np.polynomial.polynomial.polyval(h / 2, c), abs=1e-12)
        # and equals the oracle's WENO5 candidate r
        _, cand = oracle.weno5_weights(v[0], 1e-6)
        assert mlp.edge_value(theta, v)[0] == pytest.approx(cand[r], abs=1e-12)


def test_reconstruction_is_affine_invariant():
    """Normalised inputs: a v + b (a > 0) reconstructs to a * value + b."""
    rng = np.random.default_rng(8)
    theta = mlp.init_params(9)
    v = rng.normal(size=(30, 5))
    for a, b in ((3.5, -2.0), (1e-3, 7.0), (1e6, 1e9)):
        assert np.allclose(mlp.edge_value(theta, a * v + b), a * mlp.edge_value(theta, v) + b,
                           rtol=1e-9, atol=1e-9 * abs(b))


def test_relu_units_below_zero_carry_no_gradient():
    p = mlp.unpack(mlp.init_params(10))
    p["b1"][:5] = -1e3  # five dead first-layer units
    theta = mlp.pack(p)
    rng = np.random.default_rng(11)
    _, x, phat, t, mask = _batch(rng)
    _, g = mlp.loss_and_grad(theta, x, phat, t, mask, 0.1)
    gp = mlp.unpack(g)
    assert np.all(gp["W1"][:5] == 0) and np.all(gp["b1"][:5] == 0)
    assert np.all(gp["W2"][:, :5] == 0)


def test_adam_first_step_moves_each_parameter_by_the_learning_rate():
    """With bias correction the first Adam step is lr * g/|g| (eps -> 0)."""
    rng = np.random.default_rng(12)
    theta = rng.normal(size=50)
    g = rng.normal(size=50)
    new, m, v = mlp.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr=0.01, eps=0.0)
    assert np.allclose(theta - new, 0.01 * np.sign(g), rtol=1e-12, atol=1e-15)
