"""CPU pins of the learned-form reference used by the fused-inference parity
tests: with a network that returns the ideal weights (W3 = 0, b3 = log d) the
learned reconstruction is the linear fifth-order scheme, which the C oracle
computes as WENO5-JS with epsilon -> infinity; and BF16 rounding is exact on
representable values and rounds ties to even."""
import numpy as np

import oracle
import workloads
from learned_reference import bf16, learned_rhs
from oracle import mlp
from parity_util import rhs_error


def _ideal_theta():
    p = mlp.unpack(mlp.init_params(3))
    p["W3"] = np.zeros_like(p["W3"])
    p["b3"] = np.log(mlp.D_IDEAL)
    return mlp.pack(p)


def test_bf16_rounding():
    assert bf16(np.array([1.0, -2.5, 0.0]))[1] == -2.5
    one_ulp = 2.0 ** -7                  # BF16 spacing in [1, 2)
    x = np.array([1.0 + one_ulp / 2, 1.0 + 1.5 * one_ulp, 1.0 + 0.49 * one_ulp])
    # ties go to the even mantissa: 1 (even) and 1 + 2 ulp
    assert np.array_equal(bf16(x), [1.0, 1.0 + 2 * one_ulp, 1.0])


def test_reference_with_ideal_network_is_linear_weno5():
    n, nf = (12, 10, 8), 2
    gam, pin = workloads.fluids(nf)
    pb = oracle.Problem(n, (0,) * 3, (1,) * 3, (0,) * 6, gam, pin, eps=1e30, fallback=False)
    w = workloads.random_prims(n, nf, seed=5, jumps=False)
    q = oracle.cons_from_prims(pb, w)
    R_cpu, fmax, _ = oracle.rhs(pb, q, return_info=True)
    for rounded in (False, True):
        R, _ = learned_rhs(pb, q, _ideal_theta(), rounded=rounded)
        err = rhs_error(pb, q, R, R_cpu, fmax)
        assert err.max() <= 1e-11, (rounded, err)
