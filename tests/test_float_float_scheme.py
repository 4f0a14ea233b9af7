"""CPU check of the float-float arithmetic the FP64 path uses for its WENO5
weights: a float32 model of the scheme (error-free transformations, the
integer split of a double into hi + lo, the min-normalised weights) against
the oracle's FP64 WENO5-JS on stencils of every kind the solver meets.  It
models the arithmetic, not the kernel: the CUDA path's own parity is tested
on the GPU.  Exact FMA is modelled by one rounding of a float64 product-sum
(exact for float32 operands)."""

import numpy as np
import pytest

import oracle

f32 = np.float32


def _fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def _two_sum(a, b):
    s = (a + b).astype(f32)
    bb = (s - a).astype(f32)
    return s, ((a - (s - bb).astype(f32)).astype(f32) + (b - bb).astype(f32)).astype(f32)


def _fast_two_sum(a, b):
    s = (a + b).astype(f32)
    return s, (b - (s - a).astype(f32)).astype(f32)


def _two_prod(a, b):
    p = (a * b).astype(f32)
    return p, _fma(a, b, -p)


def add_fast(x, y):
    s, e = _two_sum(x[0], y[0])
    return _fast_two_sum(s, ((e + x[1]).astype(f32) + y[1]).astype(f32))


def add(x, y):
    s, e = _two_sum(x[0], y[0])
    t, f = _two_sum(x[1], y[1])
    s, e = _fast_two_sum(s, (e + t).astype(f32))
    return _fast_two_sum(s, (e + f).astype(f32))


def neg(x):
    return -x[0], -x[1]


def mul(x, y):
    p, e = _two_prod(x[0], y[0])
    e = _fma(x[1], y[0], _fma(x[0], y[1], e))
    return _fast_two_sum(p, e)


def mul_f(x, f):
    f = np.full_like(x[0], f32(f))
    p, e = _two_prod(x[0], f)
    return _fast_two_sum(p, _fma(x[1], f, e))


def mul_pow2(x, f):
    return (x[0] * f32(f)).astype(f32), (x[1] * f32(f)).astype(f32)


_RCP_RNG = np.random.default_rng(1234)


def rcp_approx(x):
    """The kernels take an approximate FP32 reciprocal (one hardware
    instruction, about one ulp); modelled here as the correctly rounded one
    perturbed by 2^-22 relative (two ulps) with a random sign, so the model
    bounds the scheme's error for any reciprocal that accurate."""
    sgn = np.where(_RCP_RNG.random(x.shape) < 0.5, -1.0, 1.0)
    return ((1.0 / x.astype(np.float64)) * (1.0 + sgn * 2.0 ** -22)).astype(f32)


def div_f(a, b):
    y = rcp_approx(b[0])
    q1 = (a * y).astype(f32)
    p, pe = _two_prod(q1, b[0])
    r = _fma(-q1, b[1], ((a - p).astype(f32) - pe).astype(f32))
    return _fast_two_sum(q1, (r * y).astype(f32))


def div(a, b):
    y = rcp_approx(b[0])
    q1 = (a[0] * y).astype(f32)
    r = add(a, neg(mul_f(b, q1)))
    return _fast_two_sum(q1, (r[0] * y).astype(f32))


def split(d):
    """double -> (hi, lo) by integer operations on the bit pattern."""
    u = d.astype(np.float64).view(np.uint64)
    hw = (u >> np.uint64(32)).astype(np.uint64)
    lw = (u & np.uint64(0xFFFFFFFF)).astype(np.uint64)
    sign = hw & np.uint64(0x80000000)
    ef = ((hw >> np.uint64(20)) & np.uint64(0x7FF)).astype(np.int64) - 1023 + 127
    hb = sign | (np.clip(ef, 0, 255).astype(np.uint64) << np.uint64(23)) | \
        ((hw & np.uint64(0xFFFFF)) << np.uint64(3)) | (lw >> np.uint64(29))
    hi = np.where(ef > 0, hb.astype(np.uint32).view(np.float32), f32(0))
    es = ef - 52
    scale = (np.maximum(es, 1).astype(np.uint32) << np.uint32(23)).view(np.float32)
    lo = ((lw & np.uint64(0x1FFFFFFF)).astype(f32) * scale).astype(f32)
    lo = np.where(sign > 0, -lo, lo)
    return hi.astype(f32), np.where(es > 0, lo, f32(0)).astype(f32)


def to_double(x):
    return x[0].astype(np.float64) + x[1].astype(np.float64)


def weno5_float_float(vc, D, eps34):
    """Edge values (eR at c-1/2, eL at c+1/2) as the FP64 path forms them: the
    c+1/2 formula on the stencil and, for eR, on the mirrored stencil
    (-D3, -D2, -D1, -D0), with b1, its weight and the normaliser m shared."""
    d = [split(D[:, j]) for j in range(4)]
    e = split(np.full(len(vc), eps34))
    S1, S2 = mul(d[1], d[1]), mul(d[2], d[2])
    b1 = add_fast(add_fast(S1, S2), mul_f(mul(d[1], d[2]), -1.25))
    t1 = add_fast(e, b1)

    def side(x0, x1, x2, x3):
        b0 = add_fast(add_fast(mul(x0, x0), mul_f(mul(x1, x0), -2.75)), mul_f(mul(x1, x1), 2.5))
        return x0, x1, x2, x3, add_fast(e, b0)

    L = side(d[0], d[1], d[2], d[3])
    R = side(neg(d[3]), neg(d[2]), neg(d[1]), neg(d[0]))
    m = np.minimum(np.minimum(L[4][0], t1[0]), R[4][0])
    g1 = div_f(m, t1)
    q1 = mul_f(mul(g1, g1), 6)
    gL, gR = div_f(m, L[4]), div_f(m, R[4])
    qL, qR = mul(gL, gL), mul(gR, gR)

    def increment(x, q0, q2):
        x0, x1, x2, x3 = x[:4]
        w2 = mul_f(q2, 3)
        P0 = add_fast(mul_f(x1, 5), mul_pow2(x0, -2))
        P1 = add_fast(x1, mul_pow2(x2, 2))
        P2 = add_fast(mul_pow2(x2, 4), neg(x3))
        num = add_fast(add_fast(mul(q0, P0), mul(q1, P1)), mul(w2, P2))
        den = mul_f(add_fast(add_fast(q0, q1), w2), 6)
        return div(num, den)

    iL = increment(L, qL, qR)
    iR = increment(R, qR, qL)
    return vc + to_double(iR), vc + to_double(iL)


def test_error_free_transformations_are_exact():
    rng = np.random.default_rng(0)
    a = (rng.standard_normal(10000) * 10.0 ** rng.uniform(-10, 10, 10000)).astype(f32)
    b = (rng.standard_normal(10000) * 10.0 ** rng.uniform(-10, 10, 10000)).astype(f32)
    s, e = _two_sum(a, b)
    assert np.all(s.astype(np.float64) + e.astype(np.float64) == a.astype(np.float64) + b.astype(np.float64))
    p, e = _two_prod(a, b)
    assert np.all(p.astype(np.float64) + e.astype(np.float64) == a.astype(np.float64) * b.astype(np.float64))


def test_integer_split_matches_the_double():
    rng = np.random.default_rng(1)
    d = rng.standard_normal(100000) * 10.0 ** rng.uniform(-22, 37, 100000)
    hi, lo = split(d)
    big = np.abs(d) >= 2.0 ** -74
    assert np.all(np.abs(to_double((hi, lo))[big] - d[big]) <= 2.0 ** -47 * np.abs(d[big]))
    assert np.all(np.abs(lo[big].astype(np.float64)) <= 2.0 ** -23 * np.abs(hi[big].astype(np.float64)))
    # exact for doubles that are floats; zero and values below the FP32 range give zero
    x = np.array([1.0, -3.5, 0.0, 1e-40, 2.0 ** -126])
    hx, lx = split(x)
    assert list(hx) == [1.0, -3.5, 0.0, 0.0, np.float32(2.0 ** -126)] and not lx.any()


def _stencils(kind, rng, B=20000):
    x = np.arange(-2, 3)[None, :]
    if kind == "jumps":
        k = rng.integers(0, 5, B)
        return np.where(x >= k[:, None], 1e9, 1e5) * (1 + 1e-4 * rng.standard_normal((B, 5)))
    if kind == "flat_next_to_jump":
        k = rng.integers(0, 6, B)
        return np.where(x >= k[:, None] - 2, 1e9, 1e5) + np.zeros((B, 5))
    if kind == "sign_changing":
        return rng.normal(0, 400, (B, 5))
    scale, noise = {"smooth_pressure": (1e9, 1e-3), "noisy_pressure": (1e5, 0.05), "volume_fraction": (1.0, 0.01),
                    "small": (1e-6, 0.1)}[kind]
    return scale * (1 + noise * rng.standard_normal((B, 5)) + 0.01 * rng.standard_normal((B, 1)) * x)


@pytest.mark.parametrize("kind", ["smooth_pressure", "noisy_pressure", "jumps", "flat_next_to_jump",
                                  "volume_fraction", "small", "sign_changing"])
def test_float_float_weno5_matches_the_oracle(kind):
    """Edge values within 1e-13 of the stencil magnitude of the oracle's FP64
    WENO5-JS (the FP64 path's parity tolerance is 1e-11 of much larger scales)."""
    rng = np.random.default_rng(sum(map(ord, kind)))
    v = _stencils(kind, rng, 2000)
    eps = 1e-6
    with np.errstate(all="ignore"):
        eR, eL = weno5_float_float(v[:, 2], np.diff(v, axis=1), 0.75 * eps)
    rL = np.array([oracle.weno5(s, eps) for s in v])
    rR = np.array([oracle.weno5(s[::-1], eps) for s in v])
    scale = np.abs(v).max(axis=1)
    assert np.all(np.abs(eL - rL) <= 1e-13 * scale)
    assert np.all(np.abs(eR - rR) <= 1e-13 * scale)


def narrow(d):
    """FP64 -> FP32 round-to-nearest-even by integer operations on the bit
    pattern, as the FP32 primitive recovery does (normal FP32 range)."""
    u = np.asarray(d, dtype=np.float64).view(np.uint64)
    hw = (u >> np.uint64(32)).astype(np.uint64)
    lw = (u & np.uint64(0xFFFFFFFF)).astype(np.uint64)
    sign = hw & np.uint64(0x80000000)
    e = ((hw >> np.uint64(20)) & np.uint64(0x7FF)).astype(np.int64) - 1023 + 127
    m23 = ((hw & np.uint64(0xFFFFF)) << np.uint64(3)) | (lw >> np.uint64(29))
    rem = lw & np.uint64(0x1FFFFFFF)
    half = np.uint64(0x10000000)
    up = ((rem > half) | ((rem == half) & ((m23 & np.uint64(1)) == 1))).astype(np.uint64)
    bits = sign | ((np.clip(e, 0, 255).astype(np.uint64) << np.uint64(23)) + m23 + up)
    out = (bits & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    out = np.where(e <= 0, np.where(sign > 0, np.float32(-0.0), np.float32(0.0)), out)
    return np.where(e >= 255, np.where(sign > 0, -np.inf, np.inf).astype(np.float32), out)


def test_integer_narrowing_rounds_to_nearest_even():
    """Equal to IEEE conversion (numpy) for every double whose result is a
    normal float, ties and carries into the exponent included."""
    rng = np.random.default_rng(3)
    d = rng.standard_normal(1_000_000) * 10.0 ** rng.uniform(-37, 38, 1_000_000)
    f = d.astype(np.float32)
    keep = np.isfinite(f) & (np.abs(f) >= np.float32(2.0 ** -126))
    assert np.array_equal(narrow(d[keep]), f[keep])
    # exact ties: a float plus half an FP32 ulp rounds to the even neighbour
    x = rng.uniform(1, 2, 10000).astype(np.float32).astype(np.float64)
    tie = x + 2.0 ** -24
    assert np.array_equal(narrow(tie), tie.astype(np.float32))
    # the largest significand rounds up into the next binade
    y = np.nextafter(np.float64(2.0), 0.0)
    assert narrow(np.array([y]))[0] == np.float32(2.0)


def widen_all(f):
    """float -> double by integer operations on the bit pattern, infinities
    and NaNs included (the FP32 forms' RK update widens c1 dt R this way)."""
    b = np.asarray(f, dtype=np.float32).view(np.uint32).astype(np.uint64)
    ef = (b >> np.uint64(23)) & np.uint64(0xFF)
    ed = np.where(ef == 0xFF, np.uint64(0x7FF), ef + np.uint64(1023 - 127))
    hw = (b & np.uint64(0x80000000)) | (ed << np.uint64(20)) | ((b & np.uint64(0x7FFFFF)) >> np.uint64(3))
    lw = (b << np.uint64(29)) & np.uint64(0xFFFFFFFF)
    d = ((hw << np.uint64(32)) | lw).view(np.float64)
    return np.where(ef == 0, 0.0, d)


def test_integer_widening_is_the_exact_conversion():
    """Equal to IEEE widening for every normal float, keeps infinities and
    NaNs (so a non-finite right-hand side reaches the state and the CFL
    check), and flushes FP32 subnormals to zero like the FTZ arithmetic."""
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2 ** 32, 1_000_000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    normal = np.isfinite(f) & (np.abs(f) >= np.float32(2.0 ** -126))
    assert np.array_equal(widen_all(f[normal]), f[normal].astype(np.float64))
    special = np.array([np.inf, -np.inf, np.nan, np.float32(2.0 ** -130), -np.float32(2.0 ** -140), 0.0],
                       dtype=np.float32)
    w = widen_all(special)
    assert w[0] == np.inf and w[1] == -np.inf and np.isnan(w[2])
    assert np.all(w[3:] == 0.0)
    assert np.isnan(widen_all(f[np.isnan(f)])).all()
