// Float-float ("double-single") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
// bits.  Built from the error-free transformations of Knuth (TwoSum, The Art of
// Computer Programming vol. 2, 4.2.2), Dekker (FastTwoSum, 1971) and the
// FMA form of TwoProduct, combined as in Hida, Li and Bailey's double-double
// algorithms (2001).  On GB300 an FP64 instruction costs the issue time of
// about sixty FP32 instructions, so the FP64 path evaluates its WENO weights in
// this arithmetic: each operation is 5-20 FP32 instructions with a relative
// error near 2^-46, far below the path's 1e-11 parity requirement.
//
// The explicit _rn intrinsics keep the compiler from contracting or
// reordering the transformations.  FP32 range applies (|x| < 3.4e38); callers
// keep their intermediates inside it.
#pragma once
#include <cuda_runtime.h>

namespace mfc {

struct df {
    float hi, lo;
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker).
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly (one rounding of the FMA recovers the product's error).
__device__ __forceinline__ df df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// x + y, accurate also under cancellation (both parts summed error-free).
__device__ __forceinline__ df df_add(df x, df y) {
    df s = df_two_sum(x.hi, y.hi);
    const df t = df_two_sum(x.lo, y.lo);
    s = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

// x + y with one error-free sum of the high parts ("sloppy" addition): error
// below ~2^-44 (|x| + |y|), so relative accuracy is lost only under
// cancellation.  Used where an absolute error of that size is harmless.
__device__ __forceinline__ df df_add_fast(df x, df y) {
    const df s = df_two_sum(x.hi, y.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, x.lo), y.lo));
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }

// x * 2^k (f a power of two): exact while both parts stay normal.
__device__ __forceinline__ df df_mul_pow2(df x, float f) { return {__fmul_rn(x.hi, f), __fmul_rn(x.lo, f)}; }

__device__ __forceinline__ df df_mul(df x, df y) {
    const df p = df_two_prod(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.lo, p.lo);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_fast_two_sum(p.hi, e);
}

// x * f for an FP32 f (exact small integers keep it exact up to the rounding of x).
__device__ __forceinline__ df df_mul_f(df x, float f) {
    const df p = df_two_prod(x.hi, f);
    return df_fast_two_sum(p.hi, __fmaf_rn(x.lo, f, p.lo));
}

// Approximate FP32 reciprocal (one MUFU instruction, subnormals kept): the
// divisions below correct their quotient from the exact residual, so the
// reciprocal's ~2^-23 error enters squared.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// a / b for an FP32 a: quotient from the approximate reciprocal of b.hi, then
// one correction from the exact residual a - q1 b (the FP64 256^3 step took
// 46.0 ms with the correctly rounded reciprocal, 44.3 with this one).
__device__ __forceinline__ df df_div_f(float a, df b) {
    const float y = rcp_approx(b.hi);
    const float q1 = __fmul_rn(a, y);
    const df p = df_two_prod(q1, b.hi);
    float r = __fsub_rn(__fsub_rn(a, p.hi), p.lo);
    r = __fmaf_rn(-q1, b.lo, r);
    return df_fast_two_sum(q1, __fmul_rn(r, y));
}

// a / b, the same correction with a float-float residual.
__device__ __forceinline__ df df_div(df a, df b) {
    const float y = rcp_approx(b.hi);
    const float q1 = __fmul_rn(a.hi, y);
    const df r = df_add(a, df_neg(df_mul_f(b, q1)));
    return df_fast_two_sum(q1, __fmul_rn(r.hi, y));
}

// sqrt(x) for x > 0: the correctly rounded FP32 root s of x.hi, then one
// Newton correction on the exact residual, sqrt(x) = s + (x - s^2)/(2 s)
// (Dekker 1971; Hida, Li and Bailey's double-double sqrt); ~2^-46 relative.
// x <= 0 gives 0.
__device__ __forceinline__ df df_sqrt(df x) {
    if (!(x.hi > 0.f)) return {0.f, 0.f};
    const float s = __fsqrt_rn(x.hi);
    const df r = df_add(x, df_neg(df_two_prod(s, s)));
    return df_fast_two_sum(s, __fmul_rn(r.hi, __fmul_rn(0.5f, __frcp_rn(s))));
}

// An FP64 value carried bit for bit in a float-float slot (the same 8 bytes):
// the six-equation sweeps keep their volume-fraction edges in FP64.
__device__ __forceinline__ df df_pack(double d) {
    return {__int_as_float(__double2loint(d)), __int_as_float(__double2hiint(d))};
}
__device__ __forceinline__ double df_unpack(df x) {
    return __hiloint2double(__float_as_int(x.lo), __float_as_int(x.hi));
}

// ---------------------------------------------------------------------------
// Two float-float values side by side: the same operation sequence as the
// scalar functions above, applied to both lanes of packed FP32 instructions
// (add/mul/fma .f32x2 of the sm_100 family: one issue slot per pair).  A
// difference a - b is formed as one rounding of a + (-1) b, the same value.
// ---------------------------------------------------------------------------
struct df2 {
    float2 hi, lo;
};

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }

__device__ __forceinline__ df2 df2_make(df x, df y) { return {make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)}; }
__device__ __forceinline__ df df2_x(df2 a) { return {a.hi.x, a.lo.x}; }
__device__ __forceinline__ df df2_y(df2 a) { return {a.hi.y, a.lo.y}; }
__device__ __forceinline__ df2 df2_swap(df2 a) { return {swap2(a.hi), swap2(a.lo)}; }

__device__ __forceinline__ df2 df2_two_sum(float2 a, float2 b) {
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}

__device__ __forceinline__ df2 df2_fast_two_sum(float2 a, float2 b) {
    const float2 s = add2(a, b);
    return {s, sub2(b, sub2(s, a))};
}

// the product's error as fma(a, b, -p)
__device__ __forceinline__ df2 df2_two_prod(float2 a, float2 b) {
    const float2 p = mul2(a, b);
    return {p, fma2(a, b, make_float2(-p.x, -p.y))};
}

__device__ __forceinline__ df2 df2_add(df2 x, df2 y) {
    df2 s = df2_two_sum(x.hi, y.hi);
    const df2 t = df2_two_sum(x.lo, y.lo);
    s = df2_fast_two_sum(s.hi, add2(s.lo, t.hi));
    return df2_fast_two_sum(s.hi, add2(s.lo, t.lo));
}

__device__ __forceinline__ df2 df2_add_fast(df2 x, df2 y) {
    const df2 s = df2_two_sum(x.hi, y.hi);
    return df2_fast_two_sum(s.hi, add2(add2(s.lo, x.lo), y.lo));
}

__device__ __forceinline__ df2 df2_neg(df2 x) {
    return {make_float2(-x.hi.x, -x.hi.y), make_float2(-x.lo.x, -x.lo.y)};
}

__device__ __forceinline__ df2 df2_mul_pow2(df2 x, float2 f) { return {mul2(x.hi, f), mul2(x.lo, f)}; }

__device__ __forceinline__ df2 df2_mul(df2 x, df2 y) {
    const df2 p = df2_two_prod(x.hi, y.hi);
    float2 e = fma2(x.hi, y.lo, p.lo);
    e = fma2(x.lo, y.hi, e);
    return df2_fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df2 df2_mul_f(df2 x, float2 f) {
    const df2 p = df2_two_prod(x.hi, f);
    return df2_fast_two_sum(p.hi, fma2(x.lo, f, p.lo));
}

__device__ __forceinline__ df2 df2_div_f(float2 a, df2 b) {
    const float2 y = make_float2(rcp_approx(b.hi.x), rcp_approx(b.hi.y));
    const float2 q1 = mul2(a, y);
    const df2 p = df2_two_prod(q1, b.hi);
    float2 r = sub2(sub2(a, p.hi), p.lo);
    r = fma2(make_float2(-q1.x, -q1.y), b.lo, r);
    return df2_fast_two_sum(q1, mul2(r, y));
}

__device__ __forceinline__ df2 df2_div(df2 a, df2 b) {
    const float2 y = make_float2(rcp_approx(b.hi.x), rcp_approx(b.hi.y));
    const float2 q1 = mul2(a.hi, y);
    const df2 r = df2_add(a, df2_neg(df2_mul_f(b, q1)));
    return df2_fast_two_sum(q1, mul2(r.hi, y));
}

// x < y (parts normalised: |lo| <= ulp(hi)/2).
__device__ __forceinline__ bool df_lt(df x, df y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
__device__ __forceinline__ df df_min(df x, df y) { return df_lt(y, x) ? y : x; }
__device__ __forceinline__ df df_max(df x, df y) { return df_lt(x, y) ? y : x; }

// FP64 -> float-float by integer operations on the bit pattern (FP64<->FP32
// conversion instructions run on the FP64 pipe, the scarce one on GB300): hi
// takes the sign, the rebiased exponent and the top 23 stored significand bits
// (a truncation, exact), lo the remaining 29 bits scaled by 2^(E-52), so
// hi + lo equals d to ~2^-48 relative.  |d| < 2^-126 gives 0 and for
// |d| < 2^-74 lo is dropped (absolute error < 2^-98); |d| must stay below
// 2^128.
__device__ __forceinline__ df df_from_double(double d) {
    const unsigned hw = (unsigned)__double2hiint(d), lw = (unsigned)__double2loint(d);
    const unsigned sign = hw & 0x80000000u;
    const int ef = (int)((hw >> 20) & 0x7FFu) - 1023 + 127;
    const unsigned hb = sign | ((unsigned)ef << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    const int es = ef - 52;
    const float lo = __uint2float_rn(lw & 0x1FFFFFFFu) * __int_as_float(max(es, 1) << 23);
    return {ef > 0 ? __int_as_float((int)hb) : 0.f, es > 0 ? __int_as_float(__float_as_int(lo) | (int)sign) : 0.f};
}

// FP32 -> FP64 by integer operations (exact for normal numbers; zero and FP32
// subnormals give 0; infinities and NaNs are not mapped: the float-float
// arithmetic of the FP64 path never forms them).
__device__ __forceinline__ double df_widen(float f) {
    const unsigned b = (unsigned)__float_as_int(f);
    const unsigned ef = (b >> 23) & 0xFFu;
    const unsigned hw = (b & 0x80000000u) | ((ef + (1023u - 127u)) << 20) | ((b & 0x7FFFFFu) >> 3);
    return ef ? __hiloint2double((int)hw, (int)(b << 29)) : 0.0;
}

// df_widen that also keeps infinities and NaNs (the FP32 forms' RK update,
// where a non-finite right-hand side must reach the state and the CFL check).
__device__ __forceinline__ double widen_all(float f) {
    const unsigned b = (unsigned)__float_as_int(f);
    const unsigned ef = (b >> 23) & 0xFFu;
    const unsigned ed = ef == 0xFFu ? 0x7FFu : ef + (1023u - 127u);
    const unsigned hw = (b & 0x80000000u) | (ed << 20) | ((b & 0x7FFFFFu) >> 3);
    return ef ? __hiloint2double((int)hw, (int)(b << 29)) : 0.0;
}

__device__ __forceinline__ double df_to_double(df x) { return df_widen(x.hi) + df_widen(x.lo); }

// FP64 -> FP32 rounded to nearest (ties to even) by integer operations on the
// bit pattern: the same result as the conversion instruction for every value
// in the normal FP32 range; |d| < 2^-126 gives a signed zero and |d| >= 2^128
// (after rounding) infinity.
__device__ __forceinline__ float narrow_rn(double d) {
    const unsigned hw = (unsigned)__double2hiint(d), lw = (unsigned)__double2loint(d);
    const unsigned sign = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7FFu) - 1023 + 127;
    if (e <= 0) return __int_as_float((int)sign);
    if (e >= 255) return __int_as_float((int)(sign | 0x7F800000u));
    const unsigned m23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);   // top 23 stored bits
    const unsigned rem = lw & 0x1FFFFFFFu;                       // the 29 bits below
    const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
    // a carry out of the significand moves into the exponent, as rounding does
    return __int_as_float((int)(sign | (((unsigned)e << 23) + m23 + up)));
}

}  // namespace mfc
