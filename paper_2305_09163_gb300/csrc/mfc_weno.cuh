// Reconstruction (Sec. 3.2, 3.3): WENO5-JS and WENO3-JS edge values in FP64
// (float-float weights) and FP32, and WENO5 on non-uniform grids from the
// per-cell coefficient tables.
#pragma once
#include "mfc_common.cuh"

namespace mfc {

// ---------------------------------------------------------------------------
// WENO5-JS edge values of one cell (Sec. 3.2).  D[k] = v_{c+k-1} - v_{c+k-2},
// k = 0..3, i.e. the four differences across the five-cell stencil c-2..c+2.
// Returns eR (value at c-1/2) and eL (value at c+1/2).
//
// The Jiang-Shu smoothness indicators as quadratic forms of the differences,
//   b0 = 4/3 [ 5/2 D1^2 - 11/4 D1 D0 + D0^2 ]   (stencil c-2..c)
//   b1 = 4/3 [ D1^2 + D2^2 - 5/4 D1 D2 ]        (stencil c-1..c+1)
//   b2 = 4/3 [ 5/2 D2^2 - 11/4 D2 D3 + D3^2 ]   (stencil c..c+2),
// are evaluated without the common factor 4/3, with eps scaled by 3/4 so every
// (eps + b_r) carries the same factor and the weights are unchanged.  The
// candidates are increments over v_c (constant data reconstructs exactly).
// eps34 = 3/4 eps.
//
// FP64 path: the differences D come in as FP64 and the edge values go out as
// FP64, but the smoothness indicators, weights and weighted increments are
// evaluated in float-float arithmetic (mfc_df.cuh, ~48 bits): on GB300 this
// costs 8 FP64 instructions per variable instead of ~50.  The weights are
// normalised by m = min_r (eps + b_r), g_r = m/(eps + b_r) <= 1, so that
// (eps + b)^2 (up to ~1e40 for a 1e9 Pa pressure jump) never meets the FP32
// range; with ideal weights 1 : 6 : 3 (times 10) and candidates times 6
// (integer coefficients, exact in FP32):
//   eL - v_c = (g0^2 (5 D1 - 2 D0) + 6 g1^2 (D1 + 2 D2) + 3 g2^2 (4 D2 - D3))
//              / (6 (g0^2 + 6 g1^2 + 3 g2^2)),
//   eR - v_c = (g2^2 (2 D3 - 5 D2) - 6 g1^2 (2 D1 + D2) + 3 g0^2 (D0 - 4 D1))
//              / (6 (g2^2 + 6 g1^2 + 3 g0^2)).
// ---------------------------------------------------------------------------
// Both edges run in the two lanes of packed FP32 instructions (df2): lane x
// evaluates the c+1/2 formula on the stencil, lane y the same formula on the
// mirrored stencil (-D3, -D2, -D1, -D0), which is the edge at c-1/2 (b0 and b2
// trade places, the candidates above become the eR ones).  b1, its weight and
// m are common to both edges and are formed once.  Sums use the fast
// float-float addition: its error, ~2^-44 of the operands, is relative to the
// stencil's differences, far inside the path's parity tolerance; scalings by
// powers of two are exact.  (256^3 FP64 step: 39.0 -> 35.9 ms against the same
// arithmetic in scalar FP32 instructions.)
__device__ __forceinline__ df2 weno5_increments_pair(const df (&D)[4], double eps34) {
    const df2 X0 = df2_make(D[0], df_neg(D[3])), X1 = df2_make(D[1], df_neg(D[2]));
    const df2 X2 = df2_swap(df2_neg(X1)), X3 = df2_swap(df2_neg(X0));   // (D2, -D1), (D3, -D0)
    const df2 SX1 = df2_mul(X1, X1);                                     // (D1^2, D2^2)
    const df2 B = df2_add_fast(df2_add_fast(df2_mul(X0, X0), df2_mul_f(df2_mul(X1, X0), f2(-2.75f))),
                               df2_mul_f(SX1, f2(2.5f)));                // (b0, b2)
    const df b1 = df_add_fast(df_add_fast(df2_x(SX1), df2_y(SX1)), df_mul_f(df_mul(D[1], D[2]), -1.25f));
    const df e = df_from_double(eps34);
    const df2 T = df2_add_fast(df2_make(e, e), B);                       // (t0, t2)
    const df t1 = df_add_fast(e, b1);
    const float m = fminf(T.hi.x, fminf(t1.hi, T.hi.y));
    const df2 G = df2_div_f(f2(m), T);                                   // (g0, g2)
    const df g1 = df_div_f(m, t1);
    const df2 Q = df2_mul(G, G);                                         // (q0, q2)
    const df q1 = df_mul_f(df_mul(g1, g1), 6.f);
    const df2 Q1 = df2_make(q1, q1);
    const df2 W2 = df2_mul_f(df2_swap(Q), f2(3.f));                      // (3 q2, 3 q0)
    const df2 P0 = df2_add_fast(df2_mul_f(X1, f2(5.f)), df2_mul_pow2(X0, f2(-2.f)));
    const df2 P1 = df2_add_fast(X1, df2_mul_pow2(X2, f2(2.f)));
    const df2 P2 = df2_add_fast(df2_mul_pow2(X2, f2(4.f)), df2_neg(X3));
    const df2 num = df2_add_fast(df2_add_fast(df2_mul(Q, P0), df2_mul(Q1, P1)), df2_mul(W2, P2));
    const df2 den = df2_mul_f(df2_add_fast(df2_add_fast(Q, Q1), W2), f2(6.f));
    return df2_div(num, den);   // (increment at c+1/2, increment at c-1/2)
}

__device__ __forceinline__ void weno5_increments_df(const df (&D)[4], double eps34, df& iR, df& iL) {
    const df2 I = weno5_increments_pair(D, eps34);
    iL = df2_x(I);
    iR = df2_y(I);
}

__device__ __forceinline__ void weno5_increments(const double D[4], double eps34, df& iR, df& iL) {
    const df d[4] = {df_from_double(D[0]), df_from_double(D[1]), df_from_double(D[2]), df_from_double(D[3])};
    weno5_increments_df(d, eps34, iR, iL);
}

// The two edge values in FP64 (the increments widened and added to v_c).
__device__ __forceinline__ void weno5_edges(double vc, const double D[4], double eps34,
                                            double& eR, double& eL) {
    df iR, iL;
    weno5_increments(D, eps34, iR, iL);
    eL = vc + df_to_double(iL);
    eR = vc + df_to_double(iR);
}

// FP32 variant for the mixed path.  The weights are normalised by the smallest
// eps+beta, so no intermediate overflows FP32 (beta of a 1e9 Pa jump is ~1e19).
// FP32: both edges in the two lanes of packed FP32 instructions, lane y
// evaluating the c+1/2 formula on the mirrored stencil (-D3, -D2, -D1, -D0)
// (as weno5_increments_pair); b1, its weight and m are formed once (256^3
// mixed step 6.29 -> 6.06 ms against scalar FP32 instructions).
__device__ __forceinline__ void weno5_edges(float vc, const float D[4], float eps34, float& eR, float& eL,
                                            float& b0, float& b1, float& b2) {
    const float2 X0 = make_float2(D[0], -D[3]), X1 = make_float2(D[1], -D[2]);
    const float2 X2 = make_float2(D[2], -D[1]), X3 = make_float2(D[3], -D[0]);
    const float2 S = mul2(X1, X1);                                                     // (D1^2, D2^2)
    const float2 B = fma2(f2(2.5f), S, fma2(f2(-2.75f), mul2(X1, X0), mul2(X0, X0)));  // (b0, b2)
    b0 = B.x;
    b2 = B.y;
    b1 = fmaf(-1.25f, D[1] * D[2], S.x + S.y);
    const float2 T = add2(f2(eps34), B);
    const float t1 = eps34 + b1;
    const float m = fminf(T.x, fminf(t1, T.y));
    float2 G = make_float2(__fdividef(m, T.x), __fdividef(m, T.y));
    G = mul2(G, G);
    float g1 = __fdividef(m, t1);
    g1 *= g1;
    const float2 P0 = fma2(f2(5.f / 6.f), X1, mul2(f2(-1.f / 3.f), X0));
    const float2 P1 = fma2(f2(1.f / 6.f), X1, mul2(f2(1.f / 3.f), X2));
    const float2 P2 = fma2(f2(2.f / 3.f), X2, mul2(f2(-1.f / 6.f), X3));
    const float2 W0 = mul2(f2(0.1f), G), W1 = f2(0.6f * g1), W2 = mul2(f2(0.3f), swap2(G));
    const float2 num = fma2(W0, P0, fma2(W1, P1, mul2(W2, P2)));
    const float2 den = add2(add2(W0, W1), W2);
    const float2 E = add2(f2(vc), make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y)));
    eL = E.x;
    eR = E.y;
}
// The same without the smoothness indicators (b0, b1, b2: without their 4/3
// factor, as above).
__device__ __forceinline__ void weno5_edges(float vc, const float D[4], float eps34, float& eR, float& eL) {
    float b0, b1, b2;
    weno5_edges(vc, D, eps34, eR, eL, b0, b1, b2);
}

// ---------------------------------------------------------------------------
// WENO3-JS (the third-order variant of Sec. 3.2: k = 2 candidates) for the
// edges at c+1/2 (eL) and c-1/2 (eR) from a = v_c - v_{c-1}, b = v_{c+1} - v_c.
// With t0 = eps + a^2, t1 = eps + b^2 the weights of the candidates
// v_c + a/2 (cells c-1, c; ideal 1/3) and v_c + b/2 (cells c, c+1; ideal 2/3)
// are proportional to t1^2 and 2 t0^2, so
//   eL = v_c + (t1^2 a + 2 t0^2 b) / (2 (t1^2 + 2 t0^2))
// and, mirrored, eR = v_c - (t0^2 b + 2 t1^2 a) / (2 (t0^2 + 2 t1^2)).
// FP64 path: a and b come in as FP64, the weights and weighted increments are
// float-float (mfc_df.cuh), scaled as the FP32 variant below so nothing leaves
// the FP32 range: g_r = min(t0, t1)/t_r <= 1, weights g0^2 and 2 g1^2 at
// c+1/2, g1^2 and 2 g0^2 at c-1/2.
// ---------------------------------------------------------------------------
// The two WENO3 increments (c+1/2 in lane x, c-1/2 in lane y): lane y evaluates
// the c+1/2 formula on the mirrored differences (-b, -a).
__device__ __forceinline__ df2 weno3_increments_pair(double a, double b, double eps) {
    const df A = df_from_double(a), Bd = df_from_double(b), E = df_from_double(eps);
    const df2 X = df2_make(A, df_neg(Bd)), Y = df2_make(Bd, df_neg(A));
    const df2 T = df2_add_fast(df2_make(E, E), df2_mul(df2_make(A, Bd), df2_make(A, Bd)));   // (t0, t1)
    const float m = fminf(T.hi.x, T.hi.y);
    const df2 G = df2_div_f(f2(m), T);
    const df2 S = df2_mul(G, G);                                     // (s0, s1)
    const df2 S2 = df2_mul_pow2(df2_swap(S), f2(2.f));               // (2 s1, 2 s0)
    const df2 num = df2_add_fast(df2_mul(S, X), df2_mul(S2, Y));
    const df2 den = df2_mul_pow2(df2_add_fast(S, S2), f2(2.f));
    return df2_div(num, den);
}
__device__ __forceinline__ void weno3_edges(double vc, double a, double b, double eps, double& eR, double& eL) {
    const df2 I = weno3_increments_pair(a, b, eps);
    eL = vc + df_to_double(df2_x(I));
    eR = vc + df_to_double(df2_y(I));
}
// FP32: t^2 can overflow FP32 (a pressure jump of 1e9 Pa gives t ~ 1e18), so
// both t are scaled by their minimum first: g_r = min(t0, t1)/t_r <= 1.
__device__ __forceinline__ void weno3_edges(float vc, float a, float b, float eps, float& eR, float& eL) {
    const float t0 = fmaf(a, a, eps), t1 = fmaf(b, b, eps);
    const float m = fminf(t0, t1);
    float g0 = __fdividef(m, t0), g1 = __fdividef(m, t1);
    g0 *= g0;
    g1 *= g1;
    // weights proportional to g0/3 and 2 g1/3 at c+1/2, g1/3 and 2 g0/3 at c-1/2
    eL = vc + 0.5f * __fdividef(fmaf(2.f * g1, b, g0 * a), fmaf(2.f, g1, g0));
    eR = vc - 0.5f * __fdividef(fmaf(2.f * g0, a, g1 * b), fmaf(2.f, g0, g1));
}

// Edge values of the reconstruction of order ORDER (3 or 5) from the four
// differences D across cells c-2..c+2; epsw is the epsilon as the order's
// edge function takes it (3/4 eps for WENO5, eps for WENO3).
template <int ORDER, typename Real>
__device__ __forceinline__ void weno_edges(Real vc, const Real D[4], Real epsw, Real& eR, Real& eL) {
    static_assert(ORDER == 3 || ORDER == 5, "WENO3 or WENO5");
    if constexpr (ORDER == 3) weno3_edges(vc, D[1], D[2], epsw, eR, eL);
    else weno5_edges(vc, D, epsw, eR, eL);
}

// ---------------------------------------------------------------------------
// WENO5-JS on a non-uniform grid (Sec. 4.1, with per-cell coefficients as in
// Listing 1): row = the cell's table row (mfc_grid.cu): candidate increments
// ea_r Da_r + eb_r Db_r for both edges (values 0..11), ideal weights (12..17),
// beta_r = qa Da^2 + qab Da Db + qb Db^2 (18..26), with (Da, Db) = (D0, D1),
// (D1, D2), (D2, D3) for r = 0, 1, 2.  The indicators are the exact integrals
// (no 4/3 scaling), so eps enters unscaled.  Weights normalised by
// m = min_r (eps + beta_r) as in the uniform variants.
// ---------------------------------------------------------------------------
template <class Col>
__device__ __forceinline__ df grid_df(const Col& row, int k) {
    const float2 v = row[k];
    return {v.x, v.y};
}

template <class Col>
__device__ __forceinline__ df2 weno5_increments_nu_pair(const double D[4], double eps, const Col& row) {
    // the two edges side by side in packed FP32 instructions: lane x the c+1/2
    // edge (coefficients 0-5, 12-14), lane y the c-1/2 edge (6-11, 15-17); the
    // smoothness indicators b0 and b2 side by side, b1 alone
    const df d0 = df_from_double(D[0]), d1 = df_from_double(D[1]);
    const df d2 = df_from_double(D[2]), d3 = df_from_double(D[3]);
    auto C = [&](int kx, int ky) { return df2_make(grid_df(row, kx), grid_df(row, ky)); };
    const df2 Dlo = df2_make(d0, d2), Dhi = df2_make(d1, d3);
    const df2 Slo = df2_mul(Dlo, Dlo), Shi = df2_mul(Dhi, Dhi);   // (S0, S2), (S1, S3)
    const df2 X = df2_mul(Dlo, Dhi);                               // (D0 D1, D2 D3)
    const df2 B = df2_add_fast(df2_add_fast(df2_mul(C(18, 24), Slo), df2_mul(C(19, 25), X)),
                               df2_mul(C(20, 26), Shi));           // (b0, b2)
    const df b1 = df_add_fast(df_add_fast(df_mul(grid_df(row, 21), df2_x(Shi)), df_mul(grid_df(row, 22), df_mul(d1, d2))),
                              df_mul(grid_df(row, 23), df2_y(Slo)));
    const df e = df_from_double(eps);
    const df2 T = df2_add_fast(df2_make(e, e), B);                 // (t0, t2)
    const df t1 = df_add_fast(e, b1);
    const float m = fminf(T.hi.x, fminf(t1.hi, T.hi.y));
    const df2 G = df2_div_f(f2(m), T);
    const df2 Q = df2_mul(G, G);                                   // (q0, q2)
    const df g1 = df_div_f(m, t1);
    const df q1 = df_mul(g1, g1);
    const df2 P0 = df2_add_fast(df2_mul(C(0, 6), df2_make(d0, d0)), df2_mul(C(1, 7), df2_make(d1, d1)));
    const df2 P1 = df2_add_fast(df2_mul(C(2, 8), df2_make(d1, d1)), df2_mul(C(3, 9), df2_make(d2, d2)));
    const df2 P2 = df2_add_fast(df2_mul(C(4, 10), df2_make(d2, d2)), df2_mul(C(5, 11), df2_make(d3, d3)));
    const df2 W0 = df2_mul(C(12, 15), df2_make(df2_x(Q), df2_x(Q)));
    const df2 W1 = df2_mul(C(13, 16), df2_make(q1, q1));
    const df2 W2 = df2_mul(C(14, 17), df2_make(df2_y(Q), df2_y(Q)));
    const df2 num = df2_add_fast(df2_add_fast(df2_mul(W0, P0), df2_mul(W1, P1)), df2_mul(W2, P2));
    const df2 den = df2_add_fast(df2_add_fast(W0, W1), W2);
    return df2_div(num, den);   // (increment at c+1/2, increment at c-1/2)
}
template <class Col>
__device__ __forceinline__ void weno5_edges_nu(double vc, const double D[4], double eps, const Col& row,
                                               double& eR, double& eL) {
    const df2 I = weno5_increments_nu_pair(D, eps, row);
    eL = vc + df_to_double(df2_x(I));
    eR = vc + df_to_double(df2_y(I));
}
template <class Col>
__device__ __forceinline__ void weno5_edges_nu(float vc, const float D[4], float eps, const Col& row,
                                               float& eR, float& eL) {
    auto T = [&](int k) { return row[k].x; };
    const float S0 = D[0] * D[0], S1 = D[1] * D[1], S2 = D[2] * D[2], S3 = D[3] * D[3];
    const float b0 = fmaf(T(18), S0, fmaf(T(19), D[0] * D[1], T(20) * S1));
    const float b1 = fmaf(T(21), S1, fmaf(T(22), D[1] * D[2], T(23) * S2));
    const float b2 = fmaf(T(24), S2, fmaf(T(25), D[2] * D[3], T(26) * S3));
    const float t0 = eps + b0, t1 = eps + b1, t2 = eps + b2;
    const float m = fminf(t0, fminf(t1, t2));
    float g0 = __fdividef(m, t0), g1 = __fdividef(m, t1), g2 = __fdividef(m, t2);
    g0 *= g0;
    g1 *= g1;
    g2 *= g2;
    const float P0 = fmaf(T(0), D[0], T(1) * D[1]), P1 = fmaf(T(2), D[1], T(3) * D[2]);
    const float P2 = fmaf(T(4), D[2], T(5) * D[3]);
    const float M0 = fmaf(T(6), D[0], T(7) * D[1]), M1 = fmaf(T(8), D[1], T(9) * D[2]);
    const float M2 = fmaf(T(10), D[2], T(11) * D[3]);
    const float wL0 = T(12) * g0, wL1 = T(13) * g1, wL2 = T(14) * g2;
    const float wR0 = T(15) * g0, wR1 = T(16) * g1, wR2 = T(17) * g2;
    eL = vc + __fdividef(fmaf(wL0, P0, fmaf(wL1, P1, wL2 * P2)), wL0 + wL1 + wL2);
    eR = vc + __fdividef(fmaf(wR0, M0, fmaf(wR1, M1, wR2 * M2)), wR0 + wR1 + wR2);
}

// 1/dx of cell c of a non-uniform direction, in the path's precision.
template <bool VALUE_MAJOR>
__device__ __forceinline__ double grid_inv_dx(const float* grid, int stride, int c, double) {
    return df_to_double(grid_df(GridCol<VALUE_MAJOR>(grid, stride, c), kGridInvDx));
}
template <bool VALUE_MAJOR>
__device__ __forceinline__ float grid_inv_dx(const float* grid, int stride, int c, float) {
    return GridCol<VALUE_MAJOR>(grid, stride, c)[kGridInvDx].x;
}

}  // namespace mfc
