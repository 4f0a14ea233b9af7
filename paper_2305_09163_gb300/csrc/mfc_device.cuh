// Device code for the five-equation (Allaire) diffuse-interface right-hand side
// on GB300 (sm_103a).  Templates over the arithmetic type Real (double for the
// FP64 path, float for the mixed path), the number of fluids NF, the number of
// dimensions NDIM and the sweep direction DIR.
//
// Method (arXiv 2305.09163):
//   Sec. 2.1      stiffened-gas EOS and the Allaire model (K div u dropped)
//   Sec. 3.1      semi-discrete operator, Eq. "fvmdis", with face velocities for div u
//   Sec. 3.2      WENO5-JS reconstruction of primitive variables
//   Sec. 3.2.1    HLLC approximate Riemann solver
//   Sec. 3.3      ghost cells three deep (periodic, transmissive, reflective)
//   Sec. 3.4      SSP (TVD) Runge-Kutta 3 update
//
// GB300 design: the FP64 pipe issues about 2 DFMA per SM clock, ~1/58 of FP32,
// and FP64 compares run on it too, while FP32<->FP64 conversions and integer
// work do not.  The FP64 path is therefore bound by FP64 instructions, not by
// HBM, and the kernels minimise them: each cell's two WENO edge values share one
// set of smoothness indicators and one reciprocal (a Newton-Raphson refinement
// of an FP32 seed), the ideal weights are folded into the candidate constants,
// positivity tests are integer tests on bit patterns, and every face flux is
// computed once.  Flux difference, alpha div(u) source and the RK3 stage update
// are applied in the same pass.  No atomics touch the state, so results are
// bitwise reproducible.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mfc_df.cuh"
#include "mfc_mlp.cuh"

namespace mfc {

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2, BC_CHARACTERISTIC = 3 };

struct Geometry {
    int n[3];
    long long ncell;
    int bc_lo[3], bc_hi[3];
    double inv_dx[3];
};

// Mixture closure written as Gamma = G_N + sum_{k<N} alpha_k dG_k, with
// G_k = 1/(gamma_k - 1) and P_k = gamma_k pinf_k/(gamma_k - 1); this is
// sum_k alpha_k G_k with alpha_N = 1 - sum_{k<N} alpha_k (Sec. 2.1).
// The six-equation model's frozen sound speed (Sec. 2.3), r c^2 =
// sum_k alpha_k g_k (p + pinf_k) = A p + B, is written the same way:
// A = A_N + sum_{k<N} alpha_k dA_k (A_k = g_k), B likewise (B_k = g_k pinf_k).
struct EosConst {
    double G_N, P_N;
    double dG[2], dP[2];
    double A_N, B_N;
    double dA[2], dB[2];
};

// FP32 copies of the constants the FP32 kernels use, converted once on the
// host (a conversion from FP64 in the kernel would run on the FP64 pipe, and
// the compiler may repeat it at every use).
struct EosConstF {
    float G_N, P_N;
    float dG[2], dP[2];
    float A_N, B_N;
    float dA[2], dB[2];
};

// Arguments of one directional sweep.
struct SweepArgs {
    Geometry g;
    EosConst e;
    const void* w;          // primitives [NS][ncell], Real
    void* R;                // right-hand side accumulator [NS][ncell], Real
    int mode;               // 0: R = s; 1: R += s; 2: RK stage update; 3: out = R + s
    int acc_in;             // modes 2/3: add the accumulator R (earlier sweeps)
    const double* q0;       // RK: state at t^n
    const double* qs;       // RK: current stage state
    double* qout;           // RK: output stage state (may alias qs or q0)
    double* out;            // mode 3: float64 right-hand side output
    double c0, c1, dt;      // RK: qout = c0 q0 + c1 (qs + dt (R + s))
    double eps;             // WENO epsilon
    int fallback;           // first-order fallback at non-physical faces
    int seg;                // marching kernels: cells per thread along DIR
    int nseg;               // marching kernels: segments along DIR
    long long slots_per_block;  // x-stream kernel: edge slots owned by one CTA
    unsigned long long* fallback_count;  // optional counter of fallback faces
    unsigned long long* net_rows;        // learned form: optional counter of network evaluations
    const uint4* mlp_frag;  // learned form: packed per-lane network fragments (device)
    float tau;              // learned form: discontinuity-sensor threshold
    int yz_stream;          // y/z sweeps: 1 = stream kernel, 0 = pencil marching
    int bound;              // learned form: range safeguard on learned edge values
    const float* grid[3];   // non-uniform directions: WENO5 table (GridCol layout), else null
    int grid_stride[3];     // x: cells per table value (n + 2); see GridCol
    int cbc;                // some boundary is characteristic
    const void* cbc_rates;  // their cells' normal rates (cbc_rates_kernel), Real, or null
    long long cbc_off[3][2];    // start of direction d, side s in cbc_rates (-1: not characteristic)
    int kapila;             // 1: Kapila model, K div(u) in the volume-fraction rows
    double kgam[3], kpinf[3];   // Kapila, six-equation model: gamma_k and pi_inf_k of every fluid
    double rc1[3];              // six-equation relaxation: (gamma_k - 1)/gamma_k
    float kgamf[3], kpinff[3];
    EosConstF ef;           // FP32 kernels: e, eps * 3/4 and g.inv_dx in FP32
    float eps34f;
    float epsf;
    float inv_dxf[3];
};

// Fill the FP32 constants of a from its FP64 ones (host, after e, eps and g).
inline void sweep_set_f32_constants(SweepArgs& a) {
    a.ef.G_N = (float)a.e.G_N;
    a.ef.P_N = (float)a.e.P_N;
    a.ef.A_N = (float)a.e.A_N;
    a.ef.B_N = (float)a.e.B_N;
    for (int k = 0; k < 2; ++k) {
        a.ef.dG[k] = (float)a.e.dG[k];
        a.ef.dP[k] = (float)a.e.dP[k];
        a.ef.dA[k] = (float)a.e.dA[k];
        a.ef.dB[k] = (float)a.e.dB[k];
    }
    a.eps34f = (float)(0.75 * a.eps);
    a.epsf = (float)a.eps;
    for (int k = 0; k < 3; ++k) {
        a.kgamf[k] = (float)a.kgam[k];
        a.kpinff[k] = (float)a.kpinf[k];
    }
    for (int d = 0; d < 3; ++d) a.inv_dxf[d] = (float)a.g.inv_dx[d];
}

struct PrimArgs {
    Geometry g;
    EosConst e;
    const double* q;        // conserved [NS][ncell]
    void* w;                // primitives out [NS][ncell], Real
    unsigned long long* rate_max;  // optional: max (|u_d|+c)/dx_d as ordered bits
    int* bad;               // optional: count of non-physical cells
    const float* grid[3];   // non-uniform directions: WENO5 table (GridCol layout), else null
    int grid_stride[3];
};

// Non-uniform grid table of one direction: 28 values per cell (mfc_grid.cu),
// each an FP32 pair (hi, lo), for the cells c = -1..n.  Value k of cell c is the
// pair at (c + 1) * step + k * stride: the x direction is stored value-major
// (step 1, stride n + 2) so that the lanes of an x sweep, on consecutive cells,
// read consecutive pairs; y and z row-major (step 28, stride 1), as all lanes
// of a y/z sweep read the same cell.  Value 27 is 1/dx.
constexpr int kGridInvDx = 27;
constexpr int kGridRowValues = 28;   // values per cell (mfc_grid.h: kGridRow)

// The values of one cell: value-major (x; runtime stride n + 2) or row-major
// (y, z; consecutive, so the loads take constant offsets).
template <bool VALUE_MAJOR>
struct GridCol {
    const float2* p;
    int stride;
    __device__ __forceinline__ GridCol(const float* grid, int stride_, int c)
        : p(reinterpret_cast<const float2*>(grid) + (long long)(c + 1) * (VALUE_MAJOR ? 1 : kGridRowValues)),
          stride(stride_) {}
    __device__ __forceinline__ float2 operator[](int k) const {
        return __ldg(p + (VALUE_MAJOR ? (long long)k * stride : (long long)k));
    }
};

// Variables of a cell.  The reconstructed (primitive) ones, NS of them, are
// the same for every model; the six-equation model's state appends the N
// phase internal energies a_k r_k e_k (rows NS .. NQ-1).
template <int NF, int NDIM, bool SIX = false> struct Layout {
    static constexpr int NS = 2 * NF + NDIM;
    static constexpr int NQ = NS + (SIX ? NF : 0);
    static constexpr int IM = NF;              // first momentum / velocity
    static constexpr int IE = NF + NDIM;       // energy / pressure
    static constexpr int IA = NF + NDIM + 1;   // first transported volume fraction
    static constexpr int II = NS;              // six-equation model: first phase internal energy
};

__host__ __device__ inline long long stride_of(const Geometry& g, int d) {
    return d == 0 ? 1LL : (d == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
}

// Ghost-cell index mapping along one axis (Sec. 3.3).  Valid for i in
// [-3, n+2] and n >= 3.  Sets *flip for reflective ghosts.
__device__ __forceinline__ int ghost_map(int i, int n, int bclo, int bchi, bool* flip) {
    if (i < 0) {
        if (bclo == BC_PERIODIC) return i + n;
        if (bclo == BC_TRANSMISSIVE || bclo == BC_CHARACTERISTIC) return 0;
        *flip = true;
        return -i - 1;
    }
    if (i >= n) {
        if (bchi == BC_PERIODIC) return i - n;
        if (bchi == BC_TRANSMISSIVE || bchi == BC_CHARACTERISTIC) return n - 1;
        *flip = true;
        return 2 * n - 1 - i;
    }
    return i;
}

// ---------------------------------------------------------------------------
// FP64 reciprocal by Newton-Raphson refinement (third-order step
// y <- y + y (e + e^2), e = 1 - d y) of an FP32 hardware estimate.  The seed
// is formed with integer operations only: the top 23 mantissa bits of d are
// placed in a float in [1,2), its approximate reciprocal is taken, and the
// exponent of d is subtracted back in.  The seed is good to ~2^-22, one step
// gives full FP64 precision (within 1 ulp of the correctly rounded 1/d).
// Valid for finite normal d; zero and subnormal inputs return +-inf.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp_nr(double d) {
    const long long bits = __double_as_longlong(d);
    const int hi = (int)(bits >> 32);
    const int e = (hi >> 20) & 0x7FF;
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const unsigned m23 = (((unsigned)hi & 0xFFFFFu) << 3) | ((unsigned)bits >> 29);
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__uint_as_float(0x3F800000u | m23)));
    const unsigned rb = __float_as_uint(r);
    const int ed = (int)((rb >> 23) & 0xFF) - 127 - (e - 1023) + 1023;
    const unsigned mr = rb & 0x7FFFFFu;
    const double y = __hiloint2double((int)(sign | ((unsigned)ed << 20) | (mr >> 3)), (int)(mr << 29));
    const double err = fma(-d, y, 1.0);
    const double res = fma(y, fma(err, err, err), y);
    return e == 0 ? __longlong_as_double((long long)((unsigned long long)sign << 32) | 0x7FF0000000000000LL) : res;
}

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
__device__ __forceinline__ void weno5_edges(double vc, const double D[4], double eps34,
                                            double& eR, double& eL) {
    // sums use the fast float-float addition: its error, ~2^-44 of the
    // operands, is relative to the stencil's differences, far inside the
    // path's parity tolerance; scalings by 2 and 4 are exact
    const df d0 = df_from_double(D[0]), d1 = df_from_double(D[1]);
    const df d2 = df_from_double(D[2]), d3 = df_from_double(D[3]);
    const df S1 = df_mul(d1, d1), S2 = df_mul(d2, d2);
    const df b0 = df_add_fast(df_add_fast(df_mul(d0, d0), df_mul_f(df_mul(d1, d0), -2.75f)), df_mul_f(S1, 2.5f));
    const df b1 = df_add_fast(df_add_fast(S1, S2), df_mul_f(df_mul(d1, d2), -1.25f));
    const df b2 = df_add_fast(df_add_fast(df_mul(d3, d3), df_mul_f(df_mul(d2, d3), -2.75f)), df_mul_f(S2, 2.5f));
    const df e = df_from_double(eps34);
    const df t0 = df_add_fast(e, b0), t1 = df_add_fast(e, b1), t2 = df_add_fast(e, b2);
    const float m = fminf(t0.hi, fminf(t1.hi, t2.hi));
    const df g0 = df_div_f(m, t0), g1 = df_div_f(m, t1), g2 = df_div_f(m, t2);
    const df q0 = df_mul(g0, g0), q1 = df_mul_f(df_mul(g1, g1), 6.f), q2 = df_mul(g2, g2);
    // edge at c+1/2: weights q0, q1, 3 q2
    const df wL2 = df_mul_f(q2, 3.f);
    const df P0 = df_add_fast(df_mul_f(d1, 5.f), df_mul_pow2(d0, -2.f));
    const df P1 = df_add_fast(d1, df_mul_pow2(d2, 2.f));
    const df P2 = df_add_fast(df_mul_pow2(d2, 4.f), df_neg(d3));
    const df numL = df_add_fast(df_add_fast(df_mul(q0, P0), df_mul(q1, P1)), df_mul(wL2, P2));
    const df denL = df_mul_f(df_add_fast(df_add_fast(q0, q1), wL2), 6.f);
    // edge at c-1/2: weights q2, q1, 3 q0
    const df wR2 = df_mul_f(q0, 3.f);
    const df M0 = df_add_fast(df_mul_pow2(d3, 2.f), df_mul_f(d2, -5.f));
    const df M1 = df_neg(df_add_fast(df_mul_pow2(d1, 2.f), d2));
    const df M2 = df_add_fast(d0, df_mul_pow2(d1, -4.f));
    const df numR = df_add_fast(df_add_fast(df_mul(q2, M0), df_mul(q1, M1)), df_mul(wR2, M2));
    const df denR = df_mul_f(df_add_fast(df_add_fast(q2, q1), wR2), 6.f);
    eL = vc + df_to_double(df_div(numL, denL));
    eR = vc + df_to_double(df_div(numR, denR));
}

// FP32 variant for the mixed path.  The weights are normalised by the smallest
// eps+beta, so no intermediate overflows FP32 (beta of a 1e9 Pa jump is ~1e19).
__device__ __forceinline__ void weno5_edges(float vc, const float D[4], float eps34,
                                            float& eR, float& eL) {
    const float S0 = D[0] * D[0], S1 = D[1] * D[1], S2 = D[2] * D[2], S3 = D[3] * D[3];
    const float b0 = fmaf(2.5f, S1, fmaf(-2.75f, D[1] * D[0], S0));
    const float b1 = fmaf(-1.25f, D[1] * D[2], S1 + S2);
    const float b2 = fmaf(2.5f, S2, fmaf(-2.75f, D[2] * D[3], S3));
    const float t0 = eps34 + b0, t1 = eps34 + b1, t2 = eps34 + b2;
    const float m = fminf(t0, fminf(t1, t2));
    float g0 = __fdividef(m, t0), g1 = __fdividef(m, t1), g2 = __fdividef(m, t2);
    g0 *= g0; g1 *= g1; g2 *= g2;
    const float p0 = fmaf(5.f / 6.f, D[1], (-1.f / 3.f) * D[0]);
    const float p1 = fmaf(1.f / 6.f, D[1], (1.f / 3.f) * D[2]);
    const float p2 = fmaf(2.f / 3.f, D[2], (-1.f / 6.f) * D[3]);
    const float m0 = fmaf(-5.f / 6.f, D[2], (1.f / 3.f) * D[3]);
    const float m1 = fmaf(-1.f / 6.f, D[2], (-1.f / 3.f) * D[1]);
    const float m2 = fmaf(-2.f / 3.f, D[1], (1.f / 6.f) * D[0]);
    const float wl0 = 0.1f * g0, wl1 = 0.6f * g1, wl2 = 0.3f * g2;
    const float wr0 = 0.1f * g2, wr2 = 0.3f * g0;
    eL = vc + __fdividef(fmaf(wl0, p0, fmaf(wl1, p1, wl2 * p2)), wl0 + wl1 + wl2);
    eR = vc + __fdividef(fmaf(wr0, m0, fmaf(wl1, m1, wr2 * m2)), wr0 + wl1 + wr2);
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
__device__ __forceinline__ void weno3_edges(double vc, double a, double b, double eps, double& eR, double& eL) {
    const df A = df_from_double(a), Bd = df_from_double(b), E = df_from_double(eps);
    const df t0 = df_add_fast(E, df_mul(A, A)), t1 = df_add_fast(E, df_mul(Bd, Bd));
    const float m = fminf(t0.hi, t1.hi);
    const df g0 = df_div_f(m, t0), g1 = df_div_f(m, t1);
    const df s0 = df_mul(g0, g0), s1 = df_mul(g1, g1);
    const df s0x2 = df_mul_pow2(s0, 2.f), s1x2 = df_mul_pow2(s1, 2.f);
    const df numL = df_add_fast(df_mul(s0, A), df_mul(s1x2, Bd));
    const df numR = df_add_fast(df_mul(s1, Bd), df_mul(s0x2, A));
    const df denL = df_mul_pow2(df_add_fast(s0, s1x2), 2.f), denR = df_mul_pow2(df_add_fast(s1, s0x2), 2.f);
    eL = vc + df_to_double(df_div(numL, denL));
    eR = vc - df_to_double(df_div(numR, denR));
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
// WENO5-JS on a non-uniform grid (Sec. 3.3, with per-cell coefficients as in
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
__device__ __forceinline__ void weno5_edges_nu(double vc, const double D[4], double eps, const Col& row,
                                               double& eR, double& eL) {
    const df d0 = df_from_double(D[0]), d1 = df_from_double(D[1]);
    const df d2 = df_from_double(D[2]), d3 = df_from_double(D[3]);
    const df S0 = df_mul(d0, d0), S1 = df_mul(d1, d1), S2 = df_mul(d2, d2), S3 = df_mul(d3, d3);
    const df X01 = df_mul(d0, d1), X12 = df_mul(d1, d2), X23 = df_mul(d2, d3);
    const df b0 = df_add_fast(df_add_fast(df_mul(grid_df(row, 18), S0), df_mul(grid_df(row, 19), X01)),
                              df_mul(grid_df(row, 20), S1));
    const df b1 = df_add_fast(df_add_fast(df_mul(grid_df(row, 21), S1), df_mul(grid_df(row, 22), X12)),
                              df_mul(grid_df(row, 23), S2));
    const df b2 = df_add_fast(df_add_fast(df_mul(grid_df(row, 24), S2), df_mul(grid_df(row, 25), X23)),
                              df_mul(grid_df(row, 26), S3));
    const df e = df_from_double(eps);
    const df t0 = df_add_fast(e, b0), t1 = df_add_fast(e, b1), t2 = df_add_fast(e, b2);
    const float m = fminf(t0.hi, fminf(t1.hi, t2.hi));
    const df g0 = df_div_f(m, t0), g1 = df_div_f(m, t1), g2 = df_div_f(m, t2);
    const df q0 = df_mul(g0, g0), q1 = df_mul(g1, g1), q2 = df_mul(g2, g2);
    const df P0 = df_add_fast(df_mul(grid_df(row, 0), d0), df_mul(grid_df(row, 1), d1));
    const df P1 = df_add_fast(df_mul(grid_df(row, 2), d1), df_mul(grid_df(row, 3), d2));
    const df P2 = df_add_fast(df_mul(grid_df(row, 4), d2), df_mul(grid_df(row, 5), d3));
    const df wL0 = df_mul(grid_df(row, 12), q0), wL1 = df_mul(grid_df(row, 13), q1), wL2 = df_mul(grid_df(row, 14), q2);
    const df numL = df_add_fast(df_add_fast(df_mul(wL0, P0), df_mul(wL1, P1)), df_mul(wL2, P2));
    const df denL = df_add_fast(df_add_fast(wL0, wL1), wL2);
    const df M0 = df_add_fast(df_mul(grid_df(row, 6), d0), df_mul(grid_df(row, 7), d1));
    const df M1 = df_add_fast(df_mul(grid_df(row, 8), d1), df_mul(grid_df(row, 9), d2));
    const df M2 = df_add_fast(df_mul(grid_df(row, 10), d2), df_mul(grid_df(row, 11), d3));
    const df wR0 = df_mul(grid_df(row, 15), q0), wR1 = df_mul(grid_df(row, 16), q1), wR2 = df_mul(grid_df(row, 17), q2);
    const df numR = df_add_fast(df_add_fast(df_mul(wR0, M0), df_mul(wR1, M1)), df_mul(wR2, M2));
    const df denR = df_add_fast(df_add_fast(wR0, wR1), wR2);
    eL = vc + df_to_double(df_div(numL, denL));
    eR = vc + df_to_double(df_div(numR, denR));
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

template <typename Real> struct EosR {
    Real G_N, P_N, dG[2], dP[2];
    Real A_N, B_N, dA[2], dB[2];
    __device__ __forceinline__ explicit EosR(const EosConst& e)
        : G_N((Real)e.G_N), P_N((Real)e.P_N), A_N((Real)e.A_N), B_N((Real)e.B_N) {
        dG[0] = (Real)e.dG[0]; dG[1] = (Real)e.dG[1];
        dP[0] = (Real)e.dP[0]; dP[1] = (Real)e.dP[1];
        dA[0] = (Real)e.dA[0]; dA[1] = (Real)e.dA[1];
        dB[0] = (Real)e.dB[0]; dB[1] = (Real)e.dB[1];
    }
    __device__ __forceinline__ explicit EosR(const EosConstF& e) : G_N(e.G_N), P_N(e.P_N), A_N(e.A_N), B_N(e.B_N) {
        dG[0] = e.dG[0]; dG[1] = e.dG[1];
        dP[0] = e.dP[0]; dP[1] = e.dP[1];
        dA[0] = e.dA[0]; dA[1] = e.dA[1];
        dB[0] = e.dB[0]; dB[1] = e.dB[1];
    }
};

// The EOS constants, 3/4 eps and 1/dx of direction d in the sweep's precision.
template <typename Real>
__device__ __forceinline__ EosR<Real> sweep_eos(const SweepArgs& a) {
    if constexpr (sizeof(Real) == 4) return EosR<Real>(a.ef);
    else return EosR<Real>(a.e);
}
template <typename Real>
__device__ __forceinline__ Real sweep_eps34(const SweepArgs& a) {
    if constexpr (sizeof(Real) == 4) return a.eps34f;
    else return (Real)(0.75 * a.eps);
}
template <typename Real, int ORDER>
__device__ __forceinline__ Real sweep_epsw(const SweepArgs& a) {
    if constexpr (ORDER == 5) return sweep_eps34<Real>(a);
    else if constexpr (sizeof(Real) == 4) return a.epsf;
    else return (Real)a.eps;
}
template <typename Real>
__device__ __forceinline__ Real sweep_inv_dx(const SweepArgs& a, int d) {
    if constexpr (sizeof(Real) == 4) return a.inv_dxf[d];
    else return (Real)a.g.inv_dx[d];
}

__device__ __forceinline__ double real_rcp(double x) { return rcp_nr(x); }
__device__ __forceinline__ float real_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double real_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float real_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double real_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float real_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double real_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float real_max(float a, float b) { return fmaxf(a, b); }

// Sign tests on the bit pattern (integer pipe), equal to the IEEE comparisons
// for every input including -0, +-inf and NaN.
__device__ __forceinline__ bool nonneg(double x) {          // x >= 0
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return u <= 0x7FF0000000000000ULL || u == 0x8000000000000000ULL;
}
__device__ __forceinline__ bool unit_interval(double x) {   // 0 <= x <= 1
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return u <= 0x3FF0000000000000ULL || u == 0x8000000000000000ULL;
}
__device__ __forceinline__ bool positive(double x) {        // x > 0
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return u - 1ULL < 0x7FF0000000000000ULL;
}
__device__ __forceinline__ bool nonneg(float x) { return x >= 0.f; }
__device__ __forceinline__ bool unit_interval(float x) { return x >= 0.f && x <= 1.f; }
__device__ __forceinline__ bool positive(float x) { return x > 0.f; }

// Mixture quantities of one face state: rho, Gamma, Pi and (Gamma+1)p + Pi.
template <typename Real> struct Mix {
    Real r, G, P, n;
};

// Six-equation model (SIX): n = Gamma r c^2 with the frozen sound speed,
// r c^2 = A p + B, so that c^2 = n/(Gamma r) holds for both models.
template <typename Real, int NF, int NDIM, bool SIX = false>
__device__ __forceinline__ Mix<Real> mixture(const Real* s, const EosR<Real>& e) {
    using Lay = Layout<NF, NDIM>;
    Mix<Real> m;
    m.r = s[0];
#pragma unroll
    for (int k = 1; k < NF; ++k) m.r += s[k];
    m.G = e.G_N;
    m.P = e.P_N;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        m.G = fma(s[Lay::IA + k], e.dG[k], m.G);
        m.P = fma(s[Lay::IA + k], e.dP[k], m.P);
    }
    if constexpr (SIX) {
        Real A = e.A_N, B = e.B_N;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            A = fma(s[Lay::IA + k], e.dA[k], A);
            B = fma(s[Lay::IA + k], e.dB[k], B);
        }
        m.n = m.G * fma(A, s[Lay::IE], B);
    } else {
        m.n = fma(m.G + (Real)1, s[Lay::IE], m.P);
    }
    return m;
}

// A reconstructed face state is physical when every partial density is
// non-negative, every volume fraction (including alpha_N) lies in [0,1], the
// density is positive and (Gamma+1)p + Pi > 0 (six-equation model: the frozen
// r c^2 > 0; m.n carries either).
template <typename Real, int NF, int NDIM>
__device__ __forceinline__ bool face_state_ok(const Real* s, const Mix<Real>& m) {
    using Lay = Layout<NF, NDIM>;
    bool ok = positive(m.r) && positive(m.n);
#pragma unroll
    for (int k = 0; k < NF; ++k) ok = ok && nonneg(s[k]);
    if (NF > 1) {
        Real asum = s[Lay::IA];
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            ok = ok && unit_interval(s[Lay::IA + k]);
            if (k > 0) asum += s[Lay::IA + k];
        }
        ok = ok && unit_interval((Real)1 - asum);
    }
    return ok;
}

// HLLC flux and face velocity (Sec. 3.2.1) between primitive states L | R with
// normal direction DIR; Davis wave-speed estimates.  The branch order matches
// the four cases of the paper: 0<=sL; sL<0<=s*; s*<0<sR; sR<=0.
//
// Six-equation model (SIX): the phase internal energies are carried with the
// mass like the volume fractions, their face values being those of the
// phases at the face pressure, a_k (p + g_k pinf_k)/(g_k - 1) =
// a_k (G_k p + P_k); their flux is the upwind value times the face velocity.
template <typename Real, int NF, int NDIM, int DIR, bool SIX = false>
__device__ __forceinline__ void hllc(const Real* L, const Real* R, const Mix<Real>& mL, const Mix<Real>& mR,
                                     Real* F, Real& ut, const EosR<Real>* e6 = nullptr) {
    using Lay = Layout<NF, NDIM>;
    constexpr int IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    const Real uL = L[IM + DIR], uR = R[IM + DIR], pL = L[IE], pR = R[IE];
    // c^2 = ((Gamma+1)p + Pi)/(Gamma rho); one reciprocal for both sides
    const Real dL = mL.G * mL.r, dR = mR.G * mR.r;
    const Real xd = real_rcp(dL * dR);
    const Real cL = real_sqrt(mL.n * (dR * xd)), cR = real_sqrt(mR.n * (dL * xd));
    const Real sL = real_min(uL - cL, uR - cR);
    const Real sR = real_max(uL + cL, uR + cR);
    const Real aL = mL.r * (sL - uL), aR = mR.r * (sR - uR);
    const Real sS = (pR - pL + aL * uL - aR * uR) * real_rcp(aL - aR);
    const bool useL = ((Real)0 <= sL) || ((Real)0 <= sS);
    const bool star = useL ? !((Real)0 <= sL) : ((Real)0 < sR);
    Real K[Lay::NS];
#pragma unroll
    for (int v = 0; v < Lay::NS; ++v) K[v] = useL ? L[v] : R[v];
    const Real rK = useL ? mL.r : mR.r, uK = useL ? uL : uR, pK = useL ? pL : pR;
    const Real GK = useL ? mL.G : mR.G, PK = useL ? mL.P : mR.P, sK = useL ? sL : sR;
    // xi - 1 = (s* - u_K)/(s_K - s*) taken directly, so a contact (s* = u_K)
    // gives the face velocity u_K exactly
    Real rr = 0, xm1 = 0, sKe = 0;
    if (star) {
        rr = real_rcp(sK - sS);
        xm1 = (sS - uK) * rr;
        sKe = sK;
    }
    const Real xi = (Real)1 + xm1;
    ut = fma(sKe, xm1, uK);
    Real u2 = K[IM] * K[IM];
#pragma unroll
    for (int d = 1; d < NDIM; ++d) u2 = fma(K[IM + d], K[IM + d], u2);
    const Real rE = fma(GK, pK, PK) + (Real)0.5 * rK * u2;
#pragma unroll
    for (int k = 0; k < NF; ++k) F[k] = K[k] * ut;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        if (d == DIR) F[IM + d] = fma(rK * uK, ut, pK) + sKe * xi * rK * (sS - uK);
        else F[IM + d] = rK * K[IM + d] * ut;
    }
    F[IE] = fma(rE, ut, pK * uK) + sKe * (sS - uK) * fma(xi * rK, sS, pK * rr);
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) F[IA + k] = K[IA + k] * ut;
    if constexpr (SIX) {
        Real aN = 1;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            aN -= K[IA + k];
            F[Lay::NS + k] = K[IA + k] * fma(e6->G_N + e6->dG[k], pK, e6->P_N + e6->dP[k]) * ut;
        }
        F[Lay::NS + NF - 1] = aN * fma(e6->G_N, pK, e6->P_N) * ut;
    }
}

// The FP64 path's HLLC in float-float arithmetic (mfc_df.cuh): the same
// steps, branch order and xi - 1 form as hllc, on float-float copies of the
// FP64 face states (integer splits); only the mixture sums before it and the
// widening of each flux after it use the FP64 pipe.  On GB300 an FP64
// instruction costs the issue time of ~60 FP32 ones, and the FP64 solver's
// two square roots, three reciprocals and ~60 further FP64 operations per face
// were half of the sweeps' FP64 work.  Differences that can cancel (p_R - p_L,
// s - u) use the exact float-float addition; the error of the flux stays near
// 2^-44 of its terms, far below the FP64 path's 1e-11 parity requirement.
template <int NF, int NDIM, int DIR, bool SIX = false>
__device__ __forceinline__ void hllc_df(const double* L, const double* R, const Mix<double>& mL,
                                        const Mix<double>& mR, double* F, double& ut,
                                        const EosR<double>* e6 = nullptr) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    const df uL = df_from_double(L[IM + DIR]), uR = df_from_double(R[IM + DIR]);
    const df pL = df_from_double(L[IE]), pR = df_from_double(R[IE]);
    const df rL = df_from_double(mL.r), rR = df_from_double(mR.r);
    // c^2 = n/(Gamma rho)
    const df cL = df_sqrt(df_div(df_from_double(mL.n), df_mul(df_from_double(mL.G), rL)));
    const df cR = df_sqrt(df_div(df_from_double(mR.n), df_mul(df_from_double(mR.G), rR)));
    const df sL = df_min(df_add_fast(uL, df_neg(cL)), df_add_fast(uR, df_neg(cR)));
    const df sR = df_max(df_add_fast(uL, cL), df_add_fast(uR, cR));
    const df aL = df_mul(rL, df_add(sL, df_neg(uL))), aR = df_mul(rR, df_add(sR, df_neg(uR)));
    const df num = df_add(df_add(pR, df_neg(pL)), df_add(df_mul(aL, uL), df_neg(df_mul(aR, uR))));
    const df sS = df_div(num, df_add(aL, df_neg(aR)));
    const bool useL = sL.hi >= 0.f || sS.hi >= 0.f;
    const bool star = useL ? !(sL.hi >= 0.f) : (sR.hi > 0.f);
    const double* K = useL ? L : R;
    const df rK = useL ? rL : rR, uK = useL ? uL : uR, pK = useL ? pL : pR, sK = useL ? sL : sR;
    const double GK = useL ? mL.G : mR.G, PK = useL ? mL.P : mR.P;
    // xi - 1 = (s* - u_K)/(s_K - s*), exact face velocity u_K at a contact
    df rr = {0.f, 0.f}, xm1 = {0.f, 0.f}, sKe = {0.f, 0.f};
    const df dsu = df_add(sS, df_neg(uK));
    if (star) {
        rr = df_div({1.f, 0.f}, df_add(sK, df_neg(sS)));
        xm1 = df_mul(dsu, rr);
        sKe = sK;
    }
    const df xi = df_add_fast({1.f, 0.f}, xm1);
    const df utd = df_add_fast(uK, df_mul(sKe, xm1));
    df Kd[NS];
#pragma unroll
    for (int v = 0; v < NS; ++v) Kd[v] = df_from_double(K[v]);
    df u2 = df_mul(Kd[IM], Kd[IM]);
#pragma unroll
    for (int dd = 1; dd < NDIM; ++dd) u2 = df_add_fast(u2, df_mul(Kd[IM + dd], Kd[IM + dd]));
    const df rE = df_add_fast(df_add_fast(df_mul(df_from_double(GK), pK), df_from_double(PK)),
                              df_mul_pow2(df_mul(rK, u2), 0.5f));
#pragma unroll
    for (int k = 0; k < NF; ++k) F[k] = df_to_double(df_mul(Kd[k], utd));
    const df sKds = df_mul(sKe, dsu);   // s_K (s* - u_K)
#pragma unroll
    for (int dd = 0; dd < NDIM; ++dd) {
        if (dd == DIR)
            F[IM + dd] = df_to_double(df_add_fast(df_add_fast(df_mul(df_mul(rK, uK), utd), pK), df_mul(df_mul(sKds, xi), rK)));
        else
            F[IM + dd] = df_to_double(df_mul(df_mul(rK, Kd[IM + dd]), utd));
    }
    F[IE] = df_to_double(df_add_fast(df_add_fast(df_mul(rE, utd), df_mul(pK, uK)),
                                     df_mul(sKds, df_add_fast(df_mul(df_mul(xi, rK), sS), df_mul(pK, rr)))));
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) F[IA + k] = df_to_double(df_mul(Kd[IA + k], utd));
    ut = df_to_double(utd);
    if constexpr (SIX) {
        double aN = 1.0;
        const double pKd = K[IE];
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            aN -= K[IA + k];
            F[NS + k] = K[IA + k] * fma(e6->G_N + e6->dG[k], pKd, e6->P_N + e6->dP[k]) * ut;
        }
        F[NS + NF - 1] = aN * fma(e6->G_N, pKd, e6->P_N) * ut;
    }
}

// Count one fallback face per calling lane with one atomic per converged
// group of lanes (a single global counter takes every fallback of the grid).
__device__ __forceinline__ void count_fallback(unsigned long long* counter) {
    if (!counter) return;
    const unsigned mask = __activemask();
    if ((int)(threadIdx.x & 31) == __ffs((int)mask) - 1) atomicAdd(counter, (unsigned long long)__popc(mask));
}

// Face flux between reconstructed states (with the optional first-order
// fallback to the two cell values cl | cr).
template <typename Real, int NF, int NDIM, int DIR, bool SIX = false>
__device__ __forceinline__ void face_flux(const SweepArgs& a, const EosR<Real>& e, const Real* eLs, const Real* eRs,
                                          const Real* cl, const Real* cr, Real* F, Real& ut) {
    constexpr int NS = Layout<NF, NDIM>::NS;
    Mix<Real> mL = mixture<Real, NF, NDIM, SIX>(eLs, e);
    Mix<Real> mR = mixture<Real, NF, NDIM, SIX>(eRs, e);
    bool first = false;
    if (a.fallback) {
        first = !(face_state_ok<Real, NF, NDIM>(eLs, mL) && face_state_ok<Real, NF, NDIM>(eRs, mR));
    }
    if constexpr (sizeof(Real) == 4) {
        // FP32: a per-lane branch (the compiler schedules this form best)
        if (first) {
            count_fallback(a.fallback_count);
            Real fl[NS], fr[NS];
#pragma unroll
            for (int v = 0; v < NS; ++v) { fl[v] = cl[v]; fr[v] = cr[v]; }
            mL = mixture<Real, NF, NDIM, SIX>(fl, e);
            mR = mixture<Real, NF, NDIM, SIX>(fr, e);
            hllc<Real, NF, NDIM, DIR, SIX>(fl, fr, mL, mR, F, ut, &e);
        } else {
            hllc<Real, NF, NDIM, DIR, SIX>(eLs, eRs, mL, mR, F, ut, &e);
        }
        return;
    }
    if constexpr (sizeof(Real) == 8) {
        // FP64: select the states first so that the solver (float-float, large)
        // is inlined once and a warp with falling-back lanes runs it once
        Real sl[NS], sr[NS];
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            sl[v] = first ? cl[v] : eLs[v];
            sr[v] = first ? cr[v] : eRs[v];
        }
        if (first) {
            count_fallback(a.fallback_count);
            mL = mixture<Real, NF, NDIM, SIX>(sl, e);
            mR = mixture<Real, NF, NDIM, SIX>(sr, e);
        }
        hllc_df<NF, NDIM, DIR, SIX>(sl, sr, mL, mR, F, ut, &e);
    }
}

// ---------------------------------------------------------------------------
// Learned form (the paper has no learned part; the network replaces the
// WENO5-JS nonlinear weights of Sec. 3.2).  Per cell and variable the FP32
// WENO5 pieces are formed as in the mixed path.  WENO5-JS weights are kept
// where the discontinuity sensor trips (max_r b_r > tau (min_r b_r + 1e-6 s^2),
// b the smoothness indicators without their 4/3 factor), where the stencil is
// flat to FP32 resolution (s <= 1e-7 |v_c|), and where the learned edge value
// would leave the range of cells c-1, c, c+1.  Only the stencils whose learned
// value can be used go to the network: the warp packs them (ballot and prefix
// count) into shared memory as BF16 rows of the five normalised differences,
// one row per edge, evaluates the network on the tensor cores 16 rows per
// tile, and each lane turns its rows' logits into weights and edge values.
// All 32 lanes must call these functions.
// ---------------------------------------------------------------------------
#ifndef MFC_LEARN_TILES
#define MFC_LEARN_TILES 1
#endif
constexpr int kLearnTiles = MFC_LEARN_TILES;

template <int NS> struct LearnSmem {
    // one row per network evaluation (both edges of up to 32 cells x NS
    // variables): BF16 inputs in columns 0..4, then overwritten by the logits
    uint4 row[2 * NS * 32];
};

// Network over rows 0..nrows-1 of sm; each row's inputs are replaced by its
// three logits (FP32, words 0..2).
template <int NS>
__device__ __forceinline__ void learned_logits(const uint4* __restrict__ frag, LearnSmem<NS>& sm, int nrows,
                                               int lane) {
    const int g = lane >> 2, t = lane & 3;
    const int nt = (nrows + 15) >> 4;
    const uint32_t* rw = reinterpret_cast<const uint32_t*>(sm.row);
    float* rf = reinterpret_cast<float*>(sm.row);
    __syncwarp();
    if (nt == 0) return;
    MlpWeights W;
    mlp_weights_from_frag(frag, W, lane);
    // kLearnTiles independent tiles at a time so their tensor-core chains overlap
#pragma unroll 1
    for (int t0 = 0; t0 < nt; t0 += kLearnTiles) {
        float z[kLearnTiles][4];
#pragma unroll
        for (int u = 0; u < kLearnTiles; ++u) {
            if (t0 + u < nt) {
                const int r0 = 16 * (t0 + u);
                const uint32_t a_in[2] = {rw[4 * (r0 + g) + t], rw[4 * (r0 + g + 8) + t]};
                mlp_tile_logits(W, a_in, z[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kLearnTiles; ++u) {
            if (t0 + u < nt && t < 2) {
                const int r0 = 16 * (t0 + u);
                *reinterpret_cast<float2*>(rf + 4 * (r0 + g) + 2 * t) = make_float2(z[u][0], z[u][1]);
                *reinterpret_cast<float2*>(rf + 4 * (r0 + g + 8) + 2 * t) = make_float2(z[u][2], z[u][3]);
            }
        }
    }
    __syncwarp();
}

// Increment sum_r omega_r d_r with omega the softmax of the logits in words
// 0..2 of a row.
__device__ __forceinline__ float learned_increment(const uint4& row, float d0, float d1, float d2) {
    const float z0 = __uint_as_float(row.x), z1 = __uint_as_float(row.y), z2 = __uint_as_float(row.z);
    const float m = fmaxf(z0, fmaxf(z1, z2));
    const float e0 = __expf(z0 - m), e1 = __expf(z1 - m), e2 = __expf(z2 - m);
    return __fdividef(fmaf(e0, d0, fmaf(e1, d1, e2 * d2)), e0 + e1 + e2);
}

// Edge values of one cell for all NS variables: WENO5-JS (eRjs, eLjs) and the
// learned form (eR, eL; equal to the JS values where the sensor trips).
// stencil(v, d) returns the cell value of variable v and fills d with the four
// differences across cells c-2..c+2; it is called once per variable, and again
// for the variables whose stencils went to the network, so that the stencils
// need not stay in registers across the network.  Returns the number of
// network rows (edges) the warp evaluated.
template <int NS, typename Stencil>
__device__ __forceinline__ int learned_cell_edges(const Stencil& stencil, float eps34, float tau, bool bound,
                                                   const uint4* __restrict__ frag, LearnSmem<NS>& sm, int lane,
                                                   float (&eRjs)[NS], float (&eLjs)[NS], float (&eR)[NS],
                                                   float (&eL)[NS]) {
    const unsigned below = (1u << lane) - 1u;
    unsigned need[NS];
    int nrows = 0;
    __syncwarp();   // the previous call's logits are read before rows are rewritten
#pragma unroll
    for (int v = 0; v < NS; ++v) {
        float d[4];
        const float vc = stencil(v, d);
        weno5_edges(vc, d, eps34, eRjs[v], eLjs[v]);
        const float S0 = d[0] * d[0], S1 = d[1] * d[1], S2 = d[2] * d[2], S3 = d[3] * d[3];
        const float b0 = fmaf(2.5f, S1, fmaf(-2.75f, d[1] * d[0], S0));
        const float b1 = fmaf(-1.25f, d[1] * d[2], S1 + S2);
        const float b2 = fmaf(2.5f, S2, fmaf(-2.75f, d[2] * d[3], S3));
        const float xm2 = -(d[0] + d[1]), xm1 = -d[1], xp1 = d[2], xp2 = d[2] + d[3];
        const float sc = fmaxf(fmaxf(fabsf(xm2), fabsf(xm1)), fmaxf(fabsf(xp1), fabsf(xp2)));
        const float bmax = fmaxf(b0, fmaxf(b1, b2)), bmin = fminf(b0, fminf(b1, b2));
        const bool usejs = !(sc > 1e-7f * fabsf(vc)) || (bmax > tau * fmaf(1e-6f * sc, sc, bmin));
        need[v] = __ballot_sync(0xffffffffu, !usejs);
        if (!usejs) {
            const float is = __fdividef(1.0f, sc + 1e-30f);
            const int r = nrows + 2 * __popc(need[v] & below);
            // edge at c+1/2: stencil c-2..c+2; edge at c-1/2: the mirrored stencil
            sm.row[r] = make_uint4(pack_bf16(xm2 * is, xm1 * is), pack_bf16(0.f, xp1 * is),
                                   pack_bf16(xp2 * is, 0.f), 0u);
            sm.row[r + 1] = make_uint4(pack_bf16(xp2 * is, xp1 * is), pack_bf16(0.f, xm1 * is),
                                       pack_bf16(xm2 * is, 0.f), 0u);
        }
        nrows += 2 * __popc(need[v]);
    }
    learned_logits<NS>(frag, sm, nrows, lane);
    int r = 0;
#pragma unroll
    for (int v = 0; v < NS; ++v) {
        eL[v] = eLjs[v];
        eR[v] = eRjs[v];
        if (need[v] & (1u << lane)) {
            float d[4];
            const float vc = stencil(v, d);
            const int rr = r + 2 * __popc(need[v] & below);
            // increments at c+1/2 of the stencils c-2..c, c-1..c+1, c..c+2
            const float p0 = fmaf(5.f / 6.f, d[1], (-1.f / 3.f) * d[0]);
            const float p1 = fmaf(1.f / 6.f, d[1], (1.f / 3.f) * d[2]);
            const float p2 = fmaf(2.f / 3.f, d[2], (-1.f / 6.f) * d[3]);
            // increments at c-1/2 of the stencils c..c+2, c-1..c+1, c-2..c
            const float m0 = fmaf(-5.f / 6.f, d[2], (1.f / 3.f) * d[3]);
            const float m1 = fmaf(-1.f / 6.f, d[2], (-1.f / 3.f) * d[1]);
            const float m2 = fmaf(-2.f / 3.f, d[1], (1.f / 6.f) * d[0]);
            const float il = learned_increment(sm.row[rr], p0, p1, p2);
            const float ir = learned_increment(sm.row[rr + 1], m0, m1, m2);
            // accept a learned value only inside the range of cells c-1, c, c+1
            const float lo = fminf(0.f, fminf(-d[1], d[2])), hi = fmaxf(0.f, fmaxf(-d[1], d[2]));
            if (!(bound && (il < lo || il > hi))) eL[v] = vc + il;
            if (!(bound && (ir < lo || ir > hi))) eR[v] = vc + ir;
        }
        r += 2 * __popc(need[v]);
    }
    return nrows;
}

// Face flux of the learned form: the learned face states, else (non-physical)
// the WENO5-JS states, else the first-order cell values.
template <int NF, int NDIM, int DIR>
__device__ __forceinline__ void face_flux_learned(const SweepArgs& a, const EosR<float>& e, const float* Ll,
                                                  const float* Rl, const float* Lj, const float* Rj, const float* cl,
                                                  const float* cr, float* F, float& ut) {
    constexpr int NS = Layout<NF, NDIM>::NS;
    Mix<float> mL = mixture<float, NF, NDIM>(Ll, e);
    Mix<float> mR = mixture<float, NF, NDIM>(Rl, e);
    int choice = 0;
    if (a.fallback) {
        if (!(face_state_ok<float, NF, NDIM>(Ll, mL) && face_state_ok<float, NF, NDIM>(Rl, mR))) {
            const Mix<float> jL = mixture<float, NF, NDIM>(Lj, e);
            const Mix<float> jR = mixture<float, NF, NDIM>(Rj, e);
            if (face_state_ok<float, NF, NDIM>(Lj, jL) && face_state_ok<float, NF, NDIM>(Rj, jR)) {
                choice = 1;
                mL = jL;
                mR = jR;
            } else {
                choice = 2;
                mL = mixture<float, NF, NDIM>(cl, e);
                mR = mixture<float, NF, NDIM>(cr, e);
                count_fallback(a.fallback_count);
            }
        }
    }
    float fl[NS], fr[NS];
#pragma unroll
    for (int v = 0; v < NS; ++v) {
        fl[v] = choice == 0 ? Ll[v] : (choice == 1 ? Lj[v] : cl[v]);
        fr[v] = choice == 0 ? Rl[v] : (choice == 1 ? Rj[v] : cr[v]);
    }
    hllc<float, NF, NDIM, DIR>(fl, fr, mL, mR, F, ut);
}

// Finish one cell: flux difference + alpha div(u) source, then the epilogue
// selected by a.mode.
// Characteristic (non-reflecting) boundary (Sec. 3.3: characteristic-based
// conditions after Thompson).  Normal part of dq/dt of a boundary cell from
// the quasi-linear primitive equations along DIR, written with the wave
// amplitudes L1 = (u - c)(p_x - r c u_x), L5 = (u + c)(p_x + r c u_x),
// Lk = u ((a_k r_k)_x - a_k r_k p_x/(r c^2)) and u (.)_x for the tangential
// velocities and volume fractions; the amplitudes of waves entering the domain
// (speed > 0 at the low boundary, < 0 at the high one) are zero.  wb: the
// cell's primitives, wx: their one-sided derivative towards the interior
// neighbour.  Rates: p_t = -(L5 + L1)/2, u_t = -(L5 - L1)/(2 r c),
// (a_k r_k)_t = -Lk - a_k r_k (L5 + L1)/(2 r c^2), others -L; then conserved.
// Not inlined: only boundary cells run it.
template <typename Real, int NF, int NDIM, int DIR>
__device__ __noinline__ void cbc_rate(const EosR<Real>& e, const Real* wb, const Real* wx, bool high, Real* out) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    Real r = 0, G = e.G_N, P = e.P_N;
#pragma unroll
    for (int k = 0; k < NF; ++k) r += wb[k];
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        G = fma(e.dG[k], wb[IA + k], G);
        P = fma(e.dP[k], wb[IA + k], P);
    }
    const Real p = wb[IE], u = wb[IM + DIR];
    const Real rc2 = ((G + (Real)1) * p + P) / G;          // r c^2
    const Real c = sqrt(rc2 / r);
    const Real ux = wx[IM + DIR], px = wx[IE];
    const Real lam1 = u - c, lam5 = u + c;
    const bool in1 = high ? lam1 < (Real)0 : lam1 > (Real)0;
    const bool in5 = high ? lam5 < (Real)0 : lam5 > (Real)0;
    const bool inu = high ? u < (Real)0 : u > (Real)0;
    const Real L1 = in1 ? (Real)0 : lam1 * (px - r * c * ux);
    const Real L5 = in5 ? (Real)0 : lam5 * (px + r * c * ux);
    const Real ac = (L5 + L1) / (2 * rc2);
    Real wt[NS];
#pragma unroll
    for (int k = 0; k < NF; ++k) wt[k] = -(inu ? (Real)0 : u * (wx[k] - wb[k] * px / rc2)) - wb[k] * ac;
#pragma unroll
    for (int m = 0; m < NDIM; ++m) wt[IM + m] = m == DIR ? -(L5 - L1) / (2 * r * c) : (inu ? (Real)0 : -u * wx[IM + m]);
    wt[IE] = -(L5 + L1) / 2;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) wt[IA + k] = inu ? (Real)0 : -u * wx[IA + k];
    Real rt = 0;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        out[k] = wt[k];
        rt += wt[k];
    }
    Real ke = 0, kt = 0;
#pragma unroll
    for (int m = 0; m < NDIM; ++m) {
        const Real um = wb[IM + m];
        out[IM + m] = fma(um, rt, r * wt[IM + m]);
        ke = fma((Real)0.5 * um, um, ke);
        kt = fma(um, wt[IM + m], kt);
    }
    Real Gt = 0, Pt = 0;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        Gt = fma(e.dG[k], wt[IA + k], Gt);
        Pt = fma(e.dP[k], wt[IA + k], Pt);
        out[IA + k] = wt[IA + k];
    }
    out[IE] = G * wt[IE] + p * Gt + Pt + ke * rt + r * kt;
}

// Kapila coefficients (Sec. 2.1, 5-equation models): the volume-fraction rows
// carry (alpha_k + K_k) div(u) instead of alpha_k div(u), with
//   K_k = alpha_k (rho c_W^2 / Z_k - 1),  1/(rho c_W^2) = sum_j alpha_j / Z_j,
// Z_k = rho_k c_k^2 = gamma_k (p + pi_inf_k) for a stiffened gas (Kapila's
// N-phase form; for two phases the formula the section prints).  Written
// with one reciprocal: rho c_W^2 / Z_k = prod_{j != k} Z_j / sum_j alpha_j
// prod_{i != j} Z_i.  w is the primitive state of the cell.  Not inlined:
// the Allaire path of the sweeps keeps its instruction schedule.
template <typename Real, int NF, int NDIM>
__device__ __noinline__ void kapila_K(const SweepArgs& a, const Real* w, Real* K) {
    using Lay = Layout<NF, NDIM>;
    const Real p = w[Lay::IE];
    Real al[NF], Z[NF];
    Real last = (Real)1;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        al[k] = w[Lay::IA + k];
        last -= al[k];
    }
    al[NF - 1] = last;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        if constexpr (sizeof(Real) == 4) Z[k] = a.kgamf[k] * (p + a.kpinff[k]);
        else Z[k] = a.kgam[k] * (p + a.kpinf[k]);
    }
    Real pe[NF];   // product of the other phases' Z
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        Real t = (Real)1;
#pragma unroll
        for (int j = 0; j < NF; ++j)
            if (j != k) t *= Z[j];
        pe[k] = t;
    }
    Real D = 0;
#pragma unroll
    for (int k = 0; k < NF; ++k) D = fma(al[k], pe[k], D);
    const Real rD = real_rcp(D);
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) K[k] = al[k] * fma(pe[k], rD, (Real)-1);
}

// The same coefficients for the FP64 path, in float-float arithmetic
// (mfc_df.cuh) and inlined: the FP64 instructions of a reciprocal and the
// call would cost more than the rest of the source term.
template <int NF, int NDIM>
__device__ __forceinline__ void kapila_K_df(const SweepArgs& a, const double* w, double* K) {
    using Lay = Layout<NF, NDIM>;
    const df p = df_from_double(w[Lay::IE]);
    df al[NF], Z[NF];
    double last = 1.0;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        al[k] = df_from_double(w[Lay::IA + k]);
        last -= w[Lay::IA + k];
    }
    al[NF - 1] = df_from_double(last);
#pragma unroll
    for (int k = 0; k < NF; ++k)   // gamma_k as float-float: its FP32 rounding would show in K
        Z[k] = df_mul(df_add(p, df_from_double(a.kpinf[k])), df_from_double(a.kgam[k]));
    df pe[NF];   // product of the other phases' Z
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        df t = {1.f, 0.f};
        bool first = true;
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            if (j == k) continue;
            t = first ? Z[j] : df_mul(t, Z[j]);
            first = false;
        }
        pe[k] = t;
    }
    df D = df_mul(al[0], pe[0]);
#pragma unroll
    for (int k = 1; k < NF; ++k) D = df_add(D, df_mul(al[k], pe[k]));
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) K[k] = df_to_double(df_mul(al[k], df_add(df_div(pe[k], D), {-1.f, 0.f})));
}

// Six-equation model (Sec. 2.3): pressure relaxation of one cell's conserved
// state q[NQ] with infinite stiffness, in place, after a Runge-Kutta stage
// (Saurel, Petitpas & Berry 2009; Schmidmayer et al. 2020).  At fixed mass
// each phase's energy follows de_k = -p dv_k at the final pressure p, which for
// a stiffened gas gives the relaxed volume fraction
//     a_k(p) = (g_k - 1)(E_k0 + a_k0 p) / (g_k (p + pinf_k)),  E_k0 = a_k r_k e_k.
// The phases taking part are those with a_k0 > 0 and p_k0 + pinf_k > 0
// (E_k0 > a_k0 pinf_k); the others keep a_k0.  The relaxed pressure solves
// f(p) = sum_{taking part} a_k(p) - (1 - sum_{others} a_k0) = 0; on
// p > lo = -min pinf (over the phases taking part) f is convex and falls
// strictly from +inf to below zero, so the root is unique.
//  1. FP32 Newton from the pressure the mixture law gives for the total energy
//     with the old fractions (the root itself for a relaxed state): from the
//     left of the root Newton rises monotonically to it, from the right it
//     lands left of it unless it would leave the domain, when the step bisects
//     [lo, p] instead; at most 60 iterations, ending at a relative step of 2^-20;
//  2. two Newton steps with f in float-float arithmetic (f' in FP32 suffices:
//     its error only slows the quadratic convergence to a linear one with
//     factor ~1e-7), which bring p to ~1e-14 relative;
//  3. one FP64 Newton step, p1 = p0 - f(p0)/f'(p0), and the new fractions
//     a_k(p1) = a_k(p0) + a_k'(p0)(p1 - p0) (the second-order remainder is
//     below FP64 rounding): a fraction near 1 must be right to ~1e-16
//     absolute, since a trace phase's fraction is 1 minus it;
//  4. in FP64 the pressure of the total energy with the mixture law of the
//     new fractions and every phase's energy reset to it.
// On GB300 an FP64 instruction costs the issue time of ~60 FP32 ones; the
// iteration is the costly part, hence steps 1-2 (see mfc_df.cuh).
template <int NF, int NDIM>
__device__ __noinline__ void relax6(const SweepArgs& a, double* q) {
    using Lay = Layout<NF, NDIM, true>;
    constexpr int IM = Lay::IM, IE = Lay::IE, IA = Lay::IA, II = Lay::II;
    double a0[NF], E0[NF];
    bool in[NF];
    double asum = 0.0;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        a0[k] = q[IA + k];
        asum += a0[k];
    }
    a0[NF - 1] = 1.0 - asum;
    double target = 1.0;
    float lo = 0.f;
    bool any = false;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        E0[k] = q[II + k];
        in[k] = a0[k] > 0.0 && E0[k] > a0[k] * a.kpinf[k];
        if (!in[k]) {
            target -= a0[k];
            continue;
        }
        lo = any ? fmaxf(lo, -a.kpinff[k]) : -a.kpinff[k];
        any = true;
    }
    if (!any) return;   // no phase can relax: left as is (the CFL check flags it)
    // mixture-law pressure of the total energy (old fractions, then new ones)
    double r = q[0], m2 = 0.0;
#pragma unroll
    for (int k = 1; k < NF; ++k) r += q[k];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) m2 = fma(q[IM + d], q[IM + d], m2);
    const double eint = q[IE] - 0.5 * m2 / r;
    auto mixture_p = [&]() {
        double G = a.e.G_N, P = a.e.P_N;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            G = fma(q[IA + k], a.e.dG[k], G);
            P = fma(q[IA + k], a.e.dP[k], P);
        }
        return (eint - P) / G;
    };
    // the phases in float-float (integer splits) and FP32
    df a0d[NF], E0d[NF], pid[NF], c1d[NF];
    float a0f[NF], E0f[NF], pif[NF], c1f[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        a0d[k] = df_from_double(a0[k]);
        E0d[k] = df_from_double(E0[k]);
        pid[k] = df_from_double(a.kpinf[k]);
        c1d[k] = df_from_double(a.rc1[k]);
        a0f[k] = a0d[k].hi;
        E0f[k] = E0d[k].hi;
        pif[k] = a.kpinff[k];
        c1f[k] = c1d[k].hi;
    }
    const df targetd = df_from_double(target);
    // 1. FP32 Newton
    float p = (float)mixture_p();
    if (!(p > lo)) p = lo + fmaxf(fabsf(lo), 1.f);
    float hi = INFINITY;
    for (int it = 0; it < 60; ++it) {
        float f = -targetd.hi, fp = 0.f;
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            if (!in[k]) continue;
            const float t = 1.f / (p + pif[k]);
            f = fmaf(c1f[k] * fmaf(a0f[k], p, E0f[k]), t, f);
            fp = fmaf(c1f[k] * fmaf(a0f[k], pif[k], -E0f[k]), t * t, fp);
        }
        if (f > 0.f) lo = p;
        else hi = p;
        float pn = p - f / fp;
        if (!(pn > lo && pn < hi)) pn = 0.5f * (lo + (hi < INFINITY ? hi : p));
        const bool done = fabsf(pn - p) <= 0x1p-20f * fabsf(pn) || !(pn > lo && pn < hi);
        p = pn;
        if (done) break;
    }
    // 2. float-float Newton steps
    df pd = {p, 0.f};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        df f = df_neg(targetd);
        float fp = 0.f;
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            if (!in[k]) continue;
            const df num = df_add(E0d[k], df_mul(a0d[k], pd));
            const df den = df_add(pd, pid[k]);
            f = df_add(f, df_mul(c1d[k], df_div(num, den)));
            const float t = 1.f / den.hi;
            fp = fmaf(c1f[k] * fmaf(a0f[k], pif[k], -E0f[k]), t * t, fp);
        }
        pd = df_add(pd, {-(f.hi + f.lo) / fp, 0.f});
    }
    // 3. one FP64 Newton step and the fractions at its end (first order)
    const double p0 = df_to_double(pd);
    double ak[NF], dak[NF], f64 = -target, fp64 = 0.0;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        ak[k] = a0[k];
        dak[k] = 0.0;
        if (!in[k]) continue;
        const double pi = a.kpinf[k];
        const double t = 1.0 / (p0 + pi);
        ak[k] = a.rc1[k] * fma(a0[k], p0, E0[k]) * t;
        dak[k] = a.rc1[k] * fma(a0[k], pi, -E0[k]) * t * t;
        f64 += ak[k];
        fp64 += dak[k];
    }
    const double dp = df_widen(-(float)f64 / (float)fp64);
    // 4. new fractions, the pressure of the total energy, the phase energies
    double an = 1.0;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        if (in[k]) q[IA + k] = fma(dak[k], dp, ak[k]);
        an -= q[IA + k];
    }
    const double pe = mixture_p();
#pragma unroll
    for (int k = 0; k < NF - 1; ++k)
        q[II + k] = q[IA + k] * fma(a.e.G_N + a.e.dG[k], pe, a.e.P_N + a.e.dP[k]);
    q[II + NF - 1] = an * fma(a.e.G_N, pe, a.e.P_N);
}

// Normal rate of a characteristic boundary cell (flat index idx, neighbours
// sd apart along DIR; n cells along DIR) from its primitives and those of its
// interior neighbour.
template <typename Real, int NF, int NDIM, int DIR>
__device__ __noinline__ void cbc_cell_rate(const SweepArgs& a, long long idx, long long sd, int n, bool high,
                                           Real inv_dx, Real* out) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS;
    const Real* __restrict__ w = static_cast<const Real*>(a.w);
    const long long nc = a.g.ncell;
    const long long nb = n > 1 ? (high ? idx - sd : idx + sd) : idx;   // one cell: no gradient
    Real wb[NS], wx[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        wb[q] = w[q * nc + idx];
        const Real wn = w[q * nc + nb];
        wx[q] = (high ? wb[q] - wn : wn - wb[q]) * inv_dx;
    }
    cbc_rate<Real, NF, NDIM, DIR>(sweep_eos<Real>(a), wb, wx, high, out);
}

// Characteristic boundary rates of every boundary cell, ahead of the sweeps:
// one lane per cell, so no sweep warp waits on the FP64 boundary arithmetic.
// cbc_rates holds, for direction d and side s (0 low, 1 high) from
// cbc_off[d][s], NS rows of the plane's cells, indexed by the transverse flat
// index tr (x fastest among the two other directions).
template <typename Real, int NF, int NDIM>
__global__ void __launch_bounds__(256) cbc_rates_kernel(const SweepArgs a, long long total) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS;
    Real* out = static_cast<Real*>(const_cast<void*>(a.cbc_rates));
    const int nx = a.g.n[0], ny = a.g.n[1];
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        int dir = -1, side = 0;
        long long tr = 0, nt = 0, base = 0;
        for (int dd = 0; dd < NDIM && dir < 0; ++dd)
            for (int s = 0; s < 2 && dir < 0; ++s) {
                const long long o = a.cbc_off[dd][s];
                if (o < 0) continue;
                const long long cnt = a.g.ncell / a.g.n[dd];
                const long long first = o / NS;   // cells before this plane
                if (g < first + cnt) {
                    dir = dd;
                    side = s;
                    tr = g - first;
                    nt = cnt;
                    base = o;
                }
            }
        if (dir < 0) continue;
        const int n = a.g.n[dir];
        const int b = side ? n - 1 : 0;
        long long idx;
        if (dir == 0) idx = (long long)b + (long long)nx * tr;
        else if (dir == 1) idx = (tr % nx) + (long long)nx * (b + (long long)ny * (tr / nx));
        else idx = tr + (long long)nx * ny * b;
        const long long sd = stride_of(a.g, dir);
        Real inv = (Real)a.g.inv_dx[dir];
        if (a.grid[dir])
            inv = dir == 0 ? grid_inv_dx<true>(a.grid[0], a.grid_stride[0], b, Real(0))
                           : grid_inv_dx<false>(a.grid[dir], a.grid_stride[dir], b, Real(0));
        Real r[NS];
        if (dir == 0) cbc_cell_rate<Real, NF, NDIM, 0>(a, idx, sd, n, side == 1, inv, r);
        else if (dir == 1) {
            if constexpr (NDIM > 1) cbc_cell_rate<Real, NF, NDIM, 1>(a, idx, sd, n, side == 1, inv, r);
        } else {
            if constexpr (NDIM > 2) cbc_cell_rate<Real, NF, NDIM, 2>(a, idx, sd, n, side == 1, inv, r);
        }
#pragma unroll
        for (int v = 0; v < NS; ++v) out[base + v * nt + tr] = r[v];
    }
}

// Finish cell idx (coordinate b along DIR, neighbours sd apart, transverse
// flat index tr or -1): flux difference and alpha div(u) source, or, at a
// characteristic boundary, the boundary rate (from cbc_rates when the caller
// gives tr, else computed here); then store, accumulate or apply the RK stage.
//
// Six-equation model (SIX): NQ rows; the phase energies lose a_k p div(u)
// (cell values), and an RK stage update ends with the pressure relaxation
// (relax6) before it is stored.
template <typename Real, int NF, int NDIM, int DIR, bool SIX = false>
__device__ __forceinline__ void finish_cell(const SweepArgs& a, long long idx, const Real* Fm, const Real* Fp,
                                            Real um, Real up, const Real* cell, Real inv_dx, int b, long long sd,
                                            long long tr = -1) {
    using Lay = Layout<NF, NDIM, SIX>;
    constexpr int NS = Lay::NS, NQ = Lay::NQ, IA = Lay::IA;
    Real out[NQ];
#pragma unroll
    for (int v = 0; v < NQ; ++v) out[v] = (Fm[v] - Fp[v]) * inv_dx;
    const Real du = (up - um) * inv_dx;
    if constexpr (SIX) {
        const Real pdu = cell[Lay::IE] * du;
        Real aN = 1;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            aN -= cell[IA + k];
            out[Lay::II + k] -= cell[IA + k] * pdu;
        }
        out[Lay::II + NF - 1] -= aN * pdu;
    }
    if constexpr (NF > 1) {
        if (a.kapila) {
            Real K[NF - 1];
            if constexpr (sizeof(Real) == 8) kapila_K_df<NF, NDIM>(a, cell, K);
            else kapila_K<Real, NF, NDIM>(a, cell, K);
#pragma unroll
            for (int k = 0; k < NF - 1; ++k) out[IA + k] = fma(cell[IA + k] + K[k], du, out[IA + k]);
        } else {
#pragma unroll
            for (int k = 0; k < NF - 1; ++k) out[IA + k] = fma(cell[IA + k], du, out[IA + k]);
        }
    }
    if (a.cbc) {
        const int n = a.g.n[DIR];
        const bool lo = b == 0 && a.g.bc_lo[DIR] == BC_CHARACTERISTIC;
        const bool hi = b == n - 1 && a.g.bc_hi[DIR] == BC_CHARACTERISTIC;
        if (lo || hi) {   // the boundary rate replaces the flux difference and the source
            if (a.cbc_rates && tr >= 0) {
                const Real* rb = static_cast<const Real*>(a.cbc_rates) + a.cbc_off[DIR][lo ? 0 : 1] + tr;
                const long long nt = a.g.ncell / n;
#pragma unroll
                for (int v = 0; v < NS; ++v) out[v] = rb[v * nt];
            } else {
                Real cb[NS];
                cbc_cell_rate<Real, NF, NDIM, DIR>(a, idx, sd, n, !lo, inv_dx, cb);
#pragma unroll
                for (int v = 0; v < NS; ++v) out[v] = cb[v];
            }
        }
    }
    const long long nc = a.g.ncell;
    Real* R = static_cast<Real*>(a.R);
    if (a.mode == 0) {
#pragma unroll
        for (int v = 0; v < NQ; ++v) R[v * nc + idx] = out[v];
    } else if (a.mode == 1) {
#pragma unroll
        for (int v = 0; v < NQ; ++v) R[v * nc + idx] += out[v];
    } else if (a.mode == 2) {
        double qn[SIX ? NQ : 1];
#pragma unroll
        for (int v = 0; v < NQ; ++v) {
            const Real rv = a.acc_in ? R[v * nc + idx] + out[v] : out[v];
            // FP32 accumulator widened by integer operations (a conversion
            // instruction would take an FP64-pipe slot)
            double rd;
            if constexpr (sizeof(Real) == 4) rd = df_widen(rv);
            else rd = rv;
            const double s = fma(a.dt, rd, a.qs[v * nc + idx]);
            double o = a.c1 * s;
            if (a.c0 != 0.0) o = fma(a.c0, a.q0[v * nc + idx], o);
            if constexpr (SIX) qn[v] = o;
            else a.qout[v * nc + idx] = o;
        }
        if constexpr (SIX) {
            relax6<NF, NDIM>(a, qn);
#pragma unroll
            for (int v = 0; v < NQ; ++v) a.qout[v * nc + idx] = qn[v];
        }
    } else {
#pragma unroll
        for (int v = 0; v < NQ; ++v) {
            const Real rv = a.acc_in ? R[v * nc + idx] + out[v] : out[v];
            a.out[v * nc + idx] = (double)rv;
        }
    }
}

// ---------------------------------------------------------------------------
// Directional sweep for y and z.  One thread marches along one pencil segment
// of `seg` cells in direction DIR: it reconstructs the edges of cells
// s0-1..s1, forms faces s0-1/2..s1-1/2 and finishes cells s0..s1-1.  A warp
// covers 32 consecutive x of one segment (lanes past the end of a row work on
// a clamped copy and store nothing), so loads and stores are coalesced and all
// lanes of a warp run the same number of iterations, which the tensor-core
// network of the learned form (LEARNED) requires.
// ---------------------------------------------------------------------------
template <typename Real, int NF, int NDIM, int DIR, bool LEARNED = false, int ORDER = 5>
__global__ void __launch_bounds__(128) sweep_kernel(const SweepArgs a) {
    static_assert(!LEARNED || sizeof(Real) == 4, "the learned form runs in FP32");
    static_assert(!LEARNED || ORDER == 5, "the learned form replaces the WENO5 weights");
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM;
    constexpr int T1 = (DIR == 0) ? 1 : 0;
    constexpr int T2 = (DIR == 2) ? 1 : 2;
    const Real* __restrict__ w = static_cast<const Real*>(a.w);
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n1 = a.g.n[T1], n2 = a.g.n[T2], nd = a.g.n[DIR];
    const int nxc = (n1 + 31) >> 5;
    if (wid >= (long long)nxc * a.nseg * n2) return;  // whole warps only
    const int xc = (int)(wid % nxc);
    const long long rest = wid / nxc;
    const int sg = (int)(rest % a.nseg);
    const int t2 = (int)(rest / a.nseg);
    const bool active = xc * 32 + lane < n1;
    if (!LEARNED && !active) return;
    const int t1 = active ? xc * 32 + lane : n1 - 1;
    const long long sd = stride_of(a.g, DIR);
    const long long base = (long long)t1 * stride_of(a.g, T1) + (long long)t2 * stride_of(a.g, T2);
    const long long nc = a.g.ncell;
    const int s0 = sg * a.seg;
    const int s1 = min(s0 + a.seg, nd);
    const int bclo = a.g.bc_lo[DIR], bchi = a.g.bc_hi[DIR];
    const Real eps34 = sweep_epsw<Real, ORDER>(a);  // 3/4 eps (WENO5) or eps (WENO3)
    const EosR<Real> e = sweep_eos<Real>(a);
    const Real inv_dx = sweep_inv_dx<Real>(a, DIR);
    LearnSmem<NS>* lsm = nullptr;
    if constexpr (LEARNED) {
        __shared__ LearnSmem<NS> lbuf[4];
        lsm = &lbuf[threadIdx.x >> 5];
    }
    unsigned long long net_rows = 0;  // learned form: network rows of this warp

    auto load = [&](int i, Real* out) {
        bool flip = false;
        const int m = ghost_map(i, nd, bclo, bchi, &flip);
        const long long idx = base + (long long)m * sd;
#pragma unroll
        for (int v = 0; v < NS; ++v) out[v] = __ldg(w + v * nc + idx);
        if (flip) out[IM + DIR] = -out[IM + DIR];
    };

    // Window around the cell c being reconstructed: vc = c, vp1 = c+1,
    // vp2 = c+2, the four differences across c-2..c+2, and cm1 = c-1.
    Real vc[NS], vp1[NS], vp2[NS], D[NS][4], cm1[NS];
    {
        Real t[NS];
        load(s0 - 3, t);
        load(s0 - 2, cm1);
        load(s0 - 1, vc);
        load(s0, vp1);
        load(s0 + 1, vp2);
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            D[v][0] = cm1[v] - t[v];
            D[v][1] = vc[v] - cm1[v];
            D[v][2] = vp1[v] - vc[v];
            D[v][3] = vp2[v] - vp1[v];
        }
    }
    Real eLprev[NS], eLprevJ[NS], Fprev[NS], utprev = 0;
#pragma unroll
    for (int v = 0; v < NS; ++v) { eLprev[v] = 0; eLprevJ[v] = 0; Fprev[v] = 0; }

    for (int c = s0 - 1; c <= s1; ++c) {
        Real eR[NS], eL[NS], eRJ[NS], eLJ[NS];
        if constexpr (LEARNED) {
            auto stencil = [&](int v, float (&dd)[4]) -> float {
                dd[0] = D[v][0];
                dd[1] = D[v][1];
                dd[2] = D[v][2];
                dd[3] = D[v][3];
                return vc[v];
            };
            net_rows += learned_cell_edges<NS>(stencil, eps34, a.tau, a.bound != 0, a.mlp_frag, *lsm, lane, eRJ, eLJ, eR,
                                                  eL);
        } else {
#pragma unroll
            for (int v = 0; v < NS; ++v) weno_edges<ORDER>(vc[v], D[v], eps34, eR[v], eL[v]);
        }
        if (c >= s0) {
            Real F[NS], ut;
            if constexpr (LEARNED)
                face_flux_learned<NF, NDIM, DIR>(a, e, eLprev, eR, eLprevJ, eRJ, cm1, vc, F, ut);
            else
                face_flux<Real, NF, NDIM, DIR>(a, e, eLprev, eR, cm1, vc, F, ut);
            if (c >= s0 + 1 && active)
                finish_cell<Real, NF, NDIM, DIR>(a, base + (long long)(c - 1) * sd, Fprev, F, utprev, ut, cm1, inv_dx,
                                                 c - 1, sd);
#pragma unroll
            for (int v = 0; v < NS; ++v) Fprev[v] = F[v];
            utprev = ut;
        }
        // advance the window by one cell
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            eLprev[v] = eL[v];
            if constexpr (LEARNED) eLprevJ[v] = eLJ[v];
            cm1[v] = vc[v];
        }
        if (c < s1) {
            Real nw[NS];
            load(c + 3, nw);
#pragma unroll
            for (int v = 0; v < NS; ++v) {
                D[v][0] = D[v][1];
                D[v][1] = D[v][2];
                D[v][2] = D[v][3];
                D[v][3] = nw[v] - vp2[v];
                vc[v] = vp1[v];
                vp1[v] = vp2[v];
                vp2[v] = nw[v];
            }
        }
    }
    if constexpr (LEARNED) {
        if ((threadIdx.x & 31) == 0 && net_rows && a.net_rows) atomicAdd(a.net_rows, net_rows);
    }
}

// ---------------------------------------------------------------------------
// x sweep as a coalesced stream.  Every x-row of n cells is laid out as n+2
// "slots" for edge cells c = -1..n; the rows are concatenated and each CTA
// owns `slots_per_block` consecutive slots.  A chunk of 128 slots is one slot
// per lane: lane s reconstructs the edges of its cell c (five-cell stencil read
// straight from global memory, consecutive lanes = consecutive x), forms the
// face c-1/2 from its own right-side value and the left-side value of slot s-1
// (shared memory), and finishes cell c-1 from faces c-3/2 and c-1/2.  The last
// slot's left-side value and flux carry to the next chunk, and each CTA starts
// two slots early so that its first cell has both faces.  Every lane takes part
// in every chunk, as the learned form's warp-level network needs.
// ---------------------------------------------------------------------------
constexpr int kStreamThreads = 128;

template <typename Real, int NF, int NDIM, bool LEARNED = false, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
__device__ __forceinline__ void sweep_x_stream_body(const SweepArgs& a) {
    static_assert(!SIX || !LEARNED, "six-equation model: FP64 and mixed forms");
    static_assert(!NONUNIF || (!LEARNED && ORDER == 5), "non-uniform grids: WENO5, FP64 and mixed forms");
    static_assert(!LEARNED || sizeof(Real) == 4, "the learned form runs in FP32");
    static_assert(!LEARNED || ORDER == 5, "the learned form replaces the WENO5 weights");
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM;
    constexpr int NQ = Layout<NF, NDIM, SIX>::NQ;   // flux rows
    constexpr int NJ = LEARNED ? NS : 1;
    __shared__ Real sh_eL[NS][kStreamThreads + 1];
    __shared__ Real sh_eLJ[NJ][kStreamThreads + 1];
    __shared__ Real sh_F[NQ + 1][kStreamThreads + 1];
    const Real* __restrict__ w = static_cast<const Real*>(a.w);
    const int n = a.g.n[0];
    const long long rowlen = (long long)n + 2;
    const long long nrows = a.g.ncell / n;
    const long long total = rowlen * nrows;
    const long long own0 = (long long)blockIdx.x * a.slots_per_block;
    const long long own1 = min(own0 + a.slots_per_block, total);
    const long long nc = a.g.ncell;
    const int bclo = a.g.bc_lo[0], bchi = a.g.bc_hi[0];
    const Real eps34 = sweep_epsw<Real, ORDER>(a);  // 3/4 eps (WENO5) or eps (WENO3)
    const EosR<Real> e = sweep_eos<Real>(a);
    const Real inv_dx = sweep_inv_dx<Real>(a, 0);
    const int t = threadIdx.x;
    LearnSmem<NS>* lsm = nullptr;
    if constexpr (LEARNED) {
        __shared__ LearnSmem<NS> lbuf[kStreamThreads / 32];
        lsm = &lbuf[t >> 5];
    }
    unsigned long long net_rows = 0;  // learned form: network rows of this warp

    // (row, column) of this lane's slot: one 64-bit division when the slot first
    // becomes valid, then advanced by 128 slots per chunk with additions (a
    // 64-bit division per chunk would run on the FP64 pipe)
    long long srow = 0;
    int scol = 0;  // slot index within its row, 0..n+1
    bool placed = false;
    for (long long base = own0 - 2; base < own1; base += kStreamThreads) {
        const long long s = base + t;
        if (s >= 0 && !placed) {
            srow = s / rowlen;
            scol = (int)(s - srow * rowlen);
            placed = true;
        }
        const bool live = (s >= 0) && (s < own1);
        const long long row = srow;
        const int c = live ? scol - 1 : -1;
        const long long rowoff = row * n;
        if (placed) {
            scol += kStreamThreads;
            while (scol >= rowlen) {
                scol -= (int)rowlen;
                ++srow;
            }
        }
        Real cell[NS], cm1[NS], eL[NS], eR[NS], eLJ[NS], eRJ[NS];
        if constexpr (LEARNED) {
            // the five cells of this lane's stencil, re-read (L1) per variable
            int mk[5];
            bool fk[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                fk[k] = false;
                mk[k] = live ? ghost_map(c + k - 2, n, bclo, bchi, &fk[k]) : 0;
            }
            const Real* wr = w + rowoff;
            auto stencil = [&](int q, float (&dd)[4]) -> float {
                float v5[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    float x = live ? __ldg(wr + q * nc + mk[k]) : 0.f;
                    if (q == IM && fk[k]) x = -x;
                    v5[k] = x;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) dd[k] = v5[k + 1] - v5[k];
                return v5[2];
            };
            net_rows += learned_cell_edges<NS>(stencil, eps34, a.tau, a.bound != 0, a.mlp_frag, *lsm, t & 31, eRJ, eLJ,
                                                  eR, eL);
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                float x1 = live ? __ldg(wr + q * nc + mk[1]) : 0.f;
                float x2 = live ? __ldg(wr + q * nc + mk[2]) : 0.f;
                if (q == IM && fk[1]) x1 = -x1;
                if (q == IM && fk[2]) x2 = -x2;
                cm1[q] = x1;
                cell[q] = x2;
            }
        }
        Real vcv[NS], Dv[NS][4];
        if constexpr (!LEARNED) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                vcv[q] = 0;
                cm1[q] = 0;
                Dv[q][0] = Dv[q][1] = Dv[q][2] = Dv[q][3] = 0;
            }
        }
        if (!LEARNED && live) {
            Real v[5][NS];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                bool flip = false;
                const int m = ghost_map(c + k - 2, n, bclo, bchi, &flip);
#pragma unroll
                for (int q = 0; q < NS; ++q) v[k][q] = __ldg(w + q * nc + rowoff + m);
                if (flip) v[k][IM] = -v[k][IM];
            }
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                Dv[q][0] = v[1][q] - v[0][q];
                Dv[q][1] = v[2][q] - v[1][q];
                Dv[q][2] = v[3][q] - v[2][q];
                Dv[q][3] = v[4][q] - v[3][q];
                vcv[q] = v[2][q];
                cm1[q] = v[1][q];
            }
        }
        if (!LEARNED && live) {
            if constexpr (NONUNIF) {
                const GridCol<true> row(a.grid[0], a.grid_stride[0], c);
                const Real epsn = sweep_epsw<Real, 3>(a);   // unscaled eps
#pragma unroll
                for (int q = 0; q < NS; ++q) weno5_edges_nu(vcv[q], Dv[q], epsn, row, eR[q], eL[q]);
            } else {
#pragma unroll
                for (int q = 0; q < NS; ++q) weno_edges<ORDER>(vcv[q], Dv[q], eps34, eR[q], eL[q]);
            }
        }
        if constexpr (!LEARNED) {
#pragma unroll
            for (int q = 0; q < NS; ++q) cell[q] = vcv[q];
        }
        // left-side values of this chunk; slot 0 holds the carry from the last chunk
        if (live) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                sh_eL[q][t + 1] = eL[q];
                if constexpr (LEARNED) sh_eLJ[q][t + 1] = eLJ[q];
            }
        }
        __syncthreads();
        Real F[NQ], ut = 0;
        const bool has_face = live && c >= 0 && s >= own0 - 1;
        if (has_face) {
            Real lft[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) lft[q] = sh_eL[q][t];
            if constexpr (LEARNED) {
                Real lftJ[NS];
#pragma unroll
                for (int q = 0; q < NS; ++q) lftJ[q] = sh_eLJ[q][t];
                face_flux_learned<NF, NDIM, 0>(a, e, lft, eR, lftJ, eRJ, cm1, cell, F, ut);
            } else {
                face_flux<Real, NF, NDIM, 0, SIX>(a, e, lft, eR, cm1, cell, F, ut);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) sh_F[q][t + 1] = F[q];
            sh_F[NQ][t + 1] = ut;
        }
        __syncthreads();
        if (has_face && s >= own0 && c >= 1) {
            Real Fm[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) Fm[q] = sh_F[q][t];
            finish_cell<Real, NF, NDIM, 0, SIX>(a, rowoff + (c - 1), Fm, F, sh_F[NQ][t], ut, cm1,
                                           NONUNIF ? grid_inv_dx<true>(a.grid[0], a.grid_stride[0], c - 1, Real(0)) : inv_dx,
                                           c - 1, 1, row);
        }
        __syncthreads();
        // carry the last slot of the chunk into position 0
        if (t == kStreamThreads - 1) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                sh_eL[q][0] = sh_eL[q][kStreamThreads];
                if constexpr (LEARNED) sh_eLJ[q][0] = sh_eLJ[q][kStreamThreads];
            }
#pragma unroll
            for (int q = 0; q <= NQ; ++q) sh_F[q][0] = sh_F[q][kStreamThreads];
        }
        __syncthreads();
    }
    if constexpr (LEARNED) {
        if ((threadIdx.x & 31) == 0 && net_rows && a.net_rows) atomicAdd(a.net_rows, net_rows);
    }
}

template <typename Real, int NF, int NDIM, bool LEARNED = false, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
__global__ void __launch_bounds__(kStreamThreads) sweep_x_stream_kernel(const SweepArgs a) {
    sweep_x_stream_body<Real, NF, NDIM, LEARNED, ORDER, NONUNIF, SIX>(a);
}

// The learned form's x sweep bounded to 4 CTAs per SM (128 registers, 32
// bytes of spills; unbounded it took 168 and kept 12 warps per SM).
template <int NF, int NDIM>
__global__ void __launch_bounds__(kStreamThreads, 4) sweep_x_stream_learned_kernel(const SweepArgs a) {
    sweep_x_stream_body<float, NF, NDIM, true, 5, false, false>(a);
}

// FP64 sweeps bounded to 4 CTAs (16 warps) per SM, for the variants where
// the extra warps outweigh the spills (launch_sweep chooses).
template <int NF, int NDIM, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
__global__ void __launch_bounds__(kStreamThreads, 4) sweep_x_stream_f64_kernel(const SweepArgs a) {
    sweep_x_stream_body<double, NF, NDIM, false, ORDER, NONUNIF, SIX>(a);
}

// ---------------------------------------------------------------------------
// y or z sweep as a coalesced stream (FP32 paths).  A CTA of 4 warps covers 32
// consecutive x (lanes) of one pencil segment s0..s1-1 along DIR and walks it
// in chunks of 4 edge cells, one per warp: warp r of a chunk reconstructs the
// edges of cell c = base + r from its five-cell stencil, read from a shared
// ring of the 8 rows base-2..base+5 (each warp loads one new row per chunk,
// prefetched into registers during the previous chunk's arithmetic), forms the
// face c-1/2 with the left-side value of the previous row (shared memory, or
// the carry from the previous chunk) and finishes cell c-1.  Unlike the
// marching kernel no per-thread window is kept, so more warps stay resident to
// hide load and tensor-core latency.
// ---------------------------------------------------------------------------
constexpr int kRowsPerChunk = 4;

template <typename Real, int NF, int NDIM, int DIR, bool LEARNED, int ORDER, bool NONUNIF = false, bool SIX = false>
__device__ __forceinline__ void sweep_yz_stream_body(const SweepArgs& a) {
    static_assert(!SIX || !LEARNED, "six-equation model: FP64 and mixed forms");
    static_assert(!NONUNIF || (!LEARNED && ORDER == 5), "non-uniform grids: WENO5, FP64 and mixed forms");
    static_assert(!LEARNED || ORDER == 5, "the learned form replaces the WENO5 weights");
    static_assert(DIR == 1 || DIR == 2, "y or z");
    static_assert(!LEARNED || sizeof(Real) == 4, "the learned form runs in FP32");
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM;
    constexpr int NQ = Layout<NF, NDIM, SIX>::NQ;   // flux rows
    constexpr int NJ = LEARNED ? NS : 1;
    constexpr int T1 = 0;
    constexpr int T2 = (DIR == 2) ? 1 : 2;
    constexpr int RING = 2 * kRowsPerChunk;  // rows base-2 .. base+5 of a chunk
    __shared__ Real ring[RING][NS][32];
    __shared__ Real sh_eL[NS][kRowsPerChunk + 1][32];
    __shared__ Real sh_eLJ[NJ][kRowsPerChunk + 1][32];
    __shared__ Real sh_F[NQ + 1][kRowsPerChunk + 1][32];
    const Real* __restrict__ w = static_cast<const Real*>(a.w);
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int n1 = a.g.n[T1], n2 = a.g.n[T2], nd = a.g.n[DIR];
    const int nxc = (n1 + 31) >> 5;
    const long long bid = blockIdx.x;
    const int xc = (int)(bid % nxc);
    const long long rest = bid / nxc;
    const int sg = (int)(rest % a.nseg);
    const int t2 = (int)(rest / a.nseg);
    if (t2 >= n2) return;  // whole CTA
    const bool active = xc * 32 + lane < n1;
    const int t1 = active ? xc * 32 + lane : n1 - 1;
    const long long sd = stride_of(a.g, DIR);
    const long long basei = (long long)t1 * stride_of(a.g, T1) + (long long)t2 * stride_of(a.g, T2);
    const long long nc = a.g.ncell;
    const int s0 = sg * a.seg;
    const int s1 = min(s0 + a.seg, nd);
    const int bclo = a.g.bc_lo[DIR], bchi = a.g.bc_hi[DIR];
    const Real eps34 = sweep_epsw<Real, ORDER>(a);  // 3/4 eps (WENO5) or eps (WENO3)
    const EosR<Real> e = sweep_eos<Real>(a);
    const Real inv_dx = sweep_inv_dx<Real>(a, DIR);
    LearnSmem<NS>* lsm = nullptr;
    if constexpr (LEARNED) {
        __shared__ LearnSmem<NS> lbuf[kRowsPerChunk];
        lsm = &lbuf[row];
    }
    unsigned long long net_rows = 0;  // learned form: network rows of this warp
    // cell i along DIR (ghost-mapped) of this lane's column
    auto load = [&](int i, Real* out) {
        bool flip = false;
        const int m = ghost_map(i, nd, bclo, bchi, &flip);
        const long long idx = basei + (long long)m * sd;
#pragma unroll
        for (int q = 0; q < NS; ++q) out[q] = __ldg(w + q * nc + idx);
        if (flip) out[IM + DIR] = -out[IM + DIR];
    };
    auto slot = [](int i) { return ((i % RING) + RING) % RING; };
    // prologue: rows s0-3 .. s0+4 (cells base-2 .. base+5 of the first chunk)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = s0 - 3 + row + kRowsPerChunk * h;
        if (i <= s1 + 2) {
            Real v[NS];
            load(i, v);
#pragma unroll
            for (int q = 0; q < NS; ++q) ring[slot(i)][q][lane] = v[q];
        }
    }
    __syncthreads();

    for (int base = s0 - 1; base <= s1; base += kRowsPerChunk) {
        // prefetch the row the next chunk adds (cell base+6+row) while this one computes
        const int inext = base + RING - 2 + row;
        const bool pf = inext <= s1 + 2;
        Real nxt[NS];
        if (pf) load(inext, nxt);
        const int c = base + row;       // edge cell of this warp (warp-uniform)
        const bool live = c <= s1;
        Real cell[NS], cm1[NS], eL[NS], eR[NS], eLJ[NS], eRJ[NS];
        if (live) {
            if constexpr (LEARNED) {
                auto stencil = [&](int q, float (&dd)[4]) -> float {
                    float v5[5];
#pragma unroll
                    for (int k = 0; k < 5; ++k) v5[k] = ring[slot(c - 2 + k)][q][lane];
#pragma unroll
                    for (int k = 0; k < 4; ++k) dd[k] = v5[k + 1] - v5[k];
                    return v5[2];
                };
                net_rows += learned_cell_edges<NS>(stencil, eps34, a.tau, a.bound != 0, a.mlp_frag, *lsm, lane, eRJ,
                                                   eLJ, eR, eL);
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    cell[q] = ring[slot(c)][q][lane];
                    cm1[q] = ring[slot(c - 1)][q][lane];
                }
            } else {
                Real Dv[NS][4];
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const Real v0 = ring[slot(c - 2)][q][lane], v1 = ring[slot(c - 1)][q][lane];
                    const Real v2 = ring[slot(c)][q][lane], v3 = ring[slot(c + 1)][q][lane];
                    const Real v4 = ring[slot(c + 2)][q][lane];
                    Dv[q][0] = v1 - v0;
                    Dv[q][1] = v2 - v1;
                    Dv[q][2] = v3 - v2;
                    Dv[q][3] = v4 - v3;
                    cell[q] = v2;
                    cm1[q] = v1;
                }
                if constexpr (NONUNIF) {
                    const GridCol<false> grow(a.grid[DIR], a.grid_stride[DIR], c);
                    const Real epsn = sweep_epsw<Real, 3>(a);   // unscaled eps
#pragma unroll
                    for (int q = 0; q < NS; ++q) weno5_edges_nu(cell[q], Dv[q], epsn, grow, eR[q], eL[q]);
                } else {
#pragma unroll
                    for (int q = 0; q < NS; ++q) weno_edges<ORDER>(cell[q], Dv[q], eps34, eR[q], eL[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                sh_eL[q][row + 1][lane] = eL[q];
                if constexpr (LEARNED) sh_eLJ[q][row + 1][lane] = eLJ[q];
            }
        }
        __syncthreads();
        // rows base-2 .. base+1 are no longer needed: the prefetched rows replace them
        if (pf) {
#pragma unroll
            for (int q = 0; q < NS; ++q) ring[slot(inext)][q][lane] = nxt[q];
        }
        Real F[NQ], ut = 0;
        const bool has_face = live && c >= s0;
        if (has_face) {
            Real lft[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) lft[q] = sh_eL[q][row][lane];
            if constexpr (LEARNED) {
                Real lftJ[NS];
#pragma unroll
                for (int q = 0; q < NS; ++q) lftJ[q] = sh_eLJ[q][row][lane];
                face_flux_learned<NF, NDIM, DIR>(a, e, lft, eR, lftJ, eRJ, cm1, cell, F, ut);
            } else {
                face_flux<Real, NF, NDIM, DIR, SIX>(a, e, lft, eR, cm1, cell, F, ut);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) sh_F[q][row + 1][lane] = F[q];
            sh_F[NQ][row + 1][lane] = ut;
        }
        __syncthreads();
        if (has_face && c >= s0 + 1 && active) {
            Real Fm[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) Fm[q] = sh_F[q][row][lane];
            finish_cell<Real, NF, NDIM, DIR, SIX>(a, basei + (long long)(c - 1) * sd, Fm, F, sh_F[NQ][row][lane], ut, cm1,
                                             NONUNIF ? grid_inv_dx<false>(a.grid[DIR], a.grid_stride[DIR], c - 1, Real(0))
                                                     : inv_dx,
                                             c - 1, sd, (long long)t1 + (long long)n1 * t2);
        }
        __syncthreads();
        // carry the last row of the chunk into row 0
        if (row == kRowsPerChunk - 1) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                sh_eL[q][0][lane] = sh_eL[q][kRowsPerChunk][lane];
                if constexpr (LEARNED) sh_eLJ[q][0][lane] = sh_eLJ[q][kRowsPerChunk][lane];
            }
#pragma unroll
            for (int q = 0; q <= NQ; ++q) sh_F[q][0][lane] = sh_F[q][kRowsPerChunk][lane];
        }
        __syncthreads();
    }
    if constexpr (LEARNED) {
        if ((threadIdx.x & 31) == 0 && net_rows && a.net_rows) atomicAdd(a.net_rows, net_rows);
    }
}

// The y/z stream kernel of the FP32 forms.  The learned form gets its own
// entry with a register bound (4 CTAs per SM for two fluids) so that enough
// warps stay resident; the mixed form keeps the compiler's own allocation,
// which schedules its loads better.
template <typename Real, int NF, int NDIM, int DIR, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
__global__ void __launch_bounds__(32 * kRowsPerChunk) sweep_yz_stream_kernel(const SweepArgs a) {
    sweep_yz_stream_body<Real, NF, NDIM, DIR, false, ORDER, NONUNIF, SIX>(a);
}

// The mixed form's six-equation y/z sweep: bounded to 5 CTAs per SM (96
// registers; unbounded it took 107 and ran 45 instead of 37 ms over the 256^3
// bench).  A bound of one CTA per SM is not the same as none: it slowed the
// five-equation kernels by half, hence a separate entry.
template <int NF, int NDIM, int DIR, int ORDER = 5, bool NONUNIF = false>
__global__ void __launch_bounds__(32 * kRowsPerChunk, 5) sweep_yz_stream_six32_kernel(const SweepArgs a) {
    sweep_yz_stream_body<float, NF, NDIM, DIR, false, ORDER, NONUNIF, true>(a);
}

template <int NF, int NDIM, int DIR, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
__global__ void __launch_bounds__(32 * kRowsPerChunk, 4) sweep_yz_stream_f64_kernel(const SweepArgs a) {
    sweep_yz_stream_body<double, NF, NDIM, DIR, false, ORDER, NONUNIF, SIX>(a);
}

template <int NF, int NDIM, int DIR>
__global__ void __launch_bounds__(32 * kRowsPerChunk, NF <= 2 ? 4 : 3) sweep_yz_stream_learned_kernel(const SweepArgs a) {
    sweep_yz_stream_body<float, NF, NDIM, DIR, true, 5>(a);
}

// ---------------------------------------------------------------------------
// Conserved -> primitive (Sec. 2.1): rho = sum a_k r_k, u = (rho u)/rho,
// p = (rho E - rho|u|^2/2 - Pi)/Gamma.  FP64 path: all in FP64.  Mixed path:
// rho E - Pi (the water Pi ~ 7.8e8 Pa cancels against rho E) and the kinetic
// energy subtraction stay FP64, the rest is FP32.  Optionally the CFL rate
// max_d (|u_d| + c)/dx_d with c^2 = ((Gamma+1)p + Pi)/(Gamma rho), reduced to one
// max per launch with an order-preserving integer atomic (non-negative
// doubles), so it is exact and independent of scheduling.  Six-equation model
// (SIX): the frozen sound speed, r c^2 = A p + B (Sec. 2.3).
// ---------------------------------------------------------------------------
template <int NF, int NDIM, bool SIX = false>
__device__ __forceinline__ void prims_cell(const double* q, const EosConst& e, double* wv, double& c2) {
    using Lay = Layout<NF, NDIM>;
    constexpr int IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    double rho = q[0];
#pragma unroll
    for (int k = 1; k < NF; ++k) rho += q[k];
    double G = e.G_N, P = e.P_N;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        G = fma(q[IA + k], e.dG[k], G);
        P = fma(q[IA + k], e.dP[k], P);
    }
    const double x = rcp_nr(rho * G);   // FP32 seed + cubic Newton step: 3 FP64 instructions
    const double irho = G * x, iG = rho * x;
    double ke = 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) { wv[IM + d] = q[IM + d] * irho; ke = fma(q[IM + d], wv[IM + d], ke); }
    const double p = (q[IE] - 0.5 * ke - P) * iG;
#pragma unroll
    for (int k = 0; k < NF; ++k) wv[k] = q[k];
    wv[IE] = p;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) wv[IA + k] = q[IA + k];
    if constexpr (SIX) {
        double A = e.A_N, B = e.B_N;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            A = fma(q[IA + k], e.dA[k], A);
            B = fma(q[IA + k], e.dB[k], B);
        }
        c2 = fma(A, p, B) * irho;
    } else {
        c2 = fma(G + 1.0, p, P) * iG * irho;
    }
}

// FP32 form: the per-cell FP64 -> FP32 conversions by integer operations
// (narrow_rn, df_widen), since conversion instructions run on the FP64 pipe.
template <int NF, int NDIM, bool SIX = false>
__device__ __forceinline__ void prims_cell(const double* q, const EosConst& e, float* wv, float& c2) {
    using Lay = Layout<NF, NDIM>;
    constexpr int IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    float qf[Lay::NS];
#pragma unroll
    for (int v = 0; v < Lay::NS; ++v) qf[v] = v == IE ? 0.f : narrow_rn(q[v]);
    float rho = qf[0];
#pragma unroll
    for (int k = 1; k < NF; ++k) rho += qf[k];
    float G = (float)e.G_N;
    double P = e.P_N;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        G = fmaf(qf[IA + k], (float)e.dG[k], G);
        P = fma(q[IA + k], e.dP[k], P);
    }
    const float irho = __fdividef(1.0f, rho);
    float ke = 0.f;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const float m = qf[IM + d];
        wv[IM + d] = m * irho;
        ke = fmaf(m, wv[IM + d], ke);
    }
    const double eint = fma(-0.5, df_widen(ke), q[IE] - P);
    const float p = __fdividef(narrow_rn(eint), G);
#pragma unroll
    for (int k = 0; k < NF; ++k) wv[k] = qf[k];
    wv[IE] = p;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) wv[IA + k] = qf[IA + k];
    if constexpr (SIX) {
        float A = (float)e.A_N, B = (float)e.B_N;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            A = fmaf(qf[IA + k], (float)e.dA[k], A);
            B = fmaf(qf[IA + k], (float)e.dB[k], B);
        }
        c2 = __fdividef(fmaf(A, p, B), rho);
    } else {
        c2 = __fdividef(fmaf(G + 1.0f, p, narrow_rn(P)), G * rho);
    }
}

template <typename Real, int NF, int NDIM, bool RATE, bool SIX = false>
__global__ void __launch_bounds__(256) prims_kernel(const PrimArgs a) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM;
    const long long nc = a.g.ncell;
    double rate = 0.0;
    int bad = 0;
    Real* w = static_cast<Real*>(a.w);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc;
         i += (long long)gridDim.x * blockDim.x) {
        double q[NS];
#pragma unroll
        for (int v = 0; v < NS; ++v) q[v] = __ldg(a.q + v * nc + i);
        Real wv[NS], c2;
        prims_cell<NF, NDIM, SIX>(q, a.e, wv, c2);
#pragma unroll
        for (int v = 0; v < NS; ++v) w[v * nc + i] = wv[v];
        if (RATE) {
            // in the arithmetic of the path: FP64, or FP32 for the mixed path
            Real us = 0;
#pragma unroll
            for (int d = 0; d < NDIM; ++d) us += wv[IM + d];
            if (!(c2 > (Real)0) || !(c2 - c2 == (Real)0) || !(us - us == (Real)0)) {
                bad += 1;
            } else {
                // FP64: the root in float-float (~2^-46 relative), off the FP64 pipe
                Real cs;
                if constexpr (sizeof(Real) == 8) cs = df_to_double(df_sqrt(df_from_double(c2)));
                else cs = real_sqrt(c2);
                Real r = 0;
                int ci[3] = {0, 0, 0};
                if (a.grid[0] || a.grid[1] || a.grid[2]) {   // non-uniform: this cell's widths
                    const unsigned ii = (unsigned)i, nx = (unsigned)a.g.n[0], ny = (unsigned)a.g.n[1];
                    ci[0] = (int)(ii % nx);
                    ci[1] = (int)((ii / nx) % ny);
                    ci[2] = (int)(ii / (nx * ny));
                }
#pragma unroll
                for (int d = 0; d < NDIM; ++d) {
                    const Real inv = !a.grid[d] ? (Real)a.g.inv_dx[d]
                                     : d == 0 ? grid_inv_dx<true>(a.grid[d], a.grid_stride[d], ci[d], Real(0))
                                              : grid_inv_dx<false>(a.grid[d], a.grid_stride[d], ci[d], Real(0));
                    r = real_max(r, (fabs(wv[IM + d]) + cs) * inv);
                }
                rate = fmax(rate, (double)r);
            }
        }
    }
    if (RATE) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
            bad += __shfl_xor_sync(0xffffffffu, bad, o);
        }
        __shared__ double srate[8];
        __shared__ int sbad[8];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) { srate[wid] = rate; sbad[wid] = bad; }
        __syncthreads();
        if (wid == 0) {
            const int nw = blockDim.x >> 5;
            rate = lane < nw ? srate[lane] : 0.0;
            bad = lane < nw ? sbad[lane] : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
                bad += __shfl_xor_sync(0xffffffffu, bad, o);
            }
            if (lane == 0) {
                atomicMax(a.rate_max, (unsigned long long)__double_as_longlong(rate));
                if (bad) atomicAdd(a.bad, bad);
            }
        }
    }
}

// Primitive -> conserved (initial conditions), FP64.
template <int NF, int NDIM>
__global__ void __launch_bounds__(256) cons_kernel(Geometry g, EosConst e, const double* __restrict__ w,
                                                   double* __restrict__ q) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    const long long nc = g.ncell;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc;
         i += (long long)gridDim.x * blockDim.x) {
        double s[NS];
#pragma unroll
        for (int v = 0; v < NS; ++v) s[v] = w[v * nc + i];
        double rho = s[0];
#pragma unroll
        for (int k = 1; k < NF; ++k) rho += s[k];
        double G = e.G_N, P = e.P_N;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) { G = fma(s[IA + k], e.dG[k], G); P = fma(s[IA + k], e.dP[k], P); }
        double ke = 0.0;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) { ke = fma(s[IM + d], s[IM + d], ke); q[(IM + d) * nc + i] = rho * s[IM + d]; }
#pragma unroll
        for (int k = 0; k < NF; ++k) q[k * nc + i] = s[k];
        q[IE * nc + i] = fma(G, s[IE], P) + 0.5 * rho * ke;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) q[(IA + k) * nc + i] = s[IA + k];
    }
}

// Six-equation model: primitive (the five-equation variables, then the phase
// pressures p_k) -> conserved.  a_k r_k e_k = a_k (p_k + g_k pinf_k)/(g_k - 1)
// = a_k (G_k p_k + P_k), r E = sum_k a_k r_k e_k + r|u|^2/2; the primitive
// mixture-pressure row is not read.
template <int NF, int NDIM>
__global__ void __launch_bounds__(256) cons6_kernel(Geometry g, EosConst e, const double* __restrict__ w,
                                                    double* __restrict__ q) {
    using Lay = Layout<NF, NDIM, true>;
    constexpr int NQ = Lay::NQ, IM = Lay::IM, IE = Lay::IE, IA = Lay::IA, II = Lay::II;
    const long long nc = g.ncell;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc;
         i += (long long)gridDim.x * blockDim.x) {
        double s[NQ];
#pragma unroll
        for (int v = 0; v < NQ; ++v) s[v] = w[v * nc + i];
        double rho = s[0];
#pragma unroll
        for (int k = 1; k < NF; ++k) rho += s[k];
        double ke = 0.0;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) { ke = fma(s[IM + d], s[IM + d], ke); q[(IM + d) * nc + i] = rho * s[IM + d]; }
#pragma unroll
        for (int k = 0; k < NF; ++k) q[k * nc + i] = s[k];
        double aN = 1.0, esum = 0.0;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            q[(IA + k) * nc + i] = s[IA + k];
            aN -= s[IA + k];
            const double E = s[IA + k] * fma(e.G_N + e.dG[k], s[II + k], e.P_N + e.dP[k]);
            q[(II + k) * nc + i] = E;
            esum += E;
        }
        const double EN = aN * fma(e.G_N, s[II + NF - 1], e.P_N);
        q[(II + NF - 1) * nc + i] = EN;
        q[IE * nc + i] = esum + EN + 0.5 * rho * ke;
    }
}

}  // namespace mfc
