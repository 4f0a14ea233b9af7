// Device code for the five-equation (Allaire) diffuse-interface right-hand side
// on GB300 (sm_103a).  Templates over the arithmetic type (double for the FP64
// path, float for the mixed path), the number of fluids NF, the number of
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
// so the FP64 path is bound by double-precision instructions, not by HBM.  The
// sweep kernel therefore (a) computes each cell's two WENO edge values from one
// shared set of smoothness indicators, (b) folds the six weight divisions of a
// cell into one reciprocal, (c) computes every face flux once, marching along a
// pencil so the neighbouring cell's edge and flux stay in registers, and (d) does
// the flux difference, the alpha div(u) source and the RK3 stage update in the
// same pass.  No atomics touch the state, so results are bitwise reproducible.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mfc {

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2 };

struct Geometry {
    int n[3];
    long long ncell;
    int bc_lo[3], bc_hi[3];
    double inv_dx[3];
};

// Mixture closure written as Gamma = G_N + sum_{k<N} alpha_k dG_k, with
// G_k = 1/(gamma_k - 1) and P_k = gamma_k pinf_k/(gamma_k - 1); this is
// sum_k alpha_k G_k with alpha_N = 1 - sum_{k<N} alpha_k (Sec. 2.1).
struct EosConst {
    double G_N, P_N;
    double dG[2], dP[2];
};

// Arguments of one directional sweep.
struct SweepArgs {
    Geometry g;
    EosConst e;
    const void* w;          // primitives [NS][ncell], Real
    double* R;              // right-hand side accumulator [NS][ncell]
    int mode;               // 0: R = sweep; 1: R += sweep; 2: RK stage update
    const double* q0;       // RK: state at t^n
    const double* qs;       // RK: current stage state
    double* qout;           // RK: output stage state (may alias qs or q0)
    double c0, c1, dt;      // RK: qout = c0 q0 + c1 (qs + dt (R + sweep))
    double eps;             // WENO epsilon
    int fallback;           // first-order fallback at non-physical faces
    int seg;                // cells per thread along the sweep direction
    int nseg;               // pencil segments along the sweep direction
    unsigned long long* fallback_count;  // optional counter of fallback faces
};

struct PrimArgs {
    Geometry g;
    EosConst e;
    const double* q;        // conserved [NS][ncell]
    void* w;                // primitives out [NS][ncell], Real
    unsigned long long* rate_max;  // optional: max (|u_d|+c)/dx_d as ordered bits
    int* bad;               // optional: count of non-physical cells
};

template <int NF, int NDIM> struct Layout {
    static constexpr int NS = 2 * NF + NDIM;
    static constexpr int IM = NF;              // first momentum / velocity
    static constexpr int IE = NF + NDIM;       // energy / pressure
    static constexpr int IA = NF + NDIM + 1;   // first transported volume fraction
};

__host__ __device__ inline long long stride_of(const Geometry& g, int d) {
    return d == 0 ? 1LL : (d == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
}

// Ghost-cell index mapping along one axis (Sec. 3.3).  Valid for i in
// [-3, n+2] and n >= 3.  Sets *flip for reflective ghosts.
__device__ __forceinline__ int ghost_map(int i, int n, int bclo, int bchi, bool* flip) {
    if (i < 0) {
        if (bclo == BC_PERIODIC) return i + n;
        if (bclo == BC_TRANSMISSIVE) return 0;
        *flip = true;
        return -i - 1;
    }
    if (i >= n) {
        if (bchi == BC_PERIODIC) return i - n;
        if (bchi == BC_TRANSMISSIVE) return n - 1;
        *flip = true;
        return 2 * n - 1 - i;
    }
    return i;
}

// ---------------------------------------------------------------------------
// WENO5-JS edge values of one cell (Sec. 3.2).  D[k] = v_{c+k-1} - v_{c+k-2},
// k = 0..3, i.e. the four differences across the five-cell stencil c-2..c+2.
// Returns eR (value at c-1/2) and eL (value at c+1/2).
//
// Smoothness indicators as quadratic forms of the differences:
//   b0 = 10/3 D1^2 - 11/3 D1 D0 + 4/3 D0^2      (stencil c-2..c)
//   b1 =  4/3 (D1^2 + D2^2) - 5/3 D1 D2         (stencil c-1..c+1)
//   b2 = 10/3 D2^2 - 11/3 D2 D3 + 4/3 D3^2      (stencil c..c+2)
// Candidates as increments over v_c, so constant data reconstructs exactly.  Both edges share
// the indicators; the mirrored edge uses the ideal weights reversed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void weno5_edges(double vc, const double D[4], double eps,
                                            double& eR, double& eL) {
    const double S0 = D[0] * D[0], S1 = D[1] * D[1], S2 = D[2] * D[2], S3 = D[3] * D[3];
    const double b0 = fma(10.0 / 3.0, S1, fma(-11.0 / 3.0, D[1] * D[0], (4.0 / 3.0) * S0));
    const double b1 = fma(4.0 / 3.0, S1 + S2, (-5.0 / 3.0) * (D[1] * D[2]));
    const double b2 = fma(10.0 / 3.0, S2, fma(-11.0 / 3.0, D[2] * D[3], (4.0 / 3.0) * S3));
    const double t0 = eps + b0, t1 = eps + b1, t2 = eps + b2;
    const double a0 = t0 * t0, a1 = t1 * t1, a2 = t2 * t2;
    // alpha_r = d_r / a_r; multiplied through by 10 a0 a1 a2
    const double P12 = a1 * a2, P02x6 = 6.0 * (a0 * a2), P01 = a0 * a1;
    const double P01x3 = 3.0 * P01, P12x3 = 3.0 * P12;
    // candidate increments p_r - v_c at c+1/2 (exact zero on constant data)
    const double p0 = fma(5.0 / 6.0, D[1], (-1.0 / 3.0) * D[0]);
    const double p1 = fma(1.0 / 6.0, D[1], (1.0 / 3.0) * D[2]);
    const double p2 = fma(2.0 / 3.0, D[2], (-1.0 / 6.0) * D[3]);
    // mirrored increments at c-1/2: stencils c..c+2, c-1..c+1, c-2..c
    const double m0 = fma(-5.0 / 6.0, D[2], (1.0 / 3.0) * D[3]);
    const double m1 = fma(-1.0 / 6.0, D[2], (-1.0 / 3.0) * D[1]);
    const double m2 = fma(-2.0 / 3.0, D[1], (1.0 / 6.0) * D[0]);
    const double numL = fma(P12, p0, fma(P02x6, p1, P01x3 * p2));
    const double denL = P12 + P02x6 + P01x3;
    const double numR = fma(P01, m0, fma(P02x6, m1, P12x3 * m2));
    const double denR = P01 + P02x6 + P12x3;
    const double x = 1.0 / (denL * denR);
    eL = fma(numL, denR * x, vc);
    eR = fma(numR, denL * x, vc);
}

// FP32 variant for the mixed path: the weights are normalised by the smallest
// eps+beta so no intermediate overflows FP32 (beta of a 1e9 Pa jump is ~1e19).
__device__ __forceinline__ void weno5_edges(float vc, const float D[4], float eps,
                                            float& eR, float& eL) {
    const float S0 = D[0] * D[0], S1 = D[1] * D[1], S2 = D[2] * D[2], S3 = D[3] * D[3];
    const float b0 = fmaf(10.f / 3.f, S1, fmaf(-11.f / 3.f, D[1] * D[0], (4.f / 3.f) * S0));
    const float b1 = fmaf(4.f / 3.f, S1 + S2, (-5.f / 3.f) * (D[1] * D[2]));
    const float b2 = fmaf(10.f / 3.f, S2, fmaf(-11.f / 3.f, D[2] * D[3], (4.f / 3.f) * S3));
    const float t0 = eps + b0, t1 = eps + b1, t2 = eps + b2;
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

template <typename Real> struct EosR {
    Real G_N, P_N, dG[2], dP[2];
    __device__ __forceinline__ explicit EosR(const EosConst& e)
        : G_N((Real)e.G_N), P_N((Real)e.P_N) {
        dG[0] = (Real)e.dG[0]; dG[1] = (Real)e.dG[1];
        dP[0] = (Real)e.dP[0]; dP[1] = (Real)e.dP[1];
    }
};

__device__ __forceinline__ double real_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float real_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double real_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float real_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double real_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float real_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double real_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float real_max(float a, float b) { return fmaxf(a, b); }

// A reconstructed face state is physical when every partial density is
// non-negative, every volume fraction (including alpha_N) lies in [0,1], the
// density is positive and (Gamma+1)p + Pi > 0.
template <typename Real, int NF, int NDIM>
__device__ __forceinline__ bool face_state_ok(const Real* s, const EosR<Real>& e) {
    using Lay = Layout<NF, NDIM>;
    bool ok = true;
    Real rho = s[0];
    ok = ok && (s[0] >= (Real)0);
#pragma unroll
    for (int k = 1; k < NF; ++k) { rho += s[k]; ok = ok && (s[k] >= (Real)0); }
    Real asum = 0, G = e.G_N, P = e.P_N;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        const Real a = s[Lay::IA + k];
        ok = ok && (a >= (Real)0) && (a <= (Real)1);
        asum += a;
        G = fma(a, e.dG[k], G);
        P = fma(a, e.dP[k], P);
    }
    const Real aN = (Real)1 - asum;
    ok = ok && (aN >= (Real)0) && (aN <= (Real)1);
    ok = ok && (rho > (Real)0);
    ok = ok && (fma(G + (Real)1, s[Lay::IE], P) > (Real)0);
    return ok;
}

// HLLC flux and face velocity (Sec. 3.2.1) between primitive states L | R with
// normal direction DIR; Davis wave-speed estimates.  The branch order matches
// the four cases of the paper: 0<=sL; sL<0<=s*; s*<0<sR; sR<=0.
template <typename Real, int NF, int NDIM, int DIR>
__device__ __forceinline__ void hllc(const Real* L, const Real* R, const EosR<Real>& e,
                                     Real* F, Real& ut) {
    using Lay = Layout<NF, NDIM>;
    constexpr int IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    Real rL = L[0], rR = R[0];
#pragma unroll
    for (int k = 1; k < NF; ++k) { rL += L[k]; rR += R[k]; }
    Real GL = e.G_N, PL = e.P_N, GR = e.G_N, PR = e.P_N;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        GL = fma(L[IA + k], e.dG[k], GL); PL = fma(L[IA + k], e.dP[k], PL);
        GR = fma(R[IA + k], e.dG[k], GR); PR = fma(R[IA + k], e.dP[k], PR);
    }
    const Real uL = L[IM + DIR], uR = R[IM + DIR], pL = L[IE], pR = R[IE];
    // c^2 = ((Gamma+1)p + Pi)/(Gamma rho); one reciprocal for both sides
    const Real nL = fma(GL + (Real)1, pL, PL), nR = fma(GR + (Real)1, pR, PR);
    const Real dL = GL * rL, dR = GR * rR;
    const Real xd = real_rcp(dL * dR);
    const Real cL = real_sqrt(nL * (dR * xd)), cR = real_sqrt(nR * (dL * xd));
    const Real sL = real_min(uL - cL, uR - cR);
    const Real sR = real_max(uL + cL, uR + cR);
    const Real aL = rL * (sL - uL), aR = rR * (sR - uR);
    const Real sS = (pR - pL + aL * uL - aR * uR) * real_rcp(aL - aR);
    const bool useL = ((Real)0 <= sL) || ((Real)0 <= sS);
    const bool star = useL ? !((Real)0 <= sL) : ((Real)0 < sR);
    Real K[Lay::NS];
#pragma unroll
    for (int v = 0; v < Lay::NS; ++v) K[v] = useL ? L[v] : R[v];
    const Real rK = useL ? rL : rR, uK = useL ? uL : uR, pK = useL ? pL : pR;
    const Real GK = useL ? GL : GR, PK = useL ? PL : PR, sK = useL ? sL : sR;
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
}

// ---------------------------------------------------------------------------
// Directional sweep.  One thread marches along one pencil segment of `seg`
// cells in direction DIR: it reconstructs the edges of cells s0-1..s1, forms
// faces s0-1/2..s1-1/2 and finishes cells s0..s1-1.  For DIR = y, z the lanes
// of a warp are consecutive x, so every load and store is coalesced.
// ---------------------------------------------------------------------------
template <typename Real, int NF, int NDIM, int DIR>
__global__ void __launch_bounds__(128) sweep_kernel(const SweepArgs a) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM, IA = Lay::IA;
    constexpr int T1 = (DIR == 0) ? 1 : 0;
    constexpr int T2 = (DIR == 2) ? 1 : 2;
    const Real* __restrict__ w = static_cast<const Real*>(a.w);
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int n1 = a.g.n[T1], n2 = a.g.n[T2], nd = a.g.n[DIR];
    const long long total = (long long)n1 * a.nseg * n2;
    if (tid >= total) return;
    const int t1 = (int)(tid % n1);
    const long long rest = tid / n1;
    const int sg = (int)(rest % a.nseg);
    const int t2 = (int)(rest / a.nseg);
    const long long sd = stride_of(a.g, DIR);
    const long long base = (long long)t1 * stride_of(a.g, T1) + (long long)t2 * stride_of(a.g, T2);
    const long long nc = a.g.ncell;
    const int s0 = sg * a.seg;
    const int s1 = min(s0 + a.seg, nd);
    const int bclo = a.g.bc_lo[DIR], bchi = a.g.bc_hi[DIR];
    const Real eps = (Real)a.eps;
    const EosR<Real> e(a.e);
    const double inv_dx = a.g.inv_dx[DIR];

    auto load = [&](int i, Real* out) {
        bool flip = false;
        const int m = ghost_map(i, nd, bclo, bchi, &flip);
        const long long idx = base + (long long)m * sd;
#pragma unroll
        for (int v = 0; v < NS; ++v) out[v] = __ldg(w + v * nc + idx);
        if (flip) out[IM + DIR] = -out[IM + DIR];
    };

    // Window around the cell c being reconstructed: vm1 = c-1, vc = c,
    // vp1 = c+1, vp2 = c+2 and the four differences across c-2..c+2.
    Real vm1[NS], vc[NS], vp1[NS], vp2[NS], D[NS][4];
    {
        Real t[NS];
        load(s0 - 3, t);
        load(s0 - 2, vm1);
        load(s0 - 1, vc);
        load(s0, vp1);
        load(s0 + 1, vp2);
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            D[v][0] = vm1[v] - t[v];
            D[v][1] = vc[v] - vm1[v];
            D[v][2] = vp1[v] - vc[v];
            D[v][3] = vp2[v] - vp1[v];
        }
    }
    Real eLprev[NS], Fprev[NS], utprev = 0;
    Real cm1[NS];  // cell c-1 values (for the fallback and the alpha source)
#pragma unroll
    for (int v = 0; v < NS; ++v) { eLprev[v] = 0; Fprev[v] = 0; cm1[v] = vm1[v]; }

    for (int c = s0 - 1; c <= s1; ++c) {
        Real eR[NS], eL[NS];
#pragma unroll
        for (int v = 0; v < NS; ++v) weno5_edges(vc[v], D[v], eps, eR[v], eL[v]);
        if (c >= s0) {
            Real F[NS], ut;
            bool first = false;
            if (a.fallback) {
                first = !(face_state_ok<Real, NF, NDIM>(eLprev, e) && face_state_ok<Real, NF, NDIM>(eR, e));
                if (first && a.fallback_count) atomicAdd(a.fallback_count, 1ULL);
            }
            Real fl[NS], fr[NS];
#pragma unroll
            for (int v = 0; v < NS; ++v) {
                fl[v] = first ? cm1[v] : eLprev[v];
                fr[v] = first ? vc[v] : eR[v];
            }
            hllc<Real, NF, NDIM, DIR>(fl, fr, e, F, ut);
            if (c >= s0 + 1) {
                // finish cell c-1: flux difference and alpha div(u) source
                double out[NS];
#pragma unroll
                for (int v = 0; v < NS; ++v) out[v] = (double)(Fprev[v] - F[v]) * inv_dx;
                const double du = (double)(ut - utprev) * inv_dx;
#pragma unroll
                for (int k = 0; k < NF - 1; ++k) out[IA + k] = fma((double)cm1[IA + k], du, out[IA + k]);
                const long long idx = base + (long long)(c - 1) * sd;
                if (a.mode == 0) {
#pragma unroll
                    for (int v = 0; v < NS; ++v) a.R[v * nc + idx] = out[v];
                } else if (a.mode == 1) {
#pragma unroll
                    for (int v = 0; v < NS; ++v) a.R[v * nc + idx] += out[v];
                } else {
                    const bool acc = (NDIM > 1);
#pragma unroll
                    for (int v = 0; v < NS; ++v) {
                        double r = out[v];
                        if (acc) r += a.R[v * nc + idx];
                        double s = fma(a.dt, r, a.qs[v * nc + idx]);
                        double o = a.c1 * s;
                        if (a.c0 != 0.0) o = fma(a.c0, a.q0[v * nc + idx], o);
                        a.qout[v * nc + idx] = o;
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < NS; ++v) Fprev[v] = F[v];
            utprev = ut;
        }
        // advance the window by one cell
#pragma unroll
        for (int v = 0; v < NS; ++v) { eLprev[v] = eL[v]; cm1[v] = vc[v]; }
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
}

// ---------------------------------------------------------------------------
// Conserved -> primitive (Sec. 2.1): rho = sum a_k r_k, u = (rho u)/rho,
// p = (rho E - rho|u|^2/2 - Pi)/Gamma, always in FP64 (the water Pi ~ 7.8e8 Pa
// cancels against rho E).  Optionally the CFL rate max_d (|u_d| + c)/dx_d with
// c^2 = ((Gamma+1)p + Pi)/(Gamma rho), reduced to one max per launch with an
// order-preserving integer atomic (non-negative doubles), so it is exact and
// independent of scheduling.
// ---------------------------------------------------------------------------
template <typename Real, int NF, int NDIM, bool RATE>
__global__ void __launch_bounds__(256) prims_kernel(const PrimArgs a) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    const long long nc = a.g.ncell;
    double rate = 0.0;
    int bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc;
         i += (long long)gridDim.x * blockDim.x) {
        double q[NS];
#pragma unroll
        for (int v = 0; v < NS; ++v) q[v] = __ldg(a.q + v * nc + i);
        double rho = q[0];
#pragma unroll
        for (int k = 1; k < NF; ++k) rho += q[k];
        double G = a.e.G_N, P = a.e.P_N;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            G = fma(q[IA + k], a.e.dG[k], G);
            P = fma(q[IA + k], a.e.dP[k], P);
        }
        const double x = 1.0 / (rho * G);
        const double irho = G * x, iG = rho * x;
        double u[NDIM], ke = 0.0;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) { u[d] = q[IM + d] * irho; ke = fma(q[IM + d], u[d], ke); }
        const double p = (q[IE] - 0.5 * ke - P) * iG;
        Real* w = static_cast<Real*>(a.w);
#pragma unroll
        for (int k = 0; k < NF; ++k) w[k * nc + i] = (Real)q[k];
#pragma unroll
        for (int d = 0; d < NDIM; ++d) w[(IM + d) * nc + i] = (Real)u[d];
        w[IE * nc + i] = (Real)p;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) w[(IA + k) * nc + i] = (Real)q[IA + k];
        if (RATE) {
            const double c2 = fma(G + 1.0, p, P) * iG * irho;
            if (!(c2 > 0.0) || !(c2 < 1e300) || !(ke == ke)) {
                bad += 1;
            } else {
                const double cs = sqrt(c2);
#pragma unroll
                for (int d = 0; d < NDIM; ++d) rate = fmax(rate, (fabs(u[d]) + cs) * a.g.inv_dx[d]);
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

}  // namespace mfc
