// Face fluxes (Sec. 3.2.1): the EOS constants in the sweep's precision, mixture
// quantities, the positivity test of reconstructed states, HLLC (FP32 form and
// the FP64 path's float-float form) and the face flux with the first-order
// fallback.
#pragma once
#include "mfc_weno.cuh"

namespace mfc {

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
// steps, branch order and xi - 1 form as hllc, on float-float face states;
// only the widening of each flux after it uses the FP64 pipe.  On GB300 an
// FP64 instruction costs the issue time of ~60 FP32 ones, and the FP64
// solver's two square roots, three reciprocals and ~60 further FP64 operations
// per face were half of the sweeps' FP64 work.  Differences that can cancel
// (p_R - p_L, s - u) use the exact float-float addition; the error of the flux
// stays near 2^-44 of its terms, far below the FP64 path's 1e-11 parity
// requirement.  The states come either as FP64 values (split by integer
// operations when read) or already in float-float; `at(v)` reads variable v.
struct F64States {
    const double* p;
    __device__ __forceinline__ df at(int v) const { return df_from_double(p[v]); }
};
struct DfStates {
    const df* p;
    __device__ __forceinline__ df at(int v) const { return p[v]; }
};

// Mixture quantities of a float-float face state (see Mix).
struct MixDf {
    df r, G, P, n;
};

// Fluxes and face velocity in float-float; returns whether the flux took the
// left state (useL).
template <int NF, int NDIM, int DIR, typename States>
__device__ __forceinline__ bool hllc_df_core(const States& L, const States& R, const MixDf& mL, const MixDf& mR,
                                             df* F, df& ut) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IM = Lay::IM, IE = Lay::IE, IA = Lay::IA;
    const df uL = L.at(IM + DIR), uR = R.at(IM + DIR);
    const df pL = L.at(IE), pR = R.at(IE);
    const df rL = mL.r, rR = mR.r;
    // c^2 = n/(Gamma rho)
    const df cL = df_sqrt(df_div(mL.n, df_mul(mL.G, rL)));
    const df cR = df_sqrt(df_div(mR.n, df_mul(mR.G, rR)));
    const df sL = df_min(df_add_fast(uL, df_neg(cL)), df_add_fast(uR, df_neg(cR)));
    const df sR = df_max(df_add_fast(uL, cL), df_add_fast(uR, cR));
    const df aL = df_mul(rL, df_add(sL, df_neg(uL))), aR = df_mul(rR, df_add(sR, df_neg(uR)));
    const df num = df_add(df_add(pR, df_neg(pL)), df_add(df_mul(aL, uL), df_neg(df_mul(aR, uR))));
    const df sS = df_div(num, df_add(aL, df_neg(aR)));
    const bool useL = sL.hi >= 0.f || sS.hi >= 0.f;
    const bool star = useL ? !(sL.hi >= 0.f) : (sR.hi > 0.f);
    const df rK = useL ? rL : rR, uK = useL ? uL : uR, pK = useL ? pL : pR, sK = useL ? sL : sR;
    const df GK = useL ? mL.G : mR.G, PK = useL ? mL.P : mR.P;
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
    for (int v = 0; v < NS; ++v) Kd[v] = useL ? L.at(v) : R.at(v);   // element by element: a reference to
    // either state array placed both in local memory (FP64 y/z sweeps 149 -> 128 registers, 256^3 step
    // 36.1 -> 34.4 ms)
    df u2 = df_mul(Kd[IM], Kd[IM]);
#pragma unroll
    for (int dd = 1; dd < NDIM; ++dd) u2 = df_add_fast(u2, df_mul(Kd[IM + dd], Kd[IM + dd]));
    const df rE = df_add_fast(df_add_fast(df_mul(GK, pK), PK), df_mul_pow2(df_mul(rK, u2), 0.5f));
#pragma unroll
    for (int k = 0; k < NF; ++k) F[k] = df_mul(Kd[k], utd);
    const df sKds = df_mul(sKe, dsu);   // s_K (s* - u_K)
#pragma unroll
    for (int dd = 0; dd < NDIM; ++dd) {
        if (dd == DIR)
            F[IM + dd] = df_add_fast(df_add_fast(df_mul(df_mul(rK, uK), utd), pK), df_mul(df_mul(sKds, xi), rK));
        else
            F[IM + dd] = df_mul(df_mul(rK, Kd[IM + dd]), utd);
    }
    F[IE] = df_add_fast(df_add_fast(df_mul(rE, utd), df_mul(pK, uK)),
                        df_mul(sKds, df_add_fast(df_mul(df_mul(xi, rK), sS), df_mul(pK, rr))));
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) F[IA + k] = df_mul(Kd[IA + k], utd);
    ut = utd;
    return useL;
}

// HLLC of FP64 face states with their FP64 mixture quantities.
template <int NF, int NDIM, int DIR, bool SIX = false>
__device__ __forceinline__ void hllc_df(const double* L, const double* R, const Mix<double>& mL,
                                        const Mix<double>& mR, double* F, double& ut,
                                        const EosR<double>* e6 = nullptr) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS, IE = Lay::IE, IA = Lay::IA;
    const MixDf xL{df_from_double(mL.r), df_from_double(mL.G), df_from_double(mL.P), df_from_double(mL.n)};
    const MixDf xR{df_from_double(mR.r), df_from_double(mR.G), df_from_double(mR.P), df_from_double(mR.n)};
    df Fd[NS], utd;
    const bool useL = hllc_df_core<NF, NDIM, DIR>(F64States{L}, F64States{R}, xL, xR, Fd, utd);
#pragma unroll
    for (int v = 0; v < NS; ++v) F[v] = df_to_double(Fd[v]);
    ut = df_to_double(utd);
    if constexpr (SIX) {
        double aN = 1.0;
        const double pKd = useL ? L[IE] : R[IE];
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            const double aK = useL ? L[IA + k] : R[IA + k];
            aN -= aK;
            F[NS + k] = aK * fma(e6->G_N + e6->dG[k], pKd, e6->P_N + e6->dP[k]) * ut;
        }
        F[NS + NF - 1] = aN * fma(e6->G_N, pKd, e6->P_N) * ut;
    }
}

// The EOS constants as float-float values (split once per kernel).
struct EosDf {
    df G_N, P_N, dG[2], dP[2];
    // six-equation model: the frozen-sound-speed coefficients and the phase
    // constants G_k = G_N + dG_k, P_k = P_N + dP_k
    df A_N, B_N, dA[2], dB[2], Gk[2], Pk[2];
    template <typename E>
    __device__ __forceinline__ explicit EosDf(const E& e)
        : G_N(df_from_double((double)e.G_N)), P_N(df_from_double((double)e.P_N)),
          A_N(df_from_double((double)e.A_N)), B_N(df_from_double((double)e.B_N)) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            dG[k] = df_from_double((double)e.dG[k]);
            dP[k] = df_from_double((double)e.dP[k]);
            dA[k] = df_from_double((double)e.dA[k]);
            dB[k] = df_from_double((double)e.dB[k]);
            Gk[k] = df_from_double((double)e.G_N + (double)e.dG[k]);
            Pk[k] = df_from_double((double)e.P_N + (double)e.dP[k]);
        }
    }
};

// Mixture quantities of a float-float face state, in float-float (SIX: n =
// Gamma r c^2 with the frozen sound speed, r c^2 = A p + B, as in mixture).
template <int NF, int NDIM, bool SIX = false>
__device__ __forceinline__ MixDf mixture_df(const df* s, const EosDf& e) {
    using Lay = Layout<NF, NDIM>;
    MixDf m;
    m.r = s[0];
#pragma unroll
    for (int k = 1; k < NF; ++k) m.r = df_add(m.r, s[k]);
    m.G = e.G_N;
    m.P = e.P_N;
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
        m.G = df_add(m.G, df_mul(s[Lay::IA + k], e.dG[k]));
        m.P = df_add(m.P, df_mul(s[Lay::IA + k], e.dP[k]));
    }
    if constexpr (SIX) {
        df A = e.A_N, B = e.B_N;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            A = df_add(A, df_mul(s[Lay::IA + k], e.dA[k]));
            B = df_add(B, df_mul(s[Lay::IA + k], e.dB[k]));
        }
        m.n = df_mul(m.G, df_add(df_mul(A, s[Lay::IE]), B));
    } else {
        m.n = df_add(df_mul(df_add_fast(m.G, {1.f, 0.f}), s[Lay::IE]), m.P);
    }
    return m;
}

// face_state_ok for float-float states (normalised: the sign and the order
// against 0 and 1 follow from hi, then lo).
__device__ __forceinline__ bool df_nonneg(df x) { return x.hi >= 0.f; }
__device__ __forceinline__ bool df_positive(df x) { return x.hi > 0.f; }
__device__ __forceinline__ bool df_unit(df x) { return x.hi >= 0.f && (x.hi < 1.f || (x.hi == 1.f && x.lo <= 0.f)); }

template <int NF, int NDIM>
__device__ __forceinline__ bool face_state_ok_df(const df* s, const MixDf& m) {
    using Lay = Layout<NF, NDIM>;
    bool ok = df_positive(m.r) && df_positive(m.n);
#pragma unroll
    for (int k = 0; k < NF; ++k) ok = ok && df_nonneg(s[k]);
    if (NF > 1) {
        df asum = s[Lay::IA];
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            ok = ok && df_unit(s[Lay::IA + k]);
            if (k > 0) asum = df_add(asum, s[Lay::IA + k]);
        }
        ok = ok && df_unit(df_add({1.f, 0.f}, df_neg(asum)));
    }
    return ok;
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

// FP64 path, face states already in float-float (the reconstruction's cell
// value plus its float-float increment): mixture and positivity test in
// float-float, the first-order fallback splitting the two FP64 cell values;
// no FP64 operation before the widened fluxes.
//
// Six-equation model (SIX): the phase internal energies are carried with the
// upwind state at the face pressure, a_k (G_k p_K + P_k) times the face
// velocity (as in hllc).  The volume-fraction slots of eLs and eRs hold FP64
// edges (df_pack): alpha_N = 1 - sum_k alpha_k is formed in FP64, since where
// phase N is a trace (alpha_N ~ 1e-6) the subtraction cancels and a
// float-float alpha_k (~2^-48 of 1) would leave alpha_N ~3e-9 relative error.
template <int NF, int NDIM, int DIR, bool SIX = false>
__device__ __forceinline__ void face_flux_df(const SweepArgs& a, const EosDf& e, const df* eLs, const df* eRs,
                                             const double* cl, const double* cr, df* F, df& ut) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS;
    df sl[NS], sr[NS];
    [[maybe_unused]] double aL[SIX ? NF - 1 : 1], aR[SIX ? NF - 1 : 1];
#pragma unroll
    for (int v = 0; v < NS; ++v) {
        sl[v] = eLs[v];
        sr[v] = eRs[v];
    }
    if constexpr (SIX) {
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            aL[k] = df_unpack(eLs[Lay::IA + k]);
            aR[k] = df_unpack(eRs[Lay::IA + k]);
            sl[Lay::IA + k] = df_from_double(aL[k]);
            sr[Lay::IA + k] = df_from_double(aR[k]);
        }
    }
    MixDf mL = mixture_df<NF, NDIM, SIX>(sl, e);
    MixDf mR = mixture_df<NF, NDIM, SIX>(sr, e);
    const bool first = a.fallback && !(face_state_ok_df<NF, NDIM>(sl, mL) && face_state_ok_df<NF, NDIM>(sr, mR));
    if (first) {
        count_fallback(a.fallback_count);
#pragma unroll
        for (int v = 0; v < NS; ++v) {
            sl[v] = df_from_double(cl[v]);
            sr[v] = df_from_double(cr[v]);
        }
        if constexpr (SIX) {
#pragma unroll
            for (int k = 0; k < NF - 1; ++k) {
                aL[k] = cl[Lay::IA + k];
                aR[k] = cr[Lay::IA + k];
            }
        }
        mL = mixture_df<NF, NDIM, SIX>(sl, e);
        mR = mixture_df<NF, NDIM, SIX>(sr, e);
    }
    const bool useL = hllc_df_core<NF, NDIM, DIR>(DfStates{sl}, DfStates{sr}, mL, mR, F, ut);
    if constexpr (SIX) {
        const df pK = useL ? sl[Lay::IE] : sr[Lay::IE];
        double aN = 1.0;
#pragma unroll
        for (int k = 0; k < NF - 1; ++k) {
            const double aK = useL ? aL[k] : aR[k];
            aN -= aK;
            F[NS + k] = df_mul(df_mul(df_from_double(aK), df_add(df_mul(e.Gk[k], pK), e.Pk[k])), ut);
        }
        F[NS + NF - 1] = df_mul(df_mul(df_from_double(aN), df_add(df_mul(e.G_N, pK), e.P_N)), ut);
    }
}

}  // namespace mfc
