// Conserved -> primitive recovery with the CFL rate, and primitive -> conserved
// conversion (Sec. 2.1, 2.3).
#pragma once
#include "mfc_sweeps.cuh"

namespace mfc {

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
