// Conserved -> primitive recovery with the CFL rate, and primitive -> conserved
// conversion (Sec. 2.1, 2.3).
#pragma once
#include "mfc_sweeps.cuh"

namespace mfc {

// Conserved -> primitive recovery per cell (prims_cell) and the CFL rate of a
// cell (cell_cfl_rate) live in mfc_cell.cuh, where the RK epilogue uses them too.

template <typename Real, int NF, int NDIM, bool RATE, bool SIX = false>
__global__ void __launch_bounds__(256) prims_kernel(const PrimArgs a) {
    using Lay = Layout<NF, NDIM>;
    constexpr int NS = Lay::NS;
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
            const double r = cell_cfl_rate<Real, NF, NDIM>(wv, c2, a.g, a.grid, a.grid_stride, i);
            if (r < 0.0) bad += 1;
            else rate = fmax(rate, r);
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
