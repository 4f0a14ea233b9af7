// Host-side launchers for the device templates.  Each translation unit
// instantiates them for one (arithmetic type, number of fluids) pair so the
// build compiles in parallel.
#pragma once
#include "mfc_device.cuh"

namespace mfc {

constexpr int kSweepThreads = 128;
constexpr int kElemThreads = 256;

// Slots (edge cells) owned by one CTA of the x-stream kernel: 16 chunks of 128,
// so the two recomputed slots at its start cost about 0.1%.
constexpr long long kStreamSlotsPerBlock = 16LL * kStreamThreads;

inline size_t stage_bytes_rt(int mask, int nq, size_t real_size) {
    return (size_t)nq * kStageSlots *
           (((mask & 1) ? real_size : 0) + ((mask & 2) ? sizeof(double) : 0) + ((mask & 4) ? sizeof(double) : 0));
}

// Launch one y/z stream kernel.  An entry built with staging (STAGE) gets its
// finish operands staged, dropping q0, then qs, then R from the staging while
// its shared memory would lower the number of CTAs resident per SM (the
// kernels are latency-bound: residency comes first).
template <typename Real, bool STAGE = false, typename Kernel>
cudaError_t launch_yz_stream(Kernel kernel, unsigned blocks, SweepArgs a, int nq, cudaStream_t s) {
    constexpr int threads = 32 * kRowsPerChunk;
    int mask = STAGE ? stage_mask(a) : 0;
    size_t dyn = 0;
    if (mask) {
        int occ0 = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, kernel, threads, 0);
        if (e != cudaSuccess) return e;
        for (; mask; mask &= ~(mask & 4 ? 4 : mask & 2 ? 2 : 1)) {
            dyn = stage_bytes_rt(mask, nq, sizeof(Real));
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
            if (e != cudaSuccess) return e;
            int occ = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, dyn);
            if (e != cudaSuccess) return e;
            if (occ >= occ0) break;
        }
        if (!mask) dyn = 0;
    }
    a.stage = mask;
    kernel<<<blocks, threads, dyn, s>>>(a);
    return cudaGetLastError();
}

// SIX: the six-equation model (stream kernels, WENO5, uniform grids).
template <typename Real, int NF, bool LEARNED = false, int ORDER = 5, bool NONUNIF = false, bool SIX = false>
cudaError_t launch_sweep(SweepArgs a, int ndim, int dir, cudaStream_t s) {
    // FP64 sweeps bounded to 4 CTAs per SM (128 registers, small spills):
    // faster for the stretched-grid (83.7 -> 71.1 ms per step at 256^3),
    // six-equation (83.4 -> 80.7) and WENO3 (42.1 -> 41.5) variants, slower
    // for the uniform WENO5 ones (61.0 -> 63.8, Kapila 65.3 -> 67.2)
    constexpr bool kBoundFp64 = NONUNIF || SIX || ORDER == 3;
    if (dir == 0) {
        const long long total = (long long)(a.g.n[0] + 2) * (a.g.ncell / a.g.n[0]);
        a.slots_per_block = kStreamSlotsPerBlock;
        const unsigned blocks = (unsigned)((total + kStreamSlotsPerBlock - 1) / kStreamSlotsPerBlock);
        if constexpr (LEARNED) {
            switch (ndim) {
                case 1: sweep_x_stream_learned_kernel<NF, 1><<<blocks, kStreamThreads, 0, s>>>(a); break;
                case 2: sweep_x_stream_learned_kernel<NF, 2><<<blocks, kStreamThreads, 0, s>>>(a); break;
                case 3: sweep_x_stream_learned_kernel<NF, 3><<<blocks, kStreamThreads, 0, s>>>(a); break;
                default: return cudaErrorInvalidValue;
            }
        } else if constexpr (sizeof(Real) == 8 && kBoundFp64) {
            switch (ndim) {
                case 1: sweep_x_stream_f64_kernel<NF, 1, ORDER, NONUNIF, SIX><<<blocks, kStreamThreads, 0, s>>>(a); break;
                case 2: sweep_x_stream_f64_kernel<NF, 2, ORDER, NONUNIF, SIX><<<blocks, kStreamThreads, 0, s>>>(a); break;
                case 3: sweep_x_stream_f64_kernel<NF, 3, ORDER, NONUNIF, SIX><<<blocks, kStreamThreads, 0, s>>>(a); break;
                default: return cudaErrorInvalidValue;
            }
        } else if constexpr (sizeof(Real) == 4 && !NONUNIF && !SIX) {
            switch (ndim) {
                case 1: sweep_x_stream_f32_kernel<NF, 1, ORDER><<<blocks, kStreamThreads, 0, s>>>(a); break;
                case 2: sweep_x_stream_f32_kernel<NF, 2, ORDER><<<blocks, kStreamThreads, 0, s>>>(a); break;
                case 3: sweep_x_stream_f32_kernel<NF, 3, ORDER><<<blocks, kStreamThreads, 0, s>>>(a); break;
                default: return cudaErrorInvalidValue;
            }
        } else {
            switch (ndim) {
                case 1: sweep_x_stream_kernel<Real, NF, 1, LEARNED, ORDER, NONUNIF, SIX><<<blocks, kStreamThreads, 0, s>>>(a); break;
                case 2: sweep_x_stream_kernel<Real, NF, 2, LEARNED, ORDER, NONUNIF, SIX><<<blocks, kStreamThreads, 0, s>>>(a); break;
                case 3: sweep_x_stream_kernel<Real, NF, 3, LEARNED, ORDER, NONUNIF, SIX><<<blocks, kStreamThreads, 0, s>>>(a); break;
                default: return cudaErrorInvalidValue;
            }
        }
        return cudaGetLastError();
    }
    const int t1 = (dir == 0) ? 1 : 0, t2 = (dir == 2) ? 1 : 2;
    if (NONUNIF || SIX || a.yz_stream) {   // non-uniform grids, six-equation model: the stream kernel only
        // y/z stream kernel, one CTA per 32 x-lanes of a segment
        const unsigned blocks = (unsigned)((long long)((a.g.n[t1] + 31) / 32) * a.nseg * a.g.n[t2]);
        auto nq = [](int nd) { return 2 * NF + nd + (SIX ? NF : 0); };
        if constexpr (LEARNED) {
            switch (ndim * 4 + dir) {
                case 9: return launch_yz_stream<Real, true>(sweep_yz_stream_learned_kernel<NF, 2, 1>, blocks, a, nq(2), s);
                case 13: return launch_yz_stream<Real, true>(sweep_yz_stream_learned_kernel<NF, 3, 1>, blocks, a, nq(3), s);
                case 14: return launch_yz_stream<Real, true>(sweep_yz_stream_learned_kernel<NF, 3, 2>, blocks, a, nq(3), s);
                default: return cudaErrorInvalidValue;
            }
        } else if constexpr (sizeof(Real) == 8 && kBoundFp64) {
            switch (ndim * 4 + dir) {
                case 9: return launch_yz_stream<Real, !NONUNIF>(sweep_yz_stream_f64_kernel<NF, 2, 1, ORDER, NONUNIF, SIX>, blocks, a, nq(2), s);
                case 13: return launch_yz_stream<Real, !NONUNIF>(sweep_yz_stream_f64_kernel<NF, 3, 1, ORDER, NONUNIF, SIX>, blocks, a, nq(3), s);
                case 14: return launch_yz_stream<Real, !NONUNIF>(sweep_yz_stream_f64_kernel<NF, 3, 2, ORDER, NONUNIF, SIX>, blocks, a, nq(3), s);
                default: return cudaErrorInvalidValue;
            }
        } else if constexpr (sizeof(Real) == 8 && NF == 3 && ORDER == 5) {
            switch (ndim * 4 + dir) {
                case 9: return launch_yz_stream<Real, true>(sweep_yz_stream_f64b3_kernel<NF, 2, 1>, blocks, a, nq(2), s);
                case 13: return launch_yz_stream<Real, true>(sweep_yz_stream_f64b3_kernel<NF, 3, 1>, blocks, a, nq(3), s);
                case 14: return launch_yz_stream<Real, true>(sweep_yz_stream_f64b3_kernel<NF, 3, 2>, blocks, a, nq(3), s);
                default: return cudaErrorInvalidValue;
            }
        } else if constexpr (SIX && sizeof(Real) == 4) {
            switch (ndim * 4 + dir) {
                case 9: return launch_yz_stream<Real, true>(sweep_yz_stream_six32_kernel<NF, 2, 1, ORDER, NONUNIF>, blocks, a, nq(2), s);
                case 13: return launch_yz_stream<Real, true>(sweep_yz_stream_six32_kernel<NF, 3, 1, ORDER, NONUNIF>, blocks, a, nq(3), s);
                case 14: return launch_yz_stream<Real, true>(sweep_yz_stream_six32_kernel<NF, 3, 2, ORDER, NONUNIF>, blocks, a, nq(3), s);
                default: return cudaErrorInvalidValue;
            }
        } else if constexpr (sizeof(Real) == 4 && !NONUNIF) {
            switch (ndim * 4 + dir) {
                case 9: return launch_yz_stream<Real, true>(sweep_yz_stream_f32_kernel<NF, 2, 1, ORDER>, blocks, a, nq(2), s);
                case 13: return launch_yz_stream<Real, true>(sweep_yz_stream_f32_kernel<NF, 3, 1, ORDER>, blocks, a, nq(3), s);
                case 14: return launch_yz_stream<Real, true>(sweep_yz_stream_f32_kernel<NF, 3, 2, ORDER>, blocks, a, nq(3), s);
                default: return cudaErrorInvalidValue;
            }
        } else {
            switch (ndim * 4 + dir) {
                case 9: return launch_yz_stream<Real, sizeof(Real) == 8>(sweep_yz_stream_kernel<Real, NF, 2, 1, ORDER, NONUNIF, SIX>, blocks, a, nq(2), s);
                case 13: return launch_yz_stream<Real, sizeof(Real) == 8>(sweep_yz_stream_kernel<Real, NF, 3, 1, ORDER, NONUNIF, SIX>, blocks, a, nq(3), s);
                case 14: return launch_yz_stream<Real, sizeof(Real) == 8>(sweep_yz_stream_kernel<Real, NF, 3, 2, ORDER, NONUNIF, SIX>, blocks, a, nq(3), s);
                default: return cudaErrorInvalidValue;
            }
        }
    }
    if constexpr (NONUNIF || SIX) return cudaErrorInvalidValue;
    const long long warps = (long long)((a.g.n[t1] + 31) / 32) * a.nseg * a.g.n[t2];
    const unsigned blocks = (unsigned)((warps * 32 + kSweepThreads - 1) / kSweepThreads);
    switch (ndim * 4 + dir) {
        case 9: sweep_kernel<Real, NF, 2, 1, LEARNED, ORDER><<<blocks, kSweepThreads, 0, s>>>(a); break;
        case 13: sweep_kernel<Real, NF, 3, 1, LEARNED, ORDER><<<blocks, kSweepThreads, 0, s>>>(a); break;
        case 14: sweep_kernel<Real, NF, 3, 2, LEARNED, ORDER><<<blocks, kSweepThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

inline unsigned elem_blocks(long long n) {
    long long b = (n + kElemThreads - 1) / kElemThreads;
    const long long cap = 152LL * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <typename Real, int NF, bool SIX = false>
cudaError_t launch_prims(const PrimArgs& a, int ndim, bool rate, cudaStream_t s) {
    const unsigned blocks = elem_blocks(a.g.ncell);
    switch (ndim * 2 + (rate ? 1 : 0)) {
        case 2: prims_kernel<Real, NF, 1, false, SIX><<<blocks, kElemThreads, 0, s>>>(a); break;
        case 3: prims_kernel<Real, NF, 1, true, SIX><<<blocks, kElemThreads, 0, s>>>(a); break;
        case 4: prims_kernel<Real, NF, 2, false, SIX><<<blocks, kElemThreads, 0, s>>>(a); break;
        case 5: prims_kernel<Real, NF, 2, true, SIX><<<blocks, kElemThreads, 0, s>>>(a); break;
        case 6: prims_kernel<Real, NF, 3, false, SIX><<<blocks, kElemThreads, 0, s>>>(a); break;
        case 7: prims_kernel<Real, NF, 3, true, SIX><<<blocks, kElemThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Characteristic boundary rates (cbc_rates_kernel): total = boundary cells.
template <typename Real, int NF>
cudaError_t launch_cbc(const SweepArgs& a, int ndim, long long total, cudaStream_t s) {
    const unsigned blocks = elem_blocks(total);
    switch (ndim) {
        case 1: cbc_rates_kernel<Real, NF, 1><<<blocks, kElemThreads, 0, s>>>(a, total); break;
        case 2: cbc_rates_kernel<Real, NF, 2><<<blocks, kElemThreads, 0, s>>>(a, total); break;
        case 3: cbc_rates_kernel<Real, NF, 3><<<blocks, kElemThreads, 0, s>>>(a, total); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NF>
cudaError_t launch_cons6(const Geometry& g, const EosConst& e, const double* w, double* q, int ndim,
                         cudaStream_t s) {
    const unsigned blocks = elem_blocks(g.ncell);
    switch (ndim) {
        case 1: cons6_kernel<NF, 1><<<blocks, kElemThreads, 0, s>>>(g, e, w, q); break;
        case 2: cons6_kernel<NF, 2><<<blocks, kElemThreads, 0, s>>>(g, e, w, q); break;
        case 3: cons6_kernel<NF, 3><<<blocks, kElemThreads, 0, s>>>(g, e, w, q); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NF>
cudaError_t launch_cons(const Geometry& g, const EosConst& e, const double* w, double* q, int ndim,
                        cudaStream_t s) {
    const unsigned blocks = elem_blocks(g.ncell);
    switch (ndim) {
        case 1: cons_kernel<NF, 1><<<blocks, kElemThreads, 0, s>>>(g, e, w, q); break;
        case 2: cons_kernel<NF, 2><<<blocks, kElemThreads, 0, s>>>(g, e, w, q); break;
        case 3: cons_kernel<NF, 3><<<blocks, kElemThreads, 0, s>>>(g, e, w, q); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Host: the EOS constants of N stiffened-gas fluids (Sec. 2.1) as the kernels
// take them, relative to fluid N (whose fraction is 1 - sum of the others):
// Gamma_k = 1/(g_k - 1), Pi_k = g_k pinf_k/(g_k - 1), and for the six-equation
// model's frozen sound speed r c^2 = sum_k a_k g_k (p + pinf_k) the pairs
// (g_k, g_k pinf_k).  Every entry point builds its constants here.
inline EosConst make_eos_const(int N, const double* gamma, const double* pi_inf) {
    double G[3], P[3];
    for (int k = 0; k < N; ++k) {
        G[k] = 1.0 / (gamma[k] - 1.0);
        P[k] = gamma[k] * pi_inf[k] / (gamma[k] - 1.0);
    }
    EosConst e{};
    e.G_N = G[N - 1];
    e.P_N = P[N - 1];
    e.A_N = gamma[N - 1];
    e.B_N = gamma[N - 1] * pi_inf[N - 1];
    for (int k = 0; k < 2; ++k) {
        const bool on = k < N - 1;
        e.dG[k] = on ? G[k] - G[N - 1] : 0.0;
        e.dP[k] = on ? P[k] - P[N - 1] : 0.0;
        e.dA[k] = on ? gamma[k] - gamma[N - 1] : 0.0;
        e.dB[k] = on ? gamma[k] * pi_inf[k] - gamma[N - 1] * pi_inf[N - 1] : 0.0;
    }
    return e;
}

// Host: cells per thread along direction dir of a sweep.  The FP64 stream
// sweeps do more work per cell, so longer segments halve the recomputed edge
// cells (256^3 shock-bubble: 104.4 vs 105.5 ms per step); the length is halved
// while fewer than ~8 warps per SM would be resident.
inline int sweep_segment(long long ncell, int n_dir, bool fp64_stream) {
    const long long trans = ncell / n_dir;
    int L = fp64_stream ? 128 : 64;
    while (L > 8 && trans * ((n_dir + L - 1) / L) < 152LL * 4 * kSweepThreads) L /= 2;
    return L;
}

// Explicitly instantiated in the mfc_inst_*.cu units.
#define MFC_DECLARE_INSTANCES(Real, NF)                                                         \
    extern template cudaError_t launch_sweep<Real, NF>(SweepArgs, int, int, cudaStream_t); \
    extern template cudaError_t launch_prims<Real, NF>(const PrimArgs&, int, bool, cudaStream_t); \
    extern template cudaError_t launch_cbc<Real, NF>(const SweepArgs&, int, long long, cudaStream_t);

MFC_DECLARE_INSTANCES(double, 1)
MFC_DECLARE_INSTANCES(double, 2)
MFC_DECLARE_INSTANCES(double, 3)
MFC_DECLARE_INSTANCES(float, 1)
MFC_DECLARE_INSTANCES(float, 2)
MFC_DECLARE_INSTANCES(float, 3)
extern template cudaError_t launch_sweep<float, 1, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 2, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 3, true>(SweepArgs, int, int, cudaStream_t);
// non-uniform grids (mfc_inst_*_nu_*.cu)
extern template cudaError_t launch_sweep<double, 1, false, 5, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<double, 2, false, 5, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<double, 3, false, 5, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 1, false, 5, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 2, false, 5, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 3, false, 5, true>(SweepArgs, int, int, cudaStream_t);
// WENO3 (mfc_inst_*_w3_*.cu)
extern template cudaError_t launch_sweep<double, 1, false, 3>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<double, 2, false, 3>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<double, 3, false, 3>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 1, false, 3>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 2, false, 3>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 3, false, 3>(SweepArgs, int, int, cudaStream_t);
// six-equation model (mfc_inst_*_six_*.cu; with a stretched grid or WENO3: mfc_inst_*_six_nu_*, *_six_w3_*)
extern template cudaError_t launch_sweep<double, 2, false, 5, true, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<double, 3, false, 5, true, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 2, false, 5, true, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 3, false, 5, true, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<double, 2, false, 3, false, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<double, 3, false, 3, false, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 2, false, 3, false, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 3, false, 3, false, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<double, 2, false, 5, false, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<double, 3, false, 5, false, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 2, false, 5, false, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_sweep<float, 3, false, 5, false, true>(SweepArgs, int, int, cudaStream_t);
extern template cudaError_t launch_prims<double, 2, true>(const PrimArgs&, int, bool, cudaStream_t);
extern template cudaError_t launch_prims<double, 3, true>(const PrimArgs&, int, bool, cudaStream_t);
extern template cudaError_t launch_prims<float, 2, true>(const PrimArgs&, int, bool, cudaStream_t);
extern template cudaError_t launch_prims<float, 3, true>(const PrimArgs&, int, bool, cudaStream_t);
extern template cudaError_t launch_cons6<2>(const Geometry&, const EosConst&, const double*, double*, int, cudaStream_t);
extern template cudaError_t launch_cons6<3>(const Geometry&, const EosConst&, const double*, double*, int, cudaStream_t);
extern template cudaError_t launch_cons<1>(const Geometry&, const EosConst&, const double*, double*, int, cudaStream_t);
extern template cudaError_t launch_cons<2>(const Geometry&, const EosConst&, const double*, double*, int, cudaStream_t);
extern template cudaError_t launch_cons<3>(const Geometry&, const EosConst&, const double*, double*, int, cudaStream_t);

}  // namespace mfc
