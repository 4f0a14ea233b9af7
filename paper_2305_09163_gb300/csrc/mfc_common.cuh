// Common device types of the sweeps: boundary kinds, grid geometry, the EOS
// constants, the arguments of every kernel, the variable layout, ghost-cell
// index mapping and the FP64 Newton reciprocal.
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
    void* w_next;           // mode 2, optional: primitives of qout [NS][ncell], Real (five-equation models)
    unsigned long long* rate_max;  // with w_next, optional: CFL rate of qout, max as ordered bits
    int* bad;               // with rate_max: count of non-physical cells of qout
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
    int stage;              // y/z stream kernels: finish operands staged in dynamic shared
                            // memory by cp.async (bit 0: R, bit 1: qs, bit 2: q0; 0: none)
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

}  // namespace mfc
