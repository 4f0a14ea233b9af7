// Allocation-free right-hand side (mfc_rhs_noalloc, declared in include/mfc.h).
//
// Some callers cannot let a library call cudaMalloc: host applications and
// frameworks that hand out every byte of device memory from their own pool or
// fixed budget, and time-critical loops that cannot absorb the implicit device
// synchronisation a cudaMalloc/cudaFree may take.  For them this entry point
// evaluates R(q) without any allocation: the caller passes the conserved state
// and the output buffer, and the only scratch the computation needs (the
// primitive variables of every cell) lives in the file-scope device array
// below, which every GPU that loads this library holds until the process exits.
//
// Host code must not use the array's name as a device address (in host code it
// is a host-side stand-in).  The device address is obtained once per device with
// cudaGetSymbolAddress, on the first call made with that device current, and
// cached; that first call should therefore come before any stream capture.  The
// cached address belongs to the device's primary context as it was then: after
// cudaDeviceReset (or anything else that re-creates that context) the module is
// loaded anew and the cached address is stale, so this entry point must not be
// used across a device reset.
// All calls share the array, so calls that overlap on the GPU (different
// streams, or different host threads on one device) race on it and must be
// serialised by the caller.  Nothing in it needs clearing: every call overwrites
// the primitives of all its cells before reading them.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/mfc.h"
#include "mfc_launch.cuh"

using namespace mfc;

namespace {

constexpr long long kMaxCells = MFC_NOALLOC_MAX_CELLS;
constexpr int kMaxVars = 2 * 3 + 3;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_prim_scratch[kMaxCells * kMaxVars];

std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {nullptr};

mfc_status noalloc_fail(char* err, int err_len, mfc_status s, const char* msg) {
    if (err && err_len > 0) {
        std::strncpy(err, msg, (size_t)err_len - 1);
        err[err_len - 1] = '\0';
    }
    return s;
}

mfc_status scratch_for_current_device(double** out, char* err, int err_len) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(err, err_len, MFC_ERR_CUDA, "no usable current CUDA device");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_prim_scratch);
        if (e != cudaSuccess || !p) {
            char buf[256];
            std::snprintf(buf, sizeof buf, "cudaGetSymbolAddress of the scratch array failed: %s",
                          cudaGetErrorString(e));
            return noalloc_fail(err, err_len, MFC_ERR_CUDA, buf);
        }
        g_scratch[dev] = static_cast<double*>(p);
    }
    *out = g_scratch[dev];
    return MFC_OK;
}

template <int NF>
cudaError_t run(const Geometry& g, const EosConst& e, int ndim, const double* q, double* rhs, double* w,
                double eps, int fallback, int cbc, cudaStream_t s) {
    PrimArgs pa{};
    pa.g = g;
    pa.e = e;
    pa.q = q;
    pa.w = w;
    cudaError_t rc = launch_prims<double, NF>(pa, ndim, false, s);
    if (rc != cudaSuccess) return rc;
    for (int d = 0; d < ndim; ++d) {
        SweepArgs a{};
        a.g = g;
        a.e = e;
        a.w = w;
        a.R = rhs;
        a.mode = d == 0 ? 0 : 1;
        a.acc_in = 0;
        a.yz_stream = 1;
        a.eps = eps;
        a.fallback = fallback;
        a.fallback_count = nullptr;
        a.cbc = cbc;
        sweep_set_f32_constants(a);
        a.seg = sweep_segment(g.ncell, g.n[d], true);
        a.nseg = (g.n[d] + a.seg - 1) / a.seg;
        rc = launch_sweep<double, NF>(a, ndim, d, s);
        if (rc != cudaSuccess) return rc;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" mfc_status mfc_rhs_noalloc(const double* q, double* rhs, int nx, int ny, int nz, const double lo[3],
                                      const double hi[3], const int bc[6], int num_fluids, const double* gamma,
                                      const double* pi_inf, double weno_eps, int fallback, void* cuda_stream,
                                      char* err, int err_len) {
    if (err && err_len > 0) err[0] = '\0';
    if (!q || !rhs || !lo || !hi || !bc || !gamma || !pi_inf)
        return noalloc_fail(err, err_len, MFC_ERR_ARG, "NULL pointer argument");
    if (num_fluids < 1 || num_fluids > 3) return noalloc_fail(err, err_len, MFC_ERR_ARG, "num_fluids must be 1..3");
    const int n[3] = {nx, ny, nz};
    const int ndim = nz > 1 ? 3 : (ny > 1 ? 2 : 1);
    for (int d = 0; d < 3; ++d) {
        if (d < ndim && (n[d] < 3 || !(hi[d] > lo[d])))
            return noalloc_fail(err, err_len, MFC_ERR_ARG, "each active direction needs >= 3 cells and hi > lo");
        if (d >= ndim && n[d] != 1)
            return noalloc_fail(err, err_len, MFC_ERR_ARG, "inactive directions must have 1 cell");
    }
    int cbc = 0;
    for (int i = 0; i < 6; ++i) {
        if (bc[i] < MFC_BC_PERIODIC || bc[i] > MFC_BC_CHARACTERISTIC)
            return noalloc_fail(err, err_len, MFC_ERR_ARG, "unknown boundary type");
        cbc |= i < 2 * ndim && bc[i] == MFC_BC_CHARACTERISTIC;
    }
    for (int d = 0; d < ndim; ++d)
        if ((bc[2 * d] == MFC_BC_PERIODIC) != (bc[2 * d + 1] == MFC_BC_PERIODIC))
            return noalloc_fail(err, err_len, MFC_ERR_ARG, "periodic must be set on both faces of a direction");
    for (int k = 0; k < num_fluids; ++k)
        if (!(gamma[k] > 1.0) || !(pi_inf[k] >= 0.0) || !std::isfinite(gamma[k]) || !std::isfinite(pi_inf[k]))
            return noalloc_fail(err, err_len, MFC_ERR_ARG, "need gamma > 1 and pi_inf >= 0");
    if (!(weno_eps >= 1e-30 && weno_eps <= 1.0))
        return noalloc_fail(err, err_len, MFC_ERR_ARG, "weno_eps must lie in [1e-30, 1]");
    if (fallback != 0 && fallback != 1) return noalloc_fail(err, err_len, MFC_ERR_ARG, "fallback must be 0 or 1");
    const long long ncell = (long long)nx * ny * nz;
    if (ncell > kMaxCells) {
        char buf[256];
        std::snprintf(buf, sizeof buf,
                      "grid of %lld cells exceeds the allocation-free maximum of %lld cells (MFC_NOALLOC_MAX_CELLS); "
                      "use mfc_init/mfc_rhs for larger grids",
                      ncell, kMaxCells);
        return noalloc_fail(err, err_len, MFC_ERR_ARG, buf);
    }

    double* w = nullptr;
    mfc_status st = scratch_for_current_device(&w, err, err_len);
    if (st != MFC_OK) return st;

    Geometry g{};
    for (int d = 0; d < 3; ++d) {
        g.n[d] = n[d];
        g.bc_lo[d] = bc[2 * d];
        g.bc_hi[d] = bc[2 * d + 1];
        g.inv_dx[d] = d < ndim ? n[d] / (hi[d] - lo[d]) : 0.0;
    }
    g.ncell = ncell;
    const int N = num_fluids;
    const EosConst e = make_eos_const(N, gamma, pi_inf);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t rc;
    switch (N) {
        case 1: rc = run<1>(g, e, ndim, q, rhs, w, weno_eps, fallback, cbc, s); break;
        case 2: rc = run<2>(g, e, ndim, q, rhs, w, weno_eps, fallback, cbc, s); break;
        default: rc = run<3>(g, e, ndim, q, rhs, w, weno_eps, fallback, cbc, s); break;
    }
    if (rc != cudaSuccess) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "kernel launch failed: %s", cudaGetErrorString(rc));
        return noalloc_fail(err, err_len, MFC_ERR_CUDA, buf);
    }
    return MFC_OK;
}
