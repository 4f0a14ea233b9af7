// C ABI of the GB300 five-equation right-hand-side library (declared in
// include/mfc.h).  Owns the device state of a context and sequences the
// kernels of one RHS evaluation and one SSP-RK3 step on the context's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mfc.h"
#include "mfc_grid.h"
#include "mfc_launch.cuh"

using namespace mfc;

// The learned form's device blob: MFC_MLP_PARAMS floats, then the packed
// per-lane fragments the sweeps load (16-byte aligned).
constexpr size_t kMlpFragOffset = 8192;
static_assert(kGridRow == kGridRowValues, "host and device grid rows agree");
static_assert(sizeof(float) * MFC_MLP_PARAMS <= kMlpFragOffset, "parameters fit before the fragments");

cudaError_t mfc_launch_mlp_pack(const float* P, void* frag, cudaStream_t s);
cudaError_t mfc_launch_prims_out(const double* q, double* w, long long nc, int nf, int ndim, const EosConst& e,
                                 int six, cudaStream_t s);

namespace {

enum ProfCat { P_PRIMS = 0, P_SWEEP_X, P_SWEEP_Y, P_SWEEP_Z, P_CFL, P_CONVERT, P_MLP, P_BOUNDARY, P_NCAT };

struct ProfRec {
    int cat;
    cudaEvent_t a, b;
};

}  // namespace

struct mfc_ctx {
    int n[3] = {1, 1, 1};
    int ndim = 1, nf = 1, ns = 3;
    long long ncell = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    int bc[6] = {1, 1, 1, 1, 1, 1};
    double gamma[3] = {0, 0, 0}, pi_inf[3] = {0, 0, 0};
    int precision = MFC_FP64;
    cudaStream_t stream = nullptr;
    double eps = 1e-6;
    int fallback = 1;
    int seg_override = 0;
    bool profile = false;
    double tau = 10.0;        // learned form: sensor threshold
    int yz_stream = -1;       // y/z sweep kernel: -1 automatic, 0 marching, 1 stream
    int bound = 1;            // learned form: range safeguard
    int weno_order = 5;       // reconstruction: WENO5-JS or WENO3-JS
    int rk_order = 3;         // SSP Runge-Kutta order of mfc_step: 1, 2 or 3
    int kapila = 0;           // model: 0 Allaire, 1 Kapila (K div u source)
    int six = 0;              // model 2: six-equation model with pressure relaxation
    int nw = 3;               // primitive rows (2N + d); ns = state rows (+N for the six-equation model)
    float* grid[3] = {nullptr, nullptr, nullptr};   // non-uniform directions: WENO5 rows (mfc_grid.cu)
    void* cbc_rates = nullptr;    // characteristic boundaries: rates of the boundary cells
    size_t cbc_bytes = 0;

    Geometry g{};
    EosConst e{};

    double* q = nullptr;      // state q^n
    double* q1 = nullptr;     // RK stage state
    void* R = nullptr;        // RHS accumulator (double or float)
    void* w = nullptr;        // primitives (double or float)
    void* w2 = nullptr;       // the other primitive buffer: the RK epilogue writes the next stage's here
    unsigned long long* d_rate = nullptr;  // CFL max (ordered bits)
    int* d_bad = nullptr;
    unsigned long long* d_fallback = nullptr;  // [0] fallback faces, [1] learned-form network rows
    unsigned long long* h_pin = nullptr;   // pinned readback [rate, bad]
    float* mlp = nullptr;         // network parameters, then (at byte kMlpFragOffset) the packed fragments

    bool state_set = false;
    bool w_valid = false;     // w holds the primitives of q
    bool rate_valid = false;  // d_rate / d_bad hold the CFL rate of q (written by the last RK epilogue)
    bool dead = false;
    long long launches = 0;
    std::string err;
    std::vector<ProfRec> prof_pending;
    double prof_ms[P_NCAT] = {0};
    long long prof_n[P_NCAT] = {0};
};

namespace {

mfc_status fail(mfc_ctx* c, mfc_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (s == MFC_ERR_CUDA) c->dead = true;
    }
    return s;
}

#define MFC_CUDA(ctx, call)                                                                \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((ctx), MFC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

bool is_f32(const mfc_ctx* c) { return c->precision != MFC_FP64; }

size_t real_size(const mfc_ctx* c) { return is_f32(c) ? sizeof(float) : sizeof(double); }

int auto_segment(const mfc_ctx* c, int dir) {
    if (c->seg_override > 0) return c->seg_override;
    return sweep_segment(c->ncell, c->n[dir], !is_f32(c) && c->yz_stream != 0);
}

template <typename F>
mfc_status launch(mfc_ctx* c, int cat, F&& fn) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->profile) {
        MFC_CUDA(c, cudaEventCreate(&a));
        MFC_CUDA(c, cudaEventCreate(&b));
        MFC_CUDA(c, cudaEventRecord(a, c->stream));
    }
    cudaError_t e = fn();
    if (e != cudaSuccess) return fail(c, MFC_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    c->launches += 1;
    if (c->profile) {
        MFC_CUDA(c, cudaEventRecord(b, c->stream));
        c->prof_pending.push_back({cat, a, b});
    }
    return MFC_OK;
}

bool nonuniform(const mfc_ctx* c) { return c->grid[0] || c->grid[1] || c->grid[2]; }

bool has_cbc(const mfc_ctx* c) {
    for (int i = 0; i < 2 * c->ndim; ++i)
        if (c->bc[i] == MFC_BC_CHARACTERISTIC) return true;
    return false;
}

cudaError_t dispatch_sweep(const mfc_ctx* c, const SweepArgs& a, int dir) {
    if (c->six) {
        const bool two = c->nf == 2;
        if (nonuniform(c)) {
            if (is_f32(c)) return two ? launch_sweep<float, 2, false, 5, true, true>(a, c->ndim, dir, c->stream)
                                      : launch_sweep<float, 3, false, 5, true, true>(a, c->ndim, dir, c->stream);
            return two ? launch_sweep<double, 2, false, 5, true, true>(a, c->ndim, dir, c->stream)
                       : launch_sweep<double, 3, false, 5, true, true>(a, c->ndim, dir, c->stream);
        }
        if (c->weno_order == 3) {
            if (is_f32(c)) return two ? launch_sweep<float, 2, false, 3, false, true>(a, c->ndim, dir, c->stream)
                                      : launch_sweep<float, 3, false, 3, false, true>(a, c->ndim, dir, c->stream);
            return two ? launch_sweep<double, 2, false, 3, false, true>(a, c->ndim, dir, c->stream)
                       : launch_sweep<double, 3, false, 3, false, true>(a, c->ndim, dir, c->stream);
        }
        if (is_f32(c)) return two ? launch_sweep<float, 2, false, 5, false, true>(a, c->ndim, dir, c->stream)
                                  : launch_sweep<float, 3, false, 5, false, true>(a, c->ndim, dir, c->stream);
        return two ? launch_sweep<double, 2, false, 5, false, true>(a, c->ndim, dir, c->stream)
                   : launch_sweep<double, 3, false, 5, false, true>(a, c->ndim, dir, c->stream);
    }
    if (nonuniform(c)) {
        if (is_f32(c)) {
            switch (c->nf) {
                case 1: return launch_sweep<float, 1, false, 5, true>(a, c->ndim, dir, c->stream);
                case 2: return launch_sweep<float, 2, false, 5, true>(a, c->ndim, dir, c->stream);
                default: return launch_sweep<float, 3, false, 5, true>(a, c->ndim, dir, c->stream);
            }
        }
        switch (c->nf) {
            case 1: return launch_sweep<double, 1, false, 5, true>(a, c->ndim, dir, c->stream);
            case 2: return launch_sweep<double, 2, false, 5, true>(a, c->ndim, dir, c->stream);
            default: return launch_sweep<double, 3, false, 5, true>(a, c->ndim, dir, c->stream);
        }
    }
    if (c->precision == MFC_LEARNED) {
        switch (c->nf) {
            case 1: return launch_sweep<float, 1, true>(a, c->ndim, dir, c->stream);
            case 2: return launch_sweep<float, 2, true>(a, c->ndim, dir, c->stream);
            default: return launch_sweep<float, 3, true>(a, c->ndim, dir, c->stream);
        }
    }
    if (c->weno_order == 3) {
        if (is_f32(c)) {
            switch (c->nf) {
                case 1: return launch_sweep<float, 1, false, 3>(a, c->ndim, dir, c->stream);
                case 2: return launch_sweep<float, 2, false, 3>(a, c->ndim, dir, c->stream);
                default: return launch_sweep<float, 3, false, 3>(a, c->ndim, dir, c->stream);
            }
        }
        switch (c->nf) {
            case 1: return launch_sweep<double, 1, false, 3>(a, c->ndim, dir, c->stream);
            case 2: return launch_sweep<double, 2, false, 3>(a, c->ndim, dir, c->stream);
            default: return launch_sweep<double, 3, false, 3>(a, c->ndim, dir, c->stream);
        }
    }
    if (is_f32(c)) {
        switch (c->nf) {
            case 1: return launch_sweep<float, 1>(a, c->ndim, dir, c->stream);
            case 2: return launch_sweep<float, 2>(a, c->ndim, dir, c->stream);
            default: return launch_sweep<float, 3>(a, c->ndim, dir, c->stream);
        }
    }
    switch (c->nf) {
        case 1: return launch_sweep<double, 1>(a, c->ndim, dir, c->stream);
        case 2: return launch_sweep<double, 2>(a, c->ndim, dir, c->stream);
        default: return launch_sweep<double, 3>(a, c->ndim, dir, c->stream);
    }
}

cudaError_t dispatch_prims(const mfc_ctx* c, const PrimArgs& a, bool rate) {
    if (c->six) {
        if (is_f32(c)) return c->nf == 2 ? launch_prims<float, 2, true>(a, c->ndim, rate, c->stream)
                                         : launch_prims<float, 3, true>(a, c->ndim, rate, c->stream);
        return c->nf == 2 ? launch_prims<double, 2, true>(a, c->ndim, rate, c->stream)
                          : launch_prims<double, 3, true>(a, c->ndim, rate, c->stream);
    }
    if (is_f32(c)) {
        switch (c->nf) {
            case 1: return launch_prims<float, 1>(a, c->ndim, rate, c->stream);
            case 2: return launch_prims<float, 2>(a, c->ndim, rate, c->stream);
            default: return launch_prims<float, 3>(a, c->ndim, rate, c->stream);
        }
    }
    switch (c->nf) {
        case 1: return launch_prims<double, 1>(a, c->ndim, rate, c->stream);
        case 2: return launch_prims<double, 2>(a, c->ndim, rate, c->stream);
        default: return launch_prims<double, 3>(a, c->ndim, rate, c->stream);
    }
}

cudaError_t dispatch_cons(const mfc_ctx* c, const double* w, double* q) {
    if (c->six)
        return c->nf == 2 ? launch_cons6<2>(c->g, c->e, w, q, c->ndim, c->stream)
                          : launch_cons6<3>(c->g, c->e, w, q, c->ndim, c->stream);
    switch (c->nf) {
        case 1: return launch_cons<1>(c->g, c->e, w, q, c->ndim, c->stream);
        case 2: return launch_cons<2>(c->g, c->e, w, q, c->ndim, c->stream);
        default: return launch_cons<3>(c->g, c->e, w, q, c->ndim, c->stream);
    }
}

mfc_status ensure_alive(mfc_ctx* c) {
    if (!c) return MFC_ERR_ARG;
    if (c->dead) return fail(c, MFC_ERR_CUDA, "context unusable after an earlier CUDA error: %s", c->err.c_str());
    return MFC_OK;
}

// Primitive recovery of src into c->w (optionally with the CFL rate).
mfc_status run_prims(mfc_ctx* c, const double* src, bool rate) {
    PrimArgs a{};
    a.g = c->g;
    a.e = c->e;
    a.q = src;
    a.w = c->w;
    a.rate_max = rate ? c->d_rate : nullptr;
    a.bad = rate ? c->d_bad : nullptr;
    for (int d = 0; d < 3; ++d) {   // layouts as mfc_set_grid stores them
        a.grid[d] = c->grid[d];
        a.grid_stride[d] = c->n[d] + 2;
    }
    return launch(c, rate ? P_CFL : P_PRIMS, [&] { return dispatch_prims(c, a, rate); });
}

SweepArgs base_sweep(const mfc_ctx* c) {
    SweepArgs a{};
    a.g = c->g;
    a.e = c->e;
    a.w = c->w;
    a.eps = c->eps;
    a.fallback = c->fallback;
    a.fallback_count = c->d_fallback;
    a.net_rows = c->d_fallback + 1;
    a.mlp_frag = c->mlp ? reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(c->mlp) + kMlpFragOffset)
                        : nullptr;
    a.tau = (float)c->tau;
    // y/z sweeps: the stream kernel (shared-memory ring) unless asked for the
    // pencil-marching kernel; with float-float WENO weights the FP64 path is
    // faster streamed too (256^3: 104 vs 122 ms per step)
    a.yz_stream = c->yz_stream >= 0 ? c->yz_stream : 1;
    a.bound = c->bound;
    a.kapila = c->kapila;
    a.cbc = has_cbc(c);
    for (int d = 0; d < 3; ++d) {   // layouts as mfc_set_grid stores them
        a.grid[d] = c->grid[d];
        a.grid_stride[d] = c->n[d] + 2;
    }
    for (int k = 0; k < 3; ++k) {
        a.kgam[k] = k < c->nf ? c->gamma[k] : 1.0;
        a.kpinf[k] = k < c->nf ? c->pi_inf[k] : 0.0;
        a.rc1[k] = k < c->nf ? (c->gamma[k] - 1.0) / c->gamma[k] : 0.0;
    }
    sweep_set_f32_constants(a);
    return a;
}

// All directional sweeps of one RHS evaluation on c->w.  The accumulator R has
// the arithmetic type of the path (float64 or float32).  With rk == nullptr the
// last sweep writes the float64 right-hand side to out; otherwise it applies
// the RK stage update described by rk.
struct RkStage {
    const double* q0;
    const double* qs;
    double* qout;
    double c0, c1, dt;
};

// Characteristic boundaries: the boundary cells' rates for this stage, ahead
// of the sweeps (cbc_rates_kernel); fills a's side-buffer fields.
mfc_status run_cbc(mfc_ctx* c, SweepArgs& a) {
    long long cells = 0;
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) {
            a.cbc_off[d][s] = -1;
            if (d < c->ndim && c->bc[2 * d + s] == MFC_BC_CHARACTERISTIC) {
                a.cbc_off[d][s] = cells * c->nw;
                cells += c->ncell / c->n[d];
            }
        }
    const size_t bytes = (size_t)cells * (size_t)c->nw * real_size(c);
    if (bytes > c->cbc_bytes) {
        cudaFree(c->cbc_rates);
        c->cbc_rates = nullptr;
        c->cbc_bytes = 0;
        cudaError_t e = cudaMalloc(&c->cbc_rates, bytes);
        if (e != cudaSuccess) {
            c->cbc_rates = nullptr;
            return fail(c, e == cudaErrorMemoryAllocation ? MFC_ERR_OOM : MFC_ERR_CUDA, "cudaMalloc: %s",
                        cudaGetErrorString(e));
        }
        c->cbc_bytes = bytes;
    }
    a.cbc_rates = c->cbc_rates;
    return launch(c, P_BOUNDARY, [&]() -> cudaError_t {
        if (is_f32(c)) {
            switch (c->nf) {
                case 1: return launch_cbc<float, 1>(a, c->ndim, cells, c->stream);
                case 2: return launch_cbc<float, 2>(a, c->ndim, cells, c->stream);
                default: return launch_cbc<float, 3>(a, c->ndim, cells, c->stream);
            }
        }
        switch (c->nf) {
            case 1: return launch_cbc<double, 1>(a, c->ndim, cells, c->stream);
            case 2: return launch_cbc<double, 2>(a, c->ndim, cells, c->stream);
            default: return launch_cbc<double, 3>(a, c->ndim, cells, c->stream);
        }
    });
}

mfc_status run_sweeps(mfc_ctx* c, double* out, const RkStage* rk, void* w_next = nullptr, bool rate = false) {
    SweepArgs cb{};
    if (has_cbc(c)) {
        cb = base_sweep(c);
        mfc_status s = run_cbc(c, cb);
        if (s != MFC_OK) return s;
    }
    for (int d = 0; d < c->ndim; ++d) {
        SweepArgs a = base_sweep(c);
        if (cb.cbc_rates) {
            a.cbc_rates = cb.cbc_rates;
            for (int k = 0; k < 3; ++k)
                for (int s = 0; s < 2; ++s) a.cbc_off[k][s] = cb.cbc_off[k][s];
        }
        a.seg = auto_segment(c, d);
        a.nseg = (c->n[d] + a.seg - 1) / a.seg;
        a.R = c->R;
        const bool last = (d == c->ndim - 1);
        a.acc_in = c->ndim > 1 ? 1 : 0;
        if (last && rk) {
            a.mode = 2;
            a.q0 = rk->q0;
            a.qs = rk->qs;
            a.qout = rk->qout;
            a.c0 = rk->c0;
            a.c1 = rk->c1;
            a.dt = rk->dt;
            a.w_next = w_next;
            a.rate_max = rate ? c->d_rate : nullptr;
            a.bad = rate ? c->d_bad : nullptr;
        } else if (last) {
            a.mode = 3;
            a.out = out;
        } else {
            a.mode = (d == 0) ? 0 : 1;
        }
        mfc_status s = launch(c, P_SWEEP_X + d, [&] { return dispatch_sweep(c, a, d); });
        if (s != MFC_OK) return s;
    }
    return MFC_OK;
}

void collect_profile(mfc_ctx* c) {
    for (auto& r : c->prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->prof_ms[r.cat] += ms;
            c->prof_n[r.cat] += 1;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->prof_pending.clear();
}

void free_all(mfc_ctx* c) {
    collect_profile(c);
    cudaFree(c->q);
    cudaFree(c->q1);
    cudaFree(c->R);
    cudaFree(c->w);
    cudaFree(c->w2);
    cudaFree(c->d_rate);
    cudaFree(c->d_bad);
    cudaFree(c->d_fallback);
    cudaFree(c->mlp);
    for (int d = 0; d < 3; ++d) cudaFree(c->grid[d]);
    cudaFree(c->cbc_rates);
    if (c->h_pin) cudaFreeHost(c->h_pin);
}

// (Re)allocate the state, stage and accumulator buffers for ns rows.
mfc_status alloc_state(mfc_ctx* c, int ns) {
    cudaFree(c->q);
    cudaFree(c->q1);
    cudaFree(c->R);
    c->q = c->q1 = nullptr;
    c->R = nullptr;
    const size_t bytes = sizeof(double) * (size_t)ns * (size_t)c->ncell;
    const size_t rbytes = real_size(c) * (size_t)ns * (size_t)c->ncell;
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&c->q, bytes)) != cudaSuccess || (e = cudaMalloc(&c->q1, bytes)) != cudaSuccess ||
        (e = cudaMalloc(&c->R, rbytes)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->q);
        cudaFree(c->q1);
        cudaFree(c->R);
        c->q = c->q1 = nullptr;
        c->R = nullptr;
        return fail(c, e == cudaErrorMemoryAllocation ? MFC_ERR_OOM : MFC_ERR_CUDA, "cudaMalloc: %s",
                    cudaGetErrorString(e));
    }
    c->ns = ns;
    return MFC_OK;
}

}  // namespace

extern "C" {

mfc_status mfc_init(mfc_ctx** out, int nx, int ny, int nz, const double lo[3], const double hi[3],
                    const int bc[6], int num_fluids, const double* gamma, const double* pi_inf,
                    int precision, void* cuda_stream) {
    if (!out || !lo || !hi || !bc || !gamma || !pi_inf) return MFC_ERR_ARG;
    if (num_fluids < 1 || num_fluids > 3) return MFC_ERR_ARG;
    if (precision < MFC_FP64 || precision > MFC_LEARNED) return MFC_ERR_ARG;
    const int n[3] = {nx, ny, nz};
    const int ndim = nz > 1 ? 3 : (ny > 1 ? 2 : 1);
    for (int d = 0; d < 3; ++d) {
        if (d < ndim && n[d] < 3) return MFC_ERR_ARG;
        if (d >= ndim && n[d] != 1) return MFC_ERR_ARG;
        if (d < ndim && !(hi[d] > lo[d]) ) return MFC_ERR_ARG;
    }
    bool any_cbc = false;
    for (int i = 0; i < 6; ++i) {
        if (bc[i] < MFC_BC_PERIODIC || bc[i] > MFC_BC_CHARACTERISTIC) return MFC_ERR_ARG;
        any_cbc |= i < 2 * ndim && bc[i] == MFC_BC_CHARACTERISTIC;
    }
    // characteristic boundaries: FP64 and mixed forms
    if (any_cbc && precision == MFC_LEARNED) return MFC_ERR_ARG;
    for (int d = 0; d < ndim; ++d)
        if ((bc[2 * d] == MFC_BC_PERIODIC) != (bc[2 * d + 1] == MFC_BC_PERIODIC)) return MFC_ERR_ARG;
    for (int k = 0; k < num_fluids; ++k)
        if (!(gamma[k] > 1.0) || !(pi_inf[k] >= 0.0) || !std::isfinite(gamma[k]) || !std::isfinite(pi_inf[k]))
            return MFC_ERR_ARG;
    const long long ncell = (long long)nx * ny * nz;
    if (ncell > (1LL << 34)) return MFC_ERR_ARG;

    mfc_ctx* c = new mfc_ctx();
    for (int d = 0; d < 3; ++d) {
        c->n[d] = n[d];
        c->lo[d] = lo[d];
        c->hi[d] = hi[d];
    }
    c->ndim = ndim;
    c->nf = num_fluids;
    c->ns = 2 * num_fluids + ndim;
    c->nw = c->ns;
    c->ncell = ncell;
    for (int i = 0; i < 6; ++i) c->bc[i] = bc[i];
    for (int k = 0; k < num_fluids; ++k) {
        c->gamma[k] = gamma[k];
        c->pi_inf[k] = pi_inf[k];
    }
    c->precision = precision;
    c->stream = static_cast<cudaStream_t>(cuda_stream);

    Geometry& g = c->g;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = n[d];
        g.bc_lo[d] = bc[2 * d];
        g.bc_hi[d] = bc[2 * d + 1];
        g.inv_dx[d] = d < ndim ? n[d] / (hi[d] - lo[d]) : 0.0;
    }
    g.ncell = ncell;
    c->e = make_eos_const(num_fluids, gamma, pi_inf);

    const size_t bytes = sizeof(double) * (size_t)c->ns * (size_t)ncell;
    const size_t wbytes = real_size(c) * (size_t)c->ns * (size_t)ncell;
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&c->q, bytes)) != cudaSuccess || (e = cudaMalloc(&c->q1, bytes)) != cudaSuccess ||
        (e = cudaMalloc(&c->R, wbytes)) != cudaSuccess || (e = cudaMalloc(&c->w, wbytes)) != cudaSuccess ||
        (e = cudaMalloc(&c->w2, wbytes)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_rate, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_bad, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_fallback, 2 * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_pin, 2 * sizeof(unsigned long long))) != cudaSuccess) {
        const bool oom = (e == cudaErrorMemoryAllocation);
        cudaGetLastError();
        free_all(c);
        delete c;
        return oom ? MFC_ERR_OOM : MFC_ERR_CUDA;
    }
    if (cudaMemsetAsync(c->d_fallback, 0, 2 * sizeof(unsigned long long), c->stream) != cudaSuccess) {
        free_all(c);
        delete c;
        return MFC_ERR_CUDA;
    }
    *out = c;
    return MFC_OK;
}

mfc_status mfc_set_param(mfc_ctx* c, const char* name, double value) {
    mfc_status s = ensure_alive(c);
    if (s != MFC_OK) return s;
    if (!name) return fail(c, MFC_ERR_ARG, "NULL parameter name");
    if (!strcmp(name, "weno_eps")) {
        if (!(value >= 1e-30 && value <= 1.0)) return fail(c, MFC_ERR_ARG, "weno_eps out of range");
        c->eps = value;
    } else if (!strcmp(name, "fallback")) {
        if (value != 0.0 && value != 1.0) return fail(c, MFC_ERR_ARG, "fallback must be 0 or 1");
        c->fallback = (int)value;
    } else if (!strcmp(name, "segment")) {
        if (!(value == 0.0 || (value >= 8 && value <= 256))) return fail(c, MFC_ERR_ARG, "segment out of range");
        c->seg_override = (int)value;
    } else if (!strcmp(name, "yz_kernel")) {
        if (value != -1.0 && value != 0.0 && value != 1.0) return fail(c, MFC_ERR_ARG, "yz_kernel must be -1, 0 or 1");
        c->yz_stream = (int)value;
    } else if (!strcmp(name, "learned_bound")) {
        if (value != 0.0 && value != 1.0) return fail(c, MFC_ERR_ARG, "learned_bound must be 0 or 1");
        c->bound = (int)value;
    } else if (!strcmp(name, "sensor_tau")) {
        if (!(value >= 1.0 && value <= 1e30)) return fail(c, MFC_ERR_ARG, "sensor_tau must lie in [1, 1e30]");
        c->tau = value;
    } else if (!strcmp(name, "weno_order")) {
        if (value != 3.0 && value != 5.0) return fail(c, MFC_ERR_ARG, "weno_order must be 3 or 5");
        if (value == 3.0 && c->precision == MFC_LEARNED)
            return fail(c, MFC_ERR_ARG, "the learned form replaces the WENO5 weights (weno_order 5)");
        if (value == 3.0 && nonuniform(c)) return fail(c, MFC_ERR_ARG, "non-uniform grids need weno_order 5");
        c->weno_order = (int)value;
    } else if (!strcmp(name, "rk_order")) {
        if (value != 1.0 && value != 2.0 && value != 3.0) return fail(c, MFC_ERR_ARG, "rk_order must be 1, 2 or 3");
        c->rk_order = (int)value;
    } else if (!strcmp(name, "model")) {
        if (value != 0.0 && value != 1.0 && value != 2.0)
            return fail(c, MFC_ERR_ARG, "model must be 0 (Allaire), 1 (Kapila) or 2 (six-equation)");
        if (value != 0.0 && has_cbc(c))
            return fail(c, MFC_ERR_ARG, "characteristic boundaries are defined for the Allaire model (model 0)");
        const int six = value == 2.0;
        if (six) {
            if (c->precision == MFC_LEARNED) return fail(c, MFC_ERR_ARG, "six-equation model: FP64 and mixed forms");
            if (c->nf < 2) return fail(c, MFC_ERR_ARG, "six-equation model: 2 or 3 fluids");
        }
        if (six != c->six) {   // the state layout changes: set the model before the state
            if (c->state_set) return fail(c, MFC_ERR_ARG, "set the model before the state");
            mfc_status st = alloc_state(c, c->nw + (six ? c->nf : 0));
            if (st != MFC_OK) return st;
            c->six = six;
        }
        c->kapila = value == 1.0;
    } else if (!strcmp(name, "profile")) {
        if (value != 0.0 && value != 1.0) return fail(c, MFC_ERR_ARG, "profile must be 0 or 1");
        c->profile = value != 0.0;
    } else {
        return fail(c, MFC_ERR_ARG, "unknown parameter '%s'", name);
    }
    return MFC_OK;
}

mfc_status mfc_set_grid(mfc_ctx* c, int dir, const double* faces, int nfaces) {
    mfc_status s = ensure_alive(c);
    if (s != MFC_OK) return s;
    if (dir < 0 || dir >= c->ndim) return fail(c, MFC_ERR_ARG, "direction %d is not active", dir);
    if (!faces || nfaces != c->n[dir] + 1) return fail(c, MFC_ERR_ARG, "need n+1 = %d face coordinates", c->n[dir] + 1);
    if (c->precision == MFC_LEARNED) return fail(c, MFC_ERR_ARG, "non-uniform grids: FP64 and mixed forms only");
    if (c->weno_order != 5) return fail(c, MFC_ERR_ARG, "non-uniform grids need weno_order 5");
    const bool periodic = c->bc[2 * dir] == MFC_BC_PERIODIC;
    std::vector<float> rows;
    if (!grid_tables(faces, c->n[dir], periodic, rows))
        return fail(c, MFC_ERR_ARG, "faces must be finite and strictly increasing");
    // device layout: x value-major (value k of cell c at pair k * (n+2) + c + 1,
    // coalesced across the lanes of the x sweep), y and z row-major as built
    const int nc = c->n[dir] + 2;
    std::vector<float> tab(rows);
    if (dir == 0)
        for (int cell = 0; cell < nc; ++cell)
            for (int k = 0; k < kGridRow; ++k) {
                tab[2 * ((size_t)k * nc + cell)] = rows[((size_t)cell * kGridRow + k) * 2];
                tab[2 * ((size_t)k * nc + cell) + 1] = rows[((size_t)cell * kGridRow + k) * 2 + 1];
            }
    if (!c->grid[dir]) {
        cudaError_t e = cudaMalloc(&c->grid[dir], tab.size() * sizeof(float));
        if (e != cudaSuccess) {
            c->grid[dir] = nullptr;
            return fail(c, e == cudaErrorMemoryAllocation ? MFC_ERR_OOM : MFC_ERR_CUDA, "cudaMalloc: %s",
                        cudaGetErrorString(e));
        }
    }
    MFC_CUDA(c, cudaMemcpyAsync(c->grid[dir], tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice,
                                c->stream));
    MFC_CUDA(c, cudaStreamSynchronize(c->stream));
    c->rate_valid = false;   // the CFL rate depends on the widths
    return MFC_OK;
}

mfc_status mfc_set_state(mfc_ctx* c, const double* q, int on_device) {
    mfc_status s = ensure_alive(c);
    if (s != MFC_OK) return s;
    if (!q) return fail(c, MFC_ERR_ARG, "NULL state");
    const size_t bytes = sizeof(double) * (size_t)c->ns * (size_t)c->ncell;
    MFC_CUDA(c, cudaMemcpyAsync(c->q, q, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                c->stream));
    if (!on_device) MFC_CUDA(c, cudaStreamSynchronize(c->stream));
    c->state_set = true;
    c->w_valid = false;
    c->rate_valid = false;
    return MFC_OK;
}

mfc_status mfc_set_state_prim(mfc_ctx* c, const double* w, int on_device) {
    mfc_status s = ensure_alive(c);
    if (s != MFC_OK) return s;
    if (!w) return fail(c, MFC_ERR_ARG, "NULL state");
    const double* src = w;
    if (!on_device) {
        const size_t bytes = sizeof(double) * (size_t)c->ns * (size_t)c->ncell;
        MFC_CUDA(c, cudaMemcpyAsync(c->q1, w, bytes, cudaMemcpyHostToDevice, c->stream));
        src = c->q1;
    }
    s = launch(c, P_CONVERT, [&] { return dispatch_cons(c, src, c->q); });
    if (s != MFC_OK) return s;
    if (!on_device) MFC_CUDA(c, cudaStreamSynchronize(c->stream));
    c->state_set = true;
    c->w_valid = false;
    c->rate_valid = false;
    return MFC_OK;
}

mfc_status mfc_get_state(mfc_ctx* c, double* q, int on_device) {
    mfc_status s = ensure_alive(c);
    if (s != MFC_OK) return s;
    if (!q) return fail(c, MFC_ERR_ARG, "NULL buffer");
    if (!c->state_set) return fail(c, MFC_ERR_STATE_UNSET, "no state set");
    const size_t bytes = sizeof(double) * (size_t)c->ns * (size_t)c->ncell;
    MFC_CUDA(c, cudaMemcpyAsync(q, c->q, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
    if (!on_device) MFC_CUDA(c, cudaStreamSynchronize(c->stream));
    return MFC_OK;
}

mfc_status mfc_rhs(mfc_ctx* c, double* rhs, int on_device) {
    mfc_status s = ensure_alive(c);
    if (s != MFC_OK) return s;
    if (!rhs) return fail(c, MFC_ERR_ARG, "NULL rhs");
    if (!c->state_set) return fail(c, MFC_ERR_STATE_UNSET, "no state set");
    if (c->precision == MFC_LEARNED && !c->mlp) return fail(c, MFC_ERR_ARG, "learned mode needs mfc_set_mlp");
    if (!c->w_valid) {
        s = run_prims(c, c->q, false);
        if (s != MFC_OK) return s;
        c->w_valid = true;
    }
    // the float64 result goes to the caller's device buffer, or through the
    // stage buffer to host memory
    double* target = on_device ? rhs : c->q1;
    s = run_sweeps(c, target, nullptr);
    if (s != MFC_OK) return s;
    if (!on_device) {
        const size_t bytes = sizeof(double) * (size_t)c->ns * (size_t)c->ncell;
        MFC_CUDA(c, cudaMemcpyAsync(rhs, c->q1, bytes, cudaMemcpyDeviceToHost, c->stream));
        MFC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return MFC_OK;
}

mfc_status mfc_step(mfc_ctx* c, double dt) {
    mfc_status s = ensure_alive(c);
    if (s != MFC_OK) return s;
    if (!c->state_set) return fail(c, MFC_ERR_STATE_UNSET, "no state set");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, MFC_ERR_ARG, "dt must be finite and > 0");
    if (c->precision == MFC_LEARNED && !c->mlp) return fail(c, MFC_ERR_ARG, "learned mode needs mfc_set_mlp");
    if (!c->w_valid) {
        s = run_prims(c, c->q, false);
        if (s != MFC_OK) return s;
    }
    c->w_valid = false;
    c->rate_valid = false;
    // FP64 five-equation models: the last sweep of every stage writes the
    // primitives of the stage's new state into w2 (then swapped with w), and
    // the last stage also the CFL rate of q^{n+1}, so no separate recovery pass
    // runs (256^3 shock-bubble: 59.0 -> 58.2 ms per step).  The six-equation
    // model relaxes in the epilogue and the FP32 forms' memory-bound z sweep
    // gains nothing from it: they recover separately.
    const bool fused = !c->six && !is_f32(c);
    auto stage = [&](const RkStage& st, bool last) -> mfc_status {
        if (!fused) return run_sweeps(c, nullptr, &st);
        if (last) {
            MFC_CUDA(c, cudaMemsetAsync(c->d_rate, 0, sizeof(unsigned long long), c->stream));
            MFC_CUDA(c, cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->stream));
        }
        mfc_status r = run_sweeps(c, nullptr, &st, c->w2, last);
        if (r != MFC_OK) return r;
        std::swap(c->w, c->w2);
        return MFC_OK;
    };
    auto between = [&](const double* q) -> mfc_status { return fused ? MFC_OK : run_prims(c, q, false); };
    if (c->rk_order == 1) {
        // forward Euler, in place: q = q + dt R(q)
        RkStage st{c->q, c->q, c->q, 0.0, 1.0, dt};
        if ((s = stage(st, true)) != MFC_OK) return s;
    } else if (c->rk_order == 2) {
        // SSP-RK2: q1 = q + dt R(q); q = 1/2 q + 1/2 (q1 + dt R(q1))
        RkStage st1{c->q, c->q, c->q1, 0.0, 1.0, dt};
        if ((s = stage(st1, false)) != MFC_OK) return s;
        if ((s = between(c->q1)) != MFC_OK) return s;
        RkStage st2{c->q, c->q1, c->q, 0.5, 0.5, dt};
        if ((s = stage(st2, true)) != MFC_OK) return s;
    } else {
        // SSP-RK3, stage 1: q1 = q + dt R(q)
        RkStage st1{c->q, c->q, c->q1, 0.0, 1.0, dt};
        if ((s = stage(st1, false)) != MFC_OK) return s;
        // stage 2: q1 = 3/4 q + 1/4 (q1 + dt R(q1))
        if ((s = between(c->q1)) != MFC_OK) return s;
        RkStage st2{c->q, c->q1, c->q1, 0.75, 0.25, dt};
        if ((s = stage(st2, false)) != MFC_OK) return s;
        // stage 3: q = 1/3 q + 2/3 (q1 + dt R(q1))
        if ((s = between(c->q1)) != MFC_OK) return s;
        RkStage st3{c->q, c->q1, c->q, 1.0 / 3.0, 2.0 / 3.0, dt};
        if ((s = stage(st3, true)) != MFC_OK) return s;
    }
    c->w_valid = fused;
    c->rate_valid = fused;
    return MFC_OK;
}

mfc_status mfc_cfl_dt(mfc_ctx* c, double cfl, double* dt_out) {
    mfc_status s = ensure_alive(c);
    if (s != MFC_OK) return s;
    if (!dt_out || !(cfl > 0.0) || !std::isfinite(cfl)) return fail(c, MFC_ERR_ARG, "bad cfl or NULL dt_out");
    if (!c->state_set) return fail(c, MFC_ERR_STATE_UNSET, "no state set");
    if (!c->rate_valid) {   // else the last RK epilogue computed it for this state
        MFC_CUDA(c, cudaMemsetAsync(c->d_rate, 0, sizeof(unsigned long long), c->stream));
        MFC_CUDA(c, cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->stream));
        s = run_prims(c, c->q, true);
        if (s != MFC_OK) return s;
        c->w_valid = true;
        c->rate_valid = true;
    }
    MFC_CUDA(c, cudaMemcpyAsync(&c->h_pin[0], c->d_rate, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                c->stream));
    MFC_CUDA(c, cudaMemcpyAsync(&c->h_pin[1], c->d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MFC_CUDA(c, cudaStreamSynchronize(c->stream));
    const int bad = *reinterpret_cast<int*>(&c->h_pin[1]);
    double rate;
    unsigned long long bits = c->h_pin[0];
    std::memcpy(&rate, &bits, sizeof rate);
    if (bad > 0 || !(rate > 0.0) || !std::isfinite(rate)) {
        *dt_out = 0.0;
        return fail(c, MFC_ERR_NONPHYSICAL, "non-physical state in %d cell(s)", bad);
    }
    *dt_out = cfl / rate;
    return MFC_OK;
}

mfc_status mfc_set_mlp(mfc_ctx* c, const float* params, int n) {
    mfc_status s = ensure_alive(c);
    if (s != MFC_OK) return s;
    if (!params || n != MFC_MLP_PARAMS) return fail(c, MFC_ERR_ARG, "need %d parameters", MFC_MLP_PARAMS);
    if (c->precision != MFC_LEARNED) return fail(c, MFC_ERR_ARG, "context is not MFC_LEARNED");
    if (!c->mlp) {
        cudaError_t e = cudaMalloc(&c->mlp, kMlpFragOffset + kMlpFragBytes);
        if (e != cudaSuccess) {
            c->mlp = nullptr;
            return fail(c, e == cudaErrorMemoryAllocation ? MFC_ERR_OOM : MFC_ERR_CUDA, "cudaMalloc: %s",
                        cudaGetErrorString(e));
        }
    }
    MFC_CUDA(c, cudaMemcpyAsync(c->mlp, params, sizeof(float) * MFC_MLP_PARAMS, cudaMemcpyHostToDevice, c->stream));
    MFC_CUDA(c, mfc_launch_mlp_pack(c->mlp, reinterpret_cast<char*>(c->mlp) + kMlpFragOffset, c->stream));
    ++c->launches;
    MFC_CUDA(c, cudaStreamSynchronize(c->stream));
    return MFC_OK;
}

mfc_status mfc_get_prims(mfc_ctx* c, double* w, int on_device) {
    mfc_status s = ensure_alive(c);
    if (s != MFC_OK) return s;
    if (!w) return fail(c, MFC_ERR_ARG, "NULL buffer");
    if (!c->state_set) return fail(c, MFC_ERR_STATE_UNSET, "no state set");
    double* dst = on_device ? w : c->q1;
    s = launch(c, P_CONVERT,
               [&] { return mfc_launch_prims_out(c->q, dst, c->ncell, c->nf, c->ndim, c->e, c->six, c->stream); });
    if (s != MFC_OK) return s;
    if (!on_device) {
        const size_t bytes = sizeof(double) * (size_t)c->ns * (size_t)c->ncell;
        MFC_CUDA(c, cudaMemcpyAsync(w, c->q1, bytes, cudaMemcpyDeviceToHost, c->stream));
        MFC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return MFC_OK;
}

int mfc_sys_size(const mfc_ctx* c) { return c ? c->ns : 0; }

long long mfc_launch_count(const mfc_ctx* c) { return c ? c->launches : 0; }

long long mfc_fallback_count(mfc_ctx* c) {
    if (!c || c->dead) return -1;
    unsigned long long v = 0;
    if (cudaMemcpyAsync(&c->h_pin[0], c->d_fallback, sizeof v, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return -1;
    v = c->h_pin[0];
    return (long long)v;
}

long long mfc_network_rows(mfc_ctx* c) {
    if (!c || c->dead) return -1;
    if (cudaMemcpyAsync(&c->h_pin[0], c->d_fallback + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return -1;
    return (long long)c->h_pin[0];
}

int mfc_profile_read(mfc_ctx* c, double* total_ms, long long* launches, int n) {
    if (!c) return 0;
    collect_profile(c);
    for (int i = 0; i < n && i < P_NCAT; ++i) {
        if (total_ms) total_ms[i] = c->prof_ms[i];
        if (launches) launches[i] = c->prof_n[i];
    }
    return P_NCAT;
}

const char* mfc_last_error(const mfc_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

void mfc_finalize(mfc_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

}  // extern "C"
