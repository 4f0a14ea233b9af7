/*
 * mfc.h -- C ABI of the GB300 (sm_103a) right-hand-side library for the
 * five-equation diffuse-interface model with stiffened-gas fluids
 * (arXiv 2305.09163).
 *
 * One context = one uniform structured grid on one GPU, its boundary types,
 * its fluids and a CUDA stream.  All device work of a context is enqueued on
 * that stream.  Every call returns an mfc_status and never aborts; the text of
 * the last error is kept per context (mfc_last_error).  After MFC_ERR_CUDA the
 * context is unusable except for mfc_finalize.
 *
 * Layout of every state array (conserved q, primitive w, right-hand side R):
 * structure of arrays, float64, [sys_size][nz][ny][nx] with x fastest;
 * sys_size = 2*N + d for N fluids and d active dimensions.  Variable order
 * (Sec. 2.1, "5-equation models"):
 *     conserved q: a_1 r_1 .. a_N r_N, r u_x [, r u_y, r u_z], r E, a_1 .. a_{N-1}
 *     primitive w: a_1 r_1 .. a_N r_N,   u_x [,   u_y,   u_z],   p, a_1 .. a_{N-1}
 * where a_k are volume fractions (a_N = 1 - sum of the others), r_k phase
 * densities, u the mixture velocity, E the total energy and p the pressure.
 * The six-equation model ("model" 2) appends N rows, sys_size = 3*N + d:
 *     conserved q: ..., a_1 r_1 e_1 .. a_N r_N e_N   (phase internal energies)
 *     primitive w: ..., p_1 .. p_N                   (phase pressures)
 * with a_k r_k e_k = a_k (p_k + g_k pinf_k)/(g_k - 1); there the primitive p
 * is the pressure of the mixture law for the total energy.
 *
 * Pointers: "on_device" = 1 means a device pointer on the context's GPU
 * (e.g. a contiguous float64 torch tensor's data_ptr), used in stream order;
 * 0 means host memory, and the call returns after the copy completes.  The
 * caller owns every q / w / rhs buffer it passes; the library owns its own
 * device state and releases it in mfc_finalize.
 */
#ifndef MFC_GB300_H
#define MFC_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mfc_ctx mfc_ctx;

typedef enum {
    MFC_OK = 0,
    MFC_ERR_ARG = 1,          /* invalid argument; nothing was changed */
    MFC_ERR_STATE_UNSET = 2,  /* no state has been set on this context */
    MFC_ERR_OOM = 3,          /* device allocation failed */
    MFC_ERR_CUDA = 4,         /* CUDA error; the context is now unusable */
    MFC_ERR_NONPHYSICAL = 5,  /* non-finite state or c^2 <= 0 somewhere */
    MFC_ERR_TIMEOUT = 6       /* reserved: a bounded device wait expired */
} mfc_status;

typedef enum {
    MFC_BC_PERIODIC = 0,
    MFC_BC_TRANSMISSIVE = 1,
    MFC_BC_REFLECTIVE = 2,
    MFC_BC_CHARACTERISTIC = 3
} mfc_bc;

/* Arithmetic of the reconstruction and Riemann solver:
 *   MFC_FP64    float64 state, primitive recovery, stencil differences, edge
 *               sums, mixture rules, fluxes, divergence and Runge-Kutta
 *               update; the WENO nonlinear weights and the HLLC solver are
 *               evaluated in float-float arithmetic (a value is the unevaluated
 *               sum of two float32 numbers, about 48 significant bits) with the
 *               float32 exponent range, and their results are widened back to
 *               float64.  The right-hand side matches a plain float64
 *               evaluation to 1e-11 relative to each component's flux scale.
 *               Supported range (SI units): every primitive value, stencil
 *               difference and pressure jump below 1e18 in magnitude (the
 *               smoothness indicators square the differences in float32
 *               range), every product of three state values such as
 *               (rho E + p) u below 1e37; a magnitude below 2^-126 (1.2e-38)
 *               inside these solvers counts as zero, an absolute error far
 *               below any flux scale;
 *   MFC_MIXED   WENO5 and HLLC in float32; pressure recovery from total energy
 *               and the Runge-Kutta accumulation stay float64;
 *   MFC_LEARNED as MFC_MIXED, with WENO5 nonlinear weights from a small MLP
 *               (mfc_set_mlp) except where the shock/interface sensor trips or
 *               the learned edge value would leave the range of the cell and
 *               its two neighbours, where WENO5-JS weights are used; a
 *               non-physical learned face state falls back to WENO5-JS, then
 *               to first order. */
typedef enum { MFC_FP64 = 0, MFC_MIXED = 1, MFC_LEARNED = 2 } mfc_precision;

/* Create a context (Sec. 3.1: uniform structured grid; Sec. 3.3: ghost-cell
 * boundaries; Sec. 2.1: stiffened-gas fluids).
 *   nx, ny, nz   cells per direction; 1D: ny = nz = 1, 2D: nz = 1.  Every
 *                active direction needs at least 3 cells.
 *   lo, hi       domain corners [3] (only active directions are used).
 *   bc           [6] boundary types for -x,+x,-y,+y,-z,+z (mfc_bc); periodic
 *                must be set on both faces of a direction.  Characteristic
 *                (non-reflecting, Sec. 3.3 after Thompson): ghost cells as
 *                transmissive for the faces of interior cells, while the
 *                boundary cell's normal rate comes from the wave amplitudes
 *                of the quasi-linear primitive system (one-sided difference
 *                to the interior neighbour over the boundary cell's width),
 *                with the amplitudes of incoming waves set to zero.  FP64 and
 *                mixed forms, Allaire model only (MFC_ERR_ARG otherwise).
 *   num_fluids   N in 1..3; gamma[N] > 1, pi_inf[N] >= 0 (Pa).
 *   precision    mfc_precision.
 *   cuda_stream  cudaStream_t to use, or NULL for the legacy default stream.
 * Allocates the state, one stage buffer, a primitive buffer and a
 * right-hand-side accumulator on the current CUDA device.
 * Errors: MFC_ERR_ARG (bad sizes / parameters; *out untouched),
 * MFC_ERR_OOM, MFC_ERR_CUDA. */
mfc_status mfc_init(mfc_ctx** out, int nx, int ny, int nz, const double lo[3], const double hi[3],
                    const int bc[6], int num_fluids, const double* gamma, const double* pi_inf,
                    int precision, void* cuda_stream);

/* Set a numerical parameter by name:
 *   "weno_eps"   epsilon of the WENO weights (Sec. 3.2), default 1e-6,
 *                valid range [1e-30, 1];
 *   "weno_order" 5 (default): WENO5-JS; 3: WENO3-JS, the third-order variant
 *                of Sec. 3.2 (FP64 and mixed forms; the learned form needs 5);
 *   "model"      0 (default): Allaire five-equation model; 1: Kapila model
 *                (Sec. 2.1), the volume-fraction rows gain K_k div(u) with
 *                K_k = alpha_k (rho c_W^2/(rho_k c_k^2) - 1), c_W Wood's mixture
 *                sound speed (two fluids: the formula of Sec. 2.1);
 *                2: six-equation model with pressure relaxation (Sec. 2.3;
 *                2 or 3 fluids, FP64 and mixed forms, no characteristic
 *                boundaries): the state gains the phase
 *                internal energies (layout above), waves travel at the frozen
 *                sound speed r c^2 = sum_k a_k g_k (p + pinf_k), the phase
 *                energies are carried with the face velocity and lose
 *                a_k p div(u), and every Runge-Kutta stage of mfc_step ends
 *                with the relaxation to one pressure with infinite stiffness
 *                (each phase's energy follows de_k = -p dv_k at the final
 *                pressure p; sum_k a_k = 1 fixes p; then p is recomputed from
 *                the total energy and the phase energies reset to it; phases
 *                with a_k <= 0 or p_k + pinf_k <= 0 keep their a_k).  mfc_rhs
 *                returns the hyperbolic part; it takes the phases at the
 *                mixture pressure (the states it acts on are relaxed).  The
 *                state layout changes, so set the model before the state
 *                (MFC_ERR_ARG otherwise);
 *   "rk_order"   order of the SSP Runge-Kutta step of mfc_step (Sec. 3.4):
 *                3 (default), 2 (q1 = q + dt R(q), q' = 1/2 q + 1/2 (q1 + dt R(q1)))
 *                or 1 (forward Euler);
 *   "fallback"   1 (default) / 0: first-order reconstruction (Sec. 3.2) at a
 *                face whose reconstructed state is non-physical;
 *   "segment"    cells per thread along a sweep (8..256), 0 = automatic;
 *   "yz_kernel"  y/z sweep kernel: -1 automatic (default: the stream kernel),
 *                0 pencil marching, 1 stream;
 *   "sensor_tau" learned form: the discontinuity sensor trips (WENO5-JS
 *                weights are used) where max_r b_r > tau (min_r b_r + 1e-6 s^2),
 *                b the smoothness indicators without their 4/3 factor and s the
 *                stencil scale; default 10, range [1, 1e30];
 *   "learned_bound" learned form: 1 (default) / 0: keep a learned edge value
 *                only inside the range of the cell and its two neighbours
 *                (WENO5-JS value otherwise);
 *   "profile"    1 / 0: time every kernel launch with CUDA events.
 * Errors: MFC_ERR_ARG for an unknown name or out-of-range value. */
mfc_status mfc_set_param(mfc_ctx* ctx, const char* name, double value);

/* Non-uniform grid (Sec. 4.1: a structured mesh with non-uniform spacing,
 * e.g. the tanh stretching of Sec. 6.3): faces[0..n_dir] are the strictly
 * increasing face coordinates of the n_dir cells of direction dir (0 x, 1 y,
 * 2 z; an active direction).  The library builds, on the host, the per-cell
 * WENO5 coefficients of the finite-volume reconstruction on each five-cell
 * stencil (candidates, ideal weights, smoothness indicators; Listing 1 keeps
 * such per-index tables) and 1/dx per cell, used by the sweeps, the divergence
 * and the CFL rate; ghost cells mirror (or, periodic, wrap) the interior
 * widths.  The direction's lo/hi of mfc_init are then unused.  FP64 and mixed
 * forms with weno_order 5 only; the y/z sweeps use the stream kernel.
 * Host pointer, copied.  Errors: MFC_ERR_ARG (inactive direction, wrong
 * count, non-increasing or non-finite faces, learned form, weno_order 3),
 * MFC_ERR_OOM, MFC_ERR_CUDA. */
mfc_status mfc_set_grid(mfc_ctx* ctx, int dir, const double* faces, int nfaces);

/* The table mfc_set_grid uploads, on the host (no GPU needed): for the cells
 * -1..n of a direction with faces[0..n], 28 values per cell, each as an FP32
 * pair (hi, lo): candidate increments at c+1/2 (ea0, eb0, ea1, eb1, ea2, eb2;
 * p_r - v_c = ea_r Da_r + eb_r Db_r, (Da, Db) = (D0, D1), (D1, D2), (D2, D3) with
 * D_k = v_{c+k-1} - v_{c+k-2}), the same at c-1/2, the ideal weights at c+1/2
 * and at c-1/2, beta_r = qa Da^2 + qab Da Db + qb Db^2 (qa, qab, qb per r), 1/dx.
 * out receives (n + 2) * 56 floats.  Returns 0; the needed length if out is
 * NULL or out_len is too small; -1 for bad faces. */
int mfc_grid_table(const double* faces, int n, int periodic, float* out, long long out_len);

/* Copy a conserved state q (layout above) into the context: the cell
 * averages q_{i,j,k} of the conserved variables of Eq. "fvm" (Sec. 3.1; the
 * variables of Sec. 2.1's five-equation model), which mfc_step advances.
 * No check of physical validity is made here (mfc_cfl_dt does it).
 * Errors: MFC_ERR_ARG (NULL q), MFC_ERR_CUDA. */
mfc_status mfc_set_state(mfc_ctx* ctx, const double* q, int on_device);

/* Set the state from primitive variables w (layout above); the conversion
 * rho E = Gamma p + Pi + rho|u|^2/2 (Sec. 2.1, Eq. "soe" with the mixture
 * rules) runs on the GPU.  Six-equation model: the phase pressures give the
 * phase energies and r E = sum_k a_k r_k e_k + r|u|^2/2; the row p is not
 * read. */
mfc_status mfc_set_state_prim(mfc_ctx* ctx, const double* w, int on_device);

/* Copy the current conserved state out: the cell averages q_{i,j,k} of
 * Eq. "fvm" (Sec. 3.1), layout above.  With a host pointer the call waits for
 * the stream; with a device pointer the copy is enqueued on it.
 * Errors: MFC_ERR_STATE_UNSET, MFC_ERR_ARG (NULL q), MFC_ERR_CUDA. */
mfc_status mfc_get_state(mfc_ctx* ctx, double* q, int on_device);

/* R(q) of Eq. "fvmdis" (Sec. 3.1) for the current state: WENO5 reconstruction
 * of primitives, HLLC fluxes, flux divergence and the a_k div(u) source of the
 * volume-fraction rows, written to rhs (layout above).
 * Errors: MFC_ERR_STATE_UNSET, MFC_ERR_ARG (NULL rhs), MFC_ERR_CUDA. */
mfc_status mfc_rhs(mfc_ctx* ctx, double* rhs, int on_device);

/* Advance the state by one SSP Runge-Kutta step of size dt (Sec. 3.4); with
 * the default rk_order 3:
 *   q1 = q + dt R(q); q2 = 3/4 q + 1/4 (q1 + dt R(q1)); q' = 1/3 q + 2/3 (q2 + dt R(q2)).
 * (rk_order 2 and 1: see mfc_set_param.)  Enqueued on the stream; returns
 * without waiting.
 * Errors: MFC_ERR_STATE_UNSET, MFC_ERR_ARG (dt not finite or <= 0), MFC_ERR_CUDA. */
mfc_status mfc_step(mfc_ctx* ctx, double dt);

/* CFL time step of the current state (Sec. 1: the Courant-Friedrichs-Lewy
 * constraint restricts the explicit time step; the paper gives no formula, so
 * this is the usual one): dt = cfl / max over cells and directions of
 * (|u_d| + c)/dx_d, with c^2 = ((Gamma+1)p + Pi)/(Gamma rho).
 * Synchronises the stream (8-byte readback).  Errors: MFC_ERR_NONPHYSICAL if
 * any cell has a non-finite state or c^2 <= 0 (*dt_out = 0),
 * MFC_ERR_STATE_UNSET, MFC_ERR_ARG. */
mfc_status mfc_cfl_dt(mfc_ctx* ctx, double cfl, double* dt_out);

/* Number of float32 parameters of the learned-weight network. */
#define MFC_MLP_PARAMS 1347

/* Install the learned-weight network (MFC_LEARNED): host array of
 * MFC_MLP_PARAMS floats laid out as W1[32][5], b1[32], W2[32][32], b2[32],
 * W3[3][32], b3[3] (inputs 5 normalised stencil differences, two ReLU layers of
 * 32, softmax over the 3 WENO5 candidates; see mfc_mlp_forward).  The library
 * keeps a device copy.  Errors: MFC_ERR_ARG (NULL, wrong n, or the context is
 * not MFC_LEARNED), MFC_ERR_CUDA. */
mfc_status mfc_set_mlp(mfc_ctx* ctx, const float* params, int n);

/* Primitive variables of the current state (layout above), float64.  Errors:
 * MFC_ERR_STATE_UNSET, MFC_ERR_ARG, MFC_ERR_CUDA. */
mfc_status mfc_get_prims(mfc_ctx* ctx, double* w, int on_device);

/* ---- Learned WENO weights: network kernels (the paper has no learned part;
 * the network replaces the WENO5-JS nonlinear weights of Sec. 3.2).  All
 * pointers are device pointers; work is enqueued on `stream` (NULL = legacy
 * default stream).  For a five-cell stencil v_{i-2..i+2} and the edge at i+1/2
 * the inputs are x_k = (v_{i+k} - v_i)/s, k = -2..2, s = max_k |v_{i+k} - v_i|
 * (+1e-30); the outputs are softmax weights omega of the three WENO5
 * candidates; the edge value is v_i + sum_r omega_r (p_r - v_i).  Matrix
 * products run on BF16 tensor cores with FP32 accumulation. ---- */

/* omega[batch][3] of inputs x[batch][5] with parameters params[MFC_MLP_PARAMS]. */
mfc_status mfc_mlp_forward(const float* params, const float* x, long long batch, float* omega, void* stream);

/* Thread blocks of mfc_mlp_grad and the size of its caller-owned workspace. */
#define MFC_MLP_GRAD_BLOCKS 608
#define MFC_MLP_WORK_FLOATS (608LL * 4 * 1348)

/* Loss and gradient of a batch:
 *   L = (1/B) sum_b [ (sum_r omega_br phat_br - target_b)^2
 *                     + lam * mask_b * sum_r (omega_br - d_r)^2 ],  d = (0.1, 0.6, 0.3),
 * with x[B][5], phat[B][3] the normalised candidate increments (p_r - v_i)/s,
 * target[B] the normalised target edge value and mask[B] (1 in smooth
 * regions).  Writes grad[MFC_MLP_PARAMS] and *loss (loss may be NULL); work is
 * a caller-owned buffer of MFC_MLP_WORK_FLOATS floats.  Deterministic. */
mfc_status mfc_mlp_grad(const float* params, const float* x, const float* phat, const float* target,
                        const float* mask, long long batch, float lam, float* grad, float* loss, float* work,
                        void* stream);

/* mfc_mlp_grad runs on the fifth-generation tensor cores (tcgen05: one CTA
 * per 128 samples, BF16 operands in shared memory, FP32 accumulators in tensor
 * memory, the weight gradients as one MMA chain over the batch); its waits on
 * the tensor core are bounded, and a wait that gives up sets a flag that
 * mfc_mlp_tc_status reports.  mfc_mlp_grad_mma computes the same loss and
 * gradient on warp-level mma.sync tiles of 16 samples (same arguments and
 * workspace); the two agree to BF16 rounding. */
mfc_status mfc_mlp_grad_mma(const float* params, const float* x, const float* phat, const float* target,
                            const float* mask, long long batch, float lam, float* grad, float* loss, float* work,
                            void* stream);

/* omega[batch][3] as mfc_mlp_forward computes it, on the tcgen05 tensor cores
 * (M = 128 samples per MMA, FP32 accumulators in tensor memory). */
mfc_status mfc_mlp_forward_tc(const float* params, const float* x, long long batch, float* omega, void* stream);

/* Synchronises the device and reports whether a bounded tensor-core wait of
 * mfc_mlp_grad or mfc_mlp_forward_tc gave up since the last call (1; the
 * flag is then cleared), 0 if none did, -1 on a CUDA error.  The kernels that
 * gave up leave their outputs incomplete. */
int mfc_mlp_tc_status(void);

/* One Adam step (bias-corrected, step >= 1) on params[n] with moments m[n], v[n]. */
mfc_status mfc_mlp_adam(float* params, const float* grad, float* m, float* v, int n, float lr, float beta1,
                        float beta2, float eps, int step, void* stream);

/* Training samples from a fine primitive field w_fine (float64, layout above,
 * nxf x nyf x nzf cells, every active size even and >= 16).  Sample k (a
 * counter-based hash of seed and k) picks an active direction, a face of the
 * 2x-restricted grid, a variable and a side, and writes: x[k][5] normalised
 * coarse stencil, phat[k][3] normalised candidate increments, target[k] the
 * normalised fine-grid face value (mean of the fine WENO5-JS left and right
 * values at the coincident fine faces), smooth[k] = 1 unless the
 * discontinuity sensor trips (max_r b_r > tau (min_r b_r + 1e-6 s^2) on the
 * smoothness indicators without their 4/3 factor), js[k] the normalised
 * coarse WENO5-JS value.  Samples whose stencil is flat to FP32 resolution of
 * its centre value (s <= 1e-7 |v_i|), or whose normalised target exceeds 8 in
 * magnitude, are written as zeros with smooth[k] = 0. */
mfc_status mfc_harvest(const double* w_fine, int nxf, int nyf, int nzf, int num_fluids, double weno_eps, double tau,
                       long long n_samples, unsigned long long seed, float* x, float* phat, float* target,
                       float* smooth, float* js, void* stream);

/* Number of conserved variables, 2N + d. */
int mfc_sys_size(const mfc_ctx* ctx);

/* Kernel launches issued by this context so far. */
long long mfc_launch_count(const mfc_ctx* ctx);

/* Number of faces that used the first-order fallback since the context was
 * created (synchronises the stream). */
long long mfc_fallback_count(mfc_ctx* ctx);

/* Learned form: number of edge values the network evaluated since the context
 * was created (the rest kept their WENO5-JS weights: sensor trip or flat
 * stencil).  0 for the other forms; -1 on error.  Synchronises the stream. */
long long mfc_network_rows(mfc_ctx* ctx);

/* Per-kernel timing collected while "profile" is on: for category i in
 * [0, n) (0 prims, 1 sweep_x, 2 sweep_y, 3 sweep_z, 4 prims+cfl, 5 convert,
 * 6 mlp, 7 characteristic-boundary rates), total milliseconds and launch
 * counts.  Synchronises the stream.
 * Returns the number of categories (8). */
int mfc_profile_read(mfc_ctx* ctx, double* total_ms, long long* launches, int n);

/* Largest grid (in cells) that mfc_rhs_noalloc accepts. */
#define MFC_NOALLOC_MAX_CELLS 262144LL

/* Allocation-free right-hand side.  The paper has no counterpart: this entry
 * point exists for callers that cannot let a library call cudaMalloc, such as
 * host applications or frameworks that hand out all device memory from their
 * own pool or fixed budget, and time-critical loops that cannot absorb the
 * device synchronisation an allocation may take.  It computes the same R(q) as
 * mfc_rhs for a stateless problem description and allocates nothing: no
 * cudaMalloc, cudaFree or allocating library routine.
 *   q          device pointer, conserved state (layout above), caller-owned;
 *   rhs        device pointer, output R(q) (layout above), caller-owned;
 *   nx..pi_inf as in mfc_init; nx*ny*nz must not exceed MFC_NOALLOC_MAX_CELLS;
 *   weno_eps   WENO epsilon in [1e-30, 1]; fallback 0/1 as in mfc_set_param;
 *   cuda_stream the stream to enqueue on (NULL = legacy default stream);
 *   err, err_len optional caller buffer for an error message (may be NULL).
 * FP64 arithmetic.  Enqueued on the stream; returns without waiting.
 * The only scratch (the primitive variables, at most MFC_NOALLOC_MAX_CELLS x 9
 * doubles = 18.9 MB) is a static device array of the library, held by every GPU
 * that loads the library until the process exits.  The first call on a device,
 * with that device current, looks up the array's device address once; make that
 * first call before any stream capture.  The address is cached for the life of
 * the process, so do not use this entry point across a cudaDeviceReset (which
 * reloads the library's device code elsewhere).  All calls share the array:
 * calls that overlap on the GPU race on it and must be serialised by the caller.
 * Errors: MFC_ERR_ARG (bad arguments, or a grid larger than
 * MFC_NOALLOC_MAX_CELLS, with the reason in err), MFC_ERR_CUDA. */
mfc_status mfc_rhs_noalloc(const double* q, double* rhs, int nx, int ny, int nz, const double lo[3],
                           const double hi[3], const int bc[6], int num_fluids, const double* gamma,
                           const double* pi_inf, double weno_eps, int fallback, void* cuda_stream,
                           char* err, int err_len);

/* Text of the last error on this context ("" if none). */
const char* mfc_last_error(const mfc_ctx* ctx);

/* Release the context and its device memory. NULL is ignored. */
void mfc_finalize(mfc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MFC_GB300_H */
