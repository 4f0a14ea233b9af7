// Device code for the diffuse-interface right-hand side and time step on GB300
// (sm_103a).  Templates over the arithmetic type Real (double for the FP64
// path, float for the mixed and learned forms), the number of fluids NF, the
// number of dimensions NDIM, the sweep direction DIR, the reconstruction order,
// non-uniform grids and the six-equation model.
//
// Method (arXiv 2305.09163):
//   Sec. 2.1      stiffened-gas EOS; the Allaire model (default) and the Kapila
//                 K div(u) source
//   Sec. 2.3      six-equation model with infinite pressure relaxation
//   Sec. 3.1      semi-discrete operator, Eq. "fvmdis", with face velocities for div u
//   Sec. 3.2      WENO5-JS / WENO3-JS reconstruction of primitive variables
//   Sec. 3.2.1    HLLC approximate Riemann solver
//   Sec. 3.3      ghost cells three deep (periodic, transmissive, reflective),
//                 characteristic (non-reflecting) boundaries, non-uniform grids
//   Sec. 3.4      SSP (TVD) Runge-Kutta update (orders 3, 2, 1)
//
// GB300 design: the FP64 pipe issues about 2 DFMA per SM clock, ~1/58 of FP32,
// and FP64 compares and FP64<->FP32 conversions run on it too.  The FP64 path
// therefore evaluates its WENO weights and its HLLC solver in float-float
// arithmetic on the FP32 pipes (mfc_df.cuh; ~48 bits, far inside the 1e-11
// parity requirement), converts by integer operations on bit patterns, tests
// positivity on bit patterns, and computes every face flux once.  Flux
// difference, sources and the RK stage update are applied in the same pass.  No
// atomics touch the state, so results are bitwise reproducible.
//
// The code is split by concern; each header includes the one before it:
//   mfc_common.cuh   types, kernel arguments, layout, ghost cells
//   mfc_weno.cuh     WENO5 / WENO3 reconstruction, non-uniform grids
//   mfc_riemann.cuh  EOS mixtures, HLLC, face fluxes
//   mfc_learned.cuh  learned WENO weights (tensor-core network)
//   mfc_cell.cuh     boundary rates, Kapila, six-equation relaxation, finish_cell
//   mfc_sweeps.cuh   the sweep kernels
//   mfc_prims.cuh    primitive recovery, CFL rate, conversions
#pragma once
#include "mfc_prims.cuh"
