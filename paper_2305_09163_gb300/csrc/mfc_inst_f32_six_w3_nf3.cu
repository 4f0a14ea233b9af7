// Instantiates the six-equation-model sweeps with WENO3 for float arithmetic and 3 fluids.
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<float, 3, false, 3, false, true>(SweepArgs, int, int, cudaStream_t);
}  // namespace mfc
