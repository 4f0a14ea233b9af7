// Instantiates the six-equation-model sweeps on non-uniform grids for float arithmetic and 2 fluids.
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<float, 2, false, 5, true, true>(SweepArgs, int, int, cudaStream_t);
}  // namespace mfc
