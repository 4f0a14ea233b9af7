// Instantiates the six-equation-model sweeps and primitive recovery for float
// arithmetic and 2 fluids.
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<float, 2, false, 5, false, true>(SweepArgs, int, int, cudaStream_t);
template cudaError_t launch_prims<float, 2, true>(const PrimArgs&, int, bool, cudaStream_t);
}  // namespace mfc
