// Instantiates the six-equation-model sweeps and primitive recovery for double
// arithmetic and 3 fluids.
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<double, 3, false, 5, false, true>(SweepArgs, int, int, cudaStream_t);
template cudaError_t launch_prims<double, 3, true>(const PrimArgs&, int, bool, cudaStream_t);
template cudaError_t launch_cons6<3>(const Geometry&, const EosConst&, const double*, double*, int, cudaStream_t);
}  // namespace mfc
