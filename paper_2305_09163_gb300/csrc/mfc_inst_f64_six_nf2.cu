// Instantiates the six-equation-model sweeps and primitive recovery for double
// arithmetic and 2 fluids.
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<double, 2, false, 5, false, true>(SweepArgs, int, int, cudaStream_t);
template cudaError_t launch_prims<double, 2, true>(const PrimArgs&, int, bool, cudaStream_t);
template cudaError_t launch_cons6<2>(const Geometry&, const EosConst&, const double*, double*, int, cudaStream_t);
}  // namespace mfc
