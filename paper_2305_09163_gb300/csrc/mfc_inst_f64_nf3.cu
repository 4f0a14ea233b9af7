// Instantiates the sweep and primitive-recovery kernels for double arithmetic
// and 3 fluid(s).
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<double, 3>(SweepArgs, int, int, cudaStream_t);
template cudaError_t launch_prims<double, 3>(const PrimArgs&, int, bool, cudaStream_t);
template cudaError_t launch_cbc<double, 3>(const SweepArgs&, int, long long, cudaStream_t);
template cudaError_t launch_cons<3>(const Geometry&, const EosConst&, const double*, double*, int, cudaStream_t);
}  // namespace mfc
