// Instantiates the sweep and primitive-recovery kernels for double arithmetic
// and 1 fluid(s).
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<double, 1>(SweepArgs, int, int, cudaStream_t);
template cudaError_t launch_prims<double, 1>(const PrimArgs&, int, bool, cudaStream_t);
template cudaError_t launch_cbc<double, 1>(const SweepArgs&, int, long long, cudaStream_t);
template cudaError_t launch_cons<1>(const Geometry&, const EosConst&, const double*, double*, int, cudaStream_t);
}  // namespace mfc
