// Instantiates the sweep and primitive-recovery kernels for float arithmetic
// and 3 fluid(s).
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<float, 3>(SweepArgs, int, int, cudaStream_t);
template cudaError_t launch_prims<float, 3>(const PrimArgs&, int, bool, cudaStream_t);
template cudaError_t launch_cbc<float, 3>(const SweepArgs&, int, long long, cudaStream_t);

}  // namespace mfc
