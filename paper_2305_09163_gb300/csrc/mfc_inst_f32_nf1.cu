// Instantiates the sweep and primitive-recovery kernels for float arithmetic
// and 1 fluid(s).
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<float, 1>(SweepArgs, int, int, cudaStream_t);
template cudaError_t launch_prims<float, 1>(const PrimArgs&, int, bool, cudaStream_t);
template cudaError_t launch_cbc<float, 1>(const SweepArgs&, int, long long, cudaStream_t);

}  // namespace mfc
