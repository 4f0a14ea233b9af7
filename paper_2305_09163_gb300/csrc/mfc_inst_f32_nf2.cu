// Instantiates the sweep and primitive-recovery kernels for float arithmetic
// and 2 fluid(s).
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<float, 2>(SweepArgs, int, int, cudaStream_t);
template cudaError_t launch_prims<float, 2>(const PrimArgs&, int, bool, cudaStream_t);
template cudaError_t launch_cbc<float, 2>(const SweepArgs&, int, long long, cudaStream_t);

}  // namespace mfc
