// Instantiates the learned-form sweep kernels (FP32, tensor-core network) for
// 1 fluid(s).
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<float, 1, true>(SweepArgs, int, int, cudaStream_t);
}  // namespace mfc
