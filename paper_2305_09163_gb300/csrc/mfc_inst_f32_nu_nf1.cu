// Instantiates the non-uniform-grid sweeps for float arithmetic and 1 fluid(s).
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<float, 1, false, 5, true>(SweepArgs, int, int, cudaStream_t);
}  // namespace mfc
