// Instantiates the non-uniform-grid sweeps for double arithmetic and 2 fluid(s).
#include "mfc_launch.cuh"
namespace mfc {
template cudaError_t launch_sweep<double, 2, false, 5, true>(SweepArgs, int, int, cudaStream_t);
}  // namespace mfc
