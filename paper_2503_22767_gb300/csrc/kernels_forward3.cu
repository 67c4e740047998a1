// The forward particle kernels for three dimensions.
#include "particle_kernels.cuh"

namespace mpm {
template cudaError_t launch_forward_dim<3>(bool, bool, bool, bool, const Params&, const StepArgs&, int,
                                           cudaStream_t);
}  // namespace mpm
