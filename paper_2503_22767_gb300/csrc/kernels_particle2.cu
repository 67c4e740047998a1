// The particle kernels for two dimensions: forward and reverse.
#include "particle_kernels.cuh"

namespace mpm {
template cudaError_t launch_forward_dim<2>(bool, bool, bool, bool, const Params&, const StepArgs&, int,
                                           cudaStream_t);
template cudaError_t launch_adjoint_dim<2>(bool, bool, bool, bool, const Params&, const StepArgs&, int,
                                           cudaStream_t);
}  // namespace mpm
