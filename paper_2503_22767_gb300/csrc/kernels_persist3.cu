// 3D instantiation of the persistent passes (kernels_persist.cuh), a
// translation unit of its own so that it compiles beside the others.
#include "kernels_persist.cuh"

namespace mpm {
template cudaError_t launch_persist_dim<3>(PersistKind, bool, const Params&, const PersistArgs&, int, int,
                                            cudaStream_t);
}  // namespace mpm
