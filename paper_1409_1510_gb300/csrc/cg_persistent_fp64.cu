// Persistent solve kernels for FP64 inner precision.
#include "cg_persistent_body.cuh"

namespace hisq {
template cudaError_t launch_persistent_prec<HISQ_FP64>(const PersArgs &, int, bool, int, int, size_t, cudaStream_t);
template cudaError_t persistent_occupancy<HISQ_FP64>(int, bool, int, size_t, int *);
}  // namespace hisq
