// Persistent solve kernels for FP32 inner precision.
#include "cg_persistent_body.cuh"

namespace hisq {
template cudaError_t launch_persistent_prec<HISQ_FP32>(const PersArgs &, int, bool, int, int, size_t, cudaStream_t);
template cudaError_t persistent_occupancy<HISQ_FP32>(int, bool, int, size_t, int *);
}  // namespace hisq
