// Persistent solve kernels for FP16 inner precision.
#include "cg_persistent_body.cuh"

namespace hisq {
template cudaError_t launch_persistent_prec<HISQ_FP16>(const PersArgs &, int, bool, int, int, size_t, cudaStream_t);
template cudaError_t persistent_occupancy<HISQ_FP16>(int, bool, int, size_t, int *);
}  // namespace hisq
