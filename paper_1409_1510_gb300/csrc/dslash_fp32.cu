// Dslash instantiations for FP32 storage.
#include "dslash_launch.cuh"

namespace hisq {

template <>
cudaError_t launch_dslash_prec<HISQ_FP32>(const KArgs &a, int recon, int epi, int R, int S, int threads, size_t smem,
                                        int num_sms, cudaStream_t s, int *grid) {
    if (recon == 13) return launch_epi<HISQ_FP32, 13>(a, epi, R, S, threads, smem, num_sms, s, grid);
    if (recon == 9) return launch_epi<HISQ_FP32, 9>(a, epi, R, S, threads, smem, num_sms, s, grid);
    return launch_epi<HISQ_FP32, 18>(a, epi, R, S, threads, smem, num_sms, s, grid);
}

}  // namespace hisq
