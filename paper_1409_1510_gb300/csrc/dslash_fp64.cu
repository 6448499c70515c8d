// Dslash instantiations for FP64 storage.
#include "dslash_launch.cuh"

namespace hisq {

template <>
cudaError_t launch_dslash_prec<HISQ_FP64>(const KArgs &a, int recon, int epi, int R, int S, int threads, size_t smem,
                                        int num_sms, cudaStream_t s, int *grid) {
    (void)recon;
    return launch_epi<HISQ_FP64, 18>(a, epi, R, S, threads, smem, num_sms, s, grid);
}

}  // namespace hisq
