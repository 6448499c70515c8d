// Dispatch from run-time (Naik recon, right-hand sides per thread, epilogue) to the compiled
// Dslash instantiations of one storage precision.  Each precision lives in its own
// translation unit so the instantiations compile in parallel.
#pragma once
#include "dslash_kernel.cuh"

namespace hisq {

// grid = whole waves: num_sms x resident blocks per SM (capped by the number of site tiles)
template <typename K>
inline int wave_grid(K kernel, int threads, size_t smem, int num_sms, long tiles) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    long g = (long)per_sm * num_sms;
    if (g > tiles) g = tiles;
    return (int)(g < 1 ? 1 : g);
}

template <int P, int NR, int R, int EPI, int S>
inline cudaError_t launch_one(const KArgs &a, int threads, size_t smem, int num_sms, cudaStream_t stream, int *grid_out) {
    auto k = dslash_kernel<P, NR, R, EPI, S>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    long tiles = (a.s1 - a.s0 + a.spb - 1) / a.spb;
    int grid = wave_grid(k, threads, smem, num_sms, tiles);
    // one full wave, every block with the same number of tiles
    grid = (int)balanced_grid(tiles, grid);
    if (grid_out) *grid_out = grid;
    k<<<grid, threads, smem, stream>>>(a);
    return cudaGetLastError();
}

// The staged kernel (S = 8: four lanes per site, link records of a tile staged in shared memory
// by the bulk-copy engine); one launch shape = sites per tile a.spb, threads = 4 t a.spb.
template <int P, int R, int EPI>
inline cudaError_t launch_staged(const KArgs &a, int threads, size_t smem, int num_sms, cudaStream_t stream,
                                 int *grid_out) {
    auto k = dslash_staged_kernel<P, R, EPI>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    long tiles = (a.g.Vh + a.spb - 1) / a.spb;
    int grid = wave_grid(k, threads, smem, num_sms, tiles);
    if (grid_out) *grid_out = grid;
    k<<<grid, threads, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int P, int NR, int EPI>
inline cudaError_t launch_r(const KArgs &a, int R, int S, int threads, size_t smem, int num_sms, cudaStream_t s, int *grid) {
    if constexpr (NR == 18 && P != HISQ_FP64 && EPI != EPI_RESID) {
        if (S == 8) {
            if (R == 1) return launch_staged<P, 1, EPI>(a, threads, smem, num_sms, s, grid);
            return launch_staged<P, 2, EPI>(a, threads, smem, num_sms, s, grid);
        }
    }
    if constexpr (NR == 18) {
        if (S == 4) {
            if (R == 1) return launch_one<P, NR, 1, EPI, 4>(a, threads, smem, num_sms, s, grid);
            return launch_one<P, NR, 2, EPI, 4>(a, threads, smem, num_sms, s, grid);
        }
        if (S == 2) {
            switch (R) {
            case 1: return launch_one<P, NR, 1, EPI, 2>(a, threads, smem, num_sms, s, grid);
            case 2: return launch_one<P, NR, 2, EPI, 2>(a, threads, smem, num_sms, s, grid);
            default: return launch_one<P, NR, 4, EPI, 2>(a, threads, smem, num_sms, s, grid);
            }
        }
    }
    switch (R) {
    case 1: return launch_one<P, NR, 1, EPI, 1>(a, threads, smem, num_sms, s, grid);
    case 2: return launch_one<P, NR, 2, EPI, 1>(a, threads, smem, num_sms, s, grid);
    case 4: return launch_one<P, NR, 4, EPI, 1>(a, threads, smem, num_sms, s, grid);
    default:
        // eight right-hand sides per thread would spill in FP64; FP64 shapes stop at four
        if constexpr (P == HISQ_FP64) return launch_one<P, NR, 4, EPI, 1>(a, threads, smem, num_sms, s, grid);
        else return launch_one<P, NR, 8, EPI, 1>(a, threads, smem, num_sms, s, grid);
    }
}

template <int P, int NR>
inline cudaError_t launch_epi(const KArgs &a, int epi, int R, int S, int threads, size_t smem, int num_sms, cudaStream_t s,
                              int *grid) {
    if (epi == EPI_PLAIN) return launch_r<P, NR, EPI_PLAIN>(a, R, S, threads, smem, num_sms, s, grid);
    if constexpr (P == HISQ_FP64 && NR == 18) {
        if (epi == EPI_RESID) return launch_r<P, NR, EPI_RESID>(a, R, S, threads, smem, num_sms, s, grid);
    }
    return launch_r<P, NR, EPI_AOP>(a, R, S, threads, smem, num_sms, s, grid);
}

// The per-precision entry (defined in dslash_<prec>.cu).
template <int P>
cudaError_t launch_dslash_prec(const KArgs &a, int recon, int epi, int R, int S, int threads, size_t smem,
                               int num_sms, cudaStream_t s, int *grid);
// The double-single entry (dslash_ds.cu): EPI_PLAIN or EPI_RESID, one or two RHS per thread.
cudaError_t launch_dslash_ds(const KArgs &a, int epi, int R, int threads, size_t smem, int num_sms, cudaStream_t s,
                             int *grid);

}  // namespace hisq
