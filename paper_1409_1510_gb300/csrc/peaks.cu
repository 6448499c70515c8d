// Arithmetic peaks of the device, measured: chains of independent fused multiply-adds on every
// SM, timed with CUDA events (the denominators of the FP32- and FP64-bound rooflines).
#include <string.h>

#include "hisq_internal.cuh"

namespace hisq {

// 8 independent accumulators per thread, `iters` rounds of 8 FMAs each; the result is written
// only if it is impossible (so the work cannot be removed).
template <typename T>
__global__ void fma_chain_kernel(int iters, T a, T b, T *sink) {
    T x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = fma(x[j], a, b);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) s += x[j];
    if (s == (T)-12345.678) *sink = s;
}

template <typename T>
static int time_fma(hisq_ctx *ctx, int iters, double *tflops) {
    T *sink = nullptr;
    HISQ_CUDA(cudaMalloc(&sink, sizeof(T)));
    const int threads = 256, grid = ctx->num_sms * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_chain_kernel<T><<<grid, threads, 0, ctx->stream>>>(iters / 10, (T)0.999, (T)1e-4, sink);  // warm-up
    cudaEventRecord(e0, ctx->stream);
    fma_chain_kernel<T><<<grid, threads, 0, ctx->stream>>>(iters, (T)0.999, (T)1e-4, sink);
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return set_error(HISQ_ERR_CUDA, "FMA timing failed: %s", cudaGetErrorString(e));
    const double flops = 2.0 * 8.0 * iters * (double)threads * grid;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_measure_fma_peaks(double *fp32_tflops, double *fp64_tflops) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!fp32_tflops || !fp64_tflops) return set_error(HISQ_ERR_ARG, "null output");
    HISQ_CHECK(time_fma<float>(ctx, 1 << 16, fp32_tflops));
    HISQ_CHECK(time_fma<double>(ctx, 1 << 12, fp64_tflops));
    return HISQ_OK;
}
