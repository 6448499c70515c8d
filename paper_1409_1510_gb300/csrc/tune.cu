// Launch-shape autotuner for the Dslash (row a6): for a given precision, Naik reconstruction
// and bundle size it times every candidate (right-hand sides per thread R dividing n, threads
// per block) with CUDA events on scratch bundles and caches the fastest in the context.
#include <string.h>
#include <algorithm>

#include "hisq_internal.cuh"

namespace hisq {

static int time_shape(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, bool use64, int n,
                      const LaunchShape &sh, void *in, void *out, float *ms_out) {
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.in = in;
    d.out = out;
    d.n = n;
    d.parity = 0;
    d.epi = EPI_PLAIN;
    cudaEvent_t e0, e1;
    HISQ_CUDA(cudaEventCreate(&e0));
    HISQ_CUDA(cudaEventCreate(&e1));
    int rc = launch_dslash(ctx, fat, naik, use64, d, &sh, ctx->stream);  // warm-up
    const int reps = 5;
    if (rc == HISQ_OK) {
        cudaEventRecord(e0, ctx->stream);
        for (int i = 0; i < reps && rc == HISQ_OK; i++) rc = launch_dslash(ctx, fat, naik, use64, d, &sh, ctx->stream);
        cudaEventRecord(e1, ctx->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess && rc == HISQ_OK) rc = set_error(HISQ_ERR_CUDA, "tuning timing failed: %s", cudaGetErrorString(e));
        *ms_out = ms / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

static int run_tuner(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int n, bool use64, LaunchShape *best) {
    int prec = use64 ? HISQ_FP64 : fat->prec;
    size_t bytes = vector_bytes(prec, ctx->geom.Vh, n);
    void *in = nullptr, *out = nullptr;
    if (cudaMalloc(&in, bytes) != cudaSuccess || cudaMalloc(&out, bytes) != cudaSuccess) {
        if (in) cudaFree(in);
        return set_error(HISQ_ERR_NOMEM, "tuner scratch allocation failed");
    }
    cudaMemsetAsync(in, 0, bytes, ctx->stream);
    *best = default_shape(prec, n);
    float best_ms = 1e30f;
    const int Rs[] = {1, 2, 4, 8};
    const int Ts[] = {64, 128, 256};
    int rc = HISQ_OK;
    for (int R : Rs) {
        if (n % R != 0) continue;
        if (prec == HISQ_FP64 && R > 4) continue;
        for (int T : Ts) {
            LaunchShape sh{R, T};
            float ms = 0;
            rc = time_shape(ctx, fat, naik, use64, n, sh, in, out, &ms);
            if (rc != HISQ_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                *best = sh;
            }
        }
        if (rc != HISQ_OK) break;
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(in);
    cudaFree(out);
    return rc;
}

LaunchShape tuned_shape(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int n, bool use64) {
    int prec = use64 ? HISQ_FP64 : fat->prec;
    int recon = use64 ? 18 : naik->recon;
    TuneKey key{prec, recon, n, 0};
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) return it->second;
    if (!ctx->params.autotune) return default_shape(prec, n);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cs);
    if (cs != cudaStreamCaptureStatusNone) return default_shape(prec, n);
    LaunchShape best;
    if (run_tuner(ctx, fat, naik, n, use64, &best) != HISQ_OK) best = default_shape(prec, n);
    ctx->tuned[key] = best;
    return best;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_autotune(const hisq_links *fat, const hisq_links *naik, int nrhs, int *rhs_per_thread,
                             int *block_threads) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!fat || !naik) return set_error(HISQ_ERR_ARG, "null links");
    if (fat->ctx != ctx || naik->ctx != ctx) return set_error(HISQ_ERR_STATE, "links of another context");
    if (nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_NRHS);
    TuneKey key{fat->prec, naik->recon, nrhs, 0};
    ctx->tuned.erase(key);
    LaunchShape best;
    HISQ_CHECK(run_tuner(ctx, fat, naik, nrhs, false, &best));
    ctx->tuned[key] = best;
    if (rhs_per_thread) *rhs_per_thread = best.R;
    if (block_threads) *block_threads = best.threads;
    return HISQ_OK;
}

extern "C" int hisq_set_launch_shape(int prec, int recon, int nrhs, int rhs_per_thread, int block_threads) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (prec < HISQ_FP64 || prec > HISQ_BF16) return set_error(HISQ_ERR_ARG, "unknown precision %d", prec);
    if (recon != 18 && recon != 13 && recon != 9) return set_error(HISQ_ERR_ARG, "recon must be 18, 13 or 9");
    if (nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_NRHS);
    int R = rhs_per_thread;
    if ((R != 1 && R != 2 && R != 4 && R != 8) || nrhs % R != 0 || (prec == HISQ_FP64 && R > 4))
        return set_error(HISQ_ERR_ARG, "rhs_per_thread %d is not available for nrhs %d", R, nrhs);
    if (block_threads < 32 || block_threads > 256) return set_error(HISQ_ERR_ARG, "block_threads must be in 32..256");
    ctx->tuned[TuneKey{prec, recon, nrhs, 0}] = LaunchShape{R, block_threads};
    return HISQ_OK;
}
