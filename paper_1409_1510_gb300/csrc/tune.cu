// Launch-shape autotuner for the Dslash: for a given precision, Naik reconstruction
// and bundle size it times every candidate (right-hand sides per thread R dividing n, threads
// per block) with CUDA events on scratch bundles and caches the fastest in the context.
#include <string.h>
#include <algorithm>

#include "hisq_internal.cuh"

namespace hisq {

// Median launch time of one shape; each timed launch follows an L2 flush (a write larger than
// L2) so the links come from HBM, as they do inside a solve, and the parity alternates.
static int time_shape(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int copy, int n,
                      const LaunchShape &sh, void *in, void *out, void *flush, size_t flush_bytes, float *ms_out) {
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.in = in;
    d.out = out;
    d.n = n;
    d.parity = 0;
    d.epi = EPI_PLAIN;
    cudaEvent_t e0[5], e1[5];
    for (int i = 0; i < 5; i++) {
        cudaEventCreate(&e0[i]);
        cudaEventCreate(&e1[i]);
    }
    int rc = launch_dslash(ctx, fat, naik, copy, d, &sh, ctx->stream);  // warm-up
    for (int i = 0; i < 5 && rc == HISQ_OK; i++) {
        if (flush) cudaMemsetAsync(flush, i, flush_bytes, ctx->stream);
        d.parity = i & 1;
        cudaEventRecord(e0[i], ctx->stream);
        rc = launch_dslash(ctx, fat, naik, copy, d, &sh, ctx->stream);
        cudaEventRecord(e1[i], ctx->stream);
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess && rc == HISQ_OK) rc = set_error(HISQ_ERR_CUDA, "tuning timing failed: %s", cudaGetErrorString(e));
    if (rc == HISQ_OK) {
        float t[5];
        for (int i = 0; i < 5; i++) cudaEventElapsedTime(&t[i], e0[i], e1[i]);
        std::sort(t, t + 5);
        *ms_out = t[2];
    }
    for (int i = 0; i < 5; i++) {
        cudaEventDestroy(e0[i]);
        cudaEventDestroy(e1[i]);
    }
    return rc;
}

static int run_tuner(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int n, int copy, LaunchShape *best,
                     float *best_ms_out) {
    int prec = copy_prec(fat, copy);
    size_t bytes = vector_bytes(prec, ctx->geom.Vh, n);
    void *in = nullptr, *out = nullptr;
    if (cudaMalloc(&in, bytes) != cudaSuccess || cudaMalloc(&out, bytes) != cudaSuccess) {
        if (in) cudaFree(in);
        return set_error(HISQ_ERR_NOMEM, "tuner scratch allocation failed");
    }
    cudaMemsetAsync(in, 0, bytes, ctx->stream);
    const size_t flush_bytes = (size_t)256 << 20;  // larger than the 129 MB L2
    void *flush = nullptr;
    if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        cudaGetLastError();
        flush = nullptr;
    }
    *best = default_shape(prec, n);
    float best_ms = 1e30f;
    const int Rs[] = {1, 2, 4, 8};
    const int Ts[] = {256, 128, 64, 32};
    int rc = HISQ_OK;
    const int recon = copy != LINKS_INNER ? 18 : naik->recon;
    for (int R : Rs) {
        if (n % R != 0) continue;
        if (prec == HISQ_FP64 && R > 4) continue;
        if (prec == HISQ_DS && R > 2) continue;  // double-single: one or two RHS per thread, no lane split
        // the staged variant (S = 8) is not a candidate: it was slower than the plain kernel at every
        // size measured (it stays available through hisq_set_launch_shape)
        for (int S = 1; S <= 4; S *= 2) {
        if (S > 1 && prec == HISQ_DS) continue;
        if (S > 1 && (recon != 18 || R > 8 / S)) continue;
        for (int T : Ts) {
            LaunchShape sh{R, T, S};
            float ms = 0;
            rc = time_shape(ctx, fat, naik, copy, n, sh, in, out, flush, flush_bytes, &ms);
            if (rc != HISQ_OK) break;
            // a candidate replaces the incumbent only if it is clearly faster (2%): the
            // candidates are ordered from the simplest shape, and noise must not pick a shape
            if (ms < 0.98f * best_ms) {
                best_ms = ms;
                *best = sh;
            }
        }
        if (rc != HISQ_OK) break;
        }
        if (rc != HISQ_OK) break;
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(in);
    cudaFree(out);
    if (flush) cudaFree(flush);
    if (best_ms_out) *best_ms_out = best_ms;
    return rc;
}

LaunchShape tuned_shape(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int n, int copy) {
    int prec = copy_prec(fat, copy);
    int recon = copy != LINKS_INNER ? 18 : naik->recon;
    TuneKey key{prec, recon, n, 0};
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) return it->second;
    if (!ctx->params.autotune) return default_shape(prec, n);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cs);
    if (cs != cudaStreamCaptureStatusNone) return default_shape(prec, n);
    LaunchShape best;
    float ms = 0.0f;
    if (run_tuner(ctx, fat, naik, n, copy, &best, &ms) != HISQ_OK) {
        best = default_shape(prec, n);
        ms = 0.0f;
    }
    ctx->tuned[key] = best;
    if (ms > 0.0f && ms < 1e29f) ctx->tuned_ms[key] = ms;
    ctx->tune_generation++;
    return best;
}

// Bundle size for nrhs right-hand sides: the candidate (1, 2, 4, 8, 12, 16 below
// min(nrhs, 16), and min(nrhs, 16) itself) that
// minimises the summed tuned Dslash time of the bundles it splits nrhs into (full bundles plus
// one for the remainder).  Every solver kernel streams the links once per bundle step and the
// vectors once per right-hand side, as the Dslash does, so its time is the model.  Falls back to
// the largest bundle when a time is unknown (tuning off or failed).
int choose_bundle(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int nrhs, int copy) {
    const int cap = std::min(nrhs, HISQ_MAX_BUNDLE);
    if (!ctx->params.autotune) return cap;
    const int prec = copy_prec(fat, copy);
    const int recon = copy != LINKS_INNER ? 18 : naik->recon;
    auto time_of = [&](int n, float *ms) {
        tuned_shape(ctx, fat, naik, n, copy);
        auto it = ctx->tuned_ms.find(TuneKey{prec, recon, n, 0});
        if (it == ctx->tuned_ms.end()) return false;
        *ms = it->second;
        return true;
    };
    int cands[8], nc = 0;
    for (int n : {1, 2, 4, 8, 12, 16})
        if (n < cap) cands[nc++] = n;
    cands[nc++] = cap;  // one bundle of everything (up to the maximum) is always a candidate
    int best = cap;
    double best_t = 1e300;
    for (int i = 0; i < nc; i++) {
        const int n = cands[i];
        float tn = 0.0f, tr = 0.0f;
        if (!time_of(n, &tn)) return cap;
        const int full = nrhs / n, rem = nrhs % n;
        if (rem && !time_of(rem, &tr)) return cap;
        const double t = (double)full * tn + (rem ? tr : 0.0);
        if (t < 0.98 * best_t) {  // a larger bundle must be clearly faster (timing noise)
            best_t = t;
            best = n;
        }
    }
    return best;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_autotune(const hisq_links *fat, const hisq_links *naik, int nrhs, int *rhs_per_thread,
                             int *block_threads, int *lanes_per_site) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!fat || !naik) return set_error(HISQ_ERR_ARG, "null links");
    if (fat->ctx != ctx || naik->ctx != ctx) return set_error(HISQ_ERR_STATE, "links of another context");
    if (nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_NRHS);
    TuneKey key{fat->prec, naik->recon, nrhs, 0};
    ctx->tuned.erase(key);
    LaunchShape best;
    float ms = 0.0f;
    HISQ_CHECK(run_tuner(ctx, fat, naik, nrhs, LINKS_INNER, &best, &ms));
    ctx->tuned[key] = best;
    if (ms > 0.0f && ms < 1e29f) ctx->tuned_ms[key] = ms;
    ctx->tune_generation++;
    if (rhs_per_thread) *rhs_per_thread = best.R;
    if (block_threads) *block_threads = best.threads;
    if (lanes_per_site) *lanes_per_site = best.S;
    return HISQ_OK;
}

extern "C" int hisq_set_launch_shape(int prec, int recon, int nrhs, int rhs_per_thread, int block_threads,
                                     int lanes_per_site) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (prec < HISQ_FP64 || prec > HISQ_BF16) return set_error(HISQ_ERR_ARG, "unknown precision %d", prec);
    if (recon != 18 && recon != 13 && recon != 9) return set_error(HISQ_ERR_ARG, "recon must be 18, 13 or 9");
    if (nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_NRHS);
    int R = rhs_per_thread;
    if ((R != 1 && R != 2 && R != 4 && R != 8) || nrhs % R != 0 || (prec == HISQ_FP64 && R > 4))
        return set_error(HISQ_ERR_ARG, "rhs_per_thread %d is not available for nrhs %d", R, nrhs);
    if (block_threads < 32 || block_threads > (lanes_per_site == 8 ? 512 : 256))
        return set_error(HISQ_ERR_ARG, "block_threads must be in 32..256 (32..512 staged)");
    if (lanes_per_site != 1 && !(lanes_per_site == 2 && recon == 18 && R <= 4) &&
        !(lanes_per_site == 4 && recon == 18 && R <= 2) &&
        !(lanes_per_site == 8 && recon == 18 && R <= 2 && prec != HISQ_FP64))
        return set_error(HISQ_ERR_ARG,
                         "lanes_per_site must be 1, 2 (18-real Naik links, rhs_per_thread <= 4), 4 (18-real Naik "
                         "links, rhs_per_thread <= 2) or 8 (as 4, with staged link records; not FP64)");
    if (lanes_per_site == 8) {
        const int t = nrhs / R, words = link_words(prec, 18) + link_words(prec, recon);
        if (block_threads % (4 * t) || block_threads % 32 || block_threads > 512 ||
            staged_smem(words, block_threads / (4 * t), block_threads, nrhs, true) > 227 * 1024)
            return set_error(HISQ_ERR_ARG, "staged shape: block_threads must be a multiple of 4 * nrhs / "
                                           "rhs_per_thread and of 32, at most 512, within shared memory");
    }
    ctx->tuned[TuneKey{prec, recon, nrhs, 0}] = LaunchShape{R, block_threads, lanes_per_site};
    ctx->tune_generation++;
    return HISQ_OK;
}
