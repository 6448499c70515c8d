// hisq_aop_noalloc: the A-operator with its fused dot, for callers that cannot allocate device
// memory.  All of its scratch lives in one file-scope static device array; nothing is allocated.
#include <string.h>
#include <mutex>
#include <algorithm>

#include "hisq_internal.cuh"

namespace hisq {

// Layout of the static scratch: [counter | dots | reduction partials | odd-parity intermediate]
constexpr size_t NOALLOC_COUNTER_OFF = 0;
constexpr size_t NOALLOC_DOTS_OFF = 256;
constexpr size_t NOALLOC_PARTIALS_OFF = 1024;
constexpr size_t NOALLOC_PARTIALS_DOUBLES = 128 * 1024;  // 1 MiB
constexpr size_t NOALLOC_TMP_OFF = NOALLOC_PARTIALS_OFF + NOALLOC_PARTIALS_DOUBLES * sizeof(double);
constexpr size_t NOALLOC_TMP_BYTES = HISQ_AOP_NOALLOC_SCRATCH_BYTES - NOALLOC_TMP_OFF;

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_aop_scratch[HISQ_AOP_NOALLOC_SCRATCH_BYTES];

// Device address of g_aop_scratch per device ordinal, looked up once with that device current.
// In host code the array's name is only a host-side stand-in, never a device address.
static std::mutex g_scratch_mutex;
static void *g_scratch_addr[128];

static int scratch_address(int device, unsigned char **out) {
    if (device < 0 || device >= 128) return set_error(HISQ_ERR_ARG, "device ordinal %d out of range", device);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_aop_scratch);
        if (e != cudaSuccess || !p)
            return set_error(HISQ_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        g_scratch_addr[device] = p;
    }
    *out = reinterpret_cast<unsigned char *>(g_scratch_addr[device]);
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_aop_noalloc(const hisq_links *fat, const hisq_links *naik, double mass, const void *in, void *out,
                                int nrhs, double *pAp) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    HISQ_CHECK(check_pair(ctx, fat, naik));
    if (!in || !out) return set_error(HISQ_ERR_ARG, "null vector");
    if (in == out) return set_error(HISQ_ERR_ARG, "in and out must not overlap");
    if (nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_NRHS);

    // the launch shape is fixed (no autotuning: the tuner allocates its timing buffers)
    const LaunchShape shape = default_shape(fat->prec, nrhs);
    const size_t tmp_bytes = vector_bytes(fat->prec, ctx->geom.Vh, nrhs);
    if (tmp_bytes > NOALLOC_TMP_BYTES)
        return set_error(HISQ_ERR_ARG,
                         "hisq_aop_noalloc: the odd-parity intermediate needs %zu bytes, more than the %zu bytes of "
                         "static scratch (HISQ_AOP_NOALLOC_SCRATCH_BYTES); use hisq_aop",
                         tmp_bytes, NOALLOC_TMP_BYTES);
    // the partials the reducing launch will write, sized by the helper launch_dslash itself uses,
    // so a request is rejected before anything is launched
    int spb = 0, threads = 0;
    dslash_block_shape(nrhs, shape.R, shape.S, shape.threads, true, &spb, &threads);
    const size_t partials = dslash_partials_needed(ctx->geom.Vh, ctx->num_sms, spb, nrhs);
    if (partials > NOALLOC_PARTIALS_DOUBLES)
        return set_error(HISQ_ERR_ARG,
                         "hisq_aop_noalloc: %zu reduction partials exceed the %zu of the static scratch; use hisq_aop",
                         partials, NOALLOC_PARTIALS_DOUBLES);

    unsigned char *base = nullptr;
    HISQ_CHECK(scratch_address(ctx->device, &base));
    unsigned int *counter = reinterpret_cast<unsigned int *>(base + NOALLOC_COUNTER_OFF);
    double *dots = reinterpret_cast<double *>(base + NOALLOC_DOTS_OFF);
    double *part = reinterpret_cast<double *>(base + NOALLOC_PARTIALS_OFF);
    void *tmp = base + NOALLOC_TMP_OFF;

    // the last-block ticket must start at zero; the array keeps whatever the previous call left
    HISQ_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned int) * 4, ctx->stream));

    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.in = in;
    d.out = tmp;
    d.n = nrhs;
    d.parity = 1;
    d.epi = EPI_PLAIN;
    HISQ_CHECK(launch_dslash(ctx, fat, naik, false, d, &shape, ctx->stream));
    d.in = tmp;
    d.out = out;
    d.parity = 0;
    d.epi = EPI_AOP;
    d.mass2 = mass * mass;
    d.axpy_in = in;
    d.partials = part;
    d.partials_cap = NOALLOC_PARTIALS_DOUBLES;
    d.counter = counter;
    d.dot_out = dots;
    HISQ_CHECK(launch_dslash(ctx, fat, naik, false, d, &shape, ctx->stream));
    if (pAp) {
        HISQ_CUDA(cudaMemcpyAsync(pAp, dots, sizeof(double) * nrhs, cudaMemcpyDefault, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return HISQ_OK;
}
