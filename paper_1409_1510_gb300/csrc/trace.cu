// Stochastic trace estimation (Eq. (2) without derivative factors): Tr A^{-1} over the even sites
// as the mean of eta^dag A^{-1} eta over Z2 noise vectors eta.  The noise comes from splitmix64
// (Steele, Lea & Flood 2014), evaluated at a counter per (vector, colour component), so any range
// of vectors can be generated on the device in any order; the solves are the bundled
// mixed-precision CG; the products are FP64 block reductions, one block per noise vector.
#include <string.h>
#include <math.h>
#include <chrono>
#include <algorithm>
#include <vector>

#include "hisq_internal.cuh"

namespace hisq {

// output i (i = 0, 1, ...) of splitmix64 started from `seed`: the state after i + 1 steps of the
// Weyl increment gamma, through the generator's mixing function
__device__ __forceinline__ unsigned long long splitmix64_output(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// vectors first .. first + n - 1, canonical [n][per] complex numbers (per = 3 V/2): element e of
// vector k is -1 when the top bit of output per k + e is set, else +1
__global__ void __launch_bounds__(256) z2_noise_kernel(double2 *out, long per, int n, unsigned long long seed,
                                                       unsigned long long first) {
    const long total = per * n;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long k = i / per, e = i - k * per;
        const unsigned long long z = splitmix64_output(seed, (first + (unsigned long long)k) * (unsigned long long)per + e);
        out[i] = make_double2((z >> 63) ? -1.0 : 1.0, 0.0);
    }
}

// samples[k] = Re <eta_k, x_k> = sum_e Re(conj(eta_e) x_e), one block per vector, FP64 tree sums
__global__ void __launch_bounds__(256) noise_dot_kernel(const double2 *eta, const double2 *x, long per, double *samples) {
    __shared__ double red[256];
    const int k = blockIdx.x, tid = threadIdx.x;
    const double2 *e = eta + (size_t)k * per, *v = x + (size_t)k * per;
    double s = 0.0;
    for (long i = tid; i < per; i += blockDim.x) {
        const double2 a = e[i], b = v[i];
        s = fma(a.x, b.x, fma(a.y, b.y, s));
    }
    red[tid] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    if (tid == 0) samples[k] = red[0];
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_z2_noise(double *out, int n, unsigned long long seed, unsigned long long first) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!out) return set_error(HISQ_ERR_ARG, "null output");
    if (n < 1) return set_error(HISQ_ERR_ARG, "n must be >= 1");
    if (!is_device_ptr(out)) return set_error(HISQ_ERR_ARG, "the noise buffer must be device memory");
    const long per = 3L * ctx->geom.Vh;
    const long blocks = std::min<long>((per * n + 255) / 256, (long)ctx->num_sms * 8);
    z2_noise_kernel<<<(int)blocks, 256, 0, ctx->stream>>>(reinterpret_cast<double2 *>(out), per, n, seed, first);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

extern "C" int hisq_trace_inverse(const hisq_links *fat, const hisq_links *naik, double mass, int nnoise,
                                  unsigned long long seed, double tol, double *estimate, double *std_error,
                                  double *samples) {
    auto t0 = std::chrono::steady_clock::now();
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!fat || !naik || !estimate) return set_error(HISQ_ERR_ARG, "null argument");
    if (nnoise < 1) return set_error(HISQ_ERR_ARG, "nnoise must be >= 1");
    if (!(tol > 0.0)) return set_error(HISQ_ERR_ARG, "tol must be positive");
    const long per = 3L * ctx->geom.Vh;
    const int chunk = std::min(nnoise, 64);  // noise vectors generated and solved per round
    double2 *eta = nullptr, *x = nullptr;
    double *d_samples = nullptr;
    const size_t bytes = (size_t)chunk * per * sizeof(double2);
    if (cudaMalloc(&eta, bytes) != cudaSuccess || cudaMalloc(&x, bytes) != cudaSuccess ||
        cudaMalloc(&d_samples, sizeof(double) * nnoise) != cudaSuccess) {
        if (eta) cudaFree(eta);
        if (x) cudaFree(x);
        cudaGetLastError();
        return set_error(HISQ_ERR_NOMEM, "cannot allocate %zu bytes for the trace estimate", 2 * bytes);
    }
    std::vector<int> iters(nnoise, 0);
    std::vector<double> resid(nnoise, 1.0);
    hisq_solve_stats total;
    memset(&total, 0, sizeof(total));
    int rc = HISQ_OK;
    std::vector<const double *> rp(chunk);
    std::vector<double *> xp(chunk);
    for (int k0 = 0; k0 < nnoise && rc == HISQ_OK; k0 += chunk) {
        const int c = std::min(chunk, nnoise - k0);
        rc = hisq_z2_noise(reinterpret_cast<double *>(eta), c, seed, (unsigned long long)k0);
        if (rc != HISQ_OK) break;
        for (int q = 0; q < c; q++) {
            rp[q] = reinterpret_cast<const double *>(eta + (size_t)q * per);
            xp[q] = reinterpret_cast<double *>(x + (size_t)q * per);
        }
        const int src = cg_solve_common(ctx, fat, naik, rp.data(), xp.data(), c, mass, tol, nullptr, nullptr);
        if (src != HISQ_OK && src != HISQ_ERR_NOT_CONVERGED) {
            rc = src;
            break;
        }
        const hisq_solve_stats &s = ctx->stats;
        total.converged += s.converged;
        total.bundles += s.bundles;
        total.bundle_size = s.bundle_size;
        total.max_iterations = std::max(total.max_iterations, s.max_iterations);
        total.total_iterations += s.total_iterations;
        total.bundle_iterations += s.bundle_iterations;
        total.reliable_updates += s.reliable_updates;
        total.flops += s.flops;
        total.kernel_launches += s.kernel_launches + 2;
        total.solve_kernel_ms += s.solve_kernel_ms;
        total.solve_kernel_launches += s.solve_kernel_launches;
        for (int q = 0; q < c; q++) {
            iters[k0 + q] = ctx->stat_iters[q];
            resid[k0 + q] = ctx->stat_resid[q];
        }
        noise_dot_kernel<<<c, 256, 0, ctx->stream>>>(eta, x, per, d_samples + k0);
        if (cudaGetLastError() != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "noise product launch failed");
    }
    std::vector<double> h(nnoise, 0.0);
    if (rc == HISQ_OK) {
        if (cudaMemcpyAsync(h.data(), d_samples, sizeof(double) * nnoise, cudaMemcpyDeviceToHost, ctx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            rc = set_error(HISQ_ERR_CUDA, "reading the noise products failed");
    }
    cudaFree(eta);
    cudaFree(x);
    cudaFree(d_samples);
    if (rc != HISQ_OK) return rc;
    double mean = 0.0;
    for (int k = 0; k < nnoise; k++) mean += h[k];
    mean /= nnoise;
    double var = 0.0;
    for (int k = 0; k < nnoise; k++) var += (h[k] - mean) * (h[k] - mean);
    *estimate = mean;
    if (std_error) *std_error = nnoise > 1 ? sqrt(var / (nnoise - 1) / nnoise) : 0.0;
    if (samples)
        for (int k = 0; k < nnoise; k++) samples[k] = h[k];
    total.nrhs = nnoise;
    total.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    ctx->stats = total;
    ctx->stat_iters = iters;
    ctx->stat_resid = resid;
    if (total.converged < nnoise)
        return set_error(HISQ_ERR_NOT_CONVERGED, "%d of %d noise solves missed tol %.1e", nnoise - total.converged, nnoise,
                         tol);
    return HISQ_OK;
}
