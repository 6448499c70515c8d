// The FP64-accurate Dslash of the residual recomputation in double-single arithmetic (see
// ds_arith.cuh), as separate kernels for the graph and host-driven solver drivers, the
// multi-shift refinement and hisq_residual: EPI_PLAIN (ds in -> ds out) and EPI_RESID
// (r = b - m^2 x + D t with t a ds bundle, x and b FP64; FP64 epilogue and |r|^2), plus the
// conversion of FP64 bundles into ds bundles.  The persistent solver runs the same stencil as
// phases of its launch (cg_persistent.cuh).
#include "ds_arith.cuh"
#include "dslash_kernel.cuh"
#include "dslash_launch.cuh"

namespace hisq {

// FP64 bundle (double2 per complex) -> ds bundle (float4 per complex), same element order
__global__ void ds_split_kernel(const double2 *in, float4 *out, long count) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        const double2 z = in[i];
        float a, b, c, d;
        ds_split(z.x, a, b);
        ds_split(z.y, c, d);
        out[i] = make_float4(a, b, c, d);
    }
}

template <int R, int EPI>
__global__ void __launch_bounds__(256) dslash_ds_kernel(KArgs a) {
    extern __shared__ double red[];
    if (a.gate && *a.gate == 0) return;
    const Geom &g = a.g;
    const int tid = threadIdx.x;
    const int gi = tid % a.t;
    const int sl = tid / a.t;
    const int r0 = gi * R;
    const int nvalid = min(R, a.n - r0);
    const float4 *in = reinterpret_cast<const float4 *>(a.in);
    bool act[R];
    bool any_act = false;
#pragma unroll
    for (int r = 0; r < R; r++) {
        act[r] = (r < nvalid) && (a.active == nullptr || a.active[r0 + r] != 0);
        any_act |= act[r];
    }
    double dot[R];
#pragma unroll
    for (int r = 0; r < R; r++) dot[r] = 0.0;

    const bool whole = a.s0 == 0 && a.s1 == g.Vh;  // a whole parity: visit in plane order
    for (int tile = blockIdx.x; (long)tile * a.spb < a.s1 - a.s0; tile += gridDim.x) {
        const int q = tile * a.spb + sl;
        if (!(sl < a.spb && q < a.s1 - a.s0 && any_act)) continue;
        const int s = whole ? visit_site(g, q) : a.s0 + q;
        dscplx acc[R][3];
        int rr[R];
#pragma unroll
        for (int r = 0; r < R; r++) rr[r] = r0 + r;
        ds_site_stencil<R, false, true>(g, a.fat, a.naik, a.parity, in, a.n, s, rr, act, acc);
        if constexpr (EPI == EPI_PLAIN) {
#pragma unroll
            for (int r = 0; r < R; r++)
                if (act[r]) ds_store3(reinterpret_cast<float4 *>(a.out), a.n, s, r0 + r, acc[r]);
        } else {
            static_assert(EPI == EPI_RESID, "ds kernels have the plain and residual epilogues");
            const double2 *vx = reinterpret_cast<const double2 *>(a.axpy);
            const double2 *vb = reinterpret_cast<const double2 *>(a.b);
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (!act[r]) continue;
                double d = 0.0;
                double2 w[3];
                const double m2 = a.mass2v ? a.mass2v[r0 + r] : a.mass2;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const long idx = ((long)s * 3 + c) * a.n + r0 + r;
                    const long bidx = a.b_one ? (long)s * 3 + c : idx;
                    const double2 x = __ldg(vx + idx), b = __ldg(vb + bidx);
                    w[c].x = b.x - m2 * x.x + ds_value(acc[r][c].re);
                    w[c].y = b.y - m2 * x.y + ds_value(acc[r][c].im);
                    d += w[c].x * w[c].x + w[c].y * w[c].y;
                }
                dot[r] += d;
                const long base = (long)s * 3 * a.n + r0 + r;
                if (a.out) {
                    double2 *o = reinterpret_cast<double2 *>(a.out);
#pragma unroll
                    for (int c = 0; c < 3; c++) o[base + (long)c * a.n] = w[c];
                }
                if (a.out_lo) {
                    if (a.lo_prec == HISQ_FP64) {
                        double2 *o = reinterpret_cast<double2 *>(a.out_lo);
#pragma unroll
                        for (int c = 0; c < 3; c++) o[base + (long)c * a.n] = w[c];
                    } else {
                        float2 *o = reinterpret_cast<float2 *>(a.out_lo);
#pragma unroll
                        for (int c = 0; c < 3; c++) o[base + (long)c * a.n] = make_float2((float)w[c].x, (float)w[c].y);
                    }
                }
            }
        }
    }
    if constexpr (EPI == EPI_RESID) {
        for (int i = tid; i < a.spb * a.n; i += blockDim.x) red[i] = 0.0;
        __syncthreads();
        if (sl < a.spb) {
#pragma unroll
            for (int r = 0; r < R; r++)
                if (r < nvalid) red[sl * a.n + r0 + r] = dot[r];
        }
        block_reduce_finish(red, a.spb, a.n, a.n, a.red);
    }
}

template <int R, int EPI>
static cudaError_t launch_ds_one(const KArgs &a, int threads, size_t smem, int num_sms, cudaStream_t stream,
                                 int *grid_out) {
    auto k = dslash_ds_kernel<R, EPI>;
    long tiles = (a.s1 - a.s0 + a.spb - 1) / a.spb;
    int grid = (int)balanced_grid(tiles, wave_grid(k, threads, smem, num_sms, tiles));
    if (grid_out) *grid_out = grid;
    k<<<grid, threads, smem, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dslash_ds(const KArgs &a, int epi, int R, int threads, size_t smem, int num_sms, cudaStream_t s,
                             int *grid) {
    if (epi == EPI_RESID) {
        if (R == 2) return launch_ds_one<2, EPI_RESID>(a, threads, smem, num_sms, s, grid);
        return launch_ds_one<1, EPI_RESID>(a, threads, smem, num_sms, s, grid);
    }
    if (epi != EPI_PLAIN) return cudaErrorInvalidValue;
    if (R == 2) return launch_ds_one<2, EPI_PLAIN>(a, threads, smem, num_sms, s, grid);
    return launch_ds_one<1, EPI_PLAIN>(a, threads, smem, num_sms, s, grid);
}

int split_vectors(hisq_ctx *ctx, const void *fp64_bundle, void *ds_bundle, int n, cudaStream_t st) {
    const long count = (long)ctx->geom.Vh * 3 * n;
    const int threads = 256;
    const int blocks = (int)std::min<long>((count + threads - 1) / threads, (long)ctx->num_sms * 16);
    ds_split_kernel<<<blocks, threads, 0, st>>>(reinterpret_cast<const double2 *>(fp64_bundle),
                                                reinterpret_cast<float4 *>(ds_bundle), count);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_residual(const hisq_links *fat, const hisq_links *naik, double mass, const double *rhs,
                             const double *x, double *r, int nrhs, double *res2) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!fat || !naik || !rhs || !x || !r) return set_error(HISQ_ERR_ARG, "null argument");
    if (fat->ctx != ctx || naik->ctx != ctx) return set_error(HISQ_ERR_STATE, "links of another context");
    if (fat->is_naik || !naik->is_naik) return set_error(HISQ_ERR_ARG, "expected (fat, naik) links handles");
    if (fat->prec != naik->prec) return set_error(HISQ_ERR_ARG, "fat and Naik links have different precisions");
    if (nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_NRHS);
    const int hp = links_hp(fat);
    const int Vh = ctx->geom.Vh;
    const size_t canon = (size_t)nrhs * Vh * 6 * sizeof(double), vb = vector_bytes(HISQ_FP64, Vh, nrhs);
    const size_t max_grid = (size_t)ctx->num_sms * 64;
    cudaStream_t st = ctx->stream;
    // scratch: canonical staging, b, x (FP64), x (ds), t, r (FP64), partials, counter
    char *buf = nullptr;
    const size_t pbytes = max_grid * nrhs * sizeof(double);
    const size_t total = canon + 5 * vb + pbytes + 256;
    HISQ_CUDA(cudaMalloc(&buf, total));
    double *stage = reinterpret_cast<double *>(buf);
    void *b64 = buf + canon, *x64 = buf + canon + vb, *xds = buf + canon + 2 * vb, *t = buf + canon + 3 * vb;
    void *r64 = buf + canon + 4 * vb;
    double *partials = reinterpret_cast<double *>(buf + canon + 5 * vb);
    unsigned int *counter = reinterpret_cast<unsigned int *>(buf + canon + 5 * vb + pbytes);
    int rc = HISQ_OK;
    auto cuda = [&](cudaError_t e, const char *what) {
        if (rc == HISQ_OK && e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    };
    cuda(cudaMemsetAsync(counter, 0, 256, st), "scratch reset");
    cuda(cudaMemcpyAsync(stage, rhs, canon, cudaMemcpyDefault, st), "rhs upload");
    if (rc == HISQ_OK) rc = pack_vectors(ctx, stage, b64, nrhs, HISQ_FP64, st);
    cuda(cudaMemcpyAsync(stage, x, canon, cudaMemcpyDefault, st), "x upload");
    if (rc == HISQ_OK) rc = pack_vectors(ctx, stage, x64, nrhs, HISQ_FP64, st);
    if (rc == HISQ_OK && hp == LINKS_DS) rc = split_vectors(ctx, x64, xds, nrhs, st);
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.n = nrhs;
    d.in = hp == LINKS_DS ? xds : x64;
    d.out = t;
    d.parity = 1;
    d.epi = EPI_PLAIN;
    if (rc == HISQ_OK) rc = launch_dslash(ctx, fat, naik, hp, d, nullptr, st);
    d.in = t;
    d.out = r64;
    d.parity = 0;
    d.epi = EPI_RESID;
    d.mass2 = mass * mass;
    d.axpy_in = x64;
    d.b = b64;
    d.partials = partials;
    d.partials_cap = max_grid * nrhs;
    d.counter = counter;
    d.dot_out = ctx->dot_out;
    if (rc == HISQ_OK) rc = launch_dslash(ctx, fat, naik, hp, d, nullptr, st);
    if (rc == HISQ_OK) rc = unpack_vectors(ctx, r64, stage, nrhs, HISQ_FP64, st);
    cuda(cudaMemcpyAsync(r, stage, canon, cudaMemcpyDefault, st), "r download");
    if (res2) cuda(cudaMemcpyAsync(res2, ctx->dot_out, sizeof(double) * nrhs, cudaMemcpyDefault, st), "dots download");
    cuda(cudaStreamSynchronize(st), "residual");
    cudaFree(buf);
    return rc;
}
