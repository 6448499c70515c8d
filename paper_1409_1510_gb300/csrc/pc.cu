// Learned gauge-covariant preconditioner: network forward, training loss and
// gradient by the project's own backward kernels, and Adam (Kingma & Ba 2014) on the GPU.
#include <string.h>
#include <math.h>
#include <algorithm>

#include "pc.cuh"

namespace hisq {

// ---- training loss pieces --------------------------------------------------------------------
struct LossArgs {
    int Vh, K, spb;
    const float2 *y, *e;
    const double *e2;   // [K] |r_k|^2
    float2 *G;          // [Vh][3][K]
    RedArgs red;
};

// u = y - e
__global__ void pc_sub_kernel(long n, const float2 *y, const float2 *e, float2 *u) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float2 a = y[i], b = e[i];
        u[i] = make_float2(a.x - b.x, a.y - b.y);
    }
}

// G *= 2 / (K |r_k|^2) for sample k = i % K
__global__ void pc_scale_kernel(long n, int K, const double *r2, float2 *G) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float s = (float)(2.0 / ((double)K * r2[i % K]));
        float2 g = G[i];
        G[i] = make_float2(s * g.x, s * g.y);
    }
}

// per-sample |v_k|^2 of a [Vh][3][K] FP32 field
__global__ void __launch_bounds__(256) pc_norm_kernel(LossArgs a) {
    extern __shared__ double red[];
    const int k = threadIdx.x % a.K, sl = threadIdx.x / a.K;
    const int rows = blockDim.x / a.K;
    double acc = 0.0;
    for (int tile = blockIdx.x; (long)tile * a.spb < a.Vh; tile += gridDim.x) {
        int s = tile * a.spb + sl;
        if (s >= a.Vh || sl >= a.spb) continue;
        for (int c = 0; c < 3; c++) {
            float2 e = a.e[((size_t)s * 3 + c) * a.K + k];
            acc += (double)(e.x * e.x + e.y * e.y);
        }
    }
    for (int i = threadIdx.x; i < rows * a.K; i += blockDim.x) red[i] = 0.0;
    __syncthreads();
    if (sl < rows) red[sl * a.K + k] = acc;
    block_reduce_finish(red, rows, a.K, 0, a.red);
}

// ---- Adam on the 2 * HISQ_PC_WEIGHTS real parameters ---------------------------------------
// grad of parameter i = sum of the two parity slots of its layer in gbuf[layer][parity][...]
__global__ void pc_adam_kernel(double *theta, double *m, double *v, const double *gbuf, const double *ext_grad,
                               int step, double lr, double b1, double b2, double eps, float2 *w32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * HISQ_PC_WEIGHTS) return;
    double g;
    if (ext_grad) {
        g = ext_grad[i];
    } else {
        int c = i / 2, comp = i % 2;
        int l = c < pc_layer_offset(1) ? 0 : c < pc_layer_offset(2) ? 1 : 2;
        int off = c - pc_layer_offset(l);
        const double *base = gbuf + (size_t)l * 2 * PC_PATHS * 16 * 2;
        g = base[off * 2 + comp] + base[PC_PATHS * 16 * 2 + off * 2 + comp];
    }
    m[i] = b1 * m[i] + (1.0 - b1) * g;
    v[i] = b2 * v[i] + (1.0 - b2) * g * g;
    double mhat = m[i] / (1.0 - pow(b1, (double)step));
    double vhat = v[i] / (1.0 - pow(b2, (double)step));
    theta[i] -= lr * mhat / (sqrt(vhat) + eps);
    float *w = reinterpret_cast<float *>(w32);
    w[i] = (float)theta[i];
}

__global__ void pc_sum_grad_kernel(const double *gbuf, double *grad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * HISQ_PC_WEIGHTS) return;
    int c = i / 2, comp = i % 2;
    int l = c < pc_layer_offset(1) ? 0 : c < pc_layer_offset(2) ? 1 : 2;
    int off = c - pc_layer_offset(l);
    const double *base = gbuf + (size_t)l * 2 * PC_PATHS * 16 * 2;
    grad[i] = base[off * 2 + comp] + base[PC_PATHS * 16 * 2 + off * 2 + comp];
}

// ---- workspace ------------------------------------------------------------------------------
struct PcWork {
    int K = 0;
    float2 *h1[2] = {nullptr, nullptr}, *h2[2] = {nullptr, nullptr};  // 4 channels per parity
    float2 *g1[2] = {nullptr, nullptr}, *g2[2] = {nullptr, nullptr};
    float2 *y = nullptr, *G3 = nullptr;   // 1 channel, even
    float2 *u = nullptr, *d = nullptr;    // 1 channel, even: y - e and A (y - e)
    float2 *t = nullptr;                  // 1 channel, odd: intermediate of A
    float2 *hN = nullptr, *gy = nullptr;  // 1 channel, even: M r and the output gradient (normal form)
    double *r2 = nullptr, *dots = nullptr;
    double *gbuf = nullptr;               // [3 layers][2 parity][17*16*2]
    double *gbuf2 = nullptr;              // first of the two gradient terms of the normal form
    double *e2 = nullptr, *err2 = nullptr, *grad = nullptr;
    double *partials = nullptr;
    size_t partials_cap = 0;
    unsigned int *counter = nullptr;
};

struct PcState {
    PcWork w;
};

static PcWork &pcw(hisq_pc *pc) { return reinterpret_cast<PcState *>(pc->work)->w; }

static void free_work(PcWork &w) {
    for (int p = 0; p < 2; p++) {
        if (w.h1[p]) cudaFree(w.h1[p]);
        if (w.h2[p]) cudaFree(w.h2[p]);
        if (w.g1[p]) cudaFree(w.g1[p]);
        if (w.g2[p]) cudaFree(w.g2[p]);
        w.h1[p] = w.h2[p] = w.g1[p] = w.g2[p] = nullptr;
    }
    void *bufs[] = {w.y, w.G3, w.u, w.d, w.t, w.hN, w.gy, w.r2, w.dots, w.gbuf, w.gbuf2, w.e2, w.err2, w.grad,
                    w.partials, w.counter};
    for (void *b : bufs)
        if (b) cudaFree(b);
    w = PcWork();
}

static int ensure_work(hisq_ctx *ctx, hisq_pc *pc, int K) {
    PcWork &w = pcw(pc);
    if (w.K >= K) return HISQ_OK;
    free_work(w);
    size_t Vh = ctx->geom.Vh;
    size_t f4 = Vh * 3 * K * 4 * sizeof(float2), f1 = Vh * 3 * K * sizeof(float2);
    size_t pcap = (size_t)ctx->num_sms * 8 * PC_PATHS * 16 * 2;
    bool ok = true;
    for (int p = 0; p < 2; p++)
        ok = ok && cudaMalloc(&w.h1[p], f4) == cudaSuccess && cudaMalloc(&w.h2[p], f4) == cudaSuccess &&
             cudaMalloc(&w.g1[p], f4) == cudaSuccess && cudaMalloc(&w.g2[p], f4) == cudaSuccess;
    ok = ok && cudaMalloc(&w.y, f1) == cudaSuccess && cudaMalloc(&w.G3, f1) == cudaSuccess &&
         cudaMalloc(&w.u, f1) == cudaSuccess && cudaMalloc(&w.d, f1) == cudaSuccess &&
         cudaMalloc(&w.t, f1) == cudaSuccess && cudaMalloc(&w.hN, f1) == cudaSuccess &&
         cudaMalloc(&w.gy, f1) == cudaSuccess && cudaMalloc(&w.r2, sizeof(double) * HISQ_MAX_BUNDLE) == cudaSuccess &&
         cudaMalloc(&w.dots, sizeof(double) * HISQ_MAX_BUNDLE * 4) == cudaSuccess &&
         cudaMalloc(&w.gbuf, sizeof(double) * 3 * 2 * PC_PATHS * 16 * 2) == cudaSuccess &&
         cudaMalloc(&w.gbuf2, sizeof(double) * 3 * 2 * PC_PATHS * 16 * 2) == cudaSuccess &&
         cudaMalloc(&w.e2, sizeof(double) * HISQ_MAX_BUNDLE) == cudaSuccess &&
         cudaMalloc(&w.err2, sizeof(double) * HISQ_MAX_BUNDLE) == cudaSuccess &&
         cudaMalloc(&w.grad, sizeof(double) * 2 * HISQ_PC_WEIGHTS) == cudaSuccess &&
         cudaMalloc(&w.partials, sizeof(double) * pcap) == cudaSuccess &&
         cudaMalloc(&w.counter, sizeof(unsigned int) * 4) == cudaSuccess;
    if (!ok) {
        free_work(w);
        return set_error(HISQ_ERR_NOMEM, "preconditioner workspace allocation failed");
    }
    w.partials_cap = pcap;
    cudaMemset(w.counter, 0, sizeof(unsigned int) * 4);
    w.K = K;
    return HISQ_OK;
}

// ---- launches -------------------------------------------------------------------------------
static int pow2_floor_pc(int x) {
    int p = 1;
    while (p * 2 <= x) p *= 2;
    return p;
}

static PcLayerArgs layer_args(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int K, int parity) {
    PcLayerArgs p;
    memset(&p, 0, sizeof(p));
    p.g = ctx->geom;
    p.fat = fat->field();
    p.naik = naik->field();
    p.K = K;
    p.spb = pow2_floor_pc(256 / K);  // kernels run 256 threads; threads with sl >= spb idle
    p.parity = parity;
    return p;
}

template <typename Kern>
static int grid_of(hisq_ctx *ctx, Kern k, size_t smem, int spb) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem);
    long tiles = (ctx->geom.Vh + spb - 1) / spb;
    return (int)std::max(1L, std::min<long>(tiles, (long)std::max(per_sm, 1) * ctx->num_sms));
}

template <int A, int B, bool ADJ>
static int run_layer(hisq_ctx *ctx, const hisq_links *naik, const PcLayerArgs &p, cudaStream_t st) {
    switch (naik->recon) {
    case 13: {
        auto k = pc_layer_kernel<A, B, ADJ, 13>;
        k<<<grid_of(ctx, k, 0, p.spb), 256, 0, st>>>(p);
        break;
    }
    case 9: {
        auto k = pc_layer_kernel<A, B, ADJ, 9>;
        k<<<grid_of(ctx, k, 0, p.spb), 256, 0, st>>>(p);
        break;
    }
    default: {
        auto k = pc_layer_kernel<A, B, ADJ, 18>;
        k<<<grid_of(ctx, k, 0, p.spb), 256, 0, st>>>(p);
    }
    }
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

template <int A, int B>
static int run_grad(hisq_ctx *ctx, const hisq_links *naik, PcWork &w, const PcGradArgs &ga, cudaStream_t st) {
    constexpr int ND = PC_PATHS * A * B * 2;
    size_t smem = (size_t)8 * ND * sizeof(double);
    auto launch = [&](auto k) -> int {
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int grid = grid_of(ctx, k, smem, ga.L.spb);
        if ((size_t)grid * ND > w.partials_cap) grid = (int)(w.partials_cap / ND);
        k<<<grid, 256, smem, st>>>(ga);
        return HISQ_OK;
    };
    switch (naik->recon) {
    case 13: launch(pc_grad_kernel<A, B, 13>); break;
    case 9: launch(pc_grad_kernel<A, B, 9>); break;
    default: launch(pc_grad_kernel<A, B, 18>);
    }
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

static const float2 *layer_w(const hisq_pc *pc, int l) { return pc->d_weights + pc_layer_offset(l); }

// forward: r (even, [Vh][3][K]) -> y (even); keeps h1, h2 of both parities in the workspace
static int forward(hisq_ctx *ctx, hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const float2 *r,
                   float2 *y, int K, cudaStream_t st) {
    PcWork &w = pcw(pc);
    for (int par = 0; par < 2; par++) {
        PcLayerArgs p = layer_args(ctx, fat, naik, K, par);
        p.W = layer_w(pc, 0);
        p.in_same = par == 0 ? r : nullptr;
        p.in_opp = par == 1 ? r : nullptr;
        p.out = w.h1[par];
        HISQ_CHECK((run_layer<1, 4, false>(ctx, naik, p, st)));
    }
    for (int par = 0; par < 2; par++) {
        PcLayerArgs p = layer_args(ctx, fat, naik, K, par);
        p.W = layer_w(pc, 1);
        p.in_same = w.h1[par];
        p.in_opp = w.h1[1 - par];
        p.out = w.h2[par];
        HISQ_CHECK((run_layer<4, 4, false>(ctx, naik, p, st)));
    }
    PcLayerArgs p = layer_args(ctx, fat, naik, K, 0);
    p.W = layer_w(pc, 2);
    p.in_same = w.h2[0];
    p.in_opp = w.h2[1];
    p.out = y;
    return run_layer<4, 1, false>(ctx, naik, p, st);
}

// y = M^dag r on even sites: the adjoint layers in reverse order (L1^dag L2^dag L3^dag),
// input r on even sites (zero on odd), output projected to even sites
static int forward_adjoint(hisq_ctx *ctx, hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const float2 *r,
                           float2 *y, int K, cudaStream_t st) {
    PcWork &w = pcw(pc);
    for (int par = 0; par < 2; par++) {
        PcLayerArgs p = layer_args(ctx, fat, naik, K, par);
        p.W = layer_w(pc, 2);
        p.in_same = par == 0 ? r : nullptr;
        p.in_opp = par == 1 ? r : nullptr;
        p.out = w.g2[par];
        HISQ_CHECK((run_layer<1, 4, true>(ctx, naik, p, st)));
    }
    for (int par = 0; par < 2; par++) {
        PcLayerArgs p = layer_args(ctx, fat, naik, K, par);
        p.W = layer_w(pc, 1);
        p.in_same = w.g2[par];
        p.in_opp = w.g2[1 - par];
        p.out = w.g1[par];
        HISQ_CHECK((run_layer<4, 4, true>(ctx, naik, p, st)));
    }
    PcLayerArgs p = layer_args(ctx, fat, naik, K, 0);
    p.W = layer_w(pc, 0);
    p.in_same = w.g1[0];
    p.in_opp = w.g1[1];
    p.out = y;
    return run_layer<4, 1, true>(ctx, naik, p, st);
}

// out = (a + b) / 2
__global__ void pc_average_kernel(long n, const float2 *a, const float2 *b, float2 *out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float2 x = a[i], y = b[i];
        out[i] = make_float2(0.5f * (x.x + y.x), 0.5f * (x.y + y.y));
    }
}

// out = M_H in with M_H = (M + M^dag) / 2, the Hermitian part of the network
static int forward_hermitian(hisq_ctx *ctx, hisq_pc *pc, const hisq_links *fat, const hisq_links *naik,
                             const float2 *in, float2 *out, int K, cudaStream_t st) {
    PcWork &w = pcw(pc);
    HISQ_CHECK(forward(ctx, pc, fat, naik, in, w.y, K, st));
    HISQ_CHECK(forward_adjoint(ctx, pc, fat, naik, in, w.u, K, st));
    const long n = (long)ctx->geom.Vh * 3 * K;
    pc_average_kernel<<<(int)std::min<long>((n + 255) / 256, (long)ctx->num_sms * 8), 256, 0, st>>>(n, w.y, w.u, out);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

// out = M^dag M in, the normal form of the network
static int forward_normal(hisq_ctx *ctx, hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const float2 *in,
                          float2 *out, int K, cudaStream_t st) {
    PcWork &w = pcw(pc);
    HISQ_CHECK(forward(ctx, pc, fat, naik, in, w.y, K, st));
    return forward_adjoint(ctx, pc, fat, naik, w.y, out, K, st);
}

// the preconditioner of the handle's form
static int forward_precond(hisq_ctx *ctx, hisq_pc *pc, const hisq_links *fat, const hisq_links *naik,
                           const float2 *in, float2 *out, int K, cudaStream_t st) {
    if (pc->form == HISQ_PC_NORMAL) return forward_normal(ctx, pc, fat, naik, in, out, K, st);
    return forward_hermitian(ctx, pc, fat, naik, in, out, K, st);
}

__global__ void pc_add_kernel(int n, double *a, const double *b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] += b[i];
}

static RedArgs red_of(PcWork &w, double *dot_out) {
    RedArgs r;
    r.partials = w.partials;
    r.counter = w.counter;
    r.dot_out = dot_out;
    r.hook = 0;
    r.st = nullptr;
    r.partials_only = 0;
    return r;
}

// backward from G3 (even, 1 channel): fills gbuf[layer][parity]
static int backward(hisq_ctx *ctx, hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const float2 *r, int K,
                    cudaStream_t st) {
    PcWork &w = pcw(pc);
    const size_t slot = PC_PATHS * 16 * 2;
    HISQ_CUDA(cudaMemsetAsync(w.gbuf, 0, sizeof(double) * 3 * 2 * slot, st));
    // layer 3 (4 -> 1): weight gradient at parity 0
    {
        PcGradArgs ga;
        ga.L = layer_args(ctx, fat, naik, K, 0);
        ga.L.in_same = w.h2[0];
        ga.L.in_opp = w.h2[1];
        ga.G = w.G3;
        ga.red = red_of(w, w.gbuf + (2 * 2 + 0) * slot);
        HISQ_CHECK((run_grad<4, 1>(ctx, naik, w, ga, st)));
    }
    // G2 = adjoint of layer 3 applied to G3
    for (int par = 0; par < 2; par++) {
        PcLayerArgs p = layer_args(ctx, fat, naik, K, par);
        p.W = layer_w(pc, 2);
        p.in_same = par == 0 ? w.G3 : nullptr;
        p.in_opp = par == 1 ? w.G3 : nullptr;
        p.out = w.g2[par];
        HISQ_CHECK((run_layer<1, 4, true>(ctx, naik, p, st)));
    }
    // layer 2 (4 -> 4): weight gradient at both parities
    for (int par = 0; par < 2; par++) {
        PcGradArgs ga;
        ga.L = layer_args(ctx, fat, naik, K, par);
        ga.L.in_same = w.h1[par];
        ga.L.in_opp = w.h1[1 - par];
        ga.G = w.g2[par];
        ga.red = red_of(w, w.gbuf + (1 * 2 + par) * slot);
        HISQ_CHECK((run_grad<4, 4>(ctx, naik, w, ga, st)));
    }
    // G1 = adjoint of layer 2 applied to G2
    for (int par = 0; par < 2; par++) {
        PcLayerArgs p = layer_args(ctx, fat, naik, K, par);
        p.W = layer_w(pc, 1);
        p.in_same = w.g2[par];
        p.in_opp = w.g2[1 - par];
        p.out = w.g1[par];
        HISQ_CHECK((run_layer<4, 4, true>(ctx, naik, p, st)));
    }
    // layer 1 (1 -> 4): weight gradient at both parities (input r lives on even sites)
    for (int par = 0; par < 2; par++) {
        PcGradArgs ga;
        ga.L = layer_args(ctx, fat, naik, K, par);
        ga.L.in_same = par == 0 ? r : nullptr;
        ga.L.in_opp = par == 1 ? r : nullptr;
        ga.G = w.g1[par];
        ga.red = red_of(w, w.gbuf + (0 * 2 + par) * slot);
        HISQ_CHECK((run_grad<1, 4>(ctx, naik, w, ga, st)));
    }
    return HISQ_OK;
}

static int reduce_launch(hisq_ctx *ctx, void (*k)(LossArgs), LossArgs a, cudaStream_t st) {
    int threads = (a.spb * a.K + 31) / 32 * 32;  // whole warps; rows beyond spb idle
    size_t smem = (threads + 64) * sizeof(double);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    long tiles = (a.Vh + a.spb - 1) / a.spb;
    int grid = (int)std::max(1L, std::min<long>(tiles, (long)std::max(per_sm, 1) * ctx->num_sms));
    k<<<grid, threads, smem, st>>>(a);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

// out = A in = m^2 in - D_eo D_oe in for K FP32 even-site vectors (t: odd intermediate)
static int apply_a(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, PcWork &w, double mass,
                   const float2 *in, float2 *out, int K, cudaStream_t st) {
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.in = in;
    d.out = w.t;
    d.n = K;
    d.parity = 1;
    d.epi = EPI_PLAIN;
    HISQ_CHECK(launch_dslash(ctx, fat, naik, false, d, nullptr, st));
    d.in = w.t;
    d.out = out;
    d.parity = 0;
    d.epi = EPI_AOP;
    d.mass2 = mass * mass;
    d.axpy_in = in;
    d.partials = w.partials;
    d.partials_cap = w.partials_cap;
    d.counter = w.counter;
    d.dot_out = w.dots;
    return launch_dslash(ctx, fat, naik, false, d, nullptr, st);
}

// loss = mean_k |A (M r_k - e_k)|^2 / |r_k|^2 and its weight gradient (gbuf)
static int loss_and_grad(hisq_ctx *ctx, hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, double mass,
                         const float2 *r, const float2 *e, int K, cudaStream_t st) {
    PcWork &w = pcw(pc);
    const long n = (long)ctx->geom.Vh * 3 * K;
    const int blocks = (int)std::min<long>((n + 255) / 256, (long)ctx->num_sms * 8);
    LossArgs a;
    memset(&a, 0, sizeof(a));
    a.Vh = ctx->geom.Vh;
    a.K = K;
    a.spb = pow2_floor_pc(256 / K);
    a.e = r;
    a.red = red_of(w, w.r2);
    HISQ_CHECK(reduce_launch(ctx, pc_norm_kernel, a, st));                 // |r_k|^2
    HISQ_CHECK(forward(ctx, pc, fat, naik, r, w.y, K, st));                 // y = M r
    pc_sub_kernel<<<blocks, 256, 0, st>>>(n, w.y, e, w.u);                  // u = y - e
    HISQ_CHECK(apply_a(ctx, fat, naik, w, mass, w.u, w.d, K, st));          // d = A u
    a.e = w.d;
    a.red = red_of(w, w.err2);
    HISQ_CHECK(reduce_launch(ctx, pc_norm_kernel, a, st));                 // |d_k|^2
    HISQ_CHECK(apply_a(ctx, fat, naik, w, mass, w.d, w.G3, K, st));         // G3 = A d
    pc_scale_kernel<<<blocks, 256, 0, st>>>(n, K, w.r2, w.G3);              // G3 *= 2 / (K |r|^2)
    HISQ_CUDA(cudaGetLastError());
    return backward(ctx, pc, fat, naik, r, K, st);
}

// The normal form P = M^dag M: loss = mean_k |A (P r_k - e_k)|^2 / |r_k|^2.  With h = M r,
// y = M^dag h and gy = 2 A A (y - e) / (K |r|^2) the weights enter twice: through M^dag (the
// backward of M at input gy with output gradient h) and through M (the backward of M at input r
// with output gradient M gy); the two weight gradients are added.
static int loss_and_grad_normal(hisq_ctx *ctx, hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, double mass,
                                const float2 *r, const float2 *e, int K, cudaStream_t st) {
    PcWork &w = pcw(pc);
    const long n = (long)ctx->geom.Vh * 3 * K;
    const size_t fbytes = sizeof(float2) * n;
    const int blocks = (int)std::min<long>((n + 255) / 256, (long)ctx->num_sms * 8);
    const int ng = 3 * 2 * PC_PATHS * 16 * 2;
    LossArgs a;
    memset(&a, 0, sizeof(a));
    a.Vh = ctx->geom.Vh;
    a.K = K;
    a.spb = pow2_floor_pc(256 / K);
    a.e = r;
    a.red = red_of(w, w.r2);
    HISQ_CHECK(reduce_launch(ctx, pc_norm_kernel, a, st));                 // |r_k|^2
    HISQ_CHECK(forward(ctx, pc, fat, naik, r, w.hN, K, st));                // h = M r
    HISQ_CHECK(forward_adjoint(ctx, pc, fat, naik, w.hN, w.u, K, st));     // y = M^dag h
    pc_sub_kernel<<<blocks, 256, 0, st>>>(n, w.u, e, w.u);                  // u = y - e
    HISQ_CHECK(apply_a(ctx, fat, naik, w, mass, w.u, w.d, K, st));          // d = A u
    a.e = w.d;
    a.red = red_of(w, w.err2);
    HISQ_CHECK(reduce_launch(ctx, pc_norm_kernel, a, st));                 // |d_k|^2
    HISQ_CHECK(apply_a(ctx, fat, naik, w, mass, w.d, w.gy, K, st));         // gy = A d
    pc_scale_kernel<<<blocks, 256, 0, st>>>(n, K, w.r2, w.gy);              // gy *= 2 / (K |r|^2)
    HISQ_CUDA(cudaGetLastError());
    // through M^dag: forward at input gy (its activations; output M gy kept in y), gradient h
    HISQ_CHECK(forward(ctx, pc, fat, naik, w.gy, w.y, K, st));
    HISQ_CUDA(cudaMemcpyAsync(w.G3, w.hN, fbytes, cudaMemcpyDeviceToDevice, st));
    HISQ_CHECK(backward(ctx, pc, fat, naik, w.gy, K, st));
    HISQ_CUDA(cudaMemcpyAsync(w.gbuf2, w.gbuf, sizeof(double) * ng, cudaMemcpyDeviceToDevice, st));
    // through M: forward at input r again (its activations), gradient M gy
    HISQ_CHECK(forward(ctx, pc, fat, naik, r, w.u, K, st));
    HISQ_CUDA(cudaMemcpyAsync(w.G3, w.y, fbytes, cudaMemcpyDeviceToDevice, st));
    HISQ_CHECK(backward(ctx, pc, fat, naik, r, K, st));
    pc_add_kernel<<<(ng + 255) / 256, 256, 0, st>>>(ng, w.gbuf, w.gbuf2);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

static int loss_and_grad_form(hisq_ctx *ctx, hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, double mass,
                              const float2 *r, const float2 *e, int K, cudaStream_t st) {
    if (pc->form == HISQ_PC_NORMAL) return loss_and_grad_normal(ctx, pc, fat, naik, mass, r, e, K, st);
    return loss_and_grad(ctx, pc, fat, naik, mass, r, e, K, st);
}

static int check_args(hisq_ctx *ctx, const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik) {
    if (!pc || !fat || !naik) return set_error(HISQ_ERR_ARG, "null argument");
    if (pc->ctx != ctx || fat->ctx != ctx || naik->ctx != ctx) return set_error(HISQ_ERR_STATE, "handle of another context");
    if (fat->is_naik || !naik->is_naik) return set_error(HISQ_ERR_ARG, "expected (fat, naik) links");
    if (fat->prec != HISQ_FP32 || naik->prec != HISQ_FP32)
        return set_error(HISQ_ERR_ARG, "the preconditioner network runs on FP32 links");
    return HISQ_OK;
}

static int upload_weights(hisq_pc *pc, cudaStream_t st) {
    float2 w[HISQ_PC_WEIGHTS];
    for (int i = 0; i < HISQ_PC_WEIGHTS; i++) w[i] = make_float2((float)pc->weights[2 * i], (float)pc->weights[2 * i + 1]);
    HISQ_CUDA(cudaMemcpyAsync(pc->d_weights, w, sizeof(w), cudaMemcpyHostToDevice, st));
    HISQ_CUDA(cudaMemcpyAsync(pc->d_theta, pc->weights, sizeof(pc->weights), cudaMemcpyHostToDevice, st));
    HISQ_CUDA(cudaStreamSynchronize(st));
    return HISQ_OK;
}

void free_pc(hisq_pc *pc) {
    if (!pc) return;
    if (pc->work) {
        free_work(pcw(pc));
        delete reinterpret_cast<PcState *>(pc->work);
    }
    if (pc->d_weights) cudaFree(pc->d_weights);
    if (pc->d_theta) cudaFree(pc->d_theta);
    if (pc->d_m) cudaFree(pc->d_m);
    if (pc->d_v) cudaFree(pc->d_v);
    delete pc;
}

int pc_prepare(hisq_ctx *ctx, const hisq_pc *pc, int n) { return ensure_work(ctx, const_cast<hisq_pc *>(pc), n); }

int pc_forward(hisq_ctx *ctx, const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const void *in,
               void *out, int n, cudaStream_t st) {
    hisq_pc *m = const_cast<hisq_pc *>(pc);
    HISQ_CHECK(ensure_work(ctx, m, n));
    return forward(ctx, m, fat, naik, reinterpret_cast<const float2 *>(in), reinterpret_cast<float2 *>(out), n, st);
}

int pc_forward_precond(hisq_ctx *ctx, const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik,
                       const void *in, void *out, int n, cudaStream_t st) {
    hisq_pc *m = const_cast<hisq_pc *>(pc);
    HISQ_CHECK(ensure_work(ctx, m, n));
    return forward_precond(ctx, m, fat, naik, reinterpret_cast<const float2 *>(in), reinterpret_cast<float2 *>(out), n,
                           st);
}

}  // namespace hisq

using namespace hisq;

extern "C" {

int hisq_pc_create(hisq_pc **out, const double *weights) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!out) return set_error(HISQ_ERR_ARG, "null output handle");
    hisq_pc *pc = new hisq_pc();
    memset(pc->weights, 0, sizeof(pc->weights));
    if (weights) {
        memcpy(pc->weights, weights, sizeof(pc->weights));
    } else {  // identity network: only the identity path of channel 0 in every layer
        for (int l = 0; l < 3; l++) pc->weights[2 * pc_layer_offset(l)] = 1.0;
    }
    pc->ctx = ctx;
    pc->form = HISQ_PC_NORMAL;
    pc->train_steps = 0;
    pc->work = new PcState();
    bool ok = cudaMalloc(&pc->d_weights, sizeof(float2) * HISQ_PC_WEIGHTS) == cudaSuccess &&
              cudaMalloc(&pc->d_theta, sizeof(pc->weights)) == cudaSuccess &&
              cudaMalloc(&pc->d_m, sizeof(pc->weights)) == cudaSuccess &&
              cudaMalloc(&pc->d_v, sizeof(pc->weights)) == cudaSuccess;
    if (!ok) {
        free_pc(pc);
        return set_error(HISQ_ERR_NOMEM, "preconditioner allocation failed");
    }
    cudaMemsetAsync(pc->d_m, 0, sizeof(pc->weights), ctx->stream);
    cudaMemsetAsync(pc->d_v, 0, sizeof(pc->weights), ctx->stream);
    int rc = upload_weights(pc, ctx->stream);
    if (rc != HISQ_OK) {
        free_pc(pc);
        return rc;
    }
    ctx->pcs.push_back(pc);
    *out = pc;
    return HISQ_OK;
}

int hisq_pc_destroy(hisq_pc *pc) {
    if (!pc) return HISQ_OK;
    hisq_ctx *ctx = pc->ctx;
    if (ctx) {
        cudaStreamSynchronize(ctx->stream);
        ctx->pcs.erase(std::remove(ctx->pcs.begin(), ctx->pcs.end(), pc), ctx->pcs.end());
    }
    free_pc(pc);
    return HISQ_OK;
}

int hisq_pc_set_weights(hisq_pc *pc, const double *weights) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!pc || !weights) return set_error(HISQ_ERR_ARG, "null argument");
    if (pc->ctx != ctx) return set_error(HISQ_ERR_STATE, "handle of another context");
    memcpy(pc->weights, weights, sizeof(pc->weights));
    cudaMemsetAsync(pc->d_m, 0, sizeof(pc->weights), ctx->stream);
    cudaMemsetAsync(pc->d_v, 0, sizeof(pc->weights), ctx->stream);
    pc->train_steps = 0;  // new weights start a new Adam run
    return upload_weights(pc, ctx->stream);
}

int hisq_pc_get_weights(const hisq_pc *pc, double *weights) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!pc || !weights) return set_error(HISQ_ERR_ARG, "null argument");
    if (pc->ctx != ctx) return set_error(HISQ_ERR_STATE, "handle of another context");
    HISQ_CUDA(cudaMemcpyAsync(const_cast<double *>(pc->weights), pc->d_theta, sizeof(pc->weights), cudaMemcpyDeviceToHost,
                              ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    memcpy(weights, pc->weights, sizeof(pc->weights));
    return HISQ_OK;
}

int hisq_pc_apply(const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const void *in, void *out, int nrhs) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    HISQ_CHECK(check_args(ctx, pc, fat, naik));
    if (!in || !out || in == out) return set_error(HISQ_ERR_ARG, "bad vectors");
    if (nrhs < 1 || nrhs > HISQ_MAX_BUNDLE) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_BUNDLE);
    return pc_forward(ctx, pc, fat, naik, in, out, nrhs, ctx->stream);
}

// the three operators of the network beyond M itself
enum { APPLY_ADJOINT, APPLY_HERMITIAN, APPLY_NORMAL };

static int apply_op(int op, const hisq_pc *pc_c, const hisq_links *fat, const hisq_links *naik, const void *in,
                    void *out, int nrhs) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    HISQ_CHECK(check_args(ctx, pc_c, fat, naik));
    if (!in || !out || in == out) return set_error(HISQ_ERR_ARG, "bad vectors");
    if (nrhs < 1 || nrhs > HISQ_MAX_BUNDLE) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_BUNDLE);
    hisq_pc *pc = const_cast<hisq_pc *>(pc_c);
    HISQ_CHECK(ensure_work(ctx, pc, nrhs));
    const float2 *x = reinterpret_cast<const float2 *>(in);
    float2 *y = reinterpret_cast<float2 *>(out);
    if (op == APPLY_ADJOINT) return forward_adjoint(ctx, pc, fat, naik, x, y, nrhs, ctx->stream);
    if (op == APPLY_HERMITIAN) return forward_hermitian(ctx, pc, fat, naik, x, y, nrhs, ctx->stream);
    return forward_normal(ctx, pc, fat, naik, x, y, nrhs, ctx->stream);
}

int hisq_pc_apply_adjoint(const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const void *in, void *out,
                          int nrhs) {
    return apply_op(APPLY_ADJOINT, pc, fat, naik, in, out, nrhs);
}

int hisq_pc_apply_hermitian(const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const void *in,
                            void *out, int nrhs) {
    return apply_op(APPLY_HERMITIAN, pc, fat, naik, in, out, nrhs);
}

int hisq_pc_apply_normal(const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const void *in, void *out,
                         int nrhs) {
    return apply_op(APPLY_NORMAL, pc, fat, naik, in, out, nrhs);
}

int hisq_pc_set_form(hisq_pc *pc, int form) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!pc) return set_error(HISQ_ERR_ARG, "null handle");
    if (pc->ctx != ctx) return set_error(HISQ_ERR_STATE, "handle of another context");
    if (form != HISQ_PC_NORMAL && form != HISQ_PC_HERMITIAN_PART) return set_error(HISQ_ERR_ARG, "unknown form %d", form);
    pc->form = form;
    return HISQ_OK;
}

int hisq_pc_loss_grad(const hisq_pc *pc_c, const hisq_links *fat, const hisq_links *naik, double mass, const void *r,
                      const void *e, int K, double *loss, double *grad) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    HISQ_CHECK(check_args(ctx, pc_c, fat, naik));
    if (!r || !e) return set_error(HISQ_ERR_ARG, "null vectors");
    if (K < 1 || K > HISQ_MAX_BUNDLE) return set_error(HISQ_ERR_ARG, "K must be in 1..%d", HISQ_MAX_BUNDLE);
    hisq_pc *pc = const_cast<hisq_pc *>(pc_c);
    HISQ_CHECK(ensure_work(ctx, pc, K));
    PcWork &w = pcw(pc);
    cudaStream_t st = ctx->stream;
    HISQ_CHECK(loss_and_grad_form(ctx, pc, fat, naik, mass, reinterpret_cast<const float2 *>(r),
                                  reinterpret_cast<const float2 *>(e), K, st));
    double err2[HISQ_MAX_BUNDLE], e2[HISQ_MAX_BUNDLE];
    HISQ_CUDA(cudaMemcpyAsync(err2, w.err2, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
    HISQ_CUDA(cudaMemcpyAsync(e2, w.r2, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
    if (grad) {
        pc_sum_grad_kernel<<<(2 * HISQ_PC_WEIGHTS + 255) / 256, 256, 0, st>>>(w.gbuf, w.grad);
        HISQ_CUDA(cudaMemcpyAsync(grad, w.grad, sizeof(double) * 2 * HISQ_PC_WEIGHTS, cudaMemcpyDefault, st));
    }
    HISQ_CUDA(cudaStreamSynchronize(st));
    if (loss) {
        double s = 0.0;
        for (int k = 0; k < K; k++) s += err2[k] / e2[k];
        *loss = s / K;
    }
    return HISQ_OK;
}

int hisq_pc_adam_step(hisq_pc *pc, const double *grad, int step, double lr, double beta1, double beta2, double eps) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!pc || !grad) return set_error(HISQ_ERR_ARG, "null argument");
    if (pc->ctx != ctx) return set_error(HISQ_ERR_STATE, "handle of another context");
    if (step < 1) return set_error(HISQ_ERR_ARG, "step counts from 1");
    HISQ_CHECK(ensure_work(ctx, pc, 1));
    PcWork &w = pcw(pc);
    const double *g = grad;
    if (!is_device_ptr(grad)) {
        HISQ_CUDA(cudaMemcpyAsync(w.grad, grad, sizeof(double) * 2 * HISQ_PC_WEIGHTS, cudaMemcpyHostToDevice, ctx->stream));
        g = w.grad;
    }
    pc_adam_kernel<<<(2 * HISQ_PC_WEIGHTS + 255) / 256, 256, 0, ctx->stream>>>(pc->d_theta, pc->d_m, pc->d_v, nullptr, g,
                                                                               step, lr, beta1, beta2, eps, pc->d_weights);
    HISQ_CUDA(cudaGetLastError());
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return HISQ_OK;
}

int hisq_pc_train(hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, double mass, const void *r, const void *e,
                  int K, int batch, int epochs, double lr, double *loss_history) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    HISQ_CHECK(check_args(ctx, pc, fat, naik));
    if (!r || !e) return set_error(HISQ_ERR_ARG, "null vectors");
    if (K < 1 || batch < 1 || batch > HISQ_MAX_BUNDLE || epochs < 1 || !(lr > 0))
        return set_error(HISQ_ERR_ARG, "bad training arguments");
    HISQ_CHECK(ensure_work(ctx, pc, batch));
    PcWork &w = pcw(pc);
    cudaStream_t st = ctx->stream;
    // pairs are stored as bundles of 16; minibatches never straddle bundles
    const size_t bundle_elems = (size_t)ctx->geom.Vh * 3 * HISQ_MAX_BUNDLE;
    int nbundles = (K + HISQ_MAX_BUNDLE - 1) / HISQ_MAX_BUNDLE;
    // the kernels address a minibatch as a contiguous [Vh][3][batch] field, so a minibatch is a
    // whole bundle of 16 when batch == 16; smaller batches use the first `batch` of a bundle
    // through a gather into the workspace
    float2 *rb = nullptr, *eb = nullptr;
    size_t mb_bytes = (size_t)ctx->geom.Vh * 3 * batch * sizeof(float2);
    HISQ_CUDA(cudaMalloc(&rb, mb_bytes));
    if (cudaMalloc(&eb, mb_bytes) != cudaSuccess) {
        cudaFree(rb);
        return set_error(HISQ_ERR_NOMEM, "training minibatch allocation failed");
    }
    int rc = HISQ_OK;
    int step = pc->train_steps;  // a later call continues the same Adam run
    for (int ep = 0; ep < epochs && rc == HISQ_OK; ep++) {
        double loss_sum = 0.0;
        int nb = 0;
        for (int bnd = 0; bnd < nbundles && rc == HISQ_OK; bnd++) {
            int in_bundle = std::min(HISQ_MAX_BUNDLE, K - bnd * HISQ_MAX_BUNDLE);
            for (int k0 = 0; k0 + batch <= in_bundle && rc == HISQ_OK; k0 += batch) {
                const float2 *rs = reinterpret_cast<const float2 *>(r) + bnd * bundle_elems;
                const float2 *es = reinterpret_cast<const float2 *>(e) + bnd * bundle_elems;
                // gather columns k0..k0+batch-1 of each (site, colour) row
                cudaError_t ce = cudaMemcpy2DAsync(rb, batch * sizeof(float2), rs + k0, HISQ_MAX_BUNDLE * sizeof(float2),
                                                   batch * sizeof(float2), (size_t)ctx->geom.Vh * 3, cudaMemcpyDeviceToDevice, st);
                if (ce == cudaSuccess)
                    ce = cudaMemcpy2DAsync(eb, batch * sizeof(float2), es + k0, HISQ_MAX_BUNDLE * sizeof(float2),
                                           batch * sizeof(float2), (size_t)ctx->geom.Vh * 3, cudaMemcpyDeviceToDevice, st);
                if (ce != cudaSuccess) {
                    rc = set_error(HISQ_ERR_CUDA, "minibatch gather failed: %s", cudaGetErrorString(ce));
                    break;
                }
                rc = loss_and_grad_form(ctx, pc, fat, naik, mass, rb, eb, batch, st);
                if (rc != HISQ_OK) break;
                step++;
                pc_adam_kernel<<<(2 * HISQ_PC_WEIGHTS + 255) / 256, 256, 0, st>>>(pc->d_theta, pc->d_m, pc->d_v, w.gbuf,
                                                                                  nullptr, step, lr, 0.9, 0.999, 1e-8,
                                                                                  pc->d_weights);
                double err2[HISQ_MAX_BUNDLE], e2[HISQ_MAX_BUNDLE];
                cudaMemcpyAsync(err2, w.err2, sizeof(double) * batch, cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(e2, w.r2, sizeof(double) * batch, cudaMemcpyDeviceToHost, st);
                ce = cudaStreamSynchronize(st);
                if (ce != cudaSuccess) {
                    rc = set_error(HISQ_ERR_CUDA, "training step failed: %s", cudaGetErrorString(ce));
                    break;
                }
                double s = 0.0;
                for (int k = 0; k < batch; k++) s += err2[k] / e2[k];
                loss_sum += s / batch;
                nb++;
            }
        }
        if (loss_history) loss_history[ep] = nb ? loss_sum / nb : 0.0;
    }
    cudaStreamSynchronize(st);
    cudaFree(rb);
    cudaFree(eb);
    pc->train_steps = step;
    if (rc == HISQ_OK) {
        HISQ_CUDA(cudaMemcpy(pc->weights, pc->d_theta, sizeof(pc->weights), cudaMemcpyDeviceToHost));
    }
    return rc;
}

}  // extern "C"
