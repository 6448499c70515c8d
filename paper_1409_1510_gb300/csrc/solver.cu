// Conjugate-gradient solvers on A = m^2 - D_eo D_oe: fused masked BLAS-1
// kernels with FP64 bundle reductions, device-side per-right-hand-side control (hooks), FP64
// reliable updates, and two drivers: host-driven iterations (residual flags read back every
// check_every iterations, as the per-iteration residual transfer of Sec. 2) and a single
// captured CUDA graph whose WHILE/IF conditional nodes keep the whole solve on the device.
#include <string.h>
#include <math.h>
#include <chrono>
#include <algorithm>

#include "hisq_internal.cuh"
#include "dslash_kernel.cuh"
#include "ds_arith.cuh"
#include "cg_persistent.cuh"

namespace hisq {


struct BlasArgs {
    int Vh, n, spb;
    void *x;          // Q: x_lo
    void *r;          // Q: r_lo
    void *p;          // P
    void *Ap;         // P
    void *z;          // P (flexible CG: preconditioned residual) or null
    void *r_old;      // Q (flexible CG)
    const void *b;    // FP64 (init)
    void *xhi;        // FP64
    void *xds;        // x_hi in double-single form, written with x_hi (null: not kept)
    RedArgs red;
    SolverState *st;
    const int *gate;
    const double *alpha_partials;  // plain CG: per-block <p, A p> partials of the A-operator
    int alpha_nblk;                // kernel (summed by every block of the update kernel)
};

template <int P>
__device__ __forceinline__ void load3(const VecView<P> &v, int s, int r, Cplx<typename Prec<P>::real> w[3]) {
    load_vec<P>(v, s, r, w);
}

// one thread per (site, rhs); red rows = sites per block
#define BLAS_PROLOGUE                                        \
    const int tid = threadIdx.x;                             \
    const int r = tid % a.n;                                 \
    const int sl = tid / a.n;

// init: x_hi = 0, x_lo = 0, r_lo = b, p = b, |b|^2 -> HOOK_INIT
template <int P>
__global__ void __launch_bounds__(256) cg_init_kernel(BlasArgs a) {
    constexpr int Q = q_prec(P);
    using rq = typename Prec<Q>::real;
    extern __shared__ double red[];
    BLAS_PROLOGUE
    auto vb = view<HISQ_FP64>(a.b, a.Vh, a.n);
    auto vxh = view<HISQ_FP64>(a.xhi, a.Vh, a.n);
    auto vx = view<Q>(a.x, a.Vh, a.n);
    auto vr = view<Q>(a.r, a.Vh, a.n);
    auto vp = view<P>(a.p, a.Vh, a.n);
    double acc = 0.0;
    for (int tile = blockIdx.x; (long)tile * a.spb < a.Vh; tile += gridDim.x) {
        int s = tile * a.spb + sl;
        if (s >= a.Vh || sl >= a.spb) continue;
        Cplx<double> b[3];
        load3<HISQ_FP64>(vb, s, r, b);
        Cplx<double> zero[3] = {{0, 0}, {0, 0}, {0, 0}};
        Cplx<rq> bq[3], zq[3] = {{0, 0}, {0, 0}, {0, 0}};
        Cplx<typename Prec<P>::real> bp[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            acc += b[c].re * b[c].re + b[c].im * b[c].im;
            bq[c] = {(rq)b[c].re, (rq)b[c].im};
            bp[c] = {(typename Prec<P>::real)b[c].re, (typename Prec<P>::real)b[c].im};
        }
        store_vec<HISQ_FP64>(vxh, s, r, zero);
        store_vec<Q>(vx, s, r, zq);
        store_vec<Q>(vr, s, r, bq);
        store_vec<P>(vp, s, r, bp);
    }
    const int rows = blockDim.x / a.n;
    for (int i = tid; i < rows * a.n; i += blockDim.x) red[i] = 0.0;
    __syncthreads();
    if (sl < rows) red[sl * a.n + r] = acc;
    block_reduce_finish(red, rows, a.n, a.n, a.red);
}

// Every block sums the A-operator kernel's per-block partials of <p, A p> in the same fixed order,
// so all blocks hold the identical alpha = |r|^2 / <p, A p> without waiting for one another.
// Writes alpha and the breakdown mask into shared memory (s_al, s_ok); red is scratch.
__device__ __forceinline__ void alpha_from_partials(const BlasArgs &a, double *red, double *s_al, int *s_ok) {
    const int tid = threadIdx.x, n = a.n;
    int np2 = 1;
    while (np2 < n) np2 *= 2;
    const int per = blockDim.x / np2, j = tid % np2, k = tid / np2;
    const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    double s = 0.0;
    if (j < n && k < per) {
#pragma unroll 4
        for (int b = k; b < a.alpha_nblk; b += per) s += __ldcg(a.alpha_partials + (size_t)b * n + j);
    }
    for (int off = 16; off >= np2; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const int groups = np2 < 32 ? nwarps : per;
    if (np2 < 32) {
        if (lane < np2) red[warp * np2 + lane] = s;
    } else {
        red[tid] = s;
    }
    __syncthreads();
    if (tid < n) {
        double pap = 0.0;
        for (int q = 0; q < groups; q++) pap += red[q * np2 + tid];
        const bool ok = pap > 0.0 && isfinite(pap);
        const double al = ok ? a.st->rr[tid] / pap : 0.0;
        s_ok[tid] = ok;
        s_al[tid] = al;
        if (blockIdx.x == 0) {  // record alpha and a breakdown for the host and the decision step
            a.st->alpha[tid][0] = al;
            a.st->alpha[tid][1] = 0.0;
            if (!ok && a.st->active[tid]) {
                a.st->active[tid] = 0;
                a.st->status[tid] = RHS_BREAKDOWN;
            }
        }
    }
    __syncthreads();
}

// x_lo += alpha p; r_lo -= alpha Ap; |r|^2 -> HOOK_DECIDE   (alpha complex for flexible CG)
template <int P>
__global__ void __launch_bounds__(256) cg_update_kernel(BlasArgs a) {
    constexpr int Q = q_prec(P);
    using rq = typename Prec<Q>::real;
    extern __shared__ double red[];
    __shared__ double s_al[HISQ_MAX_BUNDLE];
    __shared__ int s_ok[HISQ_MAX_BUNDLE];
    BLAS_PROLOGUE
    if (a.alpha_partials) alpha_from_partials(a, red, s_al, s_ok);
    auto vx = view<Q>(a.x, a.Vh, a.n);
    auto vr = view<Q>(a.r, a.Vh, a.n);
    auto vp = view<P>(a.p, a.Vh, a.n);
    auto vap = view<P>(a.Ap, a.Vh, a.n);
    const bool act = a.st->active[r] != 0 && (a.alpha_partials == nullptr || s_ok[r]);
    const rq al_re = a.alpha_partials ? (rq)s_al[r] : (rq)a.st->alpha[r][0];
    const rq al_im = a.alpha_partials ? (rq)0 : (rq)a.st->alpha[r][1];
    double acc = 0.0;
    if (act) {
        for (int tile = blockIdx.x; (long)tile * a.spb < a.Vh; tile += gridDim.x) {
            int s = tile * a.spb + sl;
            if (s >= a.Vh || sl >= a.spb) continue;
            Cplx<typename Prec<P>::real> p[3], ap[3];
            Cplx<rq> x[3], rv[3];
            load3<P>(vp, s, r, p);
            load3<P>(vap, s, r, ap);
            load3<Q>(vx, s, r, x);
            load3<Q>(vr, s, r, rv);
            rq part = 0;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                x[c].re += al_re * (rq)p[c].re - al_im * (rq)p[c].im;
                x[c].im += al_re * (rq)p[c].im + al_im * (rq)p[c].re;
                rv[c].re -= al_re * (rq)ap[c].re - al_im * (rq)ap[c].im;
                rv[c].im -= al_re * (rq)ap[c].im + al_im * (rq)ap[c].re;
                part += rv[c].re * rv[c].re + rv[c].im * rv[c].im;
            }
            acc += (double)part;
            store_vec<Q>(vx, s, r, x);
            store_vec<Q>(vr, s, r, rv);
        }
    }
    const int rows = blockDim.x / a.n;
    for (int i = tid; i < rows * a.n; i += blockDim.x) red[i] = 0.0;
    __syncthreads();
    if (sl < rows) red[sl * a.n + r] = acc;
    block_reduce_finish(red, rows, a.n, a.n, a.red);
}

// p = r + beta p for active right-hand sides (plain CG); a pure streaming kernel
template <int P>
__global__ void __launch_bounds__(256) cg_pupdate_kernel(BlasArgs a) {
    constexpr int Q = q_prec(P);
    using rp = typename Prec<P>::real;
    BLAS_PROLOGUE
    (void)tid;
    if (!a.st->active[r]) return;
    auto vr = view<Q>(a.r, a.Vh, a.n);
    auto vp = view<P>(a.p, a.Vh, a.n);
    const rp be = (rp)a.st->beta[r][0];
    for (int tile = blockIdx.x; (long)tile * a.spb < a.Vh; tile += gridDim.x) {
        int s = tile * a.spb + sl;
        if (s >= a.Vh || sl >= a.spb) continue;
        Cplx<typename Prec<Q>::real> rv[3];
        Cplx<rp> p[3];
        load3<Q>(vr, s, r, rv);
        load3<P>(vp, s, r, p);
#pragma unroll
        for (int c = 0; c < 3; c++) p[c] = {(rp)rv[c].re + be * p[c].re, (rp)rv[c].im + be * p[c].im};
        store_vec<P>(vp, s, r, p);
    }
}

// reliable update, first step: x_hi += x_lo; x_lo = 0 for right-hand sides flagged for update
template <int P>
__global__ void __launch_bounds__(256) cg_xhi_kernel(BlasArgs a) {
    constexpr int Q = q_prec(P);
    if (a.gate && *a.gate == 0) return;
    BLAS_PROLOGUE
    if (!a.st->update[r]) return;
    auto vx = view<Q>(a.x, a.Vh, a.n);
    auto vxh = view<HISQ_FP64>(a.xhi, a.Vh, a.n);
    for (int tile = blockIdx.x; (long)tile * a.spb < a.Vh; tile += gridDim.x) {
        int s = tile * a.spb + sl;
        if (s >= a.Vh || sl >= a.spb) continue;
        Cplx<typename Prec<Q>::real> x[3];
        Cplx<double> xh[3];
        load3<Q>(vx, s, r, x);
        load3<HISQ_FP64>(vxh, s, r, xh);
        Cplx<typename Prec<Q>::real> zero[3] = {{0, 0}, {0, 0}, {0, 0}};
#pragma unroll
        for (int c = 0; c < 3; c++) xh[c] = {xh[c].re + (double)x[c].re, xh[c].im + (double)x[c].im};
        store_vec<HISQ_FP64>(vxh, s, r, xh);
        store_vec<Q>(vx, s, r, zero);
        if (a.xds) {
            float4 *o = reinterpret_cast<float4 *>(a.xds);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float rh, rl, ih, il;
                ds_split(xh[c].re, rh, rl);
                ds_split(xh[c].im, ih, il);
                o[((long)s * 3 + c) * a.n + r] = make_float4(rh, rl, ih, il);
            }
        }
    }
}

// ---- flexible CG -------------------------------------------------------------------
// zz = z (network output) or r (after a stall fallback); dots <r - r_old, zz> -> HOOK_FCG_BETA
template <int P>
__global__ void __launch_bounds__(256) fcg_beta_kernel(BlasArgs a) {
    constexpr int Q = q_prec(P);
    using rq = typename Prec<Q>::real;
    extern __shared__ double red[];
    BLAS_PROLOGUE
    auto vr = view<Q>(a.r, a.Vh, a.n);
    auto vro = view<Q>(a.r_old, a.Vh, a.n);
    auto vz = view<P>(a.z, a.Vh, a.n);
    const bool act = a.st->active[r] != 0 && !a.st->restart[r];
    const bool use_r = a.st->fallback[r] != 0;
    double acc_re = 0.0, acc_im = 0.0;
    if (act) {
        for (int tile = blockIdx.x; (long)tile * a.spb < a.Vh; tile += gridDim.x) {
            int s = tile * a.spb + sl;
            if (s >= a.Vh || sl >= a.spb) continue;
            Cplx<rq> rv[3], ro[3];
            Cplx<typename Prec<P>::real> z[3];
            load3<Q>(vr, s, r, rv);
            load3<Q>(vro, s, r, ro);
            if (use_r) {
#pragma unroll
                for (int c = 0; c < 3; c++) z[c] = {(typename Prec<P>::real)rv[c].re, (typename Prec<P>::real)rv[c].im};
            } else {
                load3<P>(vz, s, r, z);
            }
            rq pre = 0, pim = 0;
#pragma unroll
            for (int c = 0; c < 3; c++) {  // conj(r - r_old) z
                rq dre = rv[c].re - ro[c].re, dim = rv[c].im - ro[c].im;
                pre += dre * (rq)z[c].re + dim * (rq)z[c].im;
                pim += dre * (rq)z[c].im - dim * (rq)z[c].re;
            }
            acc_re += (double)pre;
            acc_im += (double)pim;
        }
    }
    const int rows = blockDim.x / a.n;
    for (int i = tid; i < rows * 2 * a.n; i += blockDim.x) red[i] = 0.0;
    __syncthreads();
    if (sl < rows) {
        red[sl * 2 * a.n + 2 * r] = acc_re;
        red[sl * 2 * a.n + 2 * r + 1] = acc_im;
    }
    block_reduce_finish(red, rows, 2 * a.n, a.n, a.red);
}

// p = zz + beta p (complex beta); r_old = r; dots <p, r> -> HOOK_FCG_PR
template <int P>
__global__ void __launch_bounds__(256) fcg_pupdate_kernel(BlasArgs a) {
    constexpr int Q = q_prec(P);
    using rq = typename Prec<Q>::real;
    using rp = typename Prec<P>::real;
    extern __shared__ double red[];
    BLAS_PROLOGUE
    auto vr = view<Q>(a.r, a.Vh, a.n);
    auto vro = view<Q>(a.r_old, a.Vh, a.n);
    auto vz = view<P>(a.z, a.Vh, a.n);
    auto vp = view<P>(a.p, a.Vh, a.n);
    const bool act = a.st->active[r] != 0;
    const bool use_r = a.st->fallback[r] != 0;
    const rp b_re = (rp)a.st->beta[r][0], b_im = (rp)a.st->beta[r][1];
    double acc_re = 0.0, acc_im = 0.0;
    if (act) {
        for (int tile = blockIdx.x; (long)tile * a.spb < a.Vh; tile += gridDim.x) {
            int s = tile * a.spb + sl;
            if (s >= a.Vh || sl >= a.spb) continue;
            Cplx<rq> rv[3];
            Cplx<rp> z[3], p[3];
            load3<Q>(vr, s, r, rv);
            load3<P>(vp, s, r, p);
            if (use_r) {
#pragma unroll
                for (int c = 0; c < 3; c++) z[c] = {(rp)rv[c].re, (rp)rv[c].im};
            } else {
                load3<P>(vz, s, r, z);
            }
            rq pre = 0, pim = 0;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                p[c] = {z[c].re + b_re * p[c].re - b_im * p[c].im, z[c].im + b_re * p[c].im + b_im * p[c].re};
                pre += (rq)p[c].re * rv[c].re + (rq)p[c].im * rv[c].im;   // conj(p) r
                pim += (rq)p[c].re * rv[c].im - (rq)p[c].im * rv[c].re;
            }
            acc_re += (double)pre;
            acc_im += (double)pim;
            store_vec<P>(vp, s, r, p);
            store_vec<Q>(vro, s, r, rv);
        }
    }
    const int rows = blockDim.x / a.n;
    for (int i = tid; i < rows * 2 * a.n; i += blockDim.x) red[i] = 0.0;
    __syncthreads();
    if (sl < rows) {
        red[sl * 2 * a.n + 2 * r] = acc_re;
        red[sl * 2 * a.n + 2 * r + 1] = acc_im;
    }
    block_reduce_finish(red, rows, 2 * a.n, a.n, a.red);
}


// ------------------------------------------------------------------------------------------
// Workspace
// ------------------------------------------------------------------------------------------
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    const hisq_links *fat = nullptr, *naik = nullptr;
    const hisq_pc *pc = nullptr;
    int pc_form = -1;
    double mass = 0;
    unsigned long long h_loop = 0, h_upd = 0;  // the graph's conditional handles
    int n = 0, prec = -1;
    unsigned tune_generation = 0;
};

struct Workspace {
    int cap_n = 0;
    int prec = -1;
    void *b_hi = nullptr, *x_hi = nullptr, *x_lo = nullptr, *r_lo = nullptr, *p = nullptr, *Ap = nullptr;
    void *t = nullptr, *t64 = nullptr, *z = nullptr, *r_old = nullptr;
    void *x_ds = nullptr;         // x_hi in double-single form: input of the residual recomputation
    double *canon = nullptr;      // canonical FP64 staging [cap_n][Vh][6]
    SolverState *st = nullptr;    // device
    SolverState *h_st = nullptr;  // pinned host mirror
    double *partials = nullptr;
    size_t partials_cap = 0;
    double *partials2 = nullptr;   // the A-operator's <p, A p> partials (summed by the update kernel)
    int d2_grid = 0;               // blocks of the last A-operator launch enqueued
    unsigned int *counter = nullptr;
    double *dots = nullptr;
    unsigned int *bar = nullptr;   // persistent solve: the grid barrier's counter word
    int *err = nullptr;            // persistent solve: a barrier wait ran out
    unsigned long long *phase_ns = nullptr;  // persistent solve: per-phase time (time_kernels)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    GraphCache gc;
};

void free_graph(GraphCache &gc) {
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    if (gc.graph) cudaGraphDestroy(gc.graph);
    gc = GraphCache();
}

static void free_buffers(Workspace *w) {
    void *bufs[] = {w->b_hi, w->x_hi, w->x_lo, w->r_lo, w->p, w->Ap, w->t, w->t64, w->z, w->r_old, w->x_ds, w->canon};
    for (void *b : bufs)
        if (b) cudaFree(b);
    w->b_hi = w->x_hi = w->x_lo = w->r_lo = w->p = w->Ap = w->t = w->t64 = w->z = w->r_old = w->x_ds = nullptr;
    w->canon = nullptr;
    w->cap_n = 0;
    w->prec = -1;
    free_graph(w->gc);
}

static int ensure_workspace(hisq_ctx *ctx, int n, int prec, bool need_pc) {
    if (!ctx->ws) {
        Workspace *w = new Workspace();
        ctx->ws = w;
        size_t pcap = (size_t)ctx->num_sms * 64 * HISQ_MAX_BUNDLE * 4;
        if (cudaMalloc(&w->st, sizeof(SolverState)) != cudaSuccess ||
            cudaMallocHost(&w->h_st, sizeof(SolverState)) != cudaSuccess ||
            cudaMalloc(&w->partials, pcap * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&w->partials2, pcap * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&w->counter, sizeof(unsigned int) * 4) != cudaSuccess ||
            cudaMalloc(&w->dots, sizeof(double) * HISQ_MAX_BUNDLE * 4) != cudaSuccess ||
            cudaMalloc(&w->bar, sizeof(unsigned int) * 4) != cudaSuccess ||
            cudaMalloc(&w->err, sizeof(int) * 4) != cudaSuccess ||
            cudaMalloc(&w->phase_ns, sizeof(unsigned long long) * 8) != cudaSuccess)
            return set_error(HISQ_ERR_NOMEM, "solver workspace allocation failed");
        w->partials_cap = pcap;
        cudaMemset(w->counter, 0, sizeof(unsigned int) * 4);
        memset(w->h_st, 0, sizeof(SolverState));
        cudaEventCreate(&w->ev0);
        cudaEventCreate(&w->ev1);
    }
    Workspace *w = ctx->ws;
    bool have_pc = w->z != nullptr;
    if (w->cap_n >= n && w->prec == prec && (!need_pc || have_pc)) return HISQ_OK;
    int cap = std::max(n, w->cap_n);
    free_buffers(w);
    int Vh = ctx->geom.Vh;
    int Q = q_prec(prec);
    struct { void **ptr; size_t bytes; } allocs[] = {
        {&w->b_hi, vector_bytes(HISQ_FP64, Vh, cap)}, {&w->x_hi, vector_bytes(HISQ_FP64, Vh, cap)},
        {&w->x_lo, vector_bytes(Q, Vh, cap)},         {&w->r_lo, vector_bytes(Q, Vh, cap)},
        {&w->p, vector_bytes(prec, Vh, cap)},         {&w->Ap, vector_bytes(prec, Vh, cap)},
        {&w->t, vector_bytes(prec, Vh, cap)},         {&w->t64, vector_bytes(HISQ_FP64, Vh, cap)},
        {&w->x_ds, vector_bytes(HISQ_DS, Vh, cap)},
        {(void **)&w->canon, (size_t)cap * Vh * 6 * sizeof(double)},
    };
    for (auto &a : allocs)
        if (cudaMalloc(a.ptr, a.bytes) != cudaSuccess) {
            free_buffers(w);
            return set_error(HISQ_ERR_NOMEM, "cannot allocate %zu bytes of solver workspace", a.bytes);
        }
    if (need_pc) {
        if (cudaMalloc(&w->z, vector_bytes(prec, Vh, cap)) != cudaSuccess ||
            cudaMalloc(&w->r_old, vector_bytes(Q, Vh, cap)) != cudaSuccess) {
            free_buffers(w);
            return set_error(HISQ_ERR_NOMEM, "cannot allocate flexible-CG workspace");
        }
    }
    w->cap_n = cap;
    w->prec = prec;
    return HISQ_OK;
}

void free_workspace(hisq_ctx *ctx) {
    if (!ctx->ws) return;
    Workspace *w = ctx->ws;
    free_buffers(w);
    if (w->st) cudaFree(w->st);
    if (w->h_st) cudaFreeHost(w->h_st);
    if (w->partials) cudaFree(w->partials);
    if (w->partials2) cudaFree(w->partials2);
    if (w->counter) cudaFree(w->counter);
    if (w->dots) cudaFree(w->dots);
    if (w->bar) cudaFree(w->bar);
    if (w->err) cudaFree(w->err);
    if (w->phase_ns) cudaFree(w->phase_ns);
    if (w->ev0) cudaEventDestroy(w->ev0);
    if (w->ev1) cudaEventDestroy(w->ev1);
    delete w;
    ctx->ws = nullptr;
}

// ------------------------------------------------------------------------------------------
// Enqueueing the steps of one bundle solve
// ------------------------------------------------------------------------------------------
struct Solve {
    hisq_ctx *ctx;
    Workspace *w;
    const hisq_links *fat, *naik;
    int n, prec;
    double mass;
    cudaStream_t st;
    bool timing;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *events;    // inner-precision Dslash
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *events64;  // FP64 Dslash
    const hisq_pc *pc;                                           // flexible CG when set
    bool persistent = false;                                     // solved by the persistent kernel
    bool pers_timing = false;        // time the persistent kernel (CUDA events) and its phases
    hisq_solve_stats *stats = nullptr;
    const double *mass2v = nullptr;  // per right-hand side m^2 (shifted systems; persistent driver only)
    const double *tolv = nullptr;    // per right-hand side relative tolerance (or null: the solve's tol)
    int hp = LINKS_FP64;             // links and arithmetic of the residual recomputation (LINKS_DS
                                     // for mixed precision, LINKS_FP64 for plain FP64 solves)
};

static BlasArgs blas_args(const Solve &S) {
    BlasArgs a;
    memset(&a, 0, sizeof(a));
    a.Vh = S.ctx->geom.Vh;
    a.n = S.n;
    a.spb = std::max(1, 256 / S.n);
    int p2 = 1;
    while (p2 * 2 <= a.spb) p2 *= 2;
    a.spb = p2;
    a.x = S.w->x_lo;
    a.r = S.w->r_lo;
    a.p = S.w->p;
    a.Ap = S.w->Ap;
    a.z = S.w->z;
    a.r_old = S.w->r_old;
    a.b = S.w->b_hi;
    a.xhi = S.w->x_hi;
    a.xds = S.hp == LINKS_DS ? S.w->x_ds : nullptr;
    a.red.partials = S.w->partials;
    a.red.counter = S.w->counter;
    a.red.dot_out = S.w->dots;
    a.red.st = S.w->st;
    a.st = S.w->st;
    return a;
}

template <typename K>
static int launch_blas(const Solve &S, K kernel, BlasArgs a, int hook, bool reduce) {
    int threads = (a.spb * a.n + 31) / 32 * 32;  // whole warps; rows beyond spb idle
    size_t smem = reduce ? (size_t)(2 * threads + 64) * sizeof(double) : 0;  // red[rows][2n] and the final sums
    long tiles = (a.Vh + a.spb - 1) / a.spb;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    long grid = balanced_grid(tiles, (long)std::min(std::max(per_sm, 1), 4) * S.ctx->num_sms);
    if ((size_t)grid * a.n * 2 > S.w->partials_cap) grid = S.w->partials_cap / (a.n * 2);
    a.red.hook = hook;
    kernel<<<(int)grid, threads, smem, S.st>>>(a);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

template <int P>
static int enqueue_blas(const Solve &S, int which) {
    BlasArgs a = blas_args(S);
    switch (which) {
    case HOOK_INIT: return launch_blas(S, cg_init_kernel<P>, a, HOOK_INIT, true);
    case HOOK_DECIDE:
        if (!S.pc) {  // plain CG: alpha from the A-operator's partials, summed in every block
            a.alpha_partials = S.w->partials2;
            a.alpha_nblk = S.w->d2_grid;
        }
        return launch_blas(S, cg_update_kernel<P>, a, HOOK_DECIDE, true);
    case HOOK_LOOP: return launch_blas(S, cg_pupdate_kernel<P>, a, HOOK_NONE, false);
    case HOOK_FCG_BETA: return launch_blas(S, fcg_beta_kernel<P>, a, HOOK_FCG_BETA, true);
    case HOOK_FCG_PR: return launch_blas(S, fcg_pupdate_kernel<P>, a, HOOK_FCG_PR, true);
    default: {
        a.gate = &S.w->st->any_update;
        return launch_blas(S, cg_xhi_kernel<P>, a, HOOK_NONE, false);
    }
    }
}

static int blas(const Solve &S, int which) {
    switch (S.prec) {
    case HISQ_FP64: return enqueue_blas<HISQ_FP64>(S, which);
    case HISQ_FP32: return enqueue_blas<HISQ_FP32>(S, which);
    case HISQ_FP16: return enqueue_blas<HISQ_FP16>(S, which);
    default: return enqueue_blas<HISQ_BF16>(S, which);
    }
}

static int dslash_step(const Solve &S, DslashArgs d, int copy, int *grid_out = nullptr) {
    if (!d.partials_only) d.partials = S.w->partials;
    d.partials_cap = S.w->partials_cap;
    d.counter = S.w->counter;
    d.dot_out = S.w->dots;
    d.hook_state = S.w->st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (S.timing) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, S.st);
    }
    int rc = launch_dslash(S.ctx, S.fat, S.naik, copy, d, nullptr, S.st, grid_out);
    if (S.timing) {
        cudaEventRecord(e1, S.st);
        (copy != LINKS_INNER ? S.events64 : S.events)->push_back({e0, e1});
    }
    return rc;
}

// the reliable update: x_hi += x_lo; t64 = D_oe x_hi; r_lo = b - A x_hi (FP64 accuracy: double-
// single Dslash on the ds copy of x_hi, FP64 epilogue; native FP64 for plain FP64 solves)
// -> HOOK_RELIABLE
static int enqueue_update(const Solve &S) {
    HISQ_CHECK(blas(S, -1));
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.n = S.n;
    d.in = S.hp == LINKS_DS ? S.w->x_ds : S.w->x_hi;
    d.out = S.w->t64;
    d.parity = 1;
    d.epi = EPI_PLAIN;
    d.active = S.w->st->update;
    d.gate = &S.w->st->any_update;
    HISQ_CHECK(dslash_step(S, d, S.hp));
    d.in = S.w->t64;
    d.out = nullptr;
    d.parity = 0;
    d.epi = EPI_RESID;
    d.mass2 = S.mass * S.mass;
    d.axpy_in = S.w->x_hi;
    d.b = S.w->b_hi;
    d.out_lo = S.w->r_lo;
    d.lo_prec = q_prec(S.prec);
    d.hook = HOOK_RELIABLE;
    return dslash_step(S, d, S.hp);
}

// one CG iteration up to the decision: t = D_oe p; Ap = m^2 p - D_eo t (pAp -> alpha);
// x += alpha p, r -= alpha Ap (|r|^2 -> decide)
static int enqueue_iteration_head(const Solve &S) {
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.n = S.n;
    d.in = S.w->p;
    d.out = S.w->t;
    d.parity = 1;
    d.epi = EPI_PLAIN;
    d.active = S.w->st->active;
    const int sloppy64 = S.prec == HISQ_FP64 ? LINKS_FP64 : LINKS_INNER;  // plain FP64 CG reads the FP64 link copy
    HISQ_CHECK(dslash_step(S, d, sloppy64));
    d.in = S.w->t;
    d.out = S.w->Ap;
    d.parity = 0;
    d.epi = EPI_AOP;
    d.mass2 = S.mass * S.mass;
    d.axpy_in = S.w->p;
    if (S.pc) {
        d.hook = HOOK_FCG_ALPHA;
        HISQ_CHECK(dslash_step(S, d, sloppy64));
    } else {
        // plain CG: publish <p, A p> per block; the update kernel finishes the sum
        d.hook = HOOK_NONE;
        d.partials_only = 1;
        d.partials = S.w->partials2;
        HISQ_CHECK(dslash_step(S, d, sloppy64, &S.w->d2_grid));
    }
    return blas(S, HOOK_DECIDE);
}

// flexible CG: z = M r (network); beta; p = z + beta p with <p, r>; then the CG head
static int enqueue_fcg_head(const Solve &S) {
    // the Hermitian part of the network keeps the preconditioned recurrence a true PCG one
    HISQ_CHECK(pc_forward_precond(S.ctx, S.pc, S.fat, S.naik, S.w->r_lo, S.w->z, S.n, S.st));
    HISQ_CHECK(blas(S, HOOK_FCG_BETA));
    HISQ_CHECK(blas(S, HOOK_FCG_PR));
    return enqueue_iteration_head(S);
}

static int enqueue_head(const Solve &S) { return S.pc ? enqueue_fcg_head(S) : enqueue_iteration_head(S); }

// end of an iteration: plain CG updates p here; flexible CG only advances the loop
static int enqueue_tail(const Solve &S) {
    if (!S.pc) return blas(S, HOOK_LOOP);
    return HISQ_OK;  // flexible CG builds its direction at the start of the next iteration
}

static int enqueue_setup(const Solve &S) {
    // b_hi from the canonical staging, then x = 0, r = p = b and |b|^2
    HISQ_CHECK(pack_vectors(S.ctx, S.w->canon, S.w->b_hi, S.n, HISQ_FP64, S.st));
    return blas(S, HOOK_INIT);
}

// The reliable-update threshold when the caller leaves it to the library.  Between updates the
// iterated residual follows b - A' x with A' the operator of the links in the storage precision,
// so it drifts from the true residual by about (A - A') x_lo, a multiple of the storage rounding;
// an update threshold below that drift makes the iterated residual reach the tolerance while the
// true one has not, and every such false convergence costs a recomputation.  Measured at 32^3 x 8
// (m = 0.01) and 64^3 x 16 (m = 0.002): FP16 storage breaks down below 0.003, BF16 below 0.03, FP32
// not down to 0.001; each default sits about ten times above its breakdown (at FP16 and 64^3 x 16,
// 0.01 already costs more in added iterations than it saves in recomputations).
static double default_delta(int prec) {
    switch (prec) {
    case HISQ_FP32: return 0.01;
    case HISQ_FP16: return 0.03;
    default: return 0.1;
    }
}

static int set_state_params(const Solve &S, unsigned long long h_loop, unsigned long long h_upd, double tol) {
    const hisq_solver_params &P = S.ctx->params;
    SolverState *h = S.w->h_st;
    memset(h, 0, sizeof(SolverState));
    h->n = S.n;
    h->max_iter = P.max_iter;
    h->inner_fp64 = S.prec == HISQ_FP64;
    h->use_pc = S.pc != nullptr;
    h->stall_window = P.stall_window;
    h->stall_factor = P.stall_factor;
    for (int k = 0; k < S.n; k++) {
        h->tolk[k] = (S.tolv ? S.tolv[k] : tol) * TOL_SAFETY;
        h->mass2[k] = S.mass2v ? S.mass2v[k] : S.mass * S.mass;
    }
    h->delta = P.delta > 0.0 ? P.delta : default_delta(S.prec);
    h->h_loop = h_loop;
    h->h_upd = h_upd;
    h->cond_loop = 1;  // the defaults the graph assigns at launch
    h->cond_upd = 0;
    HISQ_CUDA(cudaMemcpyAsync(S.w->st, h, sizeof(SolverState), cudaMemcpyHostToDevice, S.st));
    return HISQ_OK;
}

// ---- graph capture with conditional nodes ----------------------------------------------------
static int add_conditional(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                           cudaGraph_t *body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t *deps;
    const cudaGraphEdgeData *edges;
    size_t ndeps;
    HISQ_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edges, &ndeps));
    if (cs != cudaStreamCaptureStatusActive) return set_error(HISQ_ERR_CUDA, "stream is not capturing");
    cudaGraphNodeParams params = {cudaGraphNodeTypeConditional};
    params.conditional.handle = h;
    params.conditional.type = type;
    params.conditional.size = 1;
    cudaGraphNode_t node;
    HISQ_CUDA(cudaGraphAddNode(&node, g, deps, edges, ndeps, &params));
    *body = params.conditional.phGraph_out[0];
    HISQ_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return HISQ_OK;
}

static int build_graph(const Solve &S) {
    Workspace *w = S.w;
    free_graph(w->gc);
    cudaGraph_t graph;
    HISQ_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h_loop, h_upd;
    HISQ_CUDA(cudaGraphConditionalHandleCreate(&h_loop, graph, 1, cudaGraphCondAssignDefault));
    HISQ_CUDA(cudaGraphConditionalHandleCreate(&h_upd, graph, 0, cudaGraphCondAssignDefault));
    cudaStream_t cap;
    HISQ_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int rc = HISQ_OK;
    Solve C = S;
    C.st = cap;
    C.timing = false;
    // the state parameters (including the handles) are copied before the graph launch, so the
    // graph itself only holds: setup; WHILE(loop) { head; IF(update) { update }; p-update }
    cudaError_t e = cudaStreamBeginCaptureToGraph(cap, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    cudaGraph_t while_body = nullptr;
    if (rc == HISQ_OK) rc = enqueue_setup(C);
    if (rc == HISQ_OK) rc = add_conditional(cap, h_loop, cudaGraphCondTypeWhile, &while_body);
    cudaGraph_t outg;
    e = cudaStreamEndCapture(cap, &outg);
    if (rc == HISQ_OK && e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    // WHILE body: head; IF node; p-update
    cudaGraph_t if_body = nullptr;
    if (rc == HISQ_OK) {
        e = cudaStreamBeginCaptureToGraph(cap, while_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "loop capture failed: %s", cudaGetErrorString(e));
        if (rc == HISQ_OK) rc = enqueue_head(C);
        if (rc == HISQ_OK) rc = add_conditional(cap, h_upd, cudaGraphCondTypeIf, &if_body);
        if (rc == HISQ_OK) rc = enqueue_tail(C);
        e = cudaStreamEndCapture(cap, &outg);
        if (rc == HISQ_OK && e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "loop capture failed: %s", cudaGetErrorString(e));
    }
    if (rc == HISQ_OK) {
        e = cudaStreamBeginCaptureToGraph(cap, if_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "update capture failed: %s", cudaGetErrorString(e));
        if (rc == HISQ_OK) rc = enqueue_update(C);
        e = cudaStreamEndCapture(cap, &outg);
        if (rc == HISQ_OK && e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "update capture failed: %s", cudaGetErrorString(e));
    }
    cudaStreamDestroy(cap);
    if (rc == HISQ_OK) {
        e = cudaGraphInstantiate(&w->gc.exec, graph, 0);
        if (e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    if (rc != HISQ_OK) {
        cudaGraphDestroy(graph);
        w->gc = GraphCache();
        cudaGetLastError();
        return rc;
    }
    w->gc.graph = graph;
    w->gc.h_loop = (unsigned long long)h_loop;
    w->gc.h_upd = (unsigned long long)h_upd;
    w->gc.fat = S.fat;
    w->gc.naik = S.naik;
    w->gc.mass = S.mass;
    w->gc.n = S.n;
    w->gc.prec = S.prec;
    w->gc.pc = S.pc;
    w->gc.pc_form = S.pc ? S.pc->form : -1;
    w->gc.tune_generation = S.ctx->tune_generation;
    return HISQ_OK;
}

// ------------------------------------------------------------------------------------------
// Persistent driver: the whole plain-CG solve of a bundle in one cooperative launch
// ------------------------------------------------------------------------------------------
// L2 residency of one link field during a persistent solve.  Every iteration reads the inner-
// precision fat and Naik links once per Dslash, 182 times in a typical solve; when the Naik copy
// fits the device's persisting set-aside whole (at 32^3 x 8 with 16-bit storage, 75 MB of the
// 129 MB L2) it is marked persisting through the stream's access-policy window, and only the
// other field and the vectors stream from HBM.  The
// set-aside is reserved once per context (restored by hisq_finalize) and the persisting lines are
// released after each solve, so no solve starts with links left in L2 by another.
static bool l2_window_begin(hisq_ctx *ctx, cudaStream_t st, const hisq_links *links) {
    if (!ctx->params.l2_persist_links || !links->words) return false;
    if (ctx->l2_persist_max < 0) {
        int maxp = 0, maxw = 0;
        if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, ctx->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device) != cudaSuccess) {
            cudaGetLastError();
            maxp = maxw = 0;
        }
        ctx->l2_persist_max = maxp;
        ctx->l2_window_max = maxw;
    }
    if (ctx->l2_persist_max <= 0 || ctx->l2_window_max <= 0) return false;
    const size_t bytes = (size_t)2 * links->W * ctx->geom.Vh * sizeof(uint4);
    // only a field that fits the set-aside whole: a window of partial hits takes L2 from the
    // vectors for little (48^3 x 12 FP32: 764 MB of Naik links against 85 MB made the solve 7%
    // slower)
    if (bytes > (size_t)ctx->l2_persist_max) return false;
    if (!ctx->l2_limit_saved) {
        size_t old = 0;
        if (cudaDeviceGetLimit(&old, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        ctx->l2_limit_old = old;
        ctx->l2_limit_saved = true;
    }
    const size_t carve = std::min((size_t)ctx->l2_persist_max, bytes);
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) cudaGetLastError();
    if (cur != carve && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, carve) != cudaSuccess) {
        cudaGetLastError();  // the set-aside is reconfigured only when it changes
        return false;
    }
    cudaStreamAttrValue v;
    memset(&v, 0, sizeof(v));
    v.accessPolicyWindow.base_ptr = (void *)links->words;
    v.accessPolicyWindow.num_bytes = std::min(bytes, (size_t)ctx->l2_window_max);
    v.accessPolicyWindow.hitRatio = std::min(1.0f, (float)carve / (float)v.accessPolicyWindow.num_bytes);
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    if (cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &v) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

static void l2_window_end(cudaStream_t st) {
    cudaStreamAttrValue v;
    memset(&v, 0, sizeof(v));
    v.accessPolicyWindow.num_bytes = 0;
    if (cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &v) != cudaSuccess) cudaGetLastError();
}

static cudaError_t persistent_occ(int prec, int R, bool cg1, int threads, size_t smem, int *per_sm) {
    switch (prec) {
    case HISQ_FP64: return persistent_occupancy<HISQ_FP64>(R, cg1, threads, smem, per_sm);
    case HISQ_FP32: return persistent_occupancy<HISQ_FP32>(R, cg1, threads, smem, per_sm);
    case HISQ_FP16: return persistent_occupancy<HISQ_FP16>(R, cg1, threads, smem, per_sm);
    default: return persistent_occupancy<HISQ_BF16>(R, cg1, threads, smem, per_sm);
    }
}

static cudaError_t persistent_launch(int prec, const PersArgs &a, int R, bool cg1, int grid, int threads, size_t smem,
                                     cudaStream_t st) {
    switch (prec) {
    case HISQ_FP64: return launch_persistent_prec<HISQ_FP64>(a, R, cg1, grid, threads, smem, st);
    case HISQ_FP32: return launch_persistent_prec<HISQ_FP32>(a, R, cg1, grid, threads, smem, st);
    case HISQ_FP16: return launch_persistent_prec<HISQ_FP16>(a, R, cg1, grid, threads, smem, st);
    default: return launch_persistent_prec<HISQ_BF16>(a, R, cg1, grid, threads, smem, st);
    }
}

// Runs the bundle in the persistent kernel when it applies (plain CG, 18-real Naik links and a
// co-resident grid); *done = false leaves the bundle to the graph driver.
static int solve_bundle_persistent(Solve &S, double tol, bool *done) {
    *done = false;
    if (S.pc || S.naik->recon != 18) return HISQ_OK;
    Workspace *w = S.w;
    LaunchShape sh = tuned_shape(S.ctx, S.fat, S.naik, S.n, S.prec == HISQ_FP64 ? LINKS_FP64 : LINKS_INNER);
    int R = sh.R > 4 ? 4 : sh.R;
    if (S.prec == HISQ_FP64 && R > 2) R = 2;  // four FP64 right-hand sides per thread would spill
    // four FP32 right-hand sides per thread fit the separate Dslash kernel (up to 255 registers) but
    // not the persistent kernel's 128: measured at 48^3 x 12, bundles of 4 and 16, two per thread
    // run the persistent solve 1.6x and 1.3x faster than four (and faster than the graph driver);
    // BF16 (its vectors unpacked by shifts, one register per value) 5% faster at 64^3 x 16 and 16
    // right-hand sides.  FP16 keeps four (its records unpack into packed pairs): 3% faster there.
    if ((S.prec == HISQ_FP32 || S.prec == HISQ_BF16) && R > 2) R = 2;
    while (S.n % R) R /= 2;
    // block size: the parameter if set (a multiple of 32 up to the kernel's bound), else 512
    int threads = std::min(pers_threads(R), PERS_DEFAULT_THREADS);
    const int want = S.ctx->params.persistent_threads;
    if (want >= 32 && want <= pers_threads(R) && want % 32 == 0) threads = want;
    const size_t smem = (size_t)(4 * threads * R + 64) * sizeof(double);  // four dot sets (single reduction)
    int per_sm = 0;
    const bool cg1 = S.ctx->params.single_reduction != 0;
    if (persistent_occ(S.prec, R, cg1, threads, smem, &per_sm) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return HISQ_OK;
    }
    const int grid = per_sm * S.ctx->num_sms;  // one wave: every block resident (cooperative launch)
    if ((size_t)grid * PERS_ND > w->partials_cap) return HISQ_OK;
    PersArgs a;
    memset(&a, 0, sizeof(a));
    a.g = S.ctx->geom;
    a.fat = S.fat->field();
    a.naik = S.naik->field();
    if (S.prec == HISQ_FP64) {
        a.fat64 = S.fat->field64();
        a.naik64 = S.naik->field64();
        a.fat = a.fat64;
        a.naik = a.naik64;
    } else {
        // the residual recomputation in double-single arithmetic on the ds link copies
        a.fat64 = S.fat->field_ds();
        a.naik64 = S.naik->field_ds();
        a.xds = w->x_ds;
    }
    a.p = w->p;
    a.t = w->t;
    a.ap = w->Ap;
    a.x = w->x_lo;
    a.r = w->r_lo;
    a.b = w->b_hi;
    a.xhi = w->x_hi;
    a.t64 = w->t64;
    a.n = S.n;
    a.partials = w->partials;
    a.st = w->st;
    a.bar = w->bar;
    a.err = w->err;
    a.spin_limit = 1LL << 22;  // a barrier wait gives up after about a second
    a.expected = grid;
    if (S.ctx->params.debug_barrier_timeout) {  // test hook: no barrier can complete
        a.expected = grid + 1;
        a.spin_limit = 1LL << 12;
    }
    HISQ_CHECK(set_state_params(S, 0, 0, tol));
    HISQ_CHECK(pack_vectors(S.ctx, w->canon, w->b_hi, S.n, HISQ_FP64, S.st));
    HISQ_CUDA(cudaMemsetAsync(w->bar, 0, sizeof(unsigned int) * 4, S.st));
    HISQ_CUDA(cudaMemsetAsync(w->err, 0, sizeof(int) * 4, S.st));
    if (S.pers_timing) {
        a.phase_ns = w->phase_ns;
        HISQ_CUDA(cudaMemsetAsync(w->phase_ns, 0, sizeof(unsigned long long) * 8, S.st));
        HISQ_CUDA(cudaEventRecord(w->ev0, S.st));
    }
    const bool l2 = l2_window_begin(S.ctx, S.st, S.naik);
    cudaError_t e = persistent_launch(S.prec, a, R, cg1, grid, threads, smem, S.st);
    if (l2) l2_window_end(S.st);
    if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
        cudaGetLastError();
        return HISQ_OK;  // not co-resident here: the graph driver takes the bundle
    }
    if (e != cudaSuccess) return set_error(HISQ_ERR_CUDA, "persistent solve launch failed: %s", cudaGetErrorString(e));
    if (S.pers_timing) HISQ_CUDA(cudaEventRecord(w->ev1, S.st));
    int err_h = 0;
    unsigned long long ph[8] = {0};
    HISQ_CUDA(cudaMemcpyAsync(w->h_st, w->st, sizeof(SolverState), cudaMemcpyDeviceToHost, S.st));
    HISQ_CUDA(cudaMemcpyAsync(&err_h, w->err, sizeof(int), cudaMemcpyDeviceToHost, S.st));
    if (S.pers_timing) HISQ_CUDA(cudaMemcpyAsync(ph, w->phase_ns, sizeof(ph), cudaMemcpyDeviceToHost, S.st));
    HISQ_CUDA(cudaStreamSynchronize(S.st));
    if (l2) cudaCtxResetPersistingL2Cache();  // the next solve (or any other kernel) starts from a normal L2
    if (err_h) return set_error(HISQ_ERR_TIMEOUT, "a grid barrier of the persistent solve ran out of its wait budget");
    if (S.pers_timing && S.stats) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, w->ev0, w->ev1) == cudaSuccess) {
            S.stats->solve_kernel_ms += ms;
            S.stats->solve_kernel_launches++;
        }
        for (int i = 0; i < PERS_PHASES; i++) S.stats->phase_ms[i] += (double)ph[i] * 1e-6;
    }
    *done = true;
    return HISQ_OK;
}

// ------------------------------------------------------------------------------------------
// One bundle
// ------------------------------------------------------------------------------------------
static int solve_bundle(Solve &S, double tol) {
    Workspace *w = S.w;
    const hisq_solver_params &P = S.ctx->params;
    if ((P.use_graph == 2 && !S.timing) || S.mass2v) {
        bool done = false;
        HISQ_CHECK(solve_bundle_persistent(S, tol, &done));
        if (done) {
            S.persistent = true;
            return HISQ_OK;
        }
        if (S.mass2v) return set_error(HISQ_ERR_ARG, "a bundle of shifted systems needs the persistent driver");
    }
    bool graph = P.use_graph && !S.timing;
    if (graph) {
        bool reuse = w->gc.exec && w->gc.fat == S.fat && w->gc.naik == S.naik && w->gc.mass == S.mass &&
                     w->gc.n == S.n && w->gc.prec == S.prec && w->gc.pc == S.pc &&
                     w->gc.pc_form == (S.pc ? S.pc->form : -1) &&
                     w->gc.tune_generation == S.ctx->tune_generation;
        if (!reuse) HISQ_CHECK(build_graph(S));
        // the handles live with the graph, not in the state mirror (which every driver rewrites):
        // the device ends the WHILE loop only through them, so a graph never runs without both
        const unsigned long long hl = w->gc.h_loop, hu = w->gc.h_upd;
        if (!hl || !hu) return set_error(HISQ_ERR_STATE, "captured solve graph without its conditional handles");
        HISQ_CHECK(set_state_params(S, hl, hu, tol));
        HISQ_CUDA(cudaGraphLaunch(w->gc.exec, S.st));
        HISQ_CUDA(cudaMemcpyAsync(w->h_st, w->st, sizeof(SolverState), cudaMemcpyDeviceToHost, S.st));
        HISQ_CUDA(cudaStreamSynchronize(S.st));
        return HISQ_OK;
    }
    HISQ_CHECK(set_state_params(S, 0, 0, tol));
    HISQ_CHECK(enqueue_setup(S));
    int check = std::max(1, P.check_every);
    for (int it = 0; it < P.max_iter; it++) {
        HISQ_CHECK(enqueue_head(S));
        HISQ_CHECK(enqueue_update(S));
        HISQ_CHECK(enqueue_tail(S));
        if ((it + 1) % check == 0 || it + 1 == P.max_iter) {
            // the per-iteration residual/flag read-back
            HISQ_CUDA(cudaMemcpyAsync(&w->h_st->any_active, &w->st->any_active, sizeof(int), cudaMemcpyDeviceToHost, S.st));
            HISQ_CUDA(cudaStreamSynchronize(S.st));
            if (!w->h_st->any_active) break;
        }
    }
    HISQ_CUDA(cudaMemcpyAsync(w->h_st, w->st, sizeof(SolverState), cudaMemcpyDeviceToHost, S.st));
    HISQ_CUDA(cudaStreamSynchronize(S.st));
    return HISQ_OK;
}

// hisq_cg_solve, and (mass2v, tolv set) bundles of shifted systems with per-right-hand-side m^2 and
// tolerance on the persistent driver
int cg_solve_common(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, const double *const rhs[],
                    double *x[], int nrhs, double mass, double tol, const double *mass2v, const double *tolv) {
    auto t0 = std::chrono::steady_clock::now();
    if (!fat || !naik || !rhs || !x) return set_error(HISQ_ERR_ARG, "null argument");
    if (fat->ctx != ctx || naik->ctx != ctx) return set_error(HISQ_ERR_STATE, "links of another context");
    if (fat->is_naik || !naik->is_naik) return set_error(HISQ_ERR_ARG, "expected (fat, naik) links");
    if (nrhs < 1) return set_error(HISQ_ERR_ARG, "nrhs must be >= 1");
    if (!(tol > 0.0)) return set_error(HISQ_ERR_ARG, "tol must be positive");
    if (mass2v && ctx->params.pc) return set_error(HISQ_ERR_ARG, "shifted bundles run without the preconditioner");
    for (int k = 0; k < nrhs; k++)
        if (!rhs[k] || !x[k]) return set_error(HISQ_ERR_ARG, "null rhs or x pointer %d", k);
    const hisq_solver_params &P = ctx->params;
    int prec = P.inner_prec;
    if (prec != HISQ_FP64 && fat->prec != prec)
        return set_error(HISQ_ERR_ARG, "inner precision %d needs links packed in that precision (links are %d)", prec, fat->prec);
    if (fat->prec != naik->prec) return set_error(HISQ_ERR_ARG, "fat and Naik links have different precisions");
    if (P.pc) {
        if (prec != HISQ_FP32 || fat->prec != HISQ_FP32)
            return set_error(HISQ_ERR_ARG, "flexible CG with the network needs FP32 inner precision and FP32 links");
        if (P.pc->ctx != ctx) return set_error(HISQ_ERR_STATE, "preconditioner of another context");
    }
    int bundle = P.bundle > 0 ? P.bundle : choose_bundle(ctx, fat, naik, nrhs, prec == HISQ_FP64 ? LINKS_FP64 : LINKS_INNER);
    bundle = std::min(bundle, nrhs);
    HISQ_CHECK(ensure_workspace(ctx, bundle, prec, P.pc != nullptr));
    if (P.pc) HISQ_CHECK(pc_prepare(ctx, P.pc, bundle));
    Workspace *w = ctx->ws;
    const int Vh = ctx->geom.Vh;
    const size_t vbytes = (size_t)Vh * 6 * sizeof(double);

    ctx->stat_iters.assign(nrhs, 0);
    ctx->stat_resid.assign(nrhs, 1.0);
    hisq_solve_stats &stats = ctx->stats;
    memset(&stats, 0, sizeof(stats));
    stats.nrhs = nrhs;
    stats.bundle_size = bundle;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events, events64;
    int worst = HISQ_OK;

    for (int k0 = 0; k0 < nrhs; k0 += bundle) {
        int n = std::min(bundle, nrhs - k0);
        Solve S{ctx, w, fat, naik, n, prec, mass, ctx->stream, P.time_kernels != 0 && !P.use_graph, &events, &events64,
                P.pc};
        S.pers_timing = P.time_kernels != 0 && (P.use_graph == 2 || mass2v);
        S.stats = &stats;
        S.mass2v = mass2v ? mass2v + k0 : nullptr;
        S.tolv = tolv ? tolv + k0 : nullptr;
        if (mass2v) S.timing = false;  // shifted bundles run on the persistent driver only
        // tune (outside any capture) before the first use of this shape
        S.hp = prec == HISQ_FP64 ? LINKS_FP64 : links_hp(fat);
        if (P.autotune) {
            tuned_shape(ctx, fat, naik, n, prec == HISQ_FP64 ? LINKS_FP64 : LINKS_INNER);
            tuned_shape(ctx, fat, naik, n, S.hp);
        }
        for (int k = 0; k < n; k++)
            HISQ_CUDA(cudaMemcpyAsync(w->canon + (size_t)k * Vh * 6, rhs[k0 + k], vbytes, cudaMemcpyDefault, ctx->stream));
        HISQ_CHECK(solve_bundle(S, tol));
        HISQ_CHECK(unpack_vectors(ctx, w->x_hi, w->canon, n, HISQ_FP64, ctx->stream));
        for (int k = 0; k < n; k++)
            HISQ_CUDA(cudaMemcpyAsync(x[k0 + k], w->canon + (size_t)k * Vh * 6, vbytes, cudaMemcpyDefault, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
        const SolverState &h = *w->h_st;
        int bmax = 0;
        for (int k = 0; k < n; k++) {
            ctx->stat_iters[k0 + k] = h.iters[k];
            ctx->stat_resid[k0 + k] = h.true_res[k];
            stats.total_iterations += h.iters[k];
            stats.max_iterations = std::max(stats.max_iterations, h.iters[k]);
            stats.reliable_updates += h.updates[k];
            bmax = std::max(bmax, h.iters[k]);
            stats.flops += (double)h.iters[k] * Vh * (2.0 * 1146 + 72);
            if (h.status[k] == RHS_CONVERGED) stats.converged++;
            else if (h.status[k] == RHS_BREAKDOWN) worst = HISQ_ERR_BREAKDOWN;
            else if (worst == HISQ_OK) worst = HISQ_ERR_NOT_CONVERGED;
        }
        stats.fallbacks += h.fallbacks;
        // setup (pack, init) and unpack, plus per iteration two Dslash, the update and the
        // p-update; the three residual-recomputation kernels run when an update is due (graph)
        // or are launched every iteration as gated no-ops (host-driven)
        bool graph_mode = P.use_graph && !S.timing;
        // flexible CG adds the network per iteration: M and M^dag (5 layer launches each), plus
        // their average for the Hermitian part, and the beta and direction kernels
        long per_iter = !P.pc ? 4 : 3 + (P.pc->form == HISQ_PC_NORMAL ? 10 : 11) + 2;
        if (S.persistent)
            stats.kernel_launches += 3;  // pack b, the persistent solve, unpack x
        else
            stats.kernel_launches += 3 + per_iter * h.bundle_iters + 3L * (graph_mode ? h.update_rounds : h.bundle_iters);
        stats.bundle_iterations += bmax;
        stats.recompute_passes += h.update_rounds;
        stats.bundles++;
    }
    for (int which = 0; which < 2; which++) {
        for (auto &e : which ? events64 : events) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) {
                (which ? stats.dslash64_ms : stats.dslash_ms) += ms;
                (which ? stats.dslash64_launches : stats.dslash_launches)++;
            }
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    }
    stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (worst == HISQ_ERR_NOT_CONVERGED)
        return set_error(worst, "%d of %d right-hand sides missed tol %.1e within %d iterations", nrhs - stats.converged,
                         nrhs, tol, P.max_iter);
    if (worst == HISQ_ERR_BREAKDOWN) return set_error(worst, "solver breakdown in at least one right-hand side");
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" {

int hisq_set_solver_params(const hisq_solver_params *p) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!p) return set_error(HISQ_ERR_ARG, "null params");
    if (p->inner_prec < HISQ_FP64 || p->inner_prec > HISQ_BF16) return set_error(HISQ_ERR_ARG, "bad inner precision");
    if (p->max_iter < 1) return set_error(HISQ_ERR_ARG, "max_iter must be >= 1");
    if (!(p->delta == 0.0 || (p->delta > 0.0 && p->delta < 1.0)))
        return set_error(HISQ_ERR_ARG, "delta must be 0 (by precision) or in (0, 1)");
    if (p->bundle < 0 || p->bundle > HISQ_MAX_BUNDLE) return set_error(HISQ_ERR_ARG, "bundle must be in 0..%d", HISQ_MAX_BUNDLE);
    if (p->pc && p->pc->ctx != ctx) return set_error(HISQ_ERR_STATE, "preconditioner of another context");
    ctx->params = *p;
    return HISQ_OK;
}

int hisq_get_solver_params(hisq_solver_params *p) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!p) return set_error(HISQ_ERR_ARG, "null params");
    *p = ctx->params;
    return HISQ_OK;
}

int hisq_cg_solve(const hisq_links *fat, const hisq_links *naik, const double *const rhs[], double *x[], int nrhs,
                  double mass, double tol) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    return cg_solve_common(ctx, fat, naik, rhs, x, nrhs, mass, tol, nullptr, nullptr);
}

int hisq_last_stats(hisq_solve_stats *s, int *iterations, double *true_residual) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!s) return set_error(HISQ_ERR_ARG, "null stats");
    *s = ctx->stats;
    int n = (int)ctx->stat_iters.size();
    if (iterations)
        for (int k = 0; k < n; k++) iterations[k] = ctx->stat_iters[k];
    if (true_residual)
        for (int k = 0; k < n; k++) true_residual[k] = ctx->stat_resid[k];
    return HISQ_OK;
}

}  // extern "C"
