// Multi-shift conjugate gradient (Jegerlehner, hep-lat/9612014): x_j = (A + sigma_j)^{-1} b for
// up to HISQ_MAX_SHIFTS shifts from the Krylov space of one CG on the base system A + sigma_base,
// sigma_base = min_j sigma_j.  Every shifted residual is a multiple zeta_j of the base residual,
// so an iteration costs one A p (the two multi-right-hand-side Dslash kernels with the fused
// <p, A p>) plus, per shift, one fused pass over x_j and p_j.
//
// The shared iteration runs after two setup kernels as one persistent cooperative kernel
// (use_graph = 2, the default, with 18-real Naik links and a co-resident grid), whose phases are
// separated by the bounded grid barrier of the persistent CG solve and whose blocks each evolve a
// shared-memory copy of the state identically (the same summed partials, the same scalar step):
//   t = D_oe p;  A p = m_base^2 p - D_eo t with <p, A p>;
//   update: for every live shift  p_j = zeta_j r + beta_j p_j,  x_j += alpha_j p_j;
//           r -= alpha A p with |r|^2;
//   p = r + beta p; the scalar step: new zeta_j, beta, per-shift convergence, the loop condition.
// Otherwise the same iteration is one CUDA graph: setup, then a WHILE conditional node whose body
// launches the two Dslash kernels and the update and direction kernels below (the last block of
// the direction kernel runs the scalar step and sets the loop condition).
// The per-shift direction update is deferred into the next iteration's update pass, so each
// shift costs one read and one write of x_j and p_j per iteration.  The blocks of the update
// and direction kernels derive alpha, beta and the zeta's from the same state and the same
// reduced dots, so no separate scalar launches are needed; only the last block of the direction
// kernel (after every block has finished reading) writes the state.
//
// With a low-precision inner iteration (FP32 / FP16 / BF16 storage, FP32 x_j, r, p_j) the shared
// iteration stops at a looser tolerance and the shifts are refined by defect correction in FP64:
// their true residuals, solved together as one bundle of shifted systems (a mass per right-hand
// side) by the mixed-precision persistent CG, and the corrections added, until every FP64 true
// residual meets the requested tolerance.
#include <string.h>
#include <math.h>
#include <chrono>
#include <algorithm>
#include <vector>

#include "hisq_internal.cuh"
#include "dslash_kernel.cuh"
#include "cg_persistent.cuh"

namespace hisq {

constexpr int MS_MAX = HISQ_MAX_SHIFTS;
constexpr int MS_THREADS = 256;

struct MsState {
    int nshift, k, max_iter, any_live, breakdown, cond_last;
    int live[MS_MAX], stop_iter[MS_MAX];
    double s[MS_MAX];                    // sigma_j - sigma_base
    double zeta[MS_MAX], zeta_old[MS_MAX];
    double rr, rr_new, pap, bb;          // |r|^2, |r_new|^2, <p, A p>, |b|^2
    double tol, tol2;                    // relative tolerance of the shared iteration, (tol |b|)^2
    double alpha_prev, beta_prev;
    double m2[MS_MAX], res2v[MS_MAX];    // a batched refinement check: m^2 + sigma_j and |r_j|^2 per listed shift
    unsigned long long h_loop;           // the WHILE node's conditional handle
};

// zeta_j of the next iterate, from the state and this iteration's alpha
__device__ __forceinline__ double ms_zeta_next(const MsState &m, int j, double alpha) {
    const double num = m.zeta[j] * m.zeta_old[j] * m.alpha_prev;
    const double den = m.zeta_old[j] * m.alpha_prev * (1.0 + m.s[j] * alpha) +
                       alpha * m.beta_prev * (m.zeta_old[j] - m.zeta[j]);
    return num / den;
}

__device__ __forceinline__ bool ms_alpha(const MsState &m, double *alpha) {
    const bool ok = m.pap > 0.0 && isfinite(m.pap) && isfinite(m.rr);
    *alpha = ok ? m.rr / m.pap : 0.0;
    return ok;
}

struct MsArgs {
    int Vh, nshift;
    size_t qbytes;   // bytes of one x_j or p_j vector
    const void *b;   // FP64 internal
    void *r;         // Q
    void *p, *ap;    // P
    void *xs, *ps;   // Q, nshift vectors each
    MsState *st;
    RedArgs red;
};

// block sum of one double per thread into the RedArgs partials and the last-block finish
__device__ __forceinline__ void ms_reduce(double *red, double v, const RedArgs &ra) {
    red[threadIdx.x] = v;
    block_reduce_finish(red, blockDim.x, 1, 0, ra);
}

// r = b, p = b, x_j = 0, |b|^2 (last block: bb, rr, tol2, the loop condition)
template <int P>
__global__ void __launch_bounds__(MS_THREADS) ms_init_kernel(MsArgs a) {
    constexpr int Q = q_prec(P);
    using rq = typename Prec<Q>::real;
    using rp = typename Prec<P>::real;
    extern __shared__ double red[];
    const VecView<HISQ_FP64> vb{const_cast<void *>(a.b), 1};
    const VecView<Q> vr{a.r, 1};
    const VecView<P> vp{a.p, 1};
    double acc = 0.0;
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < a.Vh; s += (long)gridDim.x * blockDim.x) {
        Cplx<double> b[3];
        load_vec<HISQ_FP64>(vb, s, 0, b);
        Cplx<rq> bq[3];
        Cplx<rp> bp[3];
        const Cplx<rq> z[3] = {{0, 0}, {0, 0}, {0, 0}};
#pragma unroll
        for (int c = 0; c < 3; c++) {
            acc += b[c].re * b[c].re + b[c].im * b[c].im;
            bq[c] = {(rq)b[c].re, (rq)b[c].im};
            bp[c] = {(rp)b[c].re, (rp)b[c].im};
        }
        store_vec<Q>(vr, s, 0, bq);
        store_vec<P>(vp, s, 0, bp);
        for (int j = 0; j < a.nshift; j++) store_vec<Q>(VecView<Q>{(char *)a.xs + (size_t)j * a.qbytes, 1}, s, 0, z);
    }
    ms_reduce(red, acc, a.red);
}

// The last block of ms_init: the scalars that depend on |b|^2.
__global__ void ms_init_finish_kernel(MsState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    MsState &m = *st;
    m.rr = m.bb;
    m.tol2 = m.tol * m.tol * m.bb;
    if (!(m.bb > 0.0) || !isfinite(m.bb)) {
        // a zero (or non-finite) right-hand side: x_j = 0 is exact for zero, nothing iterates
        m.any_live = 0;
        if (!isfinite(m.bb)) m.breakdown = 1;
        for (int j = 0; j < m.nshift; j++) {
            m.live[j] = 0;
            m.stop_iter[j] = 0;
        }
    }
    set_condition(m.h_loop, &m.cond_last, (unsigned)m.any_live);
}

// update pass: for live shifts p_j = zeta_j r + beta_j p_j (beta_j = 0 at k = 0), x_j += alpha_j p_j;
// r -= alpha A p; |r|^2 -> st->rr_new
template <int P>
__global__ void __launch_bounds__(MS_THREADS) ms_update_kernel(MsArgs a) {
    constexpr int Q = q_prec(P);
    using rq = typename Prec<Q>::real;
    using rp = typename Prec<P>::real;
    extern __shared__ double red[];
    __shared__ double s_zeta[MS_MAX], s_aj[MS_MAX], s_bj[MS_MAX];
    __shared__ int s_list[MS_MAX], s_nlive;
    __shared__ double s_alpha;
    __shared__ int s_ok;
    const MsState &m = *a.st;
    if (threadIdx.x == 0) {
        double al;
        s_ok = ms_alpha(m, &al) && m.any_live;
        s_alpha = al;
        int nl = 0;
        for (int j = 0; j < a.nshift; j++) {
            if (!m.live[j]) continue;
            const double zn = ms_zeta_next(m, j, al);
            const double ratio = m.zeta[j] / m.zeta_old[j];
            s_list[nl] = j;
            s_zeta[nl] = m.zeta[j];
            s_aj[nl] = al * zn / m.zeta[j];
            s_bj[nl] = m.k == 0 ? 0.0 : m.beta_prev * ratio * ratio;
            nl++;
        }
        s_nlive = nl;
    }
    __syncthreads();
    double acc = 0.0;
    if (s_ok) {
        const rq al = (rq)s_alpha;
        const VecView<Q> vr{a.r, 1};
        const VecView<P> vap{a.ap, 1};
        const size_t vb = a.qbytes;
        const int nl = s_nlive;
        for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < a.Vh; s += (long)gridDim.x * blockDim.x) {
            Cplx<rq> rv[3];
            Cplx<rp> ap[3];
            load_vec<Q>(vr, s, 0, rv);
            load_vec<P>(vap, s, 0, ap);
            for (int i = 0; i < nl; i++) {
                const int j = s_list[i];
                const VecView<Q> vx{(char *)a.xs + (size_t)j * vb, 1}, vpj{(char *)a.ps + (size_t)j * vb, 1};
                const rq z = (rq)s_zeta[i], bj = (rq)s_bj[i], aj = (rq)s_aj[i];
                Cplx<rq> pj[3], xj[3];
                if (s_bj[i] != 0.0) {
                    load_vec<Q>(vpj, s, 0, pj);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; c++) pj[c] = {0, 0};
                }
                load_vec<Q>(vx, s, 0, xj);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    pj[c] = {z * rv[c].re + bj * pj[c].re, z * rv[c].im + bj * pj[c].im};
                    xj[c] = {xj[c].re + aj * pj[c].re, xj[c].im + aj * pj[c].im};
                }
                store_vec<Q>(vpj, s, 0, pj);
                store_vec<Q>(vx, s, 0, xj);
            }
            rq part = 0;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                rv[c] = {rv[c].re - al * (rq)ap[c].re, rv[c].im - al * (rq)ap[c].im};
                part += rv[c].re * rv[c].re + rv[c].im * rv[c].im;
            }
            acc += (double)part;
            store_vec<Q>(vr, s, 0, rv);
        }
    }
    ms_reduce(red, acc, a.red);
}

// p = r + beta p; then the last block advances the state: zeta's, beta, per-shift convergence
// on |zeta_j| |r| <= tol |b|, the iteration count and the loop condition.
template <int P>
__global__ void __launch_bounds__(MS_THREADS) ms_direction_kernel(MsArgs a) {
    constexpr int Q = q_prec(P);
    using rq = typename Prec<Q>::real;
    using rp = typename Prec<P>::real;
    MsState *st = a.st;
    __shared__ int s_ok, is_last;
    __shared__ double s_beta;
    if (threadIdx.x == 0) {
        double al;
        s_ok = ms_alpha(*st, &al) && st->any_live && isfinite(st->rr_new);
        s_beta = s_ok ? st->rr_new / st->rr : 0.0;
    }
    __syncthreads();
    if (s_ok) {
        const rp be = (rp)s_beta;
        const VecView<Q> vr{a.r, 1};
        const VecView<P> vp{a.p, 1};
        for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < a.Vh; s += (long)gridDim.x * blockDim.x) {
            Cplx<rq> rv[3];
            Cplx<rp> p[3];
            load_vec<Q>(vr, s, 0, rv);
            load_vec<P>(vp, s, 0, p);
#pragma unroll
            for (int c = 0; c < 3; c++) p[c] = {(rp)rv[c].re + be * p[c].re, (rp)rv[c].im + be * p[c].im};
            store_vec<P>(vp, s, 0, p);
        }
    }
    // last block: every block has read the state, so it may be advanced
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        is_last = atomicAdd(a.red.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last || threadIdx.x != 0) return;
    __threadfence();
    *a.red.counter = 0u;
    MsState &m = *st;
    if (!m.any_live) return;
    double al;
    const bool ok = ms_alpha(m, &al) && isfinite(m.rr_new);
    if (!ok) {
        m.breakdown = 1;
        m.any_live = 0;
        set_condition(m.h_loop, &m.cond_last, 0u);
        return;
    }
    const double rr_new = m.rr_new;
    int live = 0;
    for (int j = 0; j < m.nshift; j++) {
        if (!m.live[j]) continue;
        const double zn = ms_zeta_next(m, j, al);
        m.zeta_old[j] = m.zeta[j];
        m.zeta[j] = zn;
        if (zn * zn * rr_new <= m.tol2) {
            m.live[j] = 0;
            m.stop_iter[j] = m.k + 1;
        } else {
            live++;
        }
    }
    m.beta_prev = rr_new / m.rr;
    m.alpha_prev = al;
    m.rr = rr_new;
    m.k++;
    m.any_live = live > 0 && m.k < m.max_iter;
    set_condition(m.h_loop, &m.cond_last, (unsigned)m.any_live);
}

// ---- the shared iteration as one persistent cooperative kernel ----
struct MsPersArgs {
    PersArgs pa;   // geometry, links of the iteration, p, t, ap, n = 1, partials, barrier, error flag
    MsArgs ms;     // r, x_j, p_j, the state (read at the start, written back by block 0 at the end)
    double mass2;  // m^2 + sigma_base
};

constexpr int MS_PERS_THREADS = 512;

// Per live shift j, from the state and this iteration's alpha: its list position, zeta_j, alpha_j
// and beta_j (thread 0; the same coefficients as ms_update_kernel's)
__device__ __forceinline__ int ms_coefficients(const MsState &m, int nshift, double al, int *list, double *zeta,
                                               double *aj, double *bj) {
    int nl = 0;
    for (int j = 0; j < nshift; j++) {
        if (!m.live[j]) continue;
        const double zn = ms_zeta_next(m, j, al);
        const double ratio = m.zeta[j] / m.zeta_old[j];
        list[nl] = j;
        zeta[nl] = m.zeta[j];
        aj[nl] = al * zn / m.zeta[j];
        bj[nl] = m.k == 0 ? 0.0 : m.beta_prev * ratio * ratio;
        nl++;
    }
    return nl;
}

// The state's advance after |r_new|^2 (thread 0; ms_direction_kernel's last block does the same)
__device__ __forceinline__ void ms_advance(MsState &m) {
    if (!m.any_live) return;
    double al;
    const bool ok = ms_alpha(m, &al) && isfinite(m.rr_new);
    if (!ok) {
        m.breakdown = 1;
        m.any_live = 0;
        return;
    }
    const double rr_new = m.rr_new;
    int live = 0;
    for (int j = 0; j < m.nshift; j++) {
        if (!m.live[j]) continue;
        const double zn = ms_zeta_next(m, j, al);
        m.zeta_old[j] = m.zeta[j];
        m.zeta[j] = zn;
        if (zn * zn * rr_new <= m.tol2) {
            m.live[j] = 0;
            m.stop_iter[j] = m.k + 1;
        } else {
            live++;
        }
    }
    m.beta_prev = rr_new / m.rr;
    m.alpha_prev = al;
    m.rr = rr_new;
    m.k++;
    m.any_live = live > 0 && m.k < m.max_iter;
}

template <int P>
__global__ void __launch_bounds__(MS_PERS_THREADS, P == HISQ_FP64 ? 1 : 2) ms_persistent_kernel(const __grid_constant__ MsPersArgs A) {
    constexpr int Q = q_prec(P);
    using rq = typename Prec<Q>::real;
    using rp = typename Prec<P>::real;
    extern __shared__ double red[];
    __shared__ MsState m;
    __shared__ double dots[4], m2v[1];
    __shared__ int mask[1];
    __shared__ double s_zeta[MS_MAX], s_aj[MS_MAX], s_bj[MS_MAX];
    __shared__ int s_list[MS_MAX], s_nlive, s_ok;
    __shared__ double s_alpha, s_beta;
    const PersArgs &a = A.pa;
    const int tid = threadIdx.x;
    {
        constexpr int WORDS = sizeof(MsState) / sizeof(uint32_t);
        const uint32_t *src = reinterpret_cast<const uint32_t *>(A.ms.st);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&m);
        for (int i = tid; i < WORDS; i += blockDim.x) dst[i] = __ldcg(src + i);
        if (tid == 0) {
            mask[0] = 1;
            m2v[0] = A.mass2;
        }
    }
    __syncthreads();
    const VecView<Q> vr{A.ms.r, 1};
    const VecView<P> vap{a.ap, 1}, vp{a.p, 1};
    const size_t qb = A.ms.qbytes;
    const long stride = (long)gridDim.x * blockDim.x;
    bool ok = true;
    while (m.any_live) {
        dslash_phase<P, 1, EPI_PLAIN, Q>(a, a.fat, a.naik, PlainIn<P, true>{vp}, a.t, 1, mask, PlainIn<P, true>{vp},
                                         nullptr, nullptr, red, m2v);
        if (!(ok = grid_sync(a))) break;
        dslash_phase<P, 1, EPI_AOP, Q>(a, a.fat, a.naik, PlainIn<P, true>{VecView<P>{a.t, 1}}, a.ap, 0, mask,
                                       PlainIn<P, true>{vp}, nullptr, nullptr, red, m2v);
        if (!(ok = grid_sync(a))) break;
        sum_partials(a, red, 1, dots);
        if (tid == 0) {
            m.pap = dots[0];
            double al;
            s_ok = ms_alpha(m, &al) && m.any_live;
            s_alpha = al;
            s_nlive = ms_coefficients(m, A.ms.nshift, al, s_list, s_zeta, s_aj, s_bj);
        }
        __syncthreads();
        // update pass: p_j, x_j for the live shifts; r -= alpha A p with |r|^2
        double acc[1] = {0.0};
        if (s_ok) {
            const rq al = (rq)s_alpha;
            const int nl = s_nlive;
            for (long s = (long)blockIdx.x * blockDim.x + tid; s < a.g.Vh; s += stride) {
                Cplx<rq> rv[3];
                Cplx<rp> ap[3];
                load_vec<Q, true>(vr, s, 0, rv);
                load_vec<P, true>(vap, s, 0, ap);
                for (int i = 0; i < nl; i++) {
                    const int j = s_list[i];
                    const VecView<Q> vx{(char *)A.ms.xs + (size_t)j * qb, 1}, vpj{(char *)A.ms.ps + (size_t)j * qb, 1};
                    const rq z = (rq)s_zeta[i], bj = (rq)s_bj[i], aj = (rq)s_aj[i];
                    Cplx<rq> pj[3], xj[3];
                    if (s_bj[i] != 0.0) {
                        load_vec<Q, true>(vpj, s, 0, pj);
                    } else {
#pragma unroll
                        for (int c = 0; c < 3; c++) pj[c] = {0, 0};
                    }
                    load_vec<Q, true>(vx, s, 0, xj);
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        pj[c] = {z * rv[c].re + bj * pj[c].re, z * rv[c].im + bj * pj[c].im};
                        xj[c] = {xj[c].re + aj * pj[c].re, xj[c].im + aj * pj[c].im};
                    }
                    store_vec<Q>(vpj, s, 0, pj);
                    store_vec<Q>(vx, s, 0, xj);
                }
                rq part = 0;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    rv[c] = {rv[c].re - al * (rq)ap[c].re, rv[c].im - al * (rq)ap[c].im};
                    part += rv[c].re * rv[c].re + rv[c].im * rv[c].im;
                }
                acc[0] += (double)part;
                store_vec<Q>(vr, s, 0, rv);
            }
        }
        // |r|^2 goes to partials column 1: a block that is through its update may publish while a
        // slower one still sums column 0 (<p, A p>) of this iteration
        publish_dots<1>(a, red, acc, 1, 0, 1, 1);
        if (!(ok = grid_sync(a))) break;
        sum_partials(a, red, 2, dots);
        if (tid == 0) {
            m.rr_new = s_ok ? dots[1] : 0.0;
            double al;
            s_ok = ms_alpha(m, &al) && m.any_live && isfinite(m.rr_new);
            s_beta = s_ok ? m.rr_new / m.rr : 0.0;
        }
        __syncthreads();
        // direction: p = r + beta p, then the scalar step (every block the same)
        if (s_ok) {
            const rp be = (rp)s_beta;
            for (long s = (long)blockIdx.x * blockDim.x + tid; s < a.g.Vh; s += stride) {
                Cplx<rq> rv[3];
                Cplx<rp> p[3];
                load_vec<Q, true>(vr, s, 0, rv);
                load_vec<P, true>(vp, s, 0, p);
#pragma unroll
                for (int c = 0; c < 3; c++) p[c] = {(rp)rv[c].re + be * p[c].re, (rp)rv[c].im + be * p[c].im};
                store_vec<P>(vp, s, 0, p);
            }
        }
        if (tid == 0) ms_advance(m);
        if (!(ok = grid_sync(a))) break;  // p complete before the next D_oe; the state advanced everywhere
    }
    if (blockIdx.x == 0) {
        __syncthreads();
        constexpr int WORDS = sizeof(MsState) / sizeof(uint32_t);
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&m);
        uint32_t *dst = reinterpret_cast<uint32_t *>(A.ms.st);
        for (int i = tid; i < WORDS; i += blockDim.x) dst[i] = src[i];
    }
    (void)ok;
}

template <int P>
static cudaError_t ms_persistent_launch(const MsPersArgs &a, int grid, size_t smem, cudaStream_t st) {
    void *args[] = {const_cast<MsPersArgs *>(&a)};
    const void *k = (const void *)ms_persistent_kernel<P>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(k, grid, MS_PERS_THREADS, args, smem, st);
}

template <int P>
static cudaError_t ms_persistent_occupancy(size_t smem, int *per_sm) {
    const void *k = (const void *)ms_persistent_kernel<P>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, MS_PERS_THREADS, smem);
}

// x += y on canonical FP64 arrays of `count` doubles
__global__ void __launch_bounds__(256) ms_axpy_canon_kernel(double *x, const double *y, long count) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
        x[i] += y[i];
}

struct MsWork {
    int prec = -1, cap = 0;
    void *b64 = nullptr, *r = nullptr, *p = nullptr, *t = nullptr, *ap = nullptr, *xs = nullptr, *ps = nullptr;
    void *x64 = nullptr, *t64 = nullptr, *r64 = nullptr;
    void *x_ds = nullptr;  // x64 in double-single form (residual Dslash input for low-precision links)
    double *canon_b = nullptr, *canon_r = nullptr, *canon_e = nullptr, *canon_x = nullptr;  // canonical staging
    double *partials = nullptr;
    size_t partials_cap = 0;
    unsigned int *counter = nullptr;
    unsigned int *bar = nullptr;  // the persistent kernel's grid-barrier word
    int *err = nullptr;           // set when one of its barrier waits ran out
    MsState *st = nullptr, *h_st = nullptr;
    // the captured shared iteration and what it was captured for
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    unsigned long long h_loop = 0;
    const hisq_links *fat = nullptr, *naik = nullptr;
    double mass2_base = 0;
    int g_nshift = 0, g_prec = -1;
    unsigned tune_generation = 0;
};

static void ms_free_graph(MsWork *w) {
    if (w->exec) cudaGraphExecDestroy(w->exec);
    if (w->graph) cudaGraphDestroy(w->graph);
    w->exec = nullptr;
    w->graph = nullptr;
    w->h_loop = 0;
    w->fat = w->naik = nullptr;
}

static void ms_free_buffers(MsWork *w) {
    void *bufs[] = {w->b64, w->r, w->p, w->t, w->ap, w->xs, w->ps, w->x64, w->t64, w->r64, w->x_ds,
                    w->canon_b, w->canon_r, w->canon_e, w->canon_x};
    for (void *b : bufs)
        if (b) cudaFree(b);
    w->b64 = w->r = w->p = w->t = w->ap = w->xs = w->ps = w->x64 = w->t64 = w->r64 = w->x_ds = nullptr;
    w->canon_b = w->canon_r = w->canon_e = w->canon_x = nullptr;
    w->cap = 0;
    w->prec = -1;
    ms_free_graph(w);
}

void free_multishift(hisq_ctx *ctx) {
    MsWork *w = ctx->ms;
    if (!w) return;
    ms_free_buffers(w);
    if (w->partials) cudaFree(w->partials);
    if (w->counter) cudaFree(w->counter);
    if (w->bar) cudaFree(w->bar);
    if (w->err) cudaFree(w->err);
    if (w->st) cudaFree(w->st);
    if (w->h_st) cudaFreeHost(w->h_st);
    delete w;
    ctx->ms = nullptr;
}

static int ms_workspace(hisq_ctx *ctx, int nshift, int prec) {
    if (!ctx->ms) {
        MsWork *w = new MsWork();
        ctx->ms = w;
        w->partials_cap = (size_t)ctx->num_sms * 64 * MS_MAX;  // a batched residual of every shift
        if (cudaMalloc(&w->partials, w->partials_cap * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&w->counter, 4 * sizeof(unsigned int)) != cudaSuccess ||
            cudaMalloc(&w->bar, 4 * sizeof(unsigned int)) != cudaSuccess || cudaMalloc(&w->err, 4 * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&w->st, sizeof(MsState)) != cudaSuccess || cudaMallocHost(&w->h_st, sizeof(MsState)) != cudaSuccess)
            return set_error(HISQ_ERR_NOMEM, "multi-shift workspace allocation failed");
        cudaMemset(w->counter, 0, 4 * sizeof(unsigned int));
    }
    MsWork *w = ctx->ms;
    if (w->prec == prec && w->cap >= nshift) return HISQ_OK;
    const int cap = std::max(nshift, w->prec == prec ? w->cap : 0);
    ms_free_buffers(w);
    const int Vh = ctx->geom.Vh, Q = q_prec(prec);
    const size_t canon = (size_t)Vh * 6 * sizeof(double);
    struct { void **ptr; size_t bytes; } allocs[] = {
        {&w->b64, vector_bytes(HISQ_FP64, Vh, 1)}, {&w->r, vector_bytes(Q, Vh, 1)},
        {&w->p, vector_bytes(prec, Vh, 1)},        {&w->t, vector_bytes(prec, Vh, 1)},
        {&w->ap, vector_bytes(prec, Vh, 1)},       {&w->xs, vector_bytes(Q, Vh, 1) * cap},
        {&w->ps, vector_bytes(Q, Vh, 1) * cap},    {&w->x64, vector_bytes(HISQ_FP64, Vh, cap)},
        {&w->t64, vector_bytes(HISQ_FP64, Vh, cap)}, {&w->r64, vector_bytes(HISQ_FP64, Vh, cap)},
        {&w->x_ds, vector_bytes(HISQ_DS, Vh, cap)},
        {(void **)&w->canon_b, canon},             {(void **)&w->canon_r, canon * cap},
        {(void **)&w->canon_e, canon * cap},       {(void **)&w->canon_x, canon * cap},
    };
    for (auto &a : allocs)
        if (cudaMalloc(a.ptr, a.bytes) != cudaSuccess) {
            ms_free_buffers(w);
            return set_error(HISQ_ERR_NOMEM, "cannot allocate %zu bytes of multi-shift workspace", a.bytes);
        }
    w->cap = cap;
    w->prec = prec;
    return HISQ_OK;
}

static MsArgs ms_args(hisq_ctx *ctx, MsWork *w, int nshift) {
    MsArgs a;
    memset(&a, 0, sizeof(a));
    a.Vh = ctx->geom.Vh;
    a.nshift = nshift;
    a.qbytes = vector_bytes(q_prec(w->prec), ctx->geom.Vh, 1);
    a.b = w->b64;
    a.r = w->r;
    a.p = w->p;
    a.ap = w->ap;
    a.xs = w->xs;
    a.ps = w->ps;
    a.st = w->st;
    a.red.partials = w->partials;
    a.red.counter = w->counter;
    a.red.hook = HOOK_NONE;
    return a;
}

static int ms_grid(hisq_ctx *ctx) {
    long tiles = (ctx->geom.Vh + MS_THREADS - 1) / MS_THREADS;
    return (int)balanced_grid(tiles, (long)ctx->num_sms * 4);
}

template <int P>
static int ms_enqueue_setup(hisq_ctx *ctx, MsWork *w, int nshift, cudaStream_t st) {
    MsArgs a = ms_args(ctx, w, nshift);
    a.red.dot_out = &w->st->bb;
    const size_t smem = (MS_THREADS + 64) * sizeof(double);
    ms_init_kernel<P><<<ms_grid(ctx), MS_THREADS, smem, st>>>(a);
    HISQ_CUDA(cudaGetLastError());
    ms_init_finish_kernel<<<1, 32, 0, st>>>(w->st);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

template <int P>
static int ms_enqueue_iteration(hisq_ctx *ctx, MsWork *w, const hisq_links *fat, const hisq_links *naik, int nshift,
                                double mass2_base, cudaStream_t st) {
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.n = 1;
    d.in = w->p;
    d.out = w->t;
    d.parity = 1;
    d.epi = EPI_PLAIN;
    const int use64 = (P == HISQ_FP64 && fat->prec != HISQ_FP64) ? LINKS_FP64 : LINKS_INNER;
    HISQ_CHECK(launch_dslash(ctx, fat, naik, use64, d, nullptr, st));
    d.in = w->t;
    d.out = w->ap;
    d.parity = 0;
    d.epi = EPI_AOP;
    d.mass2 = mass2_base;
    d.axpy_in = w->p;
    d.partials = w->partials;
    d.partials_cap = w->partials_cap;
    d.counter = w->counter;
    d.dot_out = &w->st->pap;
    d.hook = HOOK_NONE;
    HISQ_CHECK(launch_dslash(ctx, fat, naik, use64, d, nullptr, st));
    MsArgs a = ms_args(ctx, w, nshift);
    a.red.dot_out = &w->st->rr_new;
    const size_t smem = (MS_THREADS + 64) * sizeof(double);
    const int grid = ms_grid(ctx);
    ms_update_kernel<P><<<grid, MS_THREADS, smem, st>>>(a);
    HISQ_CUDA(cudaGetLastError());
    ms_direction_kernel<P><<<grid, MS_THREADS, 0, st>>>(a);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

template <int P>
static int ms_build_graph(hisq_ctx *ctx, MsWork *w, const hisq_links *fat, const hisq_links *naik, int nshift,
                          double mass2_base) {
    ms_free_graph(w);
    cudaGraph_t graph;
    HISQ_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h_loop;
    HISQ_CUDA(cudaGraphConditionalHandleCreate(&h_loop, graph, 1, cudaGraphCondAssignDefault));
    cudaStream_t cap;
    HISQ_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int rc = HISQ_OK;
    cudaGraph_t body = nullptr, outg;
    cudaError_t e = cudaStreamBeginCaptureToGraph(cap, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "multi-shift capture failed: %s", cudaGetErrorString(e));
    if (rc == HISQ_OK) rc = ms_enqueue_setup<P>(ctx, w, nshift, cap);
    if (rc == HISQ_OK) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g;
        const cudaGraphNode_t *deps;
        const cudaGraphEdgeData *edges;
        size_t ndeps;
        e = cudaStreamGetCaptureInfo(cap, &cs, nullptr, &g, &deps, &edges, &ndeps);
        if (e == cudaSuccess) {
            cudaGraphNodeParams params = {cudaGraphNodeTypeConditional};
            params.conditional.handle = h_loop;
            params.conditional.type = cudaGraphCondTypeWhile;
            params.conditional.size = 1;
            cudaGraphNode_t node;
            e = cudaGraphAddNode(&node, g, deps, edges, ndeps, &params);
            if (e == cudaSuccess) {
                body = params.conditional.phGraph_out[0];
                e = cudaStreamUpdateCaptureDependencies(cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
            }
        }
        if (e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "multi-shift loop node failed: %s", cudaGetErrorString(e));
    }
    e = cudaStreamEndCapture(cap, &outg);
    if (rc == HISQ_OK && e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "multi-shift capture failed: %s", cudaGetErrorString(e));
    if (rc == HISQ_OK) {
        e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "multi-shift loop capture failed: %s", cudaGetErrorString(e));
        if (rc == HISQ_OK) rc = ms_enqueue_iteration<P>(ctx, w, fat, naik, nshift, mass2_base, cap);
        e = cudaStreamEndCapture(cap, &outg);
        if (rc == HISQ_OK && e != cudaSuccess)
            rc = set_error(HISQ_ERR_CUDA, "multi-shift loop capture failed: %s", cudaGetErrorString(e));
    }
    cudaStreamDestroy(cap);
    if (rc == HISQ_OK) {
        e = cudaGraphInstantiate(&w->exec, graph, 0);
        if (e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "multi-shift graph instantiation failed: %s", cudaGetErrorString(e));
    }
    if (rc != HISQ_OK) {
        cudaGraphDestroy(graph);
        w->exec = nullptr;
        cudaGetLastError();
        return rc;
    }
    w->graph = graph;
    w->h_loop = (unsigned long long)h_loop;
    w->fat = fat;
    w->naik = naik;
    w->mass2_base = mass2_base;
    w->g_nshift = nshift;
    w->g_prec = P;
    w->tune_generation = ctx->tune_generation;
    return HISQ_OK;
}

static int ms_build(hisq_ctx *ctx, MsWork *w, const hisq_links *fat, const hisq_links *naik, int nshift, int prec,
                    double mass2_base) {
    switch (prec) {
    case HISQ_FP64: return ms_build_graph<HISQ_FP64>(ctx, w, fat, naik, nshift, mass2_base);
    case HISQ_FP32: return ms_build_graph<HISQ_FP32>(ctx, w, fat, naik, nshift, mass2_base);
    case HISQ_FP16: return ms_build_graph<HISQ_FP16>(ctx, w, fat, naik, nshift, mass2_base);
    default: return ms_build_graph<HISQ_BF16>(ctx, w, fat, naik, nshift, mass2_base);
    }
}

// The shared iteration as the persistent kernel: the two setup kernels, then one cooperative launch.
// *done = false (nothing launched past the setup, which the graph repeats) when it does not apply:
// 13- or 9-real Naik links, or a grid that cannot be co-resident.
template <int P>
static int ms_run_persistent(hisq_ctx *ctx, MsWork *w, const hisq_links *fat, const hisq_links *naik, int nshift,
                             double mass2_base, bool *done) {
    *done = false;
    if (naik->recon != 18) return HISQ_OK;
    const size_t smem = (size_t)(4 * MS_PERS_THREADS + 64) * sizeof(double);
    int per_sm = 0;
    if (ms_persistent_occupancy<P>(smem, &per_sm) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return HISQ_OK;
    }
    const int grid = per_sm * ctx->num_sms;  // one resident wave
    if ((size_t)grid * PERS_ND > w->partials_cap) return HISQ_OK;
    MsPersArgs a;
    memset(&a, 0, sizeof(a));
    const bool links64 = P == HISQ_FP64 && fat->prec != HISQ_FP64;
    a.pa.g = ctx->geom;
    a.pa.fat = links64 ? fat->field64() : fat->field();
    a.pa.naik = links64 ? naik->field64() : naik->field();
    a.pa.p = w->p;
    a.pa.t = w->t;
    a.pa.ap = w->ap;
    a.pa.n = 1;
    a.pa.partials = w->partials;
    a.pa.bar = w->bar;
    a.pa.err = w->err;
    a.pa.spin_limit = 1LL << 22;  // a barrier wait gives up after about a second
    a.pa.expected = grid;
    a.ms = ms_args(ctx, w, nshift);
    a.mass2 = mass2_base;
    cudaStream_t st = ctx->stream;
    HISQ_CHECK(ms_enqueue_setup<P>(ctx, w, nshift, st));
    HISQ_CUDA(cudaMemsetAsync(w->bar, 0, 4 * sizeof(unsigned int), st));
    HISQ_CUDA(cudaMemsetAsync(w->err, 0, 4 * sizeof(int), st));
    const cudaError_t e = ms_persistent_launch<P>(a, grid, smem, st);
    if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
        cudaGetLastError();
        return HISQ_OK;
    }
    if (e != cudaSuccess) return set_error(HISQ_ERR_CUDA, "multi-shift persistent launch failed: %s", cudaGetErrorString(e));
    *done = true;
    return HISQ_OK;
}

static int ms_persistent(hisq_ctx *ctx, MsWork *w, const hisq_links *fat, const hisq_links *naik, int nshift, int prec,
                         double mass2_base, bool *done) {
    switch (prec) {
    case HISQ_FP64: return ms_run_persistent<HISQ_FP64>(ctx, w, fat, naik, nshift, mass2_base, done);
    case HISQ_FP32: return ms_run_persistent<HISQ_FP32>(ctx, w, fat, naik, nshift, mass2_base, done);
    case HISQ_FP16: return ms_run_persistent<HISQ_FP16>(ctx, w, fat, naik, nshift, mass2_base, done);
    default: return ms_run_persistent<HISQ_BF16>(ctx, w, fat, naik, nshift, mass2_base, done);
    }
}

// The FP64 residuals r_q = b - (m^2 + sigma_{j_q} - D_eo D_oe) x_{j_q} of m listed shifts in one
// bundle: the listed canonical x_j are gathered (device copies) and packed as an m-RHS FP64
// bundle, the residual Dslash runs once over it with a mass per right-hand side and the single b
// shared by all; the residuals are unpacked to canon_r[0..m) in list order and |r_q|^2 returned.
static int ms_residuals(hisq_ctx *ctx, MsWork *w, const hisq_links *fat, const hisq_links *naik, const int *js, int m,
                        const double *m2, double *res2) {
    cudaStream_t st = ctx->stream;
    const int Vh = ctx->geom.Vh;
    const size_t vbytes = (size_t)Vh * 6 * sizeof(double);
    const int hp = links_hp(fat);
    // canon_e is free here (the corrections of the previous round were added already)
    for (int q = 0; q < m; q++)
        HISQ_CUDA(cudaMemcpyAsync(w->canon_e + (size_t)q * Vh * 6, w->canon_x + (size_t)js[q] * Vh * 6, vbytes,
                                  cudaMemcpyDeviceToDevice, st));
    HISQ_CHECK(pack_vectors(ctx, w->canon_e, w->x64, m, HISQ_FP64, st));
    if (hp == LINKS_DS) HISQ_CHECK(split_vectors(ctx, w->x64, w->x_ds, m, st));
    double m2h[MS_MAX];
    for (int q = 0; q < m; q++) m2h[q] = m2[q];
    HISQ_CUDA(cudaMemcpyAsync(w->st->m2, m2h, sizeof(double) * m, cudaMemcpyHostToDevice, st));
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.n = m;
    d.in = hp == LINKS_DS ? w->x_ds : w->x64;
    d.out = w->t64;
    d.parity = 1;
    d.epi = EPI_PLAIN;
    HISQ_CHECK(launch_dslash(ctx, fat, naik, hp, d, nullptr, st));
    d.in = w->t64;
    d.out = w->r64;
    d.parity = 0;
    d.epi = EPI_RESID;
    d.mass2v = w->st->m2;
    d.axpy_in = w->x64;
    d.b = w->b64;
    d.b_one = 1;
    d.partials = w->partials;
    d.partials_cap = w->partials_cap;
    d.counter = w->counter;
    d.dot_out = w->st->res2v;
    d.hook = HOOK_NONE;
    HISQ_CHECK(launch_dslash(ctx, fat, naik, hp, d, nullptr, st));
    HISQ_CHECK(unpack_vectors(ctx, w->r64, w->canon_r, m, HISQ_FP64, st));
    HISQ_CUDA(cudaMemcpyAsync(res2, w->st->res2v, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    HISQ_CUDA(cudaStreamSynchronize(st));
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_cg_multishift(const hisq_links *fat, const hisq_links *naik, const double *rhs, double *x[],
                                  int nshift, const double *shifts, double mass, double tol) {
    auto t0 = std::chrono::steady_clock::now();
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!fat || !naik || !rhs || !x || !shifts) return set_error(HISQ_ERR_ARG, "null argument");
    if (fat->ctx != ctx || naik->ctx != ctx) return set_error(HISQ_ERR_STATE, "links of another context");
    if (fat->is_naik || !naik->is_naik) return set_error(HISQ_ERR_ARG, "expected (fat, naik) links");
    if (fat->prec != naik->prec) return set_error(HISQ_ERR_ARG, "fat and Naik links have different precisions");
    if (nshift < 1 || nshift > HISQ_MAX_SHIFTS) return set_error(HISQ_ERR_ARG, "nshift must be in 1..%d", HISQ_MAX_SHIFTS);
    if (!(tol > 0.0)) return set_error(HISQ_ERR_ARG, "tol must be positive");
    if (!(mass * mass > 0.0) || !isfinite(mass)) return set_error(HISQ_ERR_ARG, "mass must be non-zero and finite");
    double sigma_base = shifts[0];
    for (int j = 0; j < nshift; j++) {
        if (!x[j]) return set_error(HISQ_ERR_ARG, "null x pointer %d", j);
        if (!isfinite(shifts[j]) || !(mass * mass + shifts[j] > 0.0))
            return set_error(HISQ_ERR_ARG, "shift %d (%g) must be finite and > -mass^2", j, shifts[j]);
        sigma_base = std::min(sigma_base, shifts[j]);
    }
    const hisq_solver_params P0 = ctx->params;
    const int prec = P0.inner_prec;
    if (P0.pc) return set_error(HISQ_ERR_ARG, "multi-shift CG runs without the preconditioner (set pc = NULL)");
    if (prec != HISQ_FP64 && fat->prec != prec)
        return set_error(HISQ_ERR_ARG, "inner precision %d needs links packed in that precision (links are %d)", prec, fat->prec);
    const double mass2_base = mass * mass + sigma_base;
    // the all-FP64 iteration stops at the library's acceptance bound (0.95 tol) like a CG solve
    double tol_shared = tol * TOL_SAFETY;
    if (prec != HISQ_FP64)
        tol_shared = std::max(tol_shared, P0.multishift_tol > 0.0 ? P0.multishift_tol : (prec == HISQ_FP32 ? 1e-7 : 1e-4));
    HISQ_CHECK(ms_workspace(ctx, nshift, prec));
    MsWork *w = ctx->ms;
    cudaStream_t st = ctx->stream;
    const int Vh = ctx->geom.Vh;
    const size_t vbytes = (size_t)Vh * 6 * sizeof(double);
    if (P0.autotune) {
        tuned_shape(ctx, fat, naik, 1, prec == HISQ_FP64 ? LINKS_FP64 : LINKS_INNER);
        tuned_shape(ctx, fat, naik, 1, links_hp(fat));
    }

    // ---- the shared iteration ----
    HISQ_CUDA(cudaMemcpyAsync(w->canon_b, rhs, vbytes, cudaMemcpyDefault, st));
    HISQ_CHECK(pack_vectors(ctx, w->canon_b, w->b64, 1, HISQ_FP64, st));
    MsState *h = w->h_st;
    memset(h, 0, sizeof(MsState));
    h->nshift = nshift;
    h->max_iter = P0.max_iter;
    h->any_live = 1;
    h->cond_last = 1;  // the WHILE handle's default at every launch
    h->tol = tol_shared;
    h->alpha_prev = 1.0;
    h->beta_prev = 0.0;
    h->h_loop = 0;
    for (int j = 0; j < nshift; j++) {
        h->live[j] = 1;
        h->stop_iter[j] = -1;
        h->s[j] = shifts[j] - sigma_base;
        h->zeta[j] = h->zeta_old[j] = 1.0;
    }
    bool persistent = false;
    if (P0.use_graph == 2) {
        HISQ_CUDA(cudaMemcpyAsync(w->st, h, sizeof(MsState), cudaMemcpyHostToDevice, st));
        HISQ_CHECK(ms_persistent(ctx, w, fat, naik, nshift, prec, mass2_base, &persistent));
    }
    if (!persistent) {
        const bool reuse = w->exec && w->fat == fat && w->naik == naik && w->mass2_base == mass2_base &&
                           w->g_nshift == nshift && w->g_prec == prec && w->tune_generation == ctx->tune_generation;
        if (!reuse) HISQ_CHECK(ms_build(ctx, w, fat, naik, nshift, prec, mass2_base));
        if (!w->h_loop) return set_error(HISQ_ERR_STATE, "multi-shift graph without its loop handle");
        h->h_loop = w->h_loop;
        HISQ_CUDA(cudaMemcpyAsync(w->st, h, sizeof(MsState), cudaMemcpyHostToDevice, st));
        HISQ_CUDA(cudaGraphLaunch(w->exec, st));
    }
    const int Q = q_prec(prec);
    const size_t qbytes = vector_bytes(Q, Vh, 1);
    for (int j = 0; j < nshift; j++)
        HISQ_CHECK(unpack_vectors(ctx, (const char *)w->xs + (size_t)j * qbytes, w->canon_x + (size_t)j * Vh * 6, 1, Q, st));
    HISQ_CUDA(cudaMemcpyAsync(h, w->st, sizeof(MsState), cudaMemcpyDeviceToHost, st));
    int err_h = 0;
    if (persistent) HISQ_CUDA(cudaMemcpyAsync(&err_h, w->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    HISQ_CUDA(cudaStreamSynchronize(st));
    if (err_h) return set_error(HISQ_ERR_TIMEOUT, "a grid barrier of the persistent multi-shift iteration ran out of its wait budget");
    const double t_shared = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const MsState shared = *h;
    if (shared.breakdown) return set_error(HISQ_ERR_BREAKDOWN, "multi-shift CG breakdown (non-positive <p, A p> or NaN)");

    // ---- per-shift FP64 check and refinement by defect correction ----
    // Every shift's FP64 residual r_j = b - (A + sigma_j) x_j; those above tol are solved together
    // as one bundle of shifted systems, (m^2 + sigma_j - D_eo D_oe) e_j = r_j to 0.5 tol |b| / |r_j|,
    // by the mixed-precision CG (persistent driver), and x_j += e_j.  b - (A + sigma_j)(x_j + e_j)
    // = r_j - (A + sigma_j) e_j exactly, so the correction's own FP64 true residual gives the new
    // residual of x_j; a shift still above tol is recomputed and solved again (at most three rounds).
    std::vector<int> iters(nshift, 0);
    std::vector<double> resid(nshift, 0.0);
    long refine_iters = 0;
    const double bb = shared.bb;
    const bool bundled = naik->recon == 18;
    const double *rp[HISQ_MAX_SHIFTS];
    double *ep[HISQ_MAX_SHIFTS];
    double m2v[HISQ_MAX_SHIFTS], tolv[HISQ_MAX_SHIFTS];
    int idx[HISQ_MAX_SHIFTS];
    for (int j = 0; j < nshift; j++) {
        iters[j] = shared.stop_iter[j] >= 0 ? shared.stop_iter[j] : shared.k;
        if (!(bb > 0.0)) HISQ_CUDA(cudaMemsetAsync(w->canon_x + (size_t)j * Vh * 6, 0, vbytes, st));
        else resid[j] = 2.0 * tol + 1.0;  // not yet measured
    }
    const double tol_acc = tol * TOL_SAFETY;  // acceptance bound of the library's FP64 residual
    for (int round = 0; round < 3 && bb > 0.0; round++) {
        // the FP64 residuals of every shift not yet accepted, in one bundle
        int chk[HISQ_MAX_SHIFTS], nchk = 0;
        double chk_m2[HISQ_MAX_SHIFTS], chk_res2[HISQ_MAX_SHIFTS];
        for (int j = 0; j < nshift; j++)
            if (!(resid[j] <= tol_acc)) {
                chk[nchk] = j;
                chk_m2[nchk] = mass * mass + shifts[j];
                nchk++;
            }
        if (nchk == 0) break;
        HISQ_CHECK(ms_residuals(ctx, w, fat, naik, chk, nchk, chk_m2, chk_res2));
        int m = 0;
        for (int q = 0; q < nchk; q++) {
            const int j = chk[q];
            resid[j] = sqrt(chk_res2[q] / bb);
            if (resid[j] <= tol_acc) continue;
            idx[m] = j;
            rp[m] = w->canon_r + (size_t)q * Vh * 6;  // ms_residuals left r_j at position q
            ep[m] = w->canon_e + (size_t)j * Vh * 6;
            m2v[m] = mass * mass + shifts[j];
            tolv[m] = 0.5 * tol / resid[j];
            m++;
        }
        if (m == 0) break;
        if (bundled) {
            double tmin = tolv[0];
            for (int q = 1; q < m; q++) tmin = std::min(tmin, tolv[q]);
            const int rc = cg_solve_common(ctx, fat, naik, rp, ep, m, mass, tmin, m2v, tolv);
            if (rc != HISQ_OK && rc != HISQ_ERR_NOT_CONVERGED) return rc;
            refine_iters += ctx->stats.total_iterations;
            for (int q = 0; q < m; q++) {
                iters[idx[q]] += ctx->stat_iters[q];
                resid[idx[q]] *= ctx->stat_resid[q];
            }
        } else {
            for (int q = 0; q < m; q++) {
                const int rc = cg_solve_common(ctx, fat, naik, rp + q, ep + q, 1, sqrt(m2v[q]), tolv[q], nullptr, nullptr);
                if (rc != HISQ_OK && rc != HISQ_ERR_NOT_CONVERGED) return rc;
                refine_iters += ctx->stats.total_iterations;
                iters[idx[q]] += ctx->stat_iters[0];
                resid[idx[q]] *= ctx->stat_resid[0];
            }
        }
        for (int q = 0; q < m; q++) {
            ms_axpy_canon_kernel<<<ms_grid(ctx), 256, 0, st>>>(w->canon_x + (size_t)idx[q] * Vh * 6, ep[q], (long)Vh * 6);
            HISQ_CUDA(cudaGetLastError());
        }
    }
    int worst = HISQ_OK;
    for (int j = 0; j < nshift; j++)
        if (!(resid[j] <= tol_acc)) worst = HISQ_ERR_NOT_CONVERGED;
    for (int j = 0; j < nshift; j++)
        HISQ_CUDA(cudaMemcpyAsync(x[j], w->canon_x + (size_t)j * Vh * 6, vbytes, cudaMemcpyDefault, st));
    HISQ_CUDA(cudaStreamSynchronize(st));

    hisq_solve_stats &S = ctx->stats;
    memset(&S, 0, sizeof(S));
    S.nrhs = nshift;
    S.bundles = 1;
    S.bundle_size = 1;
    S.shared_iterations = shared.k;
    S.refine_iterations = refine_iters;
    S.shared_seconds = t_shared;
    S.total_iterations = shared.k + refine_iters;
    for (int j = 0; j < nshift; j++) {
        S.max_iterations = std::max(S.max_iterations, iters[j]);
        if (resid[j] <= tol_acc) S.converged++;
    }
    S.flops = (double)S.total_iterations * Vh * (2.0 * 1146 + 72);
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    ctx->stat_iters = iters;
    ctx->stat_resid = resid;
    if (worst != HISQ_OK)
        return set_error(worst, "%d of %d shifts missed tol %.1e", nshift - S.converged, nshift, tol);
    return HISQ_OK;
}
