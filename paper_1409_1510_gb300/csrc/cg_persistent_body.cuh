// Body of the persistent solve kernel (see cg_persistent.cuh).
#pragma once
#include "cg_persistent.cuh"

namespace hisq {

template <int P, int R, bool CG1>
__global__ void __launch_bounds__(pers_threads(R), 1) cg_persistent_kernel(const __grid_constant__ PersArgs a) {
    constexpr int Q = q_prec(P);
    using rp = typename Prec<P>::real;
    using rq = typename Prec<Q>::real;
    extern __shared__ double red[];
    __shared__ SolverState st;
    __shared__ double dots[PERS_ND];
    __shared__ PhaseClock clk;
    __shared__ int upd_list[HISQ_MAX_BUNDLE], upd_n;  // right-hand sides of an FP64 recomputation
    const int tid = threadIdx.x, n = a.n;
    {
        constexpr int WORDS = sizeof(SolverState) / sizeof(uint32_t);
        const uint32_t *src = reinterpret_cast<const uint32_t *>(a.st);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&st);
        for (int i = tid; i < WORDS; i += blockDim.x) dst[i] = __ldcg(src + i);
    }
    __syncthreads();
    // vector phases: thread (site row sl, right-hand side r) over the block's share of the sites
    const int r = tid % n, spb = blockDim.x / n, sl = tid / n;
    const int ts = tile_sites(a.g.Vh, spb);
    // views are rebuilt from the (constant-bank) arguments where they are used: nothing of them
    // stays live in registers across the Dslash phases
#define V64(f) VecView<HISQ_FP64>{a.f, n}
#define VQ(f) VecView<Q>{a.f, n}
#define VP(f) VecView<P>{a.f, n}
    const bool row_ok = sl < ts;

    // ---- setup: x_hi = 0, x = 0, r = b, p = b and |b|^2 ----
    {
        double acc[1] = {0.0};
        if (row_ok) {
            for (int tile = blockIdx.x; (long)tile * ts < a.g.Vh; tile += gridDim.x) {
                const int s = tile * ts + sl;
                if (s >= a.g.Vh) break;
                Cplx<double> b[3];
                load_vec<HISQ_FP64, true>(V64(b), s, r, b);
                const Cplx<double> z64[3] = {{0, 0}, {0, 0}, {0, 0}};
                const Cplx<rq> zq[3] = {{0, 0}, {0, 0}, {0, 0}};
                Cplx<rq> bq[3];
                Cplx<rp> bp[3];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    acc[0] += b[c].re * b[c].re + b[c].im * b[c].im;
                    bq[c] = {(rq)b[c].re, (rq)b[c].im};
                    bp[c] = {(rp)b[c].re, (rp)b[c].im};
                }
                store_vec<HISQ_FP64>(V64(xhi), s, r, z64);
                store_vec<Q>(VQ(x), s, r, zq);
                store_vec<Q>(VQ(r), s, r, bq);
                store_vec<P>(VP(p), s, r, bp);
            }
        }
        publish_dots<1>(a, red, acc, n, r, n);
    }
    bool ok = grid_sync(a);
    if (ok) {
        sum_partials(a, red, n, dots);
        if (tid == 0) run_hook(HOOK_INIT, &st, dots, n);
        __syncthreads();
    }
    clock_start(clk, a.phase_ns);

    // ---- Hestenes-Stiefel CG with one reduction: three phases an iteration ----
    while (CG1 && ok && st.any_active && st.bundle_iters < st.max_iter) {
        // t = D_oe p
        dslash_phase<P, R, EPI_PLAIN, Q>(a, a.fat, a.naik, PlainIn<P, true>{VP(p)}, a.t, 1, st.active,
                                         PlainIn<P, true>{VP(p)}, nullptr, nullptr, red, st.mass2);
        if (!(ok = grid_sync(a))) break;
        clock_mark(clk, PH_DOE);
        // A p = m^2 p - D_eo t with <p, A p> and |A p|^2 (|r|^2 came from the previous update phase)
        dslash_phase<P, R, EPI_AOP, Q, PlainIn<P, true>, PlainIn<P, true>, true>(
            a, a.fat, a.naik, PlainIn<P, true>{VP(t)}, a.ap, 0, st.active, PlainIn<P, true>{VP(p)}, nullptr, nullptr, red, st.mass2);
        if (!(ok = grid_sync(a))) break;
        sum_partials(a, red, 3 * n, dots);
        if (tid == 0) run_hook(HOOK_CG1, &st, dots, n);
        __syncthreads();
        clock_mark(clk, PH_AOP);
        // x += alpha p; r -= alpha A p with |r|^2 (for the next iteration's step); p = r + beta p,
        // except where an FP64 recomputation is due (there x_hi += x, x = 0, and p waits for the
        // true residual)
        double rr_acc[1] = {0.0};
        if (st.active[r] && row_ok) {
            const rq al = (rq)st.alpha[r][0];
            const rp be = (rp)st.beta[r][0];
            const bool upd = st.update[r] != 0;
            for (int tile = blockIdx.x; (long)tile * ts < a.g.Vh; tile += gridDim.x) {
                const int s = tile * ts + sl;
                if (s >= a.g.Vh) break;
                Cplx<rp> p[3], ap[3];
                Cplx<rq> x[3], rv[3];
                load_vec<P, true>(VP(p), s, r, p);
                load_vec<P, true>(VP(ap), s, r, ap);
                load_vec<Q, true>(VQ(x), s, r, x);
                load_vec<Q, true>(VQ(r), s, r, rv);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    x[c].re += al * (rq)p[c].re;
                    x[c].im += al * (rq)p[c].im;
                    rv[c].re -= al * (rq)ap[c].re;
                    rv[c].im -= al * (rq)ap[c].im;
                }
                store_vec<Q>(VQ(r), s, r, rv);
                rq part = 0;
#pragma unroll
                for (int c = 0; c < 3; c++) part += rv[c].re * rv[c].re + rv[c].im * rv[c].im;
                rr_acc[0] += (double)part;
                if (upd) {
                    Cplx<double> xh[3];
                    const Cplx<rq> zq[3] = {{0, 0}, {0, 0}, {0, 0}};
                    load_vec<HISQ_FP64, true>(V64(xhi), s, r, xh);
#pragma unroll
                    for (int c = 0; c < 3; c++) xh[c] = {xh[c].re + (double)x[c].re, xh[c].im + (double)x[c].im};
                    store_vec<HISQ_FP64>(V64(xhi), s, r, xh);
                    if constexpr (P != HISQ_FP64) store_xds(a, s, r, xh);
                    store_vec<Q>(VQ(x), s, r, zq);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; c++) p[c] = {(rp)rv[c].re + be * p[c].re, (rp)rv[c].im + be * p[c].im};
                    store_vec<Q>(VQ(x), s, r, x);
                    store_vec<P>(VP(p), s, r, p);
                }
            }
        }
        publish_dots<1>(a, red, rr_acc, n, r, n, n);  // partials columns n..2n-1
        if (!(ok = grid_sync(a))) break;
        clock_mark(clk, PH_UPDATE);
        if (st.any_update) {
            // r = b - A x_hi in FP64 (written to r), |r|^2; then p = r + beta p with beta from it.
            // Only the right-hand sides due for it take part (the FP64 passes are FP64-arithmetic
            // bound, so their cost follows the number of such right-hand sides)
            if (tid == 0) {
                int u = 0;
                for (int k = 0; k < n; k++)
                    if (st.update[k]) upd_list[u++] = k;
                upd_n = u;
            }
            __syncthreads();
            if constexpr (P == HISQ_FP64) {
                dslash_phase<HISQ_FP64, 1, EPI_PLAIN, Q>(a, a.fat64, a.naik64, PlainIn<HISQ_FP64, true>{V64(xhi)}, a.t64,
                                                         1, st.update, PlainIn<HISQ_FP64, true>{V64(xhi)}, nullptr,
                                                         nullptr, red, st.mass2, upd_list, upd_n);
                if (!(ok = grid_sync(a))) break;
                dslash_phase<HISQ_FP64, 1, EPI_RESID, Q>(a, a.fat64, a.naik64, PlainIn<HISQ_FP64, true>{V64(t64)},
                                                         nullptr, 0, st.update, PlainIn<HISQ_FP64, true>{V64(xhi)}, a.b,
                                                         a.r, red, st.mass2, upd_list, upd_n);
            } else {
                ds_phase<EPI_PLAIN, Q, 1, false>(a, a.xds, a.t64, 1, nullptr, nullptr, nullptr, red, st.mass2, upd_list, upd_n);
                if (!(ok = grid_sync(a))) break;
                ds_phase<EPI_RESID, Q, 1, false>(a, a.t64, nullptr, 0, a.xhi, a.b, a.r, red, st.mass2, upd_list, upd_n);
            }
            if (!(ok = grid_sync(a))) break;
            sum_partials(a, red, upd_n, dots);
            if (tid == 0) {
                for (int i = upd_n - 1; i >= 0; i--) dots[upd_list[i]] = dots[i];  // listed order -> RHS index
                run_hook(HOOK_RELIABLE, &st, dots, n);
            }
            __syncthreads();
            if (st.update[r] && st.active[r] && row_ok) {
                const rp be = (rp)st.beta[r][0];
                for (int tile = blockIdx.x; (long)tile * ts < a.g.Vh; tile += gridDim.x) {
                    const int s = tile * ts + sl;
                    if (s >= a.g.Vh) break;
                    Cplx<rq> rv[3];
                    Cplx<rp> p[3];
                    load_vec<Q, true>(VQ(r), s, r, rv);
                    load_vec<P, true>(VP(p), s, r, p);
#pragma unroll
                    for (int c = 0; c < 3; c++) p[c] = {(rp)rv[c].re + be * p[c].re, (rp)rv[c].im + be * p[c].im};
                    store_vec<P>(VP(p), s, r, p);
                }
            }
            if (!(ok = grid_sync(a))) break;
            clock_mark(clk, PH_RELIABLE);
        }
    }

    // ---- Hestenes-Stiefel CG: four phases and two reductions an iteration ----
    while (!CG1 && ok && st.any_active && st.bundle_iters < st.max_iter) {
        // t = D_oe p
        dslash_phase<P, R, EPI_PLAIN, Q>(a, a.fat, a.naik, PlainIn<P, true>{VP(p)}, a.t, 1, st.active,
                                         PlainIn<P, true>{VP(p)}, nullptr, nullptr, red, st.mass2);
        if (!(ok = grid_sync(a))) break;
        clock_mark(clk, PH_DOE);
        // A p = m^2 p - D_eo t and <p, A p>
        dslash_phase<P, R, EPI_AOP, Q>(a, a.fat, a.naik, PlainIn<P, true>{VP(t)}, a.ap, 0, st.active,
                                       PlainIn<P, true>{VP(p)}, nullptr, nullptr, red, st.mass2);
        if (!(ok = grid_sync(a))) break;
        sum_partials(a, red, n, dots);
        if (tid == 0) run_hook(HOOK_ALPHA, &st, dots, n);
        __syncthreads();
        clock_mark(clk, PH_AOP);
        // x += alpha p; r -= alpha A p; |r|^2
        {
            double acc[1] = {0.0};
            if (st.active[r] && row_ok) {
                const rq al = (rq)st.alpha[r][0];
                for (int tile = blockIdx.x; (long)tile * ts < a.g.Vh; tile += gridDim.x) {
                    const int s = tile * ts + sl;
                    if (s >= a.g.Vh) break;
                    Cplx<rp> p[3], ap[3];
                    Cplx<rq> x[3], rv[3];
                    load_vec<P, true>(VP(p), s, r, p);
                    load_vec<P, true>(VP(ap), s, r, ap);
                    load_vec<Q, true>(VQ(x), s, r, x);
                    load_vec<Q, true>(VQ(r), s, r, rv);
                    rq part = 0;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        x[c].re += al * (rq)p[c].re;
                        x[c].im += al * (rq)p[c].im;
                        rv[c].re -= al * (rq)ap[c].re;
                        rv[c].im -= al * (rq)ap[c].im;
                        part += rv[c].re * rv[c].re + rv[c].im * rv[c].im;
                    }
                    acc[0] += (double)part;
                    store_vec<Q>(VQ(x), s, r, x);
                    store_vec<Q>(VQ(r), s, r, rv);
                }
            }
            publish_dots<1>(a, red, acc, n, r, n);
        }
        if (!(ok = grid_sync(a))) break;
        sum_partials(a, red, n, dots);
        if (tid == 0) run_hook(HOOK_DECIDE, &st, dots, n);
        __syncthreads();
        clock_mark(clk, PH_UPDATE);
        if (st.any_update) {
            // reliable update: x_hi += x; x = 0; r = b - A x_hi in FP64 (written to r), |r|^2
            if (st.update[r] && row_ok) {
                for (int tile = blockIdx.x; (long)tile * ts < a.g.Vh; tile += gridDim.x) {
                    const int s = tile * ts + sl;
                    if (s >= a.g.Vh) break;
                    Cplx<rq> x[3];
                    const Cplx<rq> zq[3] = {{0, 0}, {0, 0}, {0, 0}};
                    Cplx<double> xh[3];
                    load_vec<Q, true>(VQ(x), s, r, x);
                    load_vec<HISQ_FP64, true>(V64(xhi), s, r, xh);
#pragma unroll
                    for (int c = 0; c < 3; c++) xh[c] = {xh[c].re + (double)x[c].re, xh[c].im + (double)x[c].im};
                    store_vec<HISQ_FP64>(V64(xhi), s, r, xh);
                    if constexpr (P != HISQ_FP64) store_xds(a, s, r, xh);
                    store_vec<Q>(VQ(x), s, r, zq);
                }
            }
            if (!(ok = grid_sync(a))) break;
            if constexpr (P == HISQ_FP64) {
                dslash_phase<HISQ_FP64, 1, EPI_PLAIN, Q>(a, a.fat64, a.naik64, PlainIn<HISQ_FP64, true>{V64(xhi)}, a.t64,
                                                         1, st.update, PlainIn<HISQ_FP64, true>{V64(xhi)}, nullptr,
                                                         nullptr, red, st.mass2);
                if (!(ok = grid_sync(a))) break;
                dslash_phase<HISQ_FP64, 1, EPI_RESID, Q>(a, a.fat64, a.naik64, PlainIn<HISQ_FP64, true>{V64(t64)},
                                                         nullptr, 0, st.update, PlainIn<HISQ_FP64, true>{V64(xhi)}, a.b,
                                                         a.r, red, st.mass2);
                if (!(ok = grid_sync(a))) break;
                sum_partials(a, red, n, dots);
            } else {
                // the right-hand sides due for the recomputation, listed (this form recomputes
                // bundle-wide, so every active one)
                if (tid == 0) {
                    int u = 0;
                    for (int k = 0; k < n; k++)
                        if (st.update[k]) upd_list[u++] = k;
                    upd_n = u;
                }
                __syncthreads();
                ds_phase<EPI_PLAIN, Q, 1, false>(a, a.xds, a.t64, 1, nullptr, nullptr, nullptr, red, st.mass2, upd_list, upd_n);
                if (!(ok = grid_sync(a))) break;
                ds_phase<EPI_RESID, Q, 1, false>(a, a.t64, nullptr, 0, a.xhi, a.b, a.r, red, st.mass2, upd_list, upd_n);
                if (!(ok = grid_sync(a))) break;
                sum_partials(a, red, upd_n, dots);
                if (tid == 0)
                    for (int i = upd_n - 1; i >= 0; i--) dots[upd_list[i]] = dots[i];  // listed order -> RHS index
                __syncthreads();
            }
            if (tid == 0) run_hook(HOOK_RELIABLE, &st, dots, n);
            __syncthreads();
            clock_mark(clk, PH_RELIABLE);
        }
        // p = r + beta p
        if (st.active[r] && row_ok) {
            const rp be = (rp)st.beta[r][0];
            for (int tile = blockIdx.x; (long)tile * ts < a.g.Vh; tile += gridDim.x) {
                const int s = tile * ts + sl;
                if (s >= a.g.Vh) break;
                Cplx<rq> rv[3];
                Cplx<rp> p[3];
                load_vec<Q, true>(VQ(r), s, r, rv);
                load_vec<P, true>(VP(p), s, r, p);
#pragma unroll
                for (int c = 0; c < 3; c++) p[c] = {(rp)rv[c].re + be * p[c].re, (rp)rv[c].im + be * p[c].im};
                store_vec<P>(VP(p), s, r, p);
            }
        }
        if (!(ok = grid_sync(a))) break;
        clock_mark(clk, PH_PUPDATE);
    }
#undef V64
#undef VQ
#undef VP
    clock_store(clk, a.phase_ns);
    if (blockIdx.x == 0) {  // the final bundle state for the host
        __syncthreads();
        constexpr int WORDS = sizeof(SolverState) / sizeof(uint32_t);
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&st);
        uint32_t *dst = reinterpret_cast<uint32_t *>(a.st);
        for (int i = tid; i < WORDS; i += blockDim.x) dst[i] = src[i];
    }
}

// the instantiation for R right-hand sides per thread (FP64 stops at two: four would spill) and
// the CG form
template <int P, bool CG1>
const void *persistent_kernel_ptr(int R) {
    if constexpr (P != HISQ_FP64) {
        if (R == 4) return (const void *)cg_persistent_kernel<P, 4, CG1>;
    }
    if (R >= 2) return (const void *)cg_persistent_kernel<P, 2, CG1>;
    return (const void *)cg_persistent_kernel<P, 1, CG1>;
}

template <int P>
const void *persistent_kernel_ptr(int R, bool cg1) {
    return cg1 ? persistent_kernel_ptr<P, true>(R) : persistent_kernel_ptr<P, false>(R);
}

template <int P>
cudaError_t launch_persistent_prec(const PersArgs &a, int R, bool cg1, int grid, int threads, size_t smem,
                                   cudaStream_t st) {
    void *args[] = {const_cast<PersArgs *>(&a)};
    if (P == HISQ_FP64 && R > 2) return cudaErrorInvalidValue;
    const void *k = persistent_kernel_ptr<P>(R, cg1);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(k, grid, threads, args, smem, st);
}

template <int P>
cudaError_t persistent_occupancy(int R, bool cg1, int threads, size_t smem, int *blocks_per_sm) {
    if (P == HISQ_FP64 && R > 2) return cudaErrorInvalidValue;
    const void *k = persistent_kernel_ptr<P>(R, cg1);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem);
}

}  // namespace hisq
