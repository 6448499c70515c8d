// Body of the persistent solve kernel (see cg_persistent.cuh).
#pragma once
#include "cg_persistent.cuh"

namespace hisq {

// With one right-hand side per thread, four 256-thread blocks per SM (at most 64 registers) keep
// every site of a 32^3 x 8 parity resident in a single pass of each Dslash phase.
template <int P, int R>
__global__ void __launch_bounds__(256, R == 1 ? 4 : 2) cg_persistent_kernel(PersArgs a) {
    constexpr int Q = q_prec(P);
    using rp = typename Prec<P>::real;
    using rq = typename Prec<Q>::real;
    extern __shared__ double red[];
    __shared__ SolverState st;
    __shared__ double dots[PERS_ND];
    const int tid = threadIdx.x, n = a.n;
    const long Vh = a.g.Vh;
    {
        constexpr int WORDS = sizeof(SolverState) / sizeof(uint32_t);
        const uint32_t *src = reinterpret_cast<const uint32_t *>(a.st);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&st);
        for (int i = tid; i < WORDS; i += blockDim.x) dst[i] = __ldcg(src + i);
    }
    __syncthreads();
    // BLAS phases: thread (site row sl, right-hand side r)
    const int r = tid % n, spb = blockDim.x / n, sl = tid / n;
    const VecView<HISQ_FP64> vb{a.b, n}, vxh{a.xhi, n};
    const VecView<Q> vx{a.x, n}, vr{a.r, n};
    const VecView<P> vp{a.p, n}, vap{a.ap, n};
    auto publish = [&](double acc) {
        for (int i = tid; i < spb * n; i += blockDim.x) red[i] = 0.0;
        __syncthreads();
        if (sl < spb) red[sl * n + r] = acc;
        block_partials(a, red, spb, n);
    };

    // ---- setup: x_hi = 0, x = 0, r = b, p = b and |b|^2 ----
    {
        double acc = 0.0;
        for (long tile = blockIdx.x; tile * spb < Vh; tile += gridDim.x) {
            const long s = tile * spb + sl;
            if (sl >= spb || s >= Vh) continue;
            Cplx<double> b[3];
            load_vec<HISQ_FP64, true>(vb, s, r, b);
            Cplx<double> z64[3] = {{0, 0}, {0, 0}, {0, 0}};
            Cplx<rq> zq[3] = {{0, 0}, {0, 0}, {0, 0}}, bq[3];
            Cplx<rp> bp[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                acc += b[c].re * b[c].re + b[c].im * b[c].im;
                bq[c] = {(rq)b[c].re, (rq)b[c].im};
                bp[c] = {(rp)b[c].re, (rp)b[c].im};
            }
            store_vec<HISQ_FP64>(vxh, s, r, z64);
            store_vec<Q>(vx, s, r, zq);
            store_vec<Q>(vr, s, r, bq);
            store_vec<P>(vp, s, r, bp);
        }
        publish(acc);
    }
    bool ok = grid_sync(a);
    if (ok) {
        sum_partials(a, red, n, dots);
        if (tid == 0) run_hook(HOOK_INIT, &st, dots, n);
        __syncthreads();
    }
    __shared__ PhaseClock clk;
    clock_start(clk, a.phase_ns);

    while (ok && st.any_active && st.bundle_iters < st.max_iter) {
        // t = D_oe p
        dslash_phase<P, R, EPI_PLAIN, Q>(a, a.fat, a.naik, a.p, a.t, 1, st.active, nullptr, nullptr, nullptr, red);
        if (!(ok = grid_sync(a))) break;
        clock_mark(clk, PH_DOE);
        // A p = m^2 p - D_eo t and <p, A p>
        dslash_phase<P, R, EPI_AOP, Q>(a, a.fat, a.naik, a.t, a.ap, 0, st.active, a.p, nullptr, nullptr, red);
        if (!(ok = grid_sync(a))) break;
        sum_partials(a, red, n, dots);
        if (tid == 0) run_hook(HOOK_ALPHA, &st, dots, n);
        __syncthreads();
        clock_mark(clk, PH_AOP);
        // x += alpha p; r -= alpha A p; |r|^2
        {
            double acc = 0.0;
            if (st.active[r]) {
                const rq al = (rq)st.alpha[r][0];
                for (long tile = blockIdx.x; tile * spb < Vh; tile += gridDim.x) {
                    const long s = tile * spb + sl;
                    if (sl >= spb || s >= Vh) continue;
                    Cplx<rp> p[3], ap[3];
                    Cplx<rq> x[3], rv[3];
                    load_vec<P, true>(vp, s, r, p);
                    load_vec<P, true>(vap, s, r, ap);
                    load_vec<Q, true>(vx, s, r, x);
                    load_vec<Q, true>(vr, s, r, rv);
                    rq part = 0;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        x[c].re += al * (rq)p[c].re;
                        x[c].im += al * (rq)p[c].im;
                        rv[c].re -= al * (rq)ap[c].re;
                        rv[c].im -= al * (rq)ap[c].im;
                        part += rv[c].re * rv[c].re + rv[c].im * rv[c].im;
                    }
                    acc += (double)part;
                    store_vec<Q>(vx, s, r, x);
                    store_vec<Q>(vr, s, r, rv);
                }
            }
            publish(acc);
        }
        if (!(ok = grid_sync(a))) break;
        sum_partials(a, red, n, dots);
        if (tid == 0) run_hook(HOOK_DECIDE, &st, dots, n);
        __syncthreads();
        clock_mark(clk, PH_UPDATE);
        if (st.any_update) {
            // reliable update: x_hi += x; x = 0; r = b - A x_hi in FP64 (written to r), |r|^2
            if (st.update[r]) {
                for (long tile = blockIdx.x; tile * spb < Vh; tile += gridDim.x) {
                    const long s = tile * spb + sl;
                    if (sl >= spb || s >= Vh) continue;
                    Cplx<rq> x[3], zq[3] = {{0, 0}, {0, 0}, {0, 0}};
                    Cplx<double> xh[3];
                    load_vec<Q, true>(vx, s, r, x);
                    load_vec<HISQ_FP64, true>(vxh, s, r, xh);
#pragma unroll
                    for (int c = 0; c < 3; c++) xh[c] = {xh[c].re + (double)x[c].re, xh[c].im + (double)x[c].im};
                    store_vec<HISQ_FP64>(vxh, s, r, xh);
                    store_vec<Q>(vx, s, r, zq);
                }
            }
            if (!(ok = grid_sync(a))) break;
            dslash_phase<HISQ_FP64, 1, EPI_PLAIN, Q>(a, a.fat64, a.naik64, a.xhi, a.t64, 1, st.update, nullptr, nullptr,
                                                     nullptr, red);
            if (!(ok = grid_sync(a))) break;
            dslash_phase<HISQ_FP64, 1, EPI_RESID, Q>(a, a.fat64, a.naik64, a.t64, nullptr, 0, st.update, a.xhi, a.b,
                                                     a.r, red);
            if (!(ok = grid_sync(a))) break;
            sum_partials(a, red, n, dots);
            if (tid == 0) run_hook(HOOK_RELIABLE, &st, dots, n);
            __syncthreads();
            clock_mark(clk, PH_RELIABLE);
        }
        // p = r + beta p
        if (st.active[r]) {
            const rp be = (rp)st.beta[r][0];
            for (long tile = blockIdx.x; tile * spb < Vh; tile += gridDim.x) {
                const long s = tile * spb + sl;
                if (sl >= spb || s >= Vh) continue;
                Cplx<rq> rv[3];
                Cplx<rp> p[3];
                load_vec<Q, true>(vr, s, r, rv);
                load_vec<P, true>(vp, s, r, p);
#pragma unroll
                for (int c = 0; c < 3; c++) p[c] = {(rp)rv[c].re + be * p[c].re, (rp)rv[c].im + be * p[c].im};
                store_vec<P>(vp, s, r, p);
            }
        }
        if (!(ok = grid_sync(a))) break;
        clock_mark(clk, PH_PUPDATE);
    }
    clock_store(clk, a.phase_ns);
    if (blockIdx.x == 0) {  // the final bundle state for the host
        __syncthreads();
        constexpr int WORDS = sizeof(SolverState) / sizeof(uint32_t);
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&st);
        uint32_t *dst = reinterpret_cast<uint32_t *>(a.st);
        for (int i = tid; i < WORDS; i += blockDim.x) dst[i] = src[i];
    }
}

template <int P>
cudaError_t launch_persistent_prec(const PersArgs &a, int R, int grid, size_t smem, cudaStream_t st) {
    void *args[] = {const_cast<PersArgs *>(&a)};
    const void *k = R == 4 ? (const void *)cg_persistent_kernel<P, 4>
                  : R == 2 ? (const void *)cg_persistent_kernel<P, 2>
                           : (const void *)cg_persistent_kernel<P, 1>;
    return cudaLaunchCooperativeKernel(k, grid, 256, args, smem, st);
}

template <int P>
cudaError_t persistent_occupancy(int R, size_t smem, int *blocks_per_sm) {
    const void *k = R == 4 ? (const void *)cg_persistent_kernel<P, 4>
                  : R == 2 ? (const void *)cg_persistent_kernel<P, 2>
                           : (const void *)cg_persistent_kernel<P, 1>;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 256, smem);
}

}  // namespace hisq
