// Multi-right-hand-side even-odd HISQ Dslash kernel (Eq. (3)-(4)) with fused epilogues.
//
// One thread handles R right-hand sides of one output site; t = ceil(n / R) threads share a
// site and read its links together (the same 16-byte words, so one memory transaction serves
// all of them), spb = threads / t sites per block.  Every link record is read once per site
// for the whole bundle; the neighbour vectors come through L1/L2.  Grid-stride over site tiles
// with a grid of whole waves.  Epilogues:
//   EPI_PLAIN  w = D v
//   EPI_AOP    w = m^2 p - D v and the per-RHS dot Re <p, w>          (second half of A p)
//   EPI_RESID  r = b - m^2 x + D v and |r|^2, written to a sloppy copy  (FP64 true residual)
// Reducing epilogues finish with a deterministic block tree, per-block partials in FP64 and a
// last-block-done reduction (no waiting), whose last block runs the solver hook.
#pragma once
#include "hisq_internal.cuh"
#include "link_codec.cuh"
#include "solver_state.cuh"

namespace hisq {

// Reduction plumbing shared by every reducing kernel.
struct RedArgs {
    double *partials;      // [grid][ndots]
    unsigned int *counter; // last-block-done ticket (reset to 0 by the last block)
    double *dot_out;       // [ndots] final dots (may be null)
    int hook;              // solver hook run by the last block (HOOK_NONE = none)
    SolverState *st;
};

struct KArgs {
    Geom g;
    LinkField fat, naik;
    const void *in;
    void *out;
    int n, t, spb, parity;
    double mass2;
    const void *axpy;
    const void *b;
    void *out_lo;
    int lo_prec;
    const int *active;
    const int *gate;
    RedArgs red;
};

template <int P>
__device__ __forceinline__ VecView<P> view(const void *base, int Vh, int n) {
    VecView<P> v;
    v.data = const_cast<void *>(base);
    v.n = n;
    v.scale = (P == HISQ_FP16 && base)
                  ? reinterpret_cast<float *>(reinterpret_cast<char *>(const_cast<void *>(base)) + fp16_scale_offset(Vh, n))
                  : nullptr;
    return v;
}

// Deterministic reduction of red[rows][ndots] (shared, rows a power of two) into per-block
// partials, then the last-block-done finish: the block that takes the last ticket sums the
// partials of all blocks in a fixed order, writes dot_out and runs the hook for a bundle of
// hook_n right-hand sides.  No block ever waits for another.  All threads of the block call it;
// ndots may be 0 (hook only).  red must hold max(rows * ndots, blockDim.x) doubles.
__device__ __forceinline__ void block_reduce_finish(double *red, int rows, int ndots, int hook_n, const RedArgs &ra) {
    const int tid = threadIdx.x;
    if (ndots > 0) {
        for (int stride = rows / 2; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = tid; i < stride * ndots; i += blockDim.x) {
                int row = i / ndots, j = i - row * ndots;
                red[row * ndots + j] += red[(row + stride) * ndots + j];
            }
        }
        __syncthreads();
        for (int j = tid; j < ndots; j += blockDim.x) ra.partials[(size_t)blockIdx.x * ndots + j] = red[j];
        // only the threads that published partials fence them before the ticket is taken
        if (tid < ndots) __threadfence();
    }
    __shared__ int is_last;
    __syncthreads();
    if (tid == 0) is_last = (atomicAdd(ra.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    if (tid == 0) __threadfence();
    __syncthreads();
    if (ndots > 0) {
        int nchunks = 1;
        while (nchunks * 2 * ndots <= (int)blockDim.x) nchunks *= 2;
        for (int i = tid; i < nchunks * ndots; i += blockDim.x) {
            int chunk = i / ndots, j = i - chunk * ndots;
            double s = 0.0;
            for (int b = chunk; b < (int)gridDim.x; b += nchunks) s += __ldcg(ra.partials + (size_t)b * ndots + j);
            red[chunk * ndots + j] = s;
        }
        for (int stride = nchunks / 2; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = tid; i < stride * ndots; i += blockDim.x) {
                int chunk = i / ndots, j = i - chunk * ndots;
                red[chunk * ndots + j] += red[(chunk + stride) * ndots + j];
            }
        }
        __syncthreads();
        if (ra.dot_out)
            for (int j = tid; j < ndots; j += blockDim.x) ra.dot_out[j] = red[j];
    }
    if (tid == 0) {
        if (ra.hook && ra.st) run_hook(ra.hook, ra.st, red, hook_n);
        *ra.counter = 0u;
        __threadfence();
    }
}

template <int P, int NR, int R, int EPI>
__global__ void __launch_bounds__(256) dslash_kernel(KArgs a) {
    using real = typename Prec<P>::real;
    using FatC = LinkCodec<P, 18>;
    using NaikC = LinkCodec<P, NR>;
    extern __shared__ double red[];

    if (a.gate && *a.gate == 0) return;

    const Geom &g = a.g;
    const int tid = threadIdx.x;
    const int gi = tid % a.t;
    const int sl = tid / a.t;
    const int r0 = gi * R;
    const int nvalid = min(R, a.n - r0);
    const VecView<P> vin = view<P>(a.in, g.Vh, a.n);
    const VecView<P> vout = view<P>(a.out, g.Vh, a.n);

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

    for (int tile = blockIdx.x; (long)tile * a.spb < g.Vh; tile += gridDim.x) {
        const int s = tile * a.spb + sl;
        if (s >= g.Vh || !any_act) continue;
        const SiteCoord sc = decode_site(g, s, a.parity);

        Cplx<real> acc[R][3];
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[r][c] = {0, 0};

        // ---- fat links: one hop ----
        real fscale = (real)1;
        if (a.fat.scale) fscale = (real)__ldg(a.fat.scale + (size_t)a.parity * g.Vh + s);
#pragma unroll
        for (int grp = 0; grp < FatC::GROUPS; grp++) {
            uint32_t u[FatC::WG * 4];
            FatC::load_group(a.fat, a.parity, g.Vh, s, grp, u);
#pragma unroll
            for (int l = 0; l < FatC::G; l++) {
                const int slot = grp * FatC::G + l;
                const int mu = slot >> 1;
                const int nb = neighbour(g, sc, s, mu, (slot & 1) ? -1 : 1);
                Cplx<real> M[3][3];
                FatC::decode(u, l, fscale, M);
                Cplx<real> v[R][3];
#pragma unroll
                for (int r = 0; r < R; r++) {
                    if (act[r]) {
                        float sc_in = 1.0f;
                        if (P == HISQ_FP16) sc_in = __ldg(vin.scale + (long)nb * a.n + r0 + r);
#pragma unroll
                        for (int c = 0; c < 3; c++) v[r][c] = load_elem<P>(vin, ((long)nb * 3 + c) * a.n + r0 + r, sc_in);
                    } else {
#pragma unroll
                        for (int c = 0; c < 3; c++) v[r][c] = {0, 0};
                    }
                }
                matvec_acc<real, R>(M, v, acc);
            }
        }
        // ---- Naik links: three hops ----
        real nscale = (real)1;
        if (NR == 18 && a.naik.scale) nscale = (real)__ldg(a.naik.scale + (size_t)a.parity * g.Vh + s);
#pragma unroll
        for (int grp = 0; grp < NaikC::GROUPS; grp++) {
            uint32_t u[NaikC::WG * 4];
            NaikC::load_group(a.naik, a.parity, g.Vh, s, grp, u);
#pragma unroll
            for (int l = 0; l < NaikC::G; l++) {
                const int slot = grp * NaikC::G + l;
                const int mu = slot >> 1;
                const int nb = neighbour(g, sc, s, mu, (slot & 1) ? -3 : 3);
                Cplx<real> M[3][3];
                NaikC::decode(u, l, nscale, M);
                Cplx<real> v[R][3];
#pragma unroll
                for (int r = 0; r < R; r++) {
                    if (act[r]) {
                        float sc_in = 1.0f;
                        if (P == HISQ_FP16) sc_in = __ldg(vin.scale + (long)nb * a.n + r0 + r);
#pragma unroll
                        for (int c = 0; c < 3; c++) v[r][c] = load_elem<P>(vin, ((long)nb * 3 + c) * a.n + r0 + r, sc_in);
                    } else {
#pragma unroll
                        for (int c = 0; c < 3; c++) v[r][c] = {0, 0};
                    }
                }
                matvec_acc<real, R>(M, v, acc);
            }
        }

        // ---- epilogue ----
        if constexpr (EPI == EPI_PLAIN) {
#pragma unroll
            for (int r = 0; r < R; r++)
                if (act[r]) store_site<P>(vout, s, r0 + r, acc[r]);
        } else if constexpr (EPI == EPI_AOP) {
            const VecView<P> vp = view<P>(a.axpy, g.Vh, a.n);
            const real m2 = (real)a.mass2;
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (!act[r]) continue;
                float sc_p = 1.0f;
                if (P == HISQ_FP16) sc_p = __ldg(vp.scale + (long)s * a.n + r0 + r);
                Cplx<real> w[3];
                real d = 0;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    Cplx<real> p = load_elem<P>(vp, ((long)s * 3 + c) * a.n + r0 + r, sc_p);
                    w[c] = {m2 * p.re - acc[r][c].re, m2 * p.im - acc[r][c].im};
                    d += p.re * w[c].re + p.im * w[c].im;
                }
                dot[r] += (double)d;
                store_site<P>(vout, s, r0 + r, w);
            }
        } else {
            static_assert(EPI == EPI_RESID && P == HISQ_FP64, "residual epilogue is FP64 only");
            const VecView<HISQ_FP64> vx = view<HISQ_FP64>(a.axpy, g.Vh, a.n);
            const VecView<HISQ_FP64> vb = view<HISQ_FP64>(a.b, g.Vh, a.n);
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (!act[r]) continue;
                Cplx<double> w[3];
                double d = 0.0;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    long idx = ((long)s * 3 + c) * a.n + r0 + r;
                    Cplx<double> x = load_elem<HISQ_FP64>(vx, idx, 1.0f);
                    Cplx<double> b = load_elem<HISQ_FP64>(vb, idx, 1.0f);
                    w[c] = {b.re - a.mass2 * x.re + (double)acc[r][c].re, b.im - a.mass2 * x.im + (double)acc[r][c].im};
                    d += w[c].re * w[c].re + w[c].im * w[c].im;
                }
                dot[r] += d;
                if (a.out) store_site<HISQ_FP64>(vout, s, r0 + r, w);
                if (a.out_lo) {
                    long base = (long)s * 3 * a.n + r0 + r;
                    if (a.lo_prec == HISQ_FP64) {
                        double2 *o = reinterpret_cast<double2 *>(a.out_lo);
#pragma unroll
                        for (int c = 0; c < 3; c++) o[base + (long)c * a.n] = make_double2(w[c].re, w[c].im);
                    } else {
                        float2 *o = reinterpret_cast<float2 *>(a.out_lo);
#pragma unroll
                        for (int c = 0; c < 3; c++) o[base + (long)c * a.n] = make_float2((float)w[c].re, (float)w[c].im);
                    }
                }
            }
        }
    }

    if constexpr (EPI != EPI_PLAIN) {
        // red[spb][n]: each thread writes its R partial dots
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

}  // namespace hisq
