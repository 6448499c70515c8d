// The whole mixed-precision CG solve of one bundle as one cooperative, persistent kernel.
//
// Every phase of an iteration -- t = D_oe p; A p = m^2 p - D_eo t with <p, A p>; the update of x
// and r with |r|^2 and the decision step; the FP64 residual recomputation when one is due; and
// p = r + beta p -- runs inside one launch, separated by grid barriers.  Each block owns one
// contiguous, equal share of the sites (every SM gets the same work) and keeps its own
// shared-memory copy of the bundle state, evolving it identically: after a barrier every block
// sums the same per-block partials in the same order and runs the same scalar step, so nothing
// has to be broadcast.  The barrier is one counter word whose bit 31 flips when every block has
// arrived; its wait is bounded: a block that waits longer than the spin limit sets an error flag
// and the whole grid returns
// (HISQ_ERR_TIMEOUT on the host).  Vectors written inside the launch are read with ld.global.cg
// (L2), never the read-only path.
#pragma once
#include "dslash_kernel.cuh"
#include "ds_arith.cuh"

namespace hisq {

struct PersArgs {
    Geom g;
    LinkField fat, naik;      // inner precision (18-real Naik)
    LinkField fat64, naik64;  // FP64 links of the residual recomputation: the FP64 copies (P = FP64)
                              // or the double-single copies (otherwise)
    void *p, *t, *ap;         // inner precision bundles
    void *x, *r;              // x_lo and r in the iterated precision
    void *b, *xhi, *t64;      // FP64 (t64: double-single when P != FP64)
    void *xds;                // x_hi in double-single form (P != FP64)
    int n;
    double *partials;         // [gridDim][PERS_ND]
    SolverState *st;          // initial state in, final state out (block 0)
    unsigned int *bar;        // [0] the grid barrier's word (zero at launch)
    int *err;
    long long spin_limit;
    unsigned int expected;    // arrivals that complete a barrier (gridDim.x; more only to test timeouts)
    unsigned long long *phase_ns;  // [PERS_PHASES] time per phase as seen by block 0, or null
};

// Phases of the persistent solve, timed by block 0 from one grid barrier to the next: the
// first Dslash (D_oe p), the second with its epilogue (A p, <p, A p>), the x / r update with
// |r|^2, the FP64 residual recomputations, and the direction update (each phase includes the
// scalar step and barrier that end it).
enum PersPhase { PH_DOE = 0, PH_AOP = 1, PH_UPDATE = 2, PH_RELIABLE = 3, PH_PUPDATE = 4, PERS_PHASES = 5 };

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Block 0, thread 0 charges the time since the previous mark to `phase` (no-op otherwise).  The
// clock lives in shared memory so that it costs the other threads no registers.
struct PhaseClock {
    unsigned long long last, acc[PERS_PHASES];
    int on;
};

__device__ __forceinline__ void clock_start(PhaseClock &c, const unsigned long long *out) {
    if (threadIdx.x == 0) {
        c.on = out != nullptr && blockIdx.x == 0;
        for (int i = 0; i < PERS_PHASES; i++) c.acc[i] = 0;
        c.last = c.on ? global_ns() : 0;
    }
}

__device__ __forceinline__ void clock_mark(PhaseClock &c, int phase) {
    if (threadIdx.x == 0 && c.on) {
        const unsigned long long now = global_ns();
        c.acc[phase] += now - c.last;
        c.last = now;
    }
}

__device__ __forceinline__ void clock_store(const PhaseClock &c, unsigned long long *out) {
    if (threadIdx.x == 0 && c.on)
        for (int i = 0; i < PERS_PHASES; i++) out[i] = c.acc[i];
}

constexpr int PERS_ND = 3 * HISQ_MAX_BUNDLE;  // up to three dots per right-hand side

// Grid barrier on one 32-bit word: block 0 adds 2^31 - (expected - 1) and every other block adds 1,
// so the arrivals of all blocks together flip bit 31 and leave the low bits unchanged (no reset,
// no second word, one atomic round trip).  Each block's thread 0 publishes the block's writes
// (fence, then its arrival) and polls with acquire loads until bit 31 differs from the value its
// own arrival saw.  The wait is bounded: past spin_limit polls the block raises the error flag and
// returns false.  The flag is read only inside the wait (every 1024 polls), not on the way in or
// out, so a completed barrier costs no extra memory round trip; a block whose peer gave up stops
// at its next barrier, which can no longer complete, when it sees the flag.
__device__ __forceinline__ bool grid_sync(const PersArgs &a) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (a.expected - 1u) : 1u;
        __threadfence();
        const unsigned int old = atomicAdd(a.bar, inc);
        long long spins = 0;
        int ok = 1;
        while (true) {
            unsigned int cur;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(a.bar) : "memory");
            if ((cur ^ old) & 0x80000000u) break;
            if (++spins > a.spin_limit) {
                atomicExch(a.err, 1);
                ok = 0;
                break;
            }
            if ((spins & 1023) == 0 && *reinterpret_cast<volatile int *>(a.err) != 0) {  // a peer gave up
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok;
}

// Largest block: 1024 threads at one right-hand side per thread (64 registers), 512 otherwise
// (128 registers); the launch may use fewer (a multiple of 32 dividing into the SM's resources).
__host__ __device__ constexpr int pers_threads(int R) { return R == 1 ? 1024 : 512; }
constexpr int PERS_DEFAULT_THREADS = 512;  // measured best at 32^3 x 8 (one and 16 right-hand sides)

// Sites per tile for a phase whose blocks cover spb sites at a time: when the grid covers the
// lattice in one pass, ceil(count / blocks) (every block one tile of equal size, so every SM
// gets the same work); otherwise spb (tiles strided over the blocks).  Loops over tiles keep
// the register footprint of the stencil within the 64 registers of a 1024-thread block.
__device__ __forceinline__ int tile_sites(int count, int spb) {
    return min(spb, (count + (int)gridDim.x - 1) / (int)gridDim.x);
}

// Per-block column sums of the threads' dots into partials[blockIdx.x][col0 + *].  Thread
// tid = site_row * t + gi holds dot[r] of column gi * R + r (ndots = t * R columns).  With t a
// power of two the lanes of one column meet in a shuffle tree and the warps' sums in one more
// step; otherwise the dots go through red[rows][ndots] (red holds blockDim.x * R doubles).
template <int R>
__device__ __forceinline__ void publish_dots(const PersArgs &a, double *red, double (&dot)[R], int t, int gi,
                                             int ndots, int col0 = 0) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    __syncthreads();  // red may still be read by the previous step
    if ((t & (t - 1)) == 0 && t <= 32) {
        for (int off = 16; off >= t; off >>= 1)
#pragma unroll
            for (int r = 0; r < R; r++) dot[r] += __shfl_xor_sync(0xffffffffu, dot[r], off);
        if (lane < t) {
#pragma unroll
            for (int r = 0; r < R; r++)
                if (gi * R + r < ndots) red[warp * ndots + gi * R + r] = dot[r];
        }
        __syncthreads();
        for (int j = warp; j < ndots; j += nwarps) {
            double s = lane < nwarps ? red[lane * ndots + j] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) a.partials[(size_t)blockIdx.x * PERS_ND + col0 + j] = s;
        }
        return;
    }
    const int rows = blockDim.x / t, row = tid / t;
    for (int i = tid; i < rows * ndots; i += blockDim.x) red[i] = 0.0;
    __syncthreads();
    if (row < rows) {
#pragma unroll
        for (int r = 0; r < R; r++)
            if (gi * R + r < ndots) red[row * ndots + gi * R + r] = dot[r];
    }
    __syncthreads();
    for (int j = warp; j < ndots; j += nwarps) {
        double s = 0.0;
        for (int q = lane; q < rows; q += 32) s += red[q * ndots + j];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) a.partials[(size_t)blockIdx.x * PERS_ND + col0 + j] = s;
    }
}

// The same for K sets of dots in one pass: dot[k][r] is column k step + gi R + r (n = t R,
// step >= n); red holds K blockDim.x * R doubles.
template <int R, int K>
__device__ __forceinline__ void publish_dots_k(const PersArgs &a, double *red, double (&dot)[K][R], int t, int gi,
                                               int n, int step) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int nd = K * n;
    // set k, column j of the set, lands in partials column k * step + j
    auto column = [&](int jj) { return (jj / n) * step + jj % n; };
    __syncthreads();  // red may still be read by the previous step
    if ((t & (t - 1)) == 0 && t <= 32) {
        for (int off = 16; off >= t; off >>= 1)
#pragma unroll
            for (int k = 0; k < K; k++)
#pragma unroll
                for (int r = 0; r < R; r++) dot[k][r] += __shfl_xor_sync(0xffffffffu, dot[k][r], off);
        if (lane < t) {
#pragma unroll
            for (int k = 0; k < K; k++)
#pragma unroll
                for (int r = 0; r < R; r++)
                    if (gi * R + r < n) red[warp * nd + k * n + gi * R + r] = dot[k][r];
        }
        __syncthreads();
        for (int j = warp; j < nd; j += nwarps) {
            double s = lane < nwarps ? red[lane * nd + j] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) a.partials[(size_t)blockIdx.x * PERS_ND + column(j)] = s;
        }
        return;
    }
    const int rows = blockDim.x / t, row = tid / t;
    for (int i = tid; i < rows * nd; i += blockDim.x) red[i] = 0.0;
    __syncthreads();
    if (row < rows) {
#pragma unroll
        for (int k = 0; k < K; k++)
#pragma unroll
            for (int r = 0; r < R; r++)
                if (gi * R + r < n) red[row * nd + k * n + gi * R + r] = dot[k][r];
    }
    __syncthreads();
    for (int j = warp; j < nd; j += nwarps) {
        double s = 0.0;
        for (int q = lane; q < rows; q += 32) s += red[q * nd + j];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) a.partials[(size_t)blockIdx.x * PERS_ND + column(j)] = s;
    }
}

// every block: dots[j] = sum over blocks of partials[b][j], j < ndots, in a fixed order.  Every
// sum is a tree: an FP64 add is a 64-cycle dependent operation on this part, so a chain of adds
// would cost more than the loads it follows.
__device__ __forceinline__ void sum_partials(const PersArgs &a, double *red, int ndots, double *dots) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    int np2 = 1;
    while (np2 < ndots) np2 *= 2;
    const int per = blockDim.x / np2, j = tid % np2, k = tid / np2;
    double s = 0.0;
    if (j < ndots && k < per) {
        // the partials were written by other SMs just before the barrier: four independent loads
        // at a time, then a pairwise sum
        constexpr int U = 4;
        for (int b0 = k; b0 < (int)gridDim.x; b0 += U * per) {
            double v[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int b = b0 + u * per;
                v[u] = b < (int)gridDim.x ? __ldcg(a.partials + (size_t)b * PERS_ND + j) : 0.0;
            }
#pragma unroll
            for (int w = 1; w < U; w *= 2)
#pragma unroll
                for (int u = 0; u < U; u += 2 * w) v[u] += v[u + w];
            s += v[0];
        }
    }
    for (int off = 16; off >= np2; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const int groups = np2 < 32 ? nwarps : per;  // partial sums per column (at most 32)
    __syncthreads();
    if (np2 < 32) {
        if (lane < np2) red[warp * np2 + lane] = s;
    } else {
        red[tid] = s;
    }
    __syncthreads();
    for (int jj = warp; jj < ndots; jj += nwarps) {  // one warp per column: a shuffle tree
        double t = lane < groups ? red[lane * np2 + jj] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) dots[jj] = t;
    }
    __syncthreads();
}

// One Dslash phase over the block's share of the sites of output parity `parity`, input from the
// loader `in`.  EPI_PLAIN: out = D in.  EPI_AOP: out = m^2 ax - D in with Re<ax, out> per block
// (ax from the loader `ax` at the output site); with DOTS2 also |out|^2, published as columns
// 2n..3n-1 (columns n..2n-1 are left to the update phase's |r|^2).  EPI_RESID (FP64):
// r = b - m^2 ax + D in, written to out_lo (iterated precision Q) with |r|^2 per block.  mask[r]
// selects right-hand sides; m2v[r] is the m^2 of right-hand side r (shared memory).
template <int PP, int R, int EPI, int Q, class IN, class AX, bool DOTS2 = false>
__device__ __forceinline__ void dslash_phase(const PersArgs &a, const LinkField &fat, const LinkField &naik,
                                             const IN &in, void *out, int parity, const int *mask, const AX &ax,
                                             const void *bvec, void *out_lo, double *red, const double *m2v,
                                             const int *list = nullptr, int nlist = 0) {
    using real = typename Prec<PP>::real;
    const Geom &g = a.g;
    // with a list (R = 1), one thread per (site, listed right-hand side): a pass over u of the
    // bundle's n right-hand sides costs u / n of a full pass instead of idling n - u lanes
    const int n = a.n, t = list ? nlist : n / R, spb = blockDim.x / t;
    const int tid = threadIdx.x, gi = tid % t, sl = tid / t, r0 = list ? list[gi] : gi * R;
    const VecView<PP> vout{out, n};
    bool act[R];
    bool any = false;
#pragma unroll
    for (int r = 0; r < R; r++) {
        act[r] = r0 + r < n && mask[r0 + r] != 0;
        any |= act[r];
    }
    double dot[2][R];  // Re<ax, out>; with DOTS2 also |out|^2
#pragma unroll
    for (int k = 0; k < 2; k++)
#pragma unroll
        for (int r = 0; r < R; r++) dot[k][r] = 0.0;
    const int ts = tile_sites(g.Vh, spb);
    if (any && sl < ts) {
        for (int tile = blockIdx.x; (long)tile * ts < g.Vh; tile += gridDim.x) {
            const int q = tile * ts + sl;
            if (q >= g.Vh) break;
            const int s = visit_site(g, q);
            Cplx<real> acc[R][3];
            // 16-bit storage: the epilogue's own record (one 16-byte word per site and RHS) is
            // requested before the stencil, so its L2 latency overlaps the link and neighbour
            // loads; it is decoded after them
            constexpr bool EARLY = EPI == EPI_AOP && PP == HISQ_FP16 && R == 1;
            uint4 raw = make_uint4(0, 0, 0, 0);
            if constexpr (EARLY)
                if (act[0]) raw = __ldcg(reinterpret_cast<const uint4 *>(ax.v.data) + (size_t)s * n + r0);
            site_stencil<PP, 18, R, 1>(g, fat, naik, parity, in, s, 0, r0, act, acc);
            if constexpr (EPI == EPI_PLAIN) {
#pragma unroll
                for (int r = 0; r < R; r++)
                    if (act[r]) store_vec<PP>(vout, s, r0 + r, acc[r]);
            } else if constexpr (EPI == EPI_AOP) {
                Cplx<real> p[R][3];
                if constexpr (EARLY) {
                    decode_fp16_record(raw, p[0]);
                } else {
                    ax.template load<R>(s, r0, act, p);
                }
#pragma unroll
                for (int r = 0; r < R; r++) {
                    if (!act[r]) continue;
                    const real m2 = (real)m2v[r0 + r];
                    Cplx<real> w[3];
                    real d = 0;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        w[c] = {m2 * p[r][c].re - acc[r][c].re, m2 * p[r][c].im - acc[r][c].im};
                        d += p[r][c].re * w[c].re + p[r][c].im * w[c].im;
                    }
                    dot[0][r] += (double)d;
                    store_vec<PP>(vout, s, r0 + r, w);
                    if constexpr (DOTS2) {
                        real f = 0;
#pragma unroll
                        for (int c = 0; c < 3; c++) f += w[c].re * w[c].re + w[c].im * w[c].im;
                        dot[1][r] += (double)f;
                    }
                }
            } else {
                static_assert(EPI == EPI_RESID && PP == HISQ_FP64, "residual epilogue is FP64");
                const VecView<HISQ_FP64> vb{const_cast<void *>(bvec), n};
                const VecView<Q> vlo{out_lo, n};
                Cplx<double> x[R][3];
                ax.template load<R>(s, r0, act, x);
#pragma unroll
                for (int r = 0; r < R; r++) {
                    if (!act[r]) continue;
                    Cplx<double> b[3];
                    Cplx<typename Prec<Q>::real> lo3[3];
                    load_vec<HISQ_FP64, true>(vb, s, r0 + r, b);
                    double d = 0.0;
                    const double m2 = m2v[r0 + r];
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        double wr = b[c].re - m2 * x[r][c].re + (double)acc[r][c].re;
                        double wi = b[c].im - m2 * x[r][c].im + (double)acc[r][c].im;
                        d += wr * wr + wi * wi;
                        lo3[c] = {(typename Prec<Q>::real)wr, (typename Prec<Q>::real)wi};
                    }
                    dot[0][r] += d;
                    store_vec<Q>(vlo, s, r0 + r, lo3);
                }
            }
        }
    }
    if constexpr (DOTS2) {
        publish_dots_k<R, 2>(a, red, dot, t, gi, n, 2 * n);
    } else if constexpr (EPI != EPI_PLAIN) {
        publish_dots<R>(a, red, dot[0], t, gi, list ? nlist : n);  // with a list: column i = list[i]
    }
}

// The FP64-accurate residual recomputation of a mixed-precision solve in double-single
// arithmetic (ds_arith.cuh) over the block's share of the sites, one thread per site and DR
// listed right-hand sides list[DR gi .. DR gi + DR) (nlist listed in all).  The solver uses
// DR = 1: two right-hand sides per thread, which share each link load and give a thread two
// independent accumulation chains, measured no faster at 64^3 x 16 with 16 right-hand sides.
// PF: prefetch the next link's operands (it made the persistent kernels spill, so they pass
// false; the separate kernels of dslash_ds.cu prefetch).
// EPI_PLAIN: out = D in (ds bundles).  EPI_RESID: r = b - m^2 x + D in with x, b FP64
// and an FP64 epilogue, written to out_lo in the iterated precision Q, with |r|^2 per block
// published as column i of the list.
template <int EPI, int Q, int DR, bool PF>
__device__ __forceinline__ void ds_phase(const PersArgs &a, const void *in, void *out, int parity, const void *xvec,
                                         const void *bvec, void *out_lo, double *red, const double *m2v,
                                         const int *list, int nlist) {
    const Geom &g = a.g;
    const int n = a.n, t = (nlist + DR - 1) / DR, spb = blockDim.x / t;
    const int tid = threadIdx.x, gi = tid % t, sl = tid / t;
    bool act[DR];
    int rr[DR];
#pragma unroll
    for (int r = 0; r < DR; r++) {
        act[r] = DR * gi + r < nlist;
        rr[r] = act[r] ? list[DR * gi + r] : 0;
    }
    double dot[DR];
#pragma unroll
    for (int r = 0; r < DR; r++) dot[r] = 0.0;
    const int ts = tile_sites(g.Vh, spb);
    if (sl < ts) {
        for (int tile = blockIdx.x; (long)tile * ts < g.Vh; tile += gridDim.x) {
            const int q = tile * ts + sl;
            if (q >= g.Vh) break;
            const int s = visit_site(g, q);
            dscplx acc[DR][3];
            ds_site_stencil<DR, true, PF>(g, a.fat64, a.naik64, parity, reinterpret_cast<const float4 *>(in), n, s, rr,
                                          act, acc);
#pragma unroll
            for (int r = 0; r < DR; r++) {
                if (!act[r]) continue;
                if constexpr (EPI == EPI_PLAIN) {
                    ds_store3(reinterpret_cast<float4 *>(out), n, s, rr[r], acc[r]);
                } else {
                    static_assert(EPI == EPI_RESID, "the double-single phases are D in and the residual");
                    const double m2 = m2v[rr[r]];
                    const double2 *vx = reinterpret_cast<const double2 *>(xvec);
                    const double2 *vb = reinterpret_cast<const double2 *>(bvec);
                    Cplx<typename Prec<Q>::real> lo3[3];
                    double d = 0.0;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        const long idx = ((long)s * 3 + c) * n + rr[r];
                        const double2 x = __ldcg(vx + idx), b = __ldcg(vb + idx);
                        const double wr = b.x - m2 * x.x + ds_value(acc[r][c].re);
                        const double wi = b.y - m2 * x.y + ds_value(acc[r][c].im);
                        d += wr * wr + wi * wi;
                        lo3[c] = {(typename Prec<Q>::real)wr, (typename Prec<Q>::real)wi};
                    }
                    dot[r] += d;
                    store_vec<Q>(VecView<Q>{out_lo, n}, s, rr[r], lo3);
                }
            }
        }
    }
    if constexpr (EPI == EPI_RESID) publish_dots<DR>(a, red, dot, t, gi, nlist);
}

// x_hi of one site and right-hand side, written in double-single form for the recomputation
__device__ __forceinline__ void store_xds(const PersArgs &a, int s, int r, const Cplx<double> xh[3]) {
    float4 *o = reinterpret_cast<float4 *>(a.xds);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float rh, rl, ih, il;
        ds_split(xh[c].re, rh, rl);
        ds_split(xh[c].im, ih, il);
        o[((long)s * 3 + c) * a.n + r] = make_float4(rh, rl, ih, il);
    }
}

// the solve loop (body in cg_persistent_body.cuh, instantiated per precision)
template <int P, int R, bool CG1>
__global__ void __launch_bounds__(pers_threads(R), 1) cg_persistent_kernel(const __grid_constant__ PersArgs a);

template <int P>
cudaError_t launch_persistent_prec(const PersArgs &a, int R, bool cg1, int grid, int threads, size_t smem,
                                   cudaStream_t st);
template <int P>
cudaError_t persistent_occupancy(int R, bool cg1, int threads, size_t smem, int *blocks_per_sm);

}  // namespace hisq
