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
#include "bulk_copy.cuh"

namespace hisq {

// Reduction plumbing shared by every reducing kernel.
struct RedArgs {
    double *partials;      // [grid][ndots]
    unsigned int *counter; // last-block-done ticket (reset to 0 by the last block)
    double *dot_out;       // [ndots] final dots (may be null)
    int hook;              // solver hook run by the last block (HOOK_NONE = none)
    SolverState *st;
    int partials_only;     // 1: publish the block partials and stop (a later kernel sums them)
};

struct KArgs {
    Geom g;
    LinkField fat, naik;
    const void *in;
    void *out;
    int n, t, spb, parity;
    double mass2;
    const double *mass2v;  // EPI_RESID: m^2 per right-hand side (null: mass2)
    const void *axpy;
    const void *b;
    int b_one;             // EPI_RESID: b is one right-hand side shared by the bundle
    void *out_lo;
    int lo_prec;
    const int *active;
    const int *gate;
    RedArgs red;
    int *err;        // staged kernel: set when a bounded wait for a staged tile runs out
    int s0, s1;      // output sites [s0, s1) of the parity (the whole parity: 0, Vh); the staged
                     // kernel always covers the whole parity
};

template <int P>
__device__ __forceinline__ VecView<P> view(const void *base, int Vh, int n) {
    (void)Vh;
    VecView<P> v;
    v.data = const_cast<void *>(base);
    v.n = n;
    return v;
}

// Deterministic reduction of red[rows][ndots] (shared) into per-block partials, then the
// last-block-done finish: the block that takes the last ticket sums the partials of all blocks
// in a fixed order, writes dot_out and runs the hook for a bundle of hook_n right-hand sides.
// No block ever waits for another.  All threads of the block call it; blockDim.x is a multiple
// of 32; ndots may be 0 (hook only); red holds at least blockDim.x + 64 doubles, and 2 * ndots
// when ndots > 64.  Block column sums run one warp per column (lanes stride over the rows and
// finish with a shuffle tree); the last block gives each thread one column and a stride of the
// blocks' partials, so each stage needs a single barrier.
__device__ __forceinline__ void block_reduce_finish(double *red, int rows, int ndots, int hook_n, const RedArgs &ra) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    __shared__ int is_last;
    if (ndots > 0) {
        __syncthreads();
        for (int j = warp; j < ndots; j += nwarps) {
            double s = 0.0;
            for (int row = lane; row < rows; row += 32) s += red[row * ndots + j];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) {
                ra.partials[(size_t)blockIdx.x * ndots + j] = s;
                if (!ra.partials_only) __threadfence();  // publish before the ticket is taken
            }
        }
    }
    if (ra.partials_only) return;  // the kernel boundary publishes them to the consumer
    __syncthreads();
    if (tid == 0) is_last = (atomicAdd(ra.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    if (tid == 0) __threadfence();
    __syncthreads();
    if (ndots > 0) {
        const int nb = gridDim.x;
        if (ndots <= 64) {
            // thread (k, j), j < np2 (ndots padded to a power of two), sums column j over blocks
            // k, k + per, ...; lanes of one column are np2 apart in a warp and meet in a shuffle
            // tree, then at most 8 warp sums per column are added in a fixed order
            int np2 = 1;
            while (np2 < ndots) np2 *= 2;
            const int per = blockDim.x / np2;
            const int j = tid % np2, k = tid / np2;
            double s = 0.0;
            if (j < ndots && k < per) {
#pragma unroll 4
                for (int b = k; b < nb; b += per) s += __ldcg(ra.partials + (size_t)b * ndots + j);
            }
            for (int off = 16; off >= np2; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            const int groups = np2 < 32 ? nwarps : per;           // partial sums per column
            if (np2 < 32) {
                if (lane < np2) red[warp * np2 + lane] = s;
            } else {
                red[tid] = s;
            }
            __syncthreads();
            if (tid < ndots) {
                double t = 0.0;
                for (int q = 0; q < groups; q++) t += red[q * np2 + tid];
                red[blockDim.x + tid] = t;
            }
            __syncthreads();
            if (tid < ndots) red[tid] = red[blockDim.x + tid];
        } else {
            // many columns (network weight gradients): one thread per column
            for (int j = tid; j < ndots; j += blockDim.x) {
                double t = 0.0;
#pragma unroll 8
                for (int b = 0; b < nb; b++) t += __ldcg(ra.partials + (size_t)b * ndots + j);
                red[ndots + j] = t;
            }
            __syncthreads();
            for (int j = tid; j < ndots; j += blockDim.x) red[j] = red[ndots + j];
        }
        __syncthreads();
        if (ra.dot_out)
            for (int j = tid; j < ndots; j += blockDim.x) ra.dot_out[j] = red[j];
    }
    if (ra.hook && ra.st) {
        // the scalar step works on a shared-memory copy of the bundle state: one coalesced read
        // and one write-back instead of a chain of dependent global accesses by one thread
        __shared__ SolverState sst;
        constexpr int WORDS = sizeof(SolverState) / sizeof(uint32_t);
        const uint32_t *src = reinterpret_cast<const uint32_t *>(ra.st);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sst);
#pragma unroll 4
        for (int i = tid; i < WORDS; i += blockDim.x) dst[i] = __ldcg(src + i);
        __syncthreads();
        if (tid == 0) run_hook(ra.hook, &sst, red, hook_n);
        __syncthreads();
        uint32_t *back = reinterpret_cast<uint32_t *>(ra.st);
        for (int i = tid; i < WORDS; i += blockDim.x) back[i] = dst[i];
    }
    if (tid == 0) {
        *ra.counter = 0u;
        __threadfence();
    }
}

// The R neighbour vectors of the active right-hand sides (zeros for the inactive ones).
template <int P, int R, bool COHERENT>
__device__ __forceinline__ void load_neighbours(const VecView<P> &vin, int nb, int r0, const bool act[R],
                                                Cplx<typename Prec<P>::real> v[R][3]) {
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (act[r]) {
            load_vec<P, COHERENT>(vin, nb, r0 + r, v[r]);
        } else {
#pragma unroll
            for (int c = 0; c < 3; c++) v[r][c] = {0, 0};
        }
    }
}

// Input of the stencil: the colour vectors of one bundle as stored (COHERENT: read through L2,
// for vectors written earlier in the same launch).  Other inputs (a direction formed on the fly)
// provide the same load().
template <int P, bool COHERENT>
struct PlainIn {
    static constexpr bool coherent = COHERENT;
    VecView<P> v;
    template <int R>
    __device__ __forceinline__ void load(int nb, int r0, const bool act[R], Cplx<typename Prec<P>::real> out[R][3]) const {
        load_neighbours<P, R, COHERENT>(v, nb, r0, act, out);
    }
};

// acc *= f
template <typename T, int R>
__device__ __forceinline__ void scale_acc(Cplx<T> acc[R][3], T f) {
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc[r][c] = {acc[r][c].re * f, acc[r][c].im * f};
}

// ---- paired FP32 arithmetic for 16-bit storage and an even number R of right-hand sides ----
//
// Two right-hand sides r, r + 1 share every link element, so their real parts (and their
// imaginary parts) form one float2 and each complex multiply-add of a link element with the two
// vectors is four packed fused multiply-adds (fma.rn.f32x2, two FP32 lanes per instruction) in
// place of eight scalar ones: Re w += Re M Re v - Im M Im v is kept as two sums, the second
// (Im M Im v) in its own accumulator and subtracted once at the end, so no operand is negated.
// The 16-bit vectors are decoded straight into the pairs and scaled with packed multiplies.
template <int Q2>
struct PairAcc {
    float2 re[Q2][3], im[Q2][3], neg[Q2][3];
};

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

template <int Q2>
__device__ __forceinline__ void pair_scale(PairAcc<Q2> &A, float f) {
    const float2 ff = f2(f, f);
#pragma unroll
    for (int q = 0; q < Q2; q++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            A.re[q][c] = __fmul2_rn(A.re[q][c], ff);
            A.im[q][c] = __fmul2_rn(A.im[q][c], ff);
            A.neg[q][c] = __fmul2_rn(A.neg[q][c], ff);
        }
}

// the pairs (Re v_r, Re v_{r+1}), (Im v_r, Im v_{r+1}) of the neighbour nb for r = r0 + 2q
template <int P, int Q2, bool COHERENT>
__device__ __forceinline__ void load_pairs(const void *data, int n, int nb, int r0, const bool act[2 * Q2],
                                           float2 vr[Q2][3], float2 vi[Q2][3]) {
    if constexpr (P == HISQ_FP16) {
        const uint4 *rec = reinterpret_cast<const uint4 *>(data) + (size_t)nb * n + r0;
#pragma unroll
        for (int q = 0; q < Q2; q++) {
            const uint4 z = make_uint4(0, 0, 0, 0);
            const uint4 a = act[2 * q] ? vld<COHERENT>(rec + 2 * q) : z;
            const uint4 b = act[2 * q + 1] ? vld<COHERENT>(rec + 2 * q + 1) : z;
            const float2 sc = f2(__uint_as_float(a.w), __uint_as_float(b.w));
            const uint32_t ha[3] = {a.x, a.y, a.z}, hb[3] = {b.x, b.y, b.z};
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float2 fa = __half22float2(*reinterpret_cast<const __half2 *>(&ha[c]));
                const float2 fb = __half22float2(*reinterpret_cast<const __half2 *>(&hb[c]));
                vr[q][c] = __fmul2_rn(f2(fa.x, fb.x), sc);
                vi[q][c] = __fmul2_rn(f2(fa.y, fb.y), sc);
            }
        }
    } else {
        static_assert(P == HISQ_BF16, "paired loads for 16-bit storage");
        // element (s, c, r) is the bf16 pair (re, im) at (s * 3 + c) n + r: two adjacent right-hand
        // sides are one 8-byte word; a bf16 is the top half of its float
        const uint32_t *e = reinterpret_cast<const uint32_t *>(data);
#pragma unroll
        for (int q = 0; q < Q2; q++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const size_t idx = ((size_t)nb * 3 + c) * n + r0 + 2 * q;
                const uint32_t a = act[2 * q] ? vld<COHERENT>(e + idx) : 0u;
                const uint32_t b = act[2 * q + 1] ? vld<COHERENT>(e + idx + 1) : 0u;
                vr[q][c] = f2(__uint_as_float(a << 16), __uint_as_float(b << 16));
                vi[q][c] = f2(__uint_as_float(a & 0xffff0000u), __uint_as_float(b & 0xffff0000u));
            }
    }
}

template <int Q2>
__device__ __forceinline__ void matvec_pairs(const Cplx<float> M[3][3], const float2 vr[Q2][3], const float2 vi[Q2][3],
                                             PairAcc<Q2> &A) {
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const float2 mr = f2(M[a][b].re, M[a][b].re), mi = f2(M[a][b].im, M[a][b].im);
#pragma unroll
            for (int q = 0; q < Q2; q++) {
                A.re[q][a] = __ffma2_rn(mr, vr[q][b], A.re[q][a]);
                A.neg[q][a] = __ffma2_rn(mi, vi[q][b], A.neg[q][a]);
                A.im[q][a] = __ffma2_rn(mr, vi[q][b], A.im[q][a]);
                A.im[q][a] = __ffma2_rn(mi, vr[q][b], A.im[q][a]);
            }
        }
}

// site_stencil for 16-bit 18-real records, R even, S = 1 or 2 (same fields, scales and slots)
template <int P, int R, int S, bool COHERENT>
__device__ __forceinline__ void site_stencil_pairs(const Geom &g, const LinkField &fat_f, const LinkField &naik_f,
                                                   int parity, const void *in, int n, int s, int part, int r0,
                                                   const bool act[R], Cplx<float> acc[R][3]) {
    using C = LinkCodec<P, 18>;
    constexpr int Q2 = R / 2;
    const SiteCoord sc = decode_site(g, s, parity);
    const size_t site = (size_t)parity * g.Vh + s;
    PairAcc<Q2> A;
#pragma unroll
    for (int q = 0; q < Q2; q++)
#pragma unroll
        for (int c = 0; c < 3; c++) A.re[q][c] = A.im[q][c] = A.neg[q][c] = f2(0.f, 0.f);
#pragma unroll
    for (int kind = 0; kind < (S == 1 ? 2 : 1); kind++) {
        const bool naik_kind = (S == 1) ? (kind == 1) : (part == 1);
        const LinkField f = naik_kind ? naik_f : fat_f;
        const int hop = naik_kind ? 3 : 1;
        if (S == 1 && kind == 1) pair_scale(A, __ldg(fat_f.scale + site) / __ldg(naik_f.scale + site));
#pragma unroll
        for (int grp = 0; grp < C::GROUPS; grp++) {
            uint32_t u[C::WG * 4];
            C::load_group(f, parity, g.Vh, s, grp, u);
#pragma unroll
            for (int l = 0; l < C::G; l++) {
                const int slot = grp * C::G + l;
                const int nb = neighbour(g, sc, s, slot >> 1, (slot & 1) ? -hop : hop);
                Cplx<float> M[3][3];
                C::decode(u, l, M);
                float2 vr[Q2][3], vi[Q2][3];
                load_pairs<P, Q2, COHERENT>(in, n, nb, r0, act, vr, vi);
                matvec_pairs<Q2>(M, vr, vi, A);
            }
        }
        // S = 1: after the Naik field, acc = s_N (s_X / s_N sum_X + sum_N); S = 2: the lane's field
        if (S != 1 || kind == 1) pair_scale(A, __ldg(f.scale + site));
    }
    const float2 m1 = f2(-1.f, -1.f);
#pragma unroll
    for (int q = 0; q < Q2; q++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float2 re = __ffma2_rn(A.neg[q][c], m1, A.re[q][c]);
            acc[2 * q][c] = {re.x, A.im[q][c].x};
            acc[2 * q + 1][c] = {re.y, A.im[q][c].y};
        }
}

// The stencil of Eq. (3) at output site s (parity `parity`): writes into acc the sum of the
// products of the site's links with the neighbouring input vectors (from the loader `vin`) of
// the R right-hand sides r0.. that are active.  S = 1: all 16 links.  S = 2 (18-real Naik only):
// the 8 fat (part 0) or the 8 Naik links (part 1).  S = 4 (18-real Naik only): part =
// 2 kind + half, the four links of directions 2 half and 2 half + 1 of that kind.  Record slot 2 mu holds the forward link of
// direction mu and slot 2 mu + 1 the backward one (already -U^dagger of the neighbour's link).
// 16-bit 18-real records carry one positive float scale per (parity, site) and field; it is
// applied to the field's summed contribution (6 R products) instead of to the 18 reals of each
// of its links: with both fields scaled, acc = s_N (s_X / s_N sum_X + sum_N).
template <int P, int NR, int R, int S, class IN>
__device__ __forceinline__ void site_stencil(const Geom &g, const LinkField &fat_f, const LinkField &naik_f, int parity,
                                             const IN &vin, int s, int part, int r0, const bool act[R],
                                             Cplx<typename Prec<P>::real> acc[R][3]) {
    using real = typename Prec<P>::real;
    using FatC = LinkCodec<P, 18>;
    using NaikC = LinkCodec<P, NR>;
    constexpr bool SCALED = (P == HISQ_FP16 || P == HISQ_BF16);  // 18-real records of 16-bit fields
    if constexpr (SCALED && NR == 18 && R % 2 == 0 && (S == 1 || S == 2)) {
        site_stencil_pairs<P, R, S, IN::coherent>(g, fat_f, naik_f, parity, vin.v.data, vin.v.n, s, part, r0, act, acc);
        return;
    }
    const SiteCoord sc = decode_site(g, s, parity);
    const size_t site = (size_t)parity * g.Vh + s;
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc[r][c] = {0, 0};
    if constexpr (S == 4) {
        static_assert(NR == 18, "the four-lane split needs identical fat and Naik encodings");
        const bool naik_kind = (part >> 1) != 0;
        const int half = part & 1;
        const LinkField f = naik_kind ? naik_f : fat_f;
        const int hop = naik_kind ? 3 : 1;
        constexpr int GPH = 4 / FatC::G;  // groups per half record (4 links)
#pragma unroll
        for (int gg = 0; gg < GPH; gg++) {
            uint32_t u[FatC::WG * 4];
            FatC::load_group(f, parity, g.Vh, s, half * GPH + gg, u);
#pragma unroll
            for (int l = 0; l < FatC::G; l++) {
                const int j = gg * FatC::G + l;  // 0..3 within the half
                const int nb = neighbour_rt(g, sc, s, 2 * half + (j >> 1), (j & 1) ? -hop : hop);
                Cplx<real> M[3][3];
                FatC::decode(u, l, M);
                Cplx<real> v[R][3];
                vin.template load<R>(nb, r0, act, v);
                matvec_acc<real, R>(M, v, acc);
            }
        }
        if constexpr (SCALED) scale_acc<real, R>(acc, (real)__ldg(f.scale + site));
        return;
    }
#pragma unroll
    for (int kind = 0; kind < (S == 1 ? 2 : 1); kind++) {
        const bool naik_kind = (S == 1) ? (kind == 1) : (part == 1);
        const LinkField f = naik_kind ? naik_f : fat_f;
        const int hop = naik_kind ? 3 : 1;
        if (S == 1 && kind == 1 && NR != 18) {
            // reconstructed Naik records are unscaled: finish the fat sum first
            if constexpr (SCALED) scale_acc<real, R>(acc, (real)__ldg(fat_f.scale + site));
#pragma unroll
            for (int grp = 0; grp < NaikC::GROUPS; grp++) {
                uint32_t u[NaikC::WG * 4];
                NaikC::load_group(naik_f, parity, g.Vh, s, grp, u);
#pragma unroll
                for (int l = 0; l < NaikC::G; l++) {
                    const int slot = grp * NaikC::G + l;
                    const int nb = neighbour(g, sc, s, slot >> 1, (slot & 1) ? -3 : 3);
                    Cplx<real> M[3][3];
                    NaikC::decode(u, l, M);
                    Cplx<real> v[R][3];
                    vin.template load<R>(nb, r0, act, v);
                    matvec_acc<real, R>(M, v, acc);
                }
            }
            continue;
        }
        if constexpr (SCALED && S == 1) {
            // between the fields: acc = (s_X / s_N) sum_X
            if (kind == 1) scale_acc<real, R>(acc, (real)__ldg(fat_f.scale + site) / (real)__ldg(naik_f.scale + site));
        }
#pragma unroll
        for (int grp = 0; grp < FatC::GROUPS; grp++) {
            uint32_t u[FatC::WG * 4];
            FatC::load_group(f, parity, g.Vh, s, grp, u);
#pragma unroll
            for (int l = 0; l < FatC::G; l++) {
                const int slot = grp * FatC::G + l;
                const int nb = neighbour(g, sc, s, slot >> 1, (slot & 1) ? -hop : hop);
                Cplx<real> M[3][3];
                FatC::decode(u, l, M);
                Cplx<real> v[R][3];
                vin.template load<R>(nb, r0, act, v);
                matvec_acc<real, R>(M, v, acc);
            }
        }
        if constexpr (SCALED) {
            // S = 1: after the Naik field, acc = s_N (...); S = 2: the lane's one field
            if (S != 1 || kind == 1) scale_acc<real, R>(acc, (real)__ldg(f.scale + site));
        }
    }
}

// S = 1: one thread applies all 16 links of its site.  S = 2 or 4 (18-real Naik only): S adjacent
// lanes share a site, each applying 16 / S of its links with the same instruction stream (the
// lanes differ only in which record words, hop length and directions they use), and a shuffle
// tree adds their parts: S times the threads and 1/S of the dependent-load chain per thread when
// there are few right-hand sides.
template <int P, int NR, int R, int EPI, int S>
__global__ void __launch_bounds__(256) dslash_kernel(KArgs a) {
    static_assert(S == 1 || ((S == 2 || S == 4) && NR == 18), "the lane split needs identical fat and Naik encodings");
    using real = typename Prec<P>::real;
    using FatC = LinkCodec<P, 18>;
    using NaikC = LinkCodec<P, NR>;
    extern __shared__ double red[];

    if (a.gate && *a.gate == 0) return;

    const Geom &g = a.g;
    const int tid = threadIdx.x;
    const int part = tid & (S - 1);
    const int gi = (tid / S) % a.t;
    const int sl = tid / (S * a.t);
    const int r0 = gi * R;
    const int nvalid = min(R, a.n - r0);
    const PlainIn<P, false> vin{view<P>(a.in, g.Vh, a.n)};
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

    const bool whole = a.s0 == 0 && a.s1 == g.Vh;  // a whole parity: visit in plane order
    for (int tile = blockIdx.x; (long)tile * a.spb < a.s1 - a.s0; tile += gridDim.x) {
        const int q = tile * a.spb + sl;
        const bool valid = sl < a.spb && q < a.s1 - a.s0 && any_act;
        const int s = whole ? visit_site(g, valid ? q : 0) : a.s0 + q;
        if (S == 1 && !valid) continue;

        Cplx<real> acc[R][3];
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[r][c] = {0, 0};

        if (valid) site_stencil<P, NR, R, S>(g, a.fat, a.naik, a.parity, vin, s, part, r0, act, acc);
        if constexpr (S > 1) {
            // add the lanes' parts; every lane of the warp takes part
#pragma unroll
            for (int off = 1; off < S; off <<= 1)
#pragma unroll
                for (int r = 0; r < R; r++)
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        acc[r][c].re += __shfl_xor_sync(0xffffffffu, acc[r][c].re, off);
                        acc[r][c].im += __shfl_xor_sync(0xffffffffu, acc[r][c].im, off);
                    }
        }
        if (!valid || part != 0) continue;

        // ---- epilogue ----
        if constexpr (EPI == EPI_PLAIN) {
#pragma unroll
            for (int r = 0; r < R; r++)
                if (act[r]) store_vec<P>(vout, s, r0 + r, acc[r]);
        } else if constexpr (EPI == EPI_AOP) {
            const VecView<P> vp = view<P>(a.axpy, g.Vh, a.n);
            const real m2 = (real)a.mass2;
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (!act[r]) continue;
                Cplx<real> p[3], w[3];
                load_vec<P>(vp, s, r0 + r, p);
                real d = 0;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    w[c] = {m2 * p[c].re - acc[r][c].re, m2 * p[c].im - acc[r][c].im};
                    d += p[c].re * w[c].re + p[c].im * w[c].im;
                }
                dot[r] += (double)d;
                store_vec<P>(vout, s, r0 + r, w);
            }
        } else {
            static_assert(EPI == EPI_RESID && P == HISQ_FP64, "residual epilogue is FP64 only");
            const VecView<HISQ_FP64> vx = view<HISQ_FP64>(a.axpy, g.Vh, a.n);
            const VecView<HISQ_FP64> vb = view<HISQ_FP64>(a.b, g.Vh, a.b_one ? 1 : a.n);
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (!act[r]) continue;
                Cplx<double> w[3];
                double d = 0.0;
                Cplx<double> x[3], b[3];
                load_vec<HISQ_FP64>(vx, s, r0 + r, x);
                load_vec<HISQ_FP64>(vb, s, a.b_one ? 0 : r0 + r, b);
                const double m2 = a.mass2v ? a.mass2v[r0 + r] : a.mass2;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    w[c] = {b[c].re - m2 * x[c].re + (double)acc[r][c].re, b[c].im - m2 * x[c].im + (double)acc[r][c].im};
                    d += w[c].re * w[c].re + w[c].im * w[c].im;
                }
                dot[r] += d;
                if (a.out) store_vec<HISQ_FP64>(vout, s, r0 + r, w);
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
        // every thread reaches the reduction (idle threads contributed zeros)
        block_reduce_finish(red, a.spb, a.n, a.n, a.red);
    }
}

// ---- staged variant: link records of a tile of sites brought into shared memory in bulk ----
//
// The link records of TS consecutive output sites form, for every 16-byte word plane j of the
// gathered layout, one contiguous run of TS words; a single thread copies the W_X + W_N runs of a
// tile with the bulk-copy engine into a shared-memory stage while the block computes on the other
// stage (two stages).  Memory parallelism then no longer depends on how many link loads each
// thread can keep in flight, which at one right-hand side and a few hundred sites per SM is what
// limits the plain kernel.  Four lanes share a site as in the S = 4 split (two directions of one
// link kind per lane); neighbour vectors are read from global memory (they are reused by 16 sites
// and mostly hit in L2).  18-real Naik records only.

// words of the gathered records per site: fat then Naik planes; stage k holds (W_X + W_N) * TS
// words, plane j at [j * TS, (j + 1) * TS)
template <int P, int R, bool COHERENT>
__device__ __forceinline__ void staged_stencil(const Geom &g, const LinkField &fat_f, const LinkField &naik_f,
                                               int parity, const uint4 *stage, int TS, int sl,
                                               const PlainIn<P, COHERENT> &vin, int s, int part, int r0,
                                               const bool act[R], Cplx<typename Prec<P>::real> acc[R][3]) {
    using real = typename Prec<P>::real;
    using C = LinkCodec<P, 18>;
    constexpr bool SCALED = (P == HISQ_FP16 || P == HISQ_BF16);
    const SiteCoord sc = decode_site(g, s, parity);
    const bool naik_kind = (part >> 1) != 0;
    const int half = part & 1;
    const int hop = naik_kind ? 3 : 1;
    const int plane0 = naik_kind ? fat_f.W : 0;
    constexpr int GPH = 4 / C::G;  // groups per half record (4 links)
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc[r][c] = {0, 0};
#pragma unroll
    for (int gg = 0; gg < GPH; gg++) {
        uint32_t u[C::WG * 4];
        const int w0 = plane0 + (half * GPH + gg) * C::WG;
#pragma unroll
        for (int j = 0; j < C::WG; j++) {
            const uint4 w = stage[(size_t)(w0 + j) * TS + sl];
            u[4 * j] = w.x; u[4 * j + 1] = w.y; u[4 * j + 2] = w.z; u[4 * j + 3] = w.w;
        }
#pragma unroll
        for (int l = 0; l < C::G; l++) {
            const int j = gg * C::G + l;
            const int nb = neighbour_rt(g, sc, s, 2 * half + (j >> 1), (j & 1) ? -hop : hop);
            Cplx<real> M[3][3];
            C::decode(u, l, M);
            Cplx<real> v[R][3];
            vin.template load<R>(nb, r0, act, v);
            matvec_acc<real, R>(M, v, acc);
        }
    }
    if constexpr (SCALED) {
        const LinkField &f = naik_kind ? naik_f : fat_f;
        scale_acc<real, R>(acc, (real)__ldg(f.scale + (size_t)parity * g.Vh + s));
    }
}

constexpr long STAGE_WAIT_LIMIT = 1L << 22;  // bounded wait for a staged tile (about a second)

template <int P, int R, int EPI>
__global__ void __launch_bounds__(512, 1) dslash_staged_kernel(KArgs a) {
    using real = typename Prec<P>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.gate && *a.gate == 0) return;
    const Geom &g = a.g;
    const int tid = threadIdx.x;
    const int part = tid & 3;
    const int gi = (tid >> 2) % a.t;
    const int sl = tid / (4 * a.t);
    const int TS = a.spb;  // sites per tile
    const int r0 = gi * R;
    const int nvalid = min(R, a.n - r0);
    const int Wt = a.fat.W + a.naik.W;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    uint4 *stages = reinterpret_cast<uint4 *>(smem_raw + 16);
    double *red = reinterpret_cast<double *>(smem_raw + 16 + (size_t)2 * Wt * TS * sizeof(uint4));
    const PlainIn<P, false> vin{view<P>(a.in, g.Vh, a.n)};
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

    const int tiles = (g.Vh + TS - 1) / TS;
    // thread 0 copies tile k of this block (tile index blockIdx.x + k * gridDim.x) into stage k & 1
    auto issue = [&](int k) {
        const int tile = blockIdx.x + k * gridDim.x;
        if (tile >= tiles) return;
        const int s0 = tile * TS, ns = min(TS, g.Vh - s0);
        const uint32_t bytes = (uint32_t)ns * sizeof(uint4);
        uint64_t *b = bar + (k & 1);
        uint4 *dst = stages + (size_t)(k & 1) * Wt * TS;
        mbar_arrive_expect(b, bytes * (uint32_t)Wt);
        for (int j = 0; j < a.fat.W; j++)
            bulk_copy_g2s(dst + (size_t)j * TS, a.fat.words + ((size_t)a.parity * a.fat.W + j) * g.Vh + s0, bytes, b);
        for (int j = 0; j < a.naik.W; j++)
            bulk_copy_g2s(dst + (size_t)(a.fat.W + j) * TS,
                          a.naik.words + ((size_t)a.parity * a.naik.W + j) * g.Vh + s0, bytes, b);
    };
    __shared__ int s_ok;
    if (tid == 0) {
        s_ok = 1;
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        issue(0);
        issue(1);
    }
    for (int k = 0; blockIdx.x + k * (int)gridDim.x < tiles; k++) {
        const int tile = blockIdx.x + k * gridDim.x;
        const int s = tile * TS + sl;
        // every thread waits on the stage (bounded); a wait that runs out is recorded and the
        // tile is skipped, so the kernel always ends
        const bool ready = mbar_wait(bar + (k & 1), (uint32_t)((k >> 1) & 1), STAGE_WAIT_LIMIT);
        if (!ready) s_ok = 0;
        const bool valid = ready && sl < TS && s < g.Vh && any_act;
        Cplx<real> acc[R][3];
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[r][c] = {0, 0};
        if (valid)
            staged_stencil<P, R, false>(g, a.fat, a.naik, a.parity, stages + (size_t)(k & 1) * Wt * TS, TS, sl, vin, s,
                                        part, r0, act, acc);
#pragma unroll
        for (int off = 1; off < 4; off <<= 1)
#pragma unroll
            for (int r = 0; r < R; r++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    acc[r][c].re += __shfl_xor_sync(0xffffffffu, acc[r][c].re, off);
                    acc[r][c].im += __shfl_xor_sync(0xffffffffu, acc[r][c].im, off);
                }
        if (valid && part == 0) {
            if constexpr (EPI == EPI_PLAIN) {
#pragma unroll
                for (int r = 0; r < R; r++)
                    if (act[r]) store_vec<P>(vout, s, r0 + r, acc[r]);
            } else {
                static_assert(EPI == EPI_AOP, "the staged kernel has the plain and A-operator epilogues");
                const VecView<P> vp = view<P>(a.axpy, g.Vh, a.n);
                const real m2 = (real)a.mass2;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    if (!act[r]) continue;
                    Cplx<real> p[3], w[3];
                    load_vec<P>(vp, s, r0 + r, p);
                    real d = 0;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        w[c] = {m2 * p[c].re - acc[r][c].re, m2 * p[c].im - acc[r][c].im};
                        d += p[c].re * w[c].re + p[c].im * w[c].im;
                    }
                    dot[r] += (double)d;
                    store_vec<P>(vout, s, r0 + r, w);
                }
            }
        }
        __syncthreads();  // the stage is free again
        if (tid == 0) issue(k + 2);
    }
    if (tid == 0 && !s_ok && a.err) atomicExch(a.err, 1);
    if constexpr (EPI != EPI_PLAIN) {
        for (int i = tid; i < TS * a.n; i += blockDim.x) red[i] = 0.0;
        __syncthreads();
        if (sl < TS && part == 0) {
#pragma unroll
            for (int r = 0; r < R; r++)
                if (r < nvalid) red[sl * a.n + r0 + r] = dot[r];
        }
        block_reduce_finish(red, TS, a.n, a.n, a.red);
    }
}

}  // namespace hisq
