// Internal definitions shared by the CUDA translation units of the HISQ library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <vector>
#include <map>
#include <algorithm>

#include "../../include/hisq.h"

namespace hisq {

// ------------------------------------------------------------------------------------------
// Errors
// ------------------------------------------------------------------------------------------
int set_error(int code, const char *fmt, ...);

#define HISQ_CUDA(call)                                                                     \
    do {                                                                                    \
        cudaError_t err_ = (call);                                                          \
        if (err_ != cudaSuccess)                                                            \
            return ::hisq::set_error(HISQ_ERR_CUDA, "%s failed: %s (%s:%d)", #call,          \
                                     cudaGetErrorString(err_), __FILE__, __LINE__);          \
    } while (0)

#define HISQ_CHECK(expr)                                                                    \
    do {                                                                                    \
        int st_ = (expr);                                                                   \
        if (st_ != HISQ_OK) return st_;                                                     \
    } while (0)

// ------------------------------------------------------------------------------------------
// Lattice geometry on the device.  Even-odd index s of parity p:
//   xh = s % (Lx/2), row = s / (Lx/2) = y + Ly (z + Lz t), x = 2 xh + ((y+z+t+p) & 1).
// Neighbours keep the row arithmetic local: a hop in y changes s by (y'-y) Lx/2, etc.
// ------------------------------------------------------------------------------------------
struct Geom {
    int L[4];
    int half;      // Lx / 2
    int Vh;        // V / 2
    int stride[4]; // even-odd index stride of one step in y, z, t (stride[0] unused)
    int plane_order;  // 1: stencil passes visit the xy-planes with t varying before z (visit_site)
};

struct SiteCoord {
    int c[4];
    int row_base;  // s - xh: even-odd index of the row's first site
};

__host__ __device__ __forceinline__ SiteCoord decode_site(const Geom &g, int s, int parity) {
    SiteCoord sc;
    int xh = s % g.half;
    int row = s / g.half;
    sc.c[1] = row % g.L[1];
    int zt = row / g.L[1];
    sc.c[2] = zt % g.L[2];
    sc.c[3] = zt / g.L[2];
    sc.c[0] = 2 * xh + ((sc.c[1] + sc.c[2] + sc.c[3] + parity) & 1);
    sc.row_base = s - xh;
    return sc;
}

// Site of one parity visited at position q of a stencil pass over the whole parity.  The
// even-odd index runs x fastest, then y, z, t, so a site's +-1 and +-3 neighbours in t are 1 and 3
// time planes away (Lx Ly Lz / 2 sites each): while a pass sweeps the lattice in that order, the
// vectors it read at a site's t-neighbours must stay in L2 for three planes of links and vectors,
// more than the 129 MB of L2 once a bundle of right-hand sides fills GBs.  With plane_order set
// (t shorter than z) the pass visits the xy-planes (fixed z, t: Lx Ly / 2 consecutive sites) with
// t varying before z, so t-neighbours are a few xy-planes apart in the visit and z-neighbours
// 3 Lt xy-planes apart, a quarter of the distance at 64^3 x 16.  Only the order of the visit
// changes; every site is still computed once.
__host__ __device__ __forceinline__ int visit_site(const Geom &g, int q) {
    if (!g.plane_order) return q;
    const int P = g.stride[2];                 // sites of one xy-plane
    const int plane = q / P, within = q - plane * P;
    const int z = plane / g.L[3], t = plane - z * g.L[3];
    return within + P * (z + g.L[2] * t);
}

// even-odd index of the neighbour `step` hops (|step| <= 3 < L) away in direction mu// even-odd index of the neighbour `step` hops (|step| <= 3 < L) away in direction mu
__host__ __device__ __forceinline__ int neighbour(const Geom &g, const SiteCoord &sc, int s, int mu, int step) {
    int c = sc.c[mu] + step;
    int L = g.L[mu];
    c += (c < 0) ? L : 0;
    c -= (c >= L) ? L : 0;
    if (mu == 0) return sc.row_base + (c >> 1);
    return s + (c - sc.c[mu]) * g.stride[mu];
}

// Neighbour `step` hops away along a direction mu known only at run time (the four-lane split
// picks its directions by lane; loops over the links that are not unrolled): the coordinate,
// extent and stride are selected, not indexed, so nothing spills to local memory.
__device__ __forceinline__ int neighbour_rt(const Geom &g, const SiteCoord &sc, int s, int mu, int step) {
    const int cm = mu == 0 ? sc.c[0] : mu == 1 ? sc.c[1] : mu == 2 ? sc.c[2] : sc.c[3];
    const int L = mu == 0 ? g.L[0] : mu == 1 ? g.L[1] : mu == 2 ? g.L[2] : g.L[3];
    const int st = mu == 1 ? g.stride[1] : mu == 2 ? g.stride[2] : g.stride[3];
    int c = cm + step;
    c += (c < 0) ? L : 0;
    c -= (c >= L) ? L : 0;
    if (mu == 0) return sc.row_base + (c >> 1);
    return s + (c - cm) * st;
}

// ------------------------------------------------------------------------------------------
// Storage precisions
// ------------------------------------------------------------------------------------------
template <int P> struct Prec;
template <> struct Prec<HISQ_FP64> { using real = double; using store = double; static constexpr int bytes = 8; };
template <> struct Prec<HISQ_FP32> { using real = float; using store = float; static constexpr int bytes = 4; };
template <> struct Prec<HISQ_FP16> { using real = float; using store = __half; static constexpr int bytes = 2; };
template <> struct Prec<HISQ_BF16> { using real = float; using store = __nv_bfloat16; static constexpr int bytes = 2; };

template <typename R> struct Cplx { R re, im; };

// Internal storage id of the double-single form of FP64 data (ds_arith.cuh): every real as the
// float pair (hi, lo), 8 bytes, in the FP64 layouts.  Not a precision of the C ABI.
constexpr int HISQ_DS = 4;

// Internal vector bundles of n right-hand sides.  FP64, FP32 and BF16: element (s, c, r) is the
// complex number at (s*3 + c)*n + r (double2 / float2 / bf16x2).  FP16: one 16-byte record per
// (site, rhs) at s*n + r holding the three colour components as half2 and the FP32 scale
// (value = half * scale, scale = max |component|), so a neighbour is a single 16-byte load.
inline size_t vector_bytes(int prec, int Vh, int n) {
    const size_t elems = (size_t)Vh * n;
    switch (prec) {
    case HISQ_FP64:
    case HISQ_DS: return elems * 3 * 16;
    case HISQ_FP32: return elems * 3 * 8;
    case HISQ_FP16: return elems * 16;
    default: return elems * 3 * 4;
    }
}

// A right-hand side counts as converged when the library's FP64 true residual is at most
// TOL_SAFETY * tol, so that a recomputation of the same residual with another summation order
// (the caller's own FP64 check of |b - A x| / |b|) still finds it within tol.  The two differ by
// rounding only, far less than 5% of a residual of 1e-10.
constexpr double TOL_SAFETY = 0.95;

// iterated precision of x and r for an inner (Dslash) precision: FP64 stays FP64, else FP32
__host__ __device__ constexpr int q_prec(int p) { return p == HISQ_FP64 ? HISQ_FP64 : HISQ_FP32; }

template <int P> struct VecView {
    void *data;
    int n;
};

// COHERENT = true reads through L2 (ld.global.cg) instead of the read-only path: required for
// data written earlier in the same kernel launch by other blocks (the persistent solver).
template <bool COHERENT, typename T>
__device__ __forceinline__ T vld(const T *p) {
    if constexpr (COHERENT) return __ldcg(p);
    else return __ldg(p);
}

// the colour vector held in one FP16 record (three __half2 and the float scale)
__device__ __forceinline__ void decode_fp16_record(const uint4 q, Cplx<float> w[3]) {
    const float sc = __uint_as_float(q.w);
    const uint32_t h[3] = {q.x, q.y, q.z};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&h[c]));
        w[c] = {f.x * sc, f.y * sc};
    }
}

template <int P, bool COHERENT = false>
__device__ __forceinline__ void load_vec(const VecView<P> &v, long s, int r, Cplx<typename Prec<P>::real> w[3]) {
    if constexpr (P == HISQ_FP64) {
        const double2 *d = reinterpret_cast<const double2 *>(v.data) + s * 3 * v.n + r;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            double2 x = vld<COHERENT>(d + (long)c * v.n);
            w[c] = {x.x, x.y};
        }
    } else if constexpr (P == HISQ_FP32) {
        const float2 *d = reinterpret_cast<const float2 *>(v.data) + s * 3 * v.n + r;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float2 x = vld<COHERENT>(d + (long)c * v.n);
            w[c] = {x.x, x.y};
        }
    } else if constexpr (P == HISQ_FP16) {
        decode_fp16_record(vld<COHERENT>(reinterpret_cast<const uint4 *>(v.data) + s * v.n + r), w);
    } else {
        const __nv_bfloat162 *d = reinterpret_cast<const __nv_bfloat162 *>(v.data) + s * 3 * v.n + r;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float2 f = __bfloat1622float2(vld<COHERENT>(d + (long)c * v.n));
            w[c] = {f.x, f.y};
        }
    }
}

// The values a colour vector has after store_vec then load_vec (the storage precision's
// rounding, the FP16 record's shared scale included), computed in registers.
template <int P>
__device__ __forceinline__ void round_trip(const Cplx<typename Prec<P>::real> w[3], Cplx<typename Prec<P>::real> out[3]) {
    if constexpr (P == HISQ_FP64 || P == HISQ_FP32) {
#pragma unroll
        for (int c = 0; c < 3; c++) out[c] = w[c];
    } else if constexpr (P == HISQ_FP16) {
        float m = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; c++) m = fmaxf(m, fmaxf(fabsf(w[c].re), fabsf(w[c].im)));
        const float inv = m > 0.0f ? 1.0f / m : 0.0f;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float2 f = __half22float2(__floats2half2_rn(w[c].re * inv, w[c].im * inv));
            out[c] = {f.x * m, f.y * m};
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float2 f = __bfloat1622float2(__floats2bfloat162_rn(w[c].re, w[c].im));
            out[c] = {f.x, f.y};
        }
    }
}

template <int P>
__device__ __forceinline__ void store_vec(const VecView<P> &v, long s, int r, const Cplx<typename Prec<P>::real> w[3]) {
    if constexpr (P == HISQ_FP64) {
        double2 *d = reinterpret_cast<double2 *>(v.data) + s * 3 * v.n + r;
#pragma unroll
        for (int c = 0; c < 3; c++) d[(long)c * v.n] = make_double2(w[c].re, w[c].im);
    } else if constexpr (P == HISQ_FP32) {
        float2 *d = reinterpret_cast<float2 *>(v.data) + s * 3 * v.n + r;
#pragma unroll
        for (int c = 0; c < 3; c++) d[(long)c * v.n] = make_float2(w[c].re, w[c].im);
    } else if constexpr (P == HISQ_FP16) {
        float m = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; c++) m = fmaxf(m, fmaxf(fabsf(w[c].re), fabsf(w[c].im)));
        const float inv = m > 0.0f ? 1.0f / m : 0.0f;
        uint32_t h[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            __half2 x = __floats2half2_rn(w[c].re * inv, w[c].im * inv);
            h[c] = *reinterpret_cast<uint32_t *>(&x);
        }
        reinterpret_cast<uint4 *>(v.data)[s * v.n + r] = make_uint4(h[0], h[1], h[2], __float_as_uint(m));
    } else {
        __nv_bfloat162 *d = reinterpret_cast<__nv_bfloat162 *>(v.data) + s * 3 * v.n + r;
#pragma unroll
        for (int c = 0; c < 3; c++) d[(long)c * v.n] = __floats2bfloat162_rn(w[c].re, w[c].im);
    }
}

// ------------------------------------------------------------------------------------------
// Packed links.  For every output parity p and output site s (even-odd index) a record of the
// 8 links the Dslash applies at s: slot 2mu = U_{x,mu}, slot 2mu+1 = -U^dag_{x-k mu,mu}
// (k = 1 fat, 3 Naik), so the stencil is a plain sum of 8 matrix-vector products per kind.
// A record is R reals per link (18 full; 13 = two rows of W and 24c; 9 = eight SU(3) parameters
// and 24c, for links c W with W in SU(3)), stored in 16-byte word planes:
// word j of site s of parity p at  words + ((size_t)p * W + j) * Vh + s,  W = 8 R bytes / 16.
// 16-bit 18-real records carry a per-site float scale (max |entry| of the 8 links).
// ------------------------------------------------------------------------------------------
struct LinkField {
    const uint4 *words;   // [2][W][Vh]
    const float *scale;   // [2][Vh] (16-bit, recon 18) or null
    int W;                // words per site
};

__host__ __device__ constexpr int link_words(int prec, int recon) {
    return 8 * recon * ((prec == HISQ_FP64 || prec == HISQ_DS) ? 8 : prec == HISQ_FP32 ? 4 : 2) / 16;
}

}  // namespace hisq

// Library-side objects (opaque in the ABI).
struct hisq_ctx;

struct hisq_links {
    hisq_ctx *ctx;
    int is_naik;
    int prec;
    int recon;
    int W;                 // words per site of the main copy
    uint4 *words;          // [2][W][Vh] main copy
    float *scale;          // [2][Vh] or null
    uint4 *words64;        // FP64 recon-18 copy (null when prec == FP64: use words)
    uint4 *words_ds;       // double-single recon-18 copy (null when prec == FP64)
    hisq::LinkField field() const { return {words, scale, W}; }
    hisq::LinkField field64() const {
        if (prec == HISQ_FP64 && recon == 18) return {words, nullptr, W};
        return {words64, nullptr, hisq::link_words(HISQ_FP64, 18)};
    }
    hisq::LinkField field_ds() const { return {words_ds, nullptr, hisq::link_words(hisq::HISQ_DS, 18)}; }
    // the residual recomputation of a mixed-precision solve runs in double-single arithmetic on
    // the FP32 pipe; FP64 handles keep native FP64 throughout
    bool residual_ds() const { return prec != HISQ_FP64; }
};

struct hisq_pc {
    hisq_ctx *ctx;
    double weights[HISQ_PC_WEIGHTS * 2];   // host copy (authoritative after set/get/adam)
    float2 *d_weights;                     // device FP32 copy used by the kernels
    double *d_theta, *d_m, *d_v;           // Adam state on the device (FP64, real parameters)
    void *work;                            // network workspace (pc.cu)
    int form;                              // HISQ_PC_NORMAL or HISQ_PC_HERMITIAN_PART
    int train_steps;                       // Adam steps taken by hisq_pc_train (continued across calls)
};

namespace hisq {

struct TuneKey {
    int prec, recon, n, kind;
    bool operator<(const TuneKey &o) const {
        if (prec != o.prec) return prec < o.prec;
        if (recon != o.recon) return recon < o.recon;
        if (n != o.n) return n < o.n;
        return kind < o.kind;
    }
};

struct LaunchShape {
    int R;        // right-hand sides per thread
    int threads;  // threads per block
    int S = 1;    // lanes per (site, rhs group): 2 splits the fat and Naik halves, 4 two directions
                  // of one kind per lane (18-real Naik); 8 = the 4-lane split with the tile's link
                  // records staged in shared memory by the bulk-copy engine
};

// shared memory of the staged kernel for TS sites per tile: two stages of link records, the
// mbarriers, and the reduction scratch of the reducing epilogue
inline size_t staged_smem(int words_per_site, int TS, int threads, int n, bool reducing) {
    size_t red = reducing ? std::max((size_t)TS * n, (size_t)threads + 64) * sizeof(double) : 0;
    return 16 + (size_t)2 * words_per_site * TS * 16 + red;
}

struct Workspace;  // solver workspace (solver.cu)
struct MsWork;     // multi-shift solver workspace (multishift.cu)

}  // namespace hisq

struct hisq_ctx {
    hisq::Geom geom;
    int device;
    cudaStream_t stream;
    int *dev_err = nullptr;  // set by a kernel whose bounded wait ran out (read by hisq_device_status)
    int num_sms;
    hisq_solver_params params;
    std::map<hisq::TuneKey, hisq::LaunchShape> tuned;
    std::map<hisq::TuneKey, float> tuned_ms;  // median time of the chosen shape (L2 flushed)
    unsigned tune_generation = 0;  // bumped whenever a launch shape changes (captured graphs go stale)
    // generic scratch: reductions (partials + counter) and the A-operator intermediate
    double *partials;       // [max_blocks * HISQ_MAX_NRHS * 2]
    size_t partials_cap;
    unsigned int *counter;  // last-block-done counter (reset by the last block)
    double *dot_out;        // [HISQ_MAX_NRHS * 2] device results
    void *tmp;              // odd-parity intermediate for hisq_aop
    size_t tmp_cap;
    hisq::Workspace *ws;
    hisq::MsWork *ms = nullptr;
    // L2 persisting set-aside for the link window of the persistent solve
    int l2_persist_max = -1, l2_window_max = 0;  // device limits (-1: not queried yet)
    bool l2_limit_saved = false;                 // l2_limit_old holds the context's limit before ours
    size_t l2_limit_old = 0;
    // last solve statistics
    hisq_solve_stats stats;
    std::vector<int> stat_iters;
    std::vector<double> stat_resid;
    std::vector<hisq_links *> links;
    std::vector<hisq_pc *> pcs;
};

namespace hisq {
hisq_ctx *current();
int require_ctx(hisq_ctx **ctx);
int ensure_scratch(hisq_ctx *ctx, size_t partial_doubles, size_t tmp_bytes);
bool is_device_ptr(const void *p);
// Largest grid <= max_blocks that gives every block the same number of tiles (one fewer for
// some when tiles is not a multiple), so no SM waits on a straggling extra tile.
inline long balanced_grid(long tiles, long max_blocks) {
    if (max_blocks < 1) max_blocks = 1;
    if (tiles <= max_blocks) return tiles < 1 ? 1 : tiles;
    long per_block = (tiles + max_blocks - 1) / max_blocks;
    return (tiles + per_block - 1) / per_block;
}

// Dslash family launchers (context.cu)
enum Epilogue { EPI_PLAIN = 0, EPI_AOP = 1, EPI_RESID = 2 };
struct DslashArgs {
    const void *in;        // opposite-parity input bundle
    void *out;             // output bundle (parity `parity`)
    int n;                 // right-hand sides in the bundle
    int parity;            // output parity
    Epilogue epi;
    double mass2;          // EPI_AOP / EPI_RESID
    const double *mass2v;  // EPI_RESID: device m^2 per right-hand side (null: mass2 for all)
    const void *axpy_in;   // EPI_AOP: p (same precision); EPI_RESID: x_hi (FP64)
    const void *b;         // EPI_RESID: right-hand side b (FP64 internal)
    int b_one;             // EPI_RESID: b holds one right-hand side, shared by all of the bundle
    void *out_lo;          // EPI_RESID: sloppy copy of the new residual (lo_prec) or null
    int lo_prec;
    const int *active;     // per-rhs mask (null = all)
    const int *gate;       // kernel is a no-op when *gate == 0 (null = always run)
    double *partials;      // per-block partial dots (EPI_AOP / EPI_RESID)
    size_t partials_cap;   // doubles available in partials
    unsigned int *counter;
    double *dot_out;       // reduced dots [n]
    int hook;              // solver hook run by the last block (0 = none)
    void *hook_state;
    int partials_only;     // reducing epilogues: publish per-block partials only (no finish)
    int site_begin, site_end;  // output sites [site_begin, site_end) of the parity; 0, 0 = all
    // another lattice and link records than the context's (a slab of the domain decomposition):
    // used instead of ctx->geom and the handles' copies when set; the handles then only give the
    // precision and encoding, and the caller passes the launch shape
    const Geom *geom;
    const LinkField *fields;   // [2]: fat, Naik
};
// Which copy of the links a Dslash reads, and in which arithmetic: the handle's own storage
// precision; the FP64 copy in FP64; or the double-single copy in double-single arithmetic (input
// and, for EPI_PLAIN, output bundles in the ds form; EPI_RESID keeps x, b and r in FP64).
enum LinkCopy { LINKS_INNER = 0, LINKS_FP64 = 1, LINKS_DS = 2 };
// the copy that gives FP64 accuracy for these links: double-single unless they are FP64 already
inline int links_hp(const hisq_links *fat) { return fat->residual_ds() ? LINKS_DS : LINKS_FP64; }
// Sites per block and threads per block of a (non-staged) Dslash launch of n right-hand sides,
// R per thread and S lanes per site, for the shape's block size (reducing epilogues use at
// least 128 threads); launch_dslash and every caller that sizes reduction scratch in advance use it
inline void dslash_block_shape(int n, int R, int S, int shape_threads, bool reducing, int *spb, int *threads) {
    const int t = (n + R - 1) / R;
    const int want = reducing ? std::max(shape_threads, 128) : shape_threads;
    int p = 1;
    while (p * 2 <= std::max(1, std::min(want, 256) / (S * t))) p *= 2;  // kernels are bounded to 256 threads
    *spb = p;
    *threads = (p * S * t + 31) / 32 * 32;  // whole warps; threads with site index >= spb idle
}
// the reduction partials (doubles) a reducing Dslash epilogue of that shape writes on a parity of
// Vh sites: one per block and right-hand side, the grid capped at 64 blocks per SM
inline size_t dslash_partials_needed(long Vh, int num_sms, int spb, int n) {
    const long tiles = (Vh + spb - 1) / spb;
    return (size_t)std::min<long>(tiles, (long)num_sms * 64) * n;
}
// (fat, naik) handles of this context with matching precisions (context.cu)
int check_pair(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik);
// grid_out (optional) receives the number of blocks launched (= partials written per dot)
int launch_dslash(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int copy,
                  const DslashArgs &a, const LaunchShape *shape, cudaStream_t stream, int *grid_out = nullptr);
LaunchShape default_shape(int prec, int n);
LaunchShape tuned_shape(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int n, int copy);
int choose_bundle(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int nrhs, int copy);  // tune.cu
// the precision id a copy computes in (tuning keys, vector sizes)
inline int copy_prec(const hisq_links *fat, int copy) {
    return copy == LINKS_DS ? HISQ_DS : copy == LINKS_FP64 ? HISQ_FP64 : fat->prec;
}
// Gathered link records (context.cu) of the storage lattice gs for links U of the lattice g: storage
// site (x, y, z, ts) is lattice site (x, y, z, (ts + t_off) mod Lt), only planes ts in [t_lo, t_hi)
// (gs = g, t_off = 0: the whole lattice; otherwise one slab with ghost planes)
void pack_links_into(int prec, int recon, const Geom &g, const Geom &gs, int t_off, int t_lo, int t_hi,
                     const double *U, int hop, uint4 *words, float *scale, int W, cudaStream_t st);
// FP64 bundle -> double-single bundle of n right-hand sides (dslash_ds.cu)
int split_vectors(hisq_ctx *ctx, const void *fp64_bundle, void *ds_bundle, int n, cudaStream_t st);
void free_workspace(hisq_ctx *ctx);  // solver.cu
void free_multishift(hisq_ctx *ctx); // multishift.cu
// CG solve of nrhs right-hand sides (solver.cu): hisq_cg_solve when mass2v and tolv are null;
// otherwise each right-hand side k solves (mass2v[k] - D_eo D_oe) x = b to tolv[k] (persistent
// driver, 18-real Naik links, no preconditioner)
int cg_solve_common(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, const double *const rhs[],
                    double *x[], int nrhs, double mass, double tol, const double *mass2v, const double *tolv);
void free_pc(hisq_pc *pc);           // pc.cu
int pc_forward(hisq_ctx *ctx, const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const void *in,
               void *out, int n, cudaStream_t st);
int pc_forward_precond(hisq_ctx *ctx, const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik,
                       const void *in, void *out, int n, cudaStream_t st);  // the handle's form
int pc_prepare(hisq_ctx *ctx, const hisq_pc *pc, int n);  // allocate the network workspace
int pack_vectors(hisq_ctx *ctx, const double *canon_dev, void *internal, int n, int prec, cudaStream_t st);
int unpack_vectors(hisq_ctx *ctx, const void *internal, double *canon_dev, int n, int prec, cudaStream_t st);
}  // namespace hisq
