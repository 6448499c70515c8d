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

// even-odd index of the neighbour `step` hops (|step| <= 3 < L) away in direction mu
__host__ __device__ __forceinline__ int neighbour(const Geom &g, const SiteCoord &sc, int s, int mu, int step) {
    int c = sc.c[mu] + step;
    int L = g.L[mu];
    c += (c < 0) ? L : 0;
    c -= (c >= L) ? L : 0;
    if (mu == 0) return sc.row_base + (c >> 1);
    return s + (c - sc.c[mu]) * g.stride[mu];
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

// bytes of one complex element of an internal vector
__host__ __device__ constexpr int vec_elem_bytes(int prec) {
    return prec == HISQ_FP64 ? 16 : prec == HISQ_FP32 ? 8 : 4;
}

// offset of the FP16 per-(site, rhs) scale array inside a bundle
__host__ __device__ inline size_t fp16_scale_offset(int Vh, int n) {
    size_t main = (size_t)Vh * 3 * n * 4;
    return (main + 255) & ~(size_t)255;
}

inline size_t vector_bytes(int prec, int Vh, int n) {
    if (prec == HISQ_FP16) return fp16_scale_offset(Vh, n) + (size_t)Vh * n * 4;
    return (size_t)Vh * 3 * n * vec_elem_bytes(prec);
}

// A bundle of n right-hand sides in the internal layout, typed by precision.
template <int P> struct VecView {
    void *data;
    float *scale;  // FP16 only
    int n;
};

template <int P>
__device__ __forceinline__ Cplx<typename Prec<P>::real> load_elem(const VecView<P> &v, long idx, float sc);

template <>
__device__ __forceinline__ Cplx<double> load_elem<HISQ_FP64>(const VecView<HISQ_FP64> &v, long idx, float) {
    double2 d = __ldg(reinterpret_cast<const double2 *>(v.data) + idx);
    return {d.x, d.y};
}
template <>
__device__ __forceinline__ Cplx<float> load_elem<HISQ_FP32>(const VecView<HISQ_FP32> &v, long idx, float) {
    float2 d = __ldg(reinterpret_cast<const float2 *>(v.data) + idx);
    return {d.x, d.y};
}
template <>
__device__ __forceinline__ Cplx<float> load_elem<HISQ_FP16>(const VecView<HISQ_FP16> &v, long idx, float sc) {
    __half2 h = __ldg(reinterpret_cast<const __half2 *>(v.data) + idx);
    float2 f = __half22float2(h);
    return {f.x * sc, f.y * sc};
}
template <>
__device__ __forceinline__ Cplx<float> load_elem<HISQ_BF16>(const VecView<HISQ_BF16> &v, long idx, float) {
    __nv_bfloat162 h = __ldg(reinterpret_cast<const __nv_bfloat162 *>(v.data) + idx);
    float2 f = __bfloat1622float2(h);
    return {f.x, f.y};
}

// load the 3 colours of right-hand sides r0..r0+R-1 at site s
template <int P, int R>
__device__ __forceinline__ void load_site(const VecView<P> &v, int s, int r0, int nvalid,
                                          Cplx<typename Prec<P>::real> out[R][3]) {
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (r < nvalid) {
            float sc = 1.0f;
            if (P == HISQ_FP16) sc = __ldg(v.scale + (long)s * v.n + r0 + r);
#pragma unroll
            for (int c = 0; c < 3; c++) out[r][c] = load_elem<P>(v, ((long)s * 3 + c) * v.n + r0 + r, sc);
        } else {
#pragma unroll
            for (int c = 0; c < 3; c++) out[r][c] = {0, 0};
        }
    }
}

// store the 3 colours of one right-hand side r at site s (FP16: computes the scale)
template <int P>
__device__ __forceinline__ void store_site(const VecView<P> &v, int s, int r,
                                           const Cplx<typename Prec<P>::real> w[3]) {
    long base = (long)s * 3 * v.n + r;
    if constexpr (P == HISQ_FP64) {
        double2 *d = reinterpret_cast<double2 *>(v.data);
#pragma unroll
        for (int c = 0; c < 3; c++) d[base + (long)c * v.n] = make_double2(w[c].re, w[c].im);
    } else if constexpr (P == HISQ_FP32) {
        float2 *d = reinterpret_cast<float2 *>(v.data);
#pragma unroll
        for (int c = 0; c < 3; c++) d[base + (long)c * v.n] = make_float2(w[c].re, w[c].im);
    } else if constexpr (P == HISQ_FP16) {
        float m = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; c++) m = fmaxf(m, fmaxf(fabsf(w[c].re), fabsf(w[c].im)));
        float inv = m > 0.0f ? 1.0f / m : 0.0f;
        __half2 *d = reinterpret_cast<__half2 *>(v.data);
#pragma unroll
        for (int c = 0; c < 3; c++) d[base + (long)c * v.n] = __floats2half2_rn(w[c].re * inv, w[c].im * inv);
        v.scale[(long)s * v.n + r] = m;
    } else {
        __nv_bfloat162 *d = reinterpret_cast<__nv_bfloat162 *>(v.data);
#pragma unroll
        for (int c = 0; c < 3; c++) d[base + (long)c * v.n] = __floats2bfloat162_rn(w[c].re, w[c].im);
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
    return 8 * recon * (prec == HISQ_FP64 ? 8 : prec == HISQ_FP32 ? 4 : 2) / 16;
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
    hisq::LinkField field() const { return {words, scale, W}; }
    hisq::LinkField field64() const {
        if (prec == HISQ_FP64 && recon == 18) return {words, nullptr, W};
        return {words64, nullptr, hisq::link_words(HISQ_FP64, 18)};
    }
};

struct hisq_pc {
    hisq_ctx *ctx;
    double weights[HISQ_PC_WEIGHTS * 2];   // host copy (authoritative after set/get/adam)
    float2 *d_weights;                     // device FP32 copy used by the kernels
    double *d_theta, *d_m, *d_v;           // Adam state on the device (FP64, real parameters)
    void *work;                            // network workspace (pc.cu)
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
};

struct Workspace;  // solver workspace (solver.cu)

}  // namespace hisq

struct hisq_ctx {
    hisq::Geom geom;
    int device;
    cudaStream_t stream;
    int num_sms;
    hisq_solver_params params;
    std::map<hisq::TuneKey, hisq::LaunchShape> tuned;
    // generic scratch: reductions (partials + counter) and the A-operator intermediate
    double *partials;       // [max_blocks * HISQ_MAX_NRHS * 2]
    size_t partials_cap;
    unsigned int *counter;  // last-block-done counter (reset by the last block)
    double *dot_out;        // [HISQ_MAX_NRHS * 2] device results
    void *tmp;              // odd-parity intermediate for hisq_aop
    size_t tmp_cap;
    hisq::Workspace *ws;
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
int grid_for(hisq_ctx *ctx, long work_items, int threads, int max_waves = 8);

// Dslash family launchers (context.cu)
enum Epilogue { EPI_PLAIN = 0, EPI_AOP = 1, EPI_RESID = 2 };
struct DslashArgs {
    const void *in;        // opposite-parity input bundle
    void *out;             // output bundle (parity `parity`)
    int n;                 // right-hand sides in the bundle
    int parity;            // output parity
    Epilogue epi;
    double mass2;          // EPI_AOP / EPI_RESID
    const void *axpy_in;   // EPI_AOP: p (same precision); EPI_RESID: x_hi (FP64)
    const void *b;         // EPI_RESID: right-hand side b (FP64 internal)
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
};
int launch_dslash(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, bool use64,
                  const DslashArgs &a, const LaunchShape *shape, cudaStream_t stream);
LaunchShape default_shape(int prec, int n);
LaunchShape tuned_shape(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int n, bool use64);
void free_workspace(hisq_ctx *ctx);  // solver.cu
void free_pc(hisq_pc *pc);           // pc.cu
int pc_forward(hisq_ctx *ctx, const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, const void *in,
               void *out, int n, cudaStream_t st);
int pc_prepare(hisq_ctx *ctx, const hisq_pc *pc, int n);  // allocate the network workspace
int pack_vectors(hisq_ctx *ctx, const double *canon_dev, void *internal, int n, int prec, cudaStream_t st);
int unpack_vectors(hisq_ctx *ctx, const void *internal, double *canon_dev, int n, int prec, cudaStream_t st);
}  // namespace hisq
