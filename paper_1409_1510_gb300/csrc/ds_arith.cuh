// Double-single ("ds") arithmetic: the FP64-accurate residual recomputation r = b - A x of the
// mixed-precision solver (the reliable update) on the FP32 pipe.
//
// A real x is held as two floats, hi = fl32(x) and lo = fl32(x - hi), so that hi + lo equals x to
// within 2^-48 |x|.  A product of two such numbers keeps the exact product of the high parts,
// split into its rounded value p = fl(a_hi b_hi) and its rounding error fma(a_hi, b_hi, -p)
// (Dekker 1971, with a fused multiply-add in place of operand splitting), plus the two cross
// terms a_hi b_lo and a_lo b_hi (a_lo b_lo is below 2^-48 of the product and dropped).  Sums of
// products add the rounded parts with Knuth's two-sum, which returns the rounding error of a
// float addition exactly, and gather every error and cross term in a second float accumulator:
// the cascaded summation of Ogita, Rump and Oishi (2005), whose result is as accurate as a sum
// computed in twice the working precision.  On this part the FP32 pipe issues 64 times as many
// operations per cycle as the FP64 pipe, so the twelve float operations a real multiply-add
// costs here run about five times faster than one FP64 fused multiply-add.
//
// The error-free steps use the rounding intrinsics (__fmul_rn, __fadd_rn, __fsub_rn, __fmaf_rn),
// which the compiler neither contracts into fused operations nor reorders.
//
// Storage: a ds link record has the FP64 record's layout (8 bytes per real) with every double
// replaced by its (hi, lo) float pair; a ds colour vector bundle has the FP64 bundle's layout
// with every complex number (re, im) stored as the float4 (re_hi, re_lo, im_hi, im_lo).
#pragma once
#include "hisq_internal.cuh"

namespace hisq {

struct dsacc {
    float hi, lo;
};

// s += a b for ds numbers a = (a_hi, a_lo), b = (b_hi, b_lo)
__device__ __forceinline__ void ds_mac(dsacc &s, float a_hi, float a_lo, float b_hi, float b_lo) {
    const float p = __fmul_rn(a_hi, b_hi);
    const float e = __fmaf_rn(a_hi, b_hi, -p);  // a_hi b_hi - p, exactly
    const float t = __fadd_rn(s.hi, p);
    const float z = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(p, z));  // s.hi + p - t, exactly
    float lo = __fmaf_rn(a_hi, b_lo, s.lo);
    lo = __fmaf_rn(a_lo, b_hi, lo);
    s.hi = t;
    s.lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// the pair (hi, lo) with hi = fl(hi + lo): the accumulator in the storage form
__device__ __forceinline__ dsacc ds_normalize(dsacc s) {
    const float t = __fadd_rn(s.hi, s.lo);
    const float z = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(s.lo, z));
    return {t, err};
}

__device__ __forceinline__ double ds_value(dsacc s) { return (double)s.hi + (double)s.lo; }

__device__ __forceinline__ void ds_split(double x, float &hi, float &lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
}

// A complex ds accumulator and the ds colour-vector bundle (float4 per complex number at
// (s * 3 + c) * n + r, like the FP64 bundle's double2).
struct dscplx {
    dsacc re, im;
};

template <bool COHERENT>
__device__ __forceinline__ float4 ds_load(const float4 *v, long idx) {
    if constexpr (COHERENT) return __ldcg(v + idx);
    else return __ldg(v + idx);
}

__device__ __forceinline__ void ds_store3(float4 *v, int n, long s, int r, const dscplx w[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const dsacc re = ds_normalize(w[c].re), im = ds_normalize(w[c].im);
        v[(s * 3 + c) * n + r] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
}

// acc[a] += M_ab v_b for the three rows a of column b of one ds link: m[a] = the 16-byte word of
// entry (a, b), i.e. the floats (re_hi, re_lo, im_hi, im_lo), and one ds colour component v_b.
// The six accumulators (three rows, real and imaginary part) are independent chains, so a thread
// keeps six two-sum sequences in flight instead of two.
__device__ __forceinline__ void ds_column_acc(const uint4 m[3], const float4 vb, dscplx acc[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float mr_hi = __uint_as_float(m[a].x), mr_lo = __uint_as_float(m[a].y);
        // (mr + i mi)(vr + i vi): the mr products first, the mi products below
        ds_mac(acc[a].re, mr_hi, mr_lo, vb.x, vb.y);
        ds_mac(acc[a].im, mr_hi, mr_lo, vb.z, vb.w);
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float mi_hi = __uint_as_float(m[a].z), mi_lo = __uint_as_float(m[a].w);
        ds_mac(acc[a].re, -mi_hi, -mi_lo, vb.z, vb.w);
        ds_mac(acc[a].im, mi_hi, mi_lo, vb.x, vb.y);
    }
}

// the 9 words of link `slot` of a ds record and the neighbour vectors it multiplies
template <int R, bool COHERENT>
struct DsOperands {
    uint4 m[9];        // entry (a, b) in word 3 a + b
    float4 v[R][3];
    __device__ __forceinline__ void load(const Geom &g, const SiteCoord &sc, const LinkField &f, int hop, int parity,
                                         int s, int slot, const float4 *in, int n, const int rr[R], const bool act[R]) {
        const uint4 *base = f.words + ((size_t)parity * f.W + (size_t)slot * 9) * g.Vh + s;
#pragma unroll
        for (int j = 0; j < 9; j++) m[j] = __ldg(base + (size_t)j * g.Vh);
        const int nb = neighbour_rt(g, sc, s, slot >> 1, (slot & 1) ? -hop : hop);
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int c = 0; c < 3; c++)
                v[r][c] = act[r] ? ds_load<COHERENT>(in, ((long)nb * 3 + c) * n + rr[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __device__ __forceinline__ void apply(dscplx acc[R][3]) const {
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const uint4 col[3] = {m[b], m[3 + b], m[6 + b]};
#pragma unroll
            for (int r = 0; r < R; r++) ds_column_acc(col, v[r][b], acc[r]);
        }
    }
};

// The stencil of Eq. (3) at output site s of parity `parity` in ds arithmetic for the R
// right-hand sides rr[0..R) of the ds input bundle `in` (n right-hand sides): the 8 fat and 8 Naik
// links of the site's gathered ds records (slot 2 mu forward, 2 mu + 1 the backward -U^dagger, as
// in every other precision) times the neighbouring input vectors, summed into acc.  The 16 links
// run as one sequence (fat slots 0..7, then Naik).  With PREFETCH the words and vectors of the next
// link are requested before the current one is applied, column by column (six independent
// accumulation chains): twice the operand registers for more loads in flight (the recomputation
// is bound by memory latency with one thread per site and right-hand side).  Without it (kernels
// that must stay within 64 or 128 registers) each link row is requested just before its use.
template <int R, bool COHERENT, bool PREFETCH = false>
__device__ __forceinline__ void ds_site_stencil(const Geom &g, const LinkField &fat, const LinkField &naik, int parity,
                                                const float4 *in, int n, int s, const int rr[R], const bool act[R],
                                                dscplx acc[R][3]) {
    const SiteCoord sc = decode_site(g, s, parity);
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc[r][c] = {{0.f, 0.f}, {0.f, 0.f}};
    if constexpr (PREFETCH) {
        DsOperands<R, COHERENT> cur, nxt;
        cur.load(g, sc, fat, 1, parity, s, 0, in, n, rr, act);
#pragma unroll 1
        for (int k = 0; k < 16; k++) {
            if (k + 1 < 16) {
                const bool nk = k + 1 >= 8;
                nxt.load(g, sc, nk ? naik : fat, nk ? 3 : 1, parity, s, (k + 1) & 7, in, n, rr, act);
            }
            cur.apply(acc);
            cur = nxt;
        }
    } else {
        // few registers: each link's words are requested row by row, just before their use
#pragma unroll 1
        for (int k = 0; k < 16; k++) {
            const bool nk = k >= 8;
            const LinkField &f = nk ? naik : fat;
            const int slot = k & 7, hop = nk ? 3 : 1;
            const uint4 *base = f.words + ((size_t)parity * f.W + (size_t)slot * 9) * g.Vh + s;
            const int nb = neighbour_rt(g, sc, s, slot >> 1, (slot & 1) ? -hop : hop);
            float4 v[R][3];
#pragma unroll
            for (int r = 0; r < R; r++)
#pragma unroll
                for (int c = 0; c < 3; c++)
                    v[r][c] = act[r] ? ds_load<COHERENT>(in, ((long)nb * 3 + c) * n + rr[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int a = 0; a < 3; a++) {
                uint4 m[3];
#pragma unroll
                for (int b = 0; b < 3; b++) m[b] = __ldg(base + (size_t)(3 * a + b) * g.Vh);
#pragma unroll
                for (int r = 0; r < R; r++)
#pragma unroll
                    for (int b = 0; b < 3; b++) {
                        const float mr_hi = __uint_as_float(m[b].x), mr_lo = __uint_as_float(m[b].y);
                        const float mi_hi = __uint_as_float(m[b].z), mi_lo = __uint_as_float(m[b].w);
                        ds_mac(acc[r][a].re, mr_hi, mr_lo, v[r][b].x, v[r][b].y);
                        ds_mac(acc[r][a].re, -mi_hi, -mi_lo, v[r][b].z, v[r][b].w);
                        ds_mac(acc[r][a].im, mr_hi, mr_lo, v[r][b].z, v[r][b].w);
                        ds_mac(acc[r][a].im, mi_hi, mi_lo, v[r][b].x, v[r][b].y);
                    }
            }
        }
    }
}

}  // namespace hisq
