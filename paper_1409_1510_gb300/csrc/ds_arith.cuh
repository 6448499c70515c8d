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

// acc += (M v)_a for row a of one ds link: m[b] = the 16-byte word of entry (a, b), i.e. the
// floats (re_hi, re_lo, im_hi, im_lo), and one ds colour vector v[3]
__device__ __forceinline__ void ds_row_acc(const uint4 m[3], const float4 v[3], dscplx &acc) {
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const float mr_hi = __uint_as_float(m[b].x), mr_lo = __uint_as_float(m[b].y);
        const float mi_hi = __uint_as_float(m[b].z), mi_lo = __uint_as_float(m[b].w);
        // (mr + i mi)(vr + i vi)
        ds_mac(acc.re, mr_hi, mr_lo, v[b].x, v[b].y);
        ds_mac(acc.re, -mi_hi, -mi_lo, v[b].z, v[b].w);
        ds_mac(acc.im, mr_hi, mr_lo, v[b].z, v[b].w);
        ds_mac(acc.im, mi_hi, mi_lo, v[b].x, v[b].y);
    }
}

// The stencil of Eq. (3) at output site s of parity `parity` in ds arithmetic for the R
// right-hand sides rr[0..R) of the ds input bundle `in` (n right-hand sides): the 8 fat and 8 Naik
// links of the site's gathered ds records (slot 2 mu forward, 2 mu + 1 the backward -U^dagger, as
// in every other precision) times the neighbouring input vectors, summed into acc.
template <int R, bool COHERENT>
__device__ __forceinline__ void ds_site_stencil(const Geom &g, const LinkField &fat, const LinkField &naik, int parity,
                                                const float4 *in, int n, int s, const int rr[R], const bool act[R],
                                                dscplx acc[R][3]) {
    const SiteCoord sc = decode_site(g, s, parity);
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc[r][c] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int kind = 0; kind < 2; kind++) {
        const LinkField &f = kind ? naik : fat;
        const int hop = kind ? 3 : 1;
#pragma unroll 1
        for (int slot = 0; slot < 8; slot++) {
            // a ds link is 9 words: entry (a, b) in word 3 a + b of the record's link
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
                for (int r = 0; r < R; r++) ds_row_acc(m, v[r], acc[r][a]);
            }
        }
    }
}

}  // namespace hisq
