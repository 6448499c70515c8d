// Decoding of packed link records into 3x3 complex matrices (device side).
#pragma once
#include "hisq_internal.cuh"

namespace hisq {

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

template <int P, int RECON>
struct LinkCodec {
    using real = typename Prec<P>::real;
    static constexpr int EB = Prec<P>::bytes;        // bytes per stored real
    static constexpr int LB = RECON * EB;            // bytes per link
    static constexpr int G = 16 / gcd_c(LB, 16);     // links per word-aligned group
    static constexpr int WG = G * LB / 16;           // words per group
    static constexpr int GROUPS = 8 / G;             // groups per 8-link record
    static_assert(8 % G == 0, "group size must divide the 8 links of a record");

    // element e (0 <= e < G*RECON) of a group held in u[WG*4]
    __device__ __forceinline__ static real elem(const uint32_t *u, int e) {
        if constexpr (P == HISQ_FP64) {
            return __hiloint2double((int)u[2 * e + 1], (int)u[2 * e]);
        } else if constexpr (P == HISQ_FP32) {
            return __uint_as_float(u[e]);
        } else if constexpr (P == HISQ_FP16) {
            unsigned short b = (unsigned short)(u[e >> 1] >> (16 * (e & 1)));
            return __half2float(__ushort_as_half(b));
        } else {
            unsigned short b = (unsigned short)(u[e >> 1] >> (16 * (e & 1)));
            return __bfloat162float(__ushort_as_bfloat16(b));
        }
    }

    __device__ __forceinline__ static void load_group(const LinkField &f, int parity, int Vh, int s,
                                                      int group, uint32_t u[WG * 4]) {
        const uint4 *base = f.words + ((size_t)parity * f.W + (size_t)group * WG) * Vh + s;
#pragma unroll
        for (int j = 0; j < WG; j++) {
            uint4 w = __ldg(base + (size_t)j * Vh);
            u[4 * j] = w.x; u[4 * j + 1] = w.y; u[4 * j + 2] = w.z; u[4 * j + 3] = w.w;
        }
    }

    // link l (0 <= l < G) of the group, times `scale` (18-real records only)
    __device__ __forceinline__ static void decode(const uint32_t *u, int l, real scale, Cplx<real> M[3][3]) {
        decode(u, l, M);
        if constexpr (RECON == 18) {
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) M[a][b] = {M[a][b].re * scale, M[a][b].im * scale};
        }
    }

    // link l (0 <= l < G) of the group as stored (16-bit 18-real records without their site scale)
    __device__ __forceinline__ static void decode(const uint32_t *u, int l, Cplx<real> M[3][3]) {
        const int o = l * RECON;
        if constexpr (RECON == 18) {
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) M[a][b] = {elem(u, o + 6 * a + 2 * b), elem(u, o + 6 * a + 2 * b + 1)};
        } else if constexpr (RECON == 13) {
            // rows 0, 1 of W; row 2 = conj(row0 x row1); link = c W with c = elem(12) / 24
            Cplx<real> r0[3], r1[3];
#pragma unroll
            for (int b = 0; b < 3; b++) {
                r0[b] = {elem(u, o + 2 * b), elem(u, o + 2 * b + 1)};
                r1[b] = {elem(u, o + 6 + 2 * b), elem(u, o + 7 + 2 * b)};
            }
            real c = elem(u, o + 12) * (real)(1.0 / 24.0);
#pragma unroll
            for (int b = 0; b < 3; b++) {
                int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
                // (r0 x r1)_b = r0_b1 r1_b2 - r0_b2 r1_b1
                real cre = r0[b1].re * r1[b2].re - r0[b1].im * r1[b2].im - (r0[b2].re * r1[b1].re - r0[b2].im * r1[b1].im);
                real cim = r0[b1].re * r1[b2].im + r0[b1].im * r1[b2].re - (r0[b2].re * r1[b1].im + r0[b2].im * r1[b1].re);
                M[0][b] = {c * r0[b].re, c * r0[b].im};
                M[1][b] = {c * r1[b].re, c * r1[b].im};
                M[2][b] = {c * cre, -c * cim};
            }
        } else {
            static_assert(RECON == 9, "recon must be 18, 13 or 9");
            // elements: theta0 = arg W00, theta2 = arg W20, W01, W02, W10, 24c
            real th0 = elem(u, o + 0), th2 = elem(u, o + 1);
            Cplx<real> w01 = {elem(u, o + 2), elem(u, o + 3)};
            Cplx<real> w02 = {elem(u, o + 4), elem(u, o + 5)};
            Cplx<real> w10 = {elem(u, o + 6), elem(u, o + 7)};
            real c = elem(u, o + 8) * (real)(1.0 / 24.0);
            real n2 = w01.re * w01.re + w01.im * w01.im + w02.re * w02.re + w02.im * w02.im;
            real a00 = sqrt(fmax((real)0, (real)1 - n2));
            real s0, c0, s2, c2;
            sincos_r(th0, &s0, &c0);
            sincos_r(th2, &s2, &c2);
            Cplx<real> w00 = {a00 * c0, a00 * s0};
            real a20 = sqrt(fmax((real)0, (real)1 - a00 * a00 - (w10.re * w10.re + w10.im * w10.im)));
            Cplx<real> w20 = {a20 * c2, a20 * s2};
            // e = -W00 conj(W10)
            Cplx<real> e = {-(w00.re * w10.re + w00.im * w10.im), -(w00.im * w10.re - w00.re * w10.im)};
            real inv = (real)1 / n2;
            // X = conj(W11) = (e conj(W01) - W02 W20) / n2 ;  Y = conj(W12) = (W01 W20 + e conj(W02)) / n2
            Cplx<real> X = {(e.re * w01.re + e.im * w01.im) - (w02.re * w20.re - w02.im * w20.im),
                            (e.im * w01.re - e.re * w01.im) - (w02.re * w20.im + w02.im * w20.re)};
            Cplx<real> Y = {(w01.re * w20.re - w01.im * w20.im) + (e.re * w02.re + e.im * w02.im),
                            (w01.re * w20.im + w01.im * w20.re) + (e.im * w02.re - e.re * w02.im)};
            Cplx<real> w11 = {X.re * inv, -X.im * inv};
            Cplx<real> w12 = {Y.re * inv, -Y.im * inv};
            // W21 = conj(W02 W10 - W00 W12), W22 = conj(W00 W11 - W01 W10)
            Cplx<real> w21 = {(w02.re * w10.re - w02.im * w10.im) - (w00.re * w12.re - w00.im * w12.im),
                              -((w02.re * w10.im + w02.im * w10.re) - (w00.re * w12.im + w00.im * w12.re))};
            Cplx<real> w22 = {(w00.re * w11.re - w00.im * w11.im) - (w01.re * w10.re - w01.im * w10.im),
                              -((w00.re * w11.im + w00.im * w11.re) - (w01.re * w10.im + w01.im * w10.re))};
            M[0][0] = {c * w00.re, c * w00.im}; M[0][1] = {c * w01.re, c * w01.im}; M[0][2] = {c * w02.re, c * w02.im};
            M[1][0] = {c * w10.re, c * w10.im}; M[1][1] = {c * w11.re, c * w11.im}; M[1][2] = {c * w12.re, c * w12.im};
            M[2][0] = {c * w20.re, c * w20.im}; M[2][1] = {c * w21.re, c * w21.im}; M[2][2] = {c * w22.re, c * w22.im};
        }
    }

    __device__ __forceinline__ static void sincos_r(real x, real *s, real *c) {
        if constexpr (sizeof(real) == 8) sincos(x, s, c);
        else sincosf(x, s, c);
    }
};

// acc[r] += M v[r]
template <typename T, int R>
__device__ __forceinline__ void matvec_acc(const Cplx<T> M[3][3], const Cplx<T> v[R][3], Cplx<T> acc[R][3]) {
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                acc[r][a].re = fma(M[a][b].re, v[r][b].re, fma(-M[a][b].im, v[r][b].im, acc[r][a].re));
                acc[r][a].im = fma(M[a][b].re, v[r][b].im, fma(M[a][b].im, v[r][b].re, acc[r][a].im));
            }
}

}  // namespace hisq
