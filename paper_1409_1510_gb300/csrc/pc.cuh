// Gauge-covariant parallel-transport network: layer, adjoint-layer and weight-gradient kernels.
//
// A layer maps A input channels to B output channels of full-lattice colour fields, for K
// samples, one output parity at a time:
//   h'_b(x) = sum_path sum_a W[path][b][a] (T_path h_a)(x),
// path 0 = identity, the 8 one-hop transports through the fat links and the 8 three-hop
// transports through the Naik links.  The transports use the packed (gathered) links of the
// Dslash, whose backward slots hold -U^dag, so the backward paths take the weight with a minus
// sign.  Channel fields are stored per parity as [Vh][3 colour][K][C] complex FP32.
#pragma once
#include "hisq_internal.cuh"
#include "link_codec.cuh"
#include "dslash_kernel.cuh"

namespace hisq {

constexpr int PC_PATHS = 17;
constexpr int PC_CH[4] = {1, 4, 4, 1};

// weight offset (complex numbers) of layer l in the packed weight vector
__host__ __device__ constexpr int pc_layer_offset(int l) {
    return l == 0 ? 0 : l == 1 ? PC_PATHS * 4 * 1 : PC_PATHS * 4 * 1 + PC_PATHS * 4 * 4;
}

// path taken by gathered link slot j (0..7 fat, 8..15 Naik) and the sign of its weight
__host__ __device__ constexpr int slot_path(int j) { return (j < 8 ? 1 : 9) + (j & 7); }
__host__ __device__ constexpr float slot_sign(int j) { return (j & 1) ? -1.0f : 1.0f; }
// adjoint path (T^{+k} <-> T^{-k})
__host__ __device__ constexpr int adjoint_path(int p) { return p == 0 ? 0 : (((p - 1) & 1) ? p - 1 : p + 1); }

struct PcLayerArgs {
    Geom g;
    LinkField fat, naik;
    const float2 *in_same;  // [Vh][3][K][A] at the output parity (identity path) or null
    const float2 *in_opp;   // [Vh][3][K][A] at the opposite parity (hop paths) or null
    float2 *out;            // [Vh][3][K][B]
    const float2 *W;        // layer weights (see pc_layer_kernel)
    int K, spb, parity;
};

// Weights in shared memory as ws[q][b][a] for q = 0 (identity) and q = 1 + slot (16 slots),
// with the backward-slot sign folded in.  ADJ: the adjoint of a layer with weights W[17][A][B]
// (mapping B -> A channels): ws[q][b][a] = conj(W[adj(q)][a][b]).
template <int A, int B, bool ADJ>
__device__ __forceinline__ void stage_weights(const float2 *W, float2 *ws) {
    for (int i = threadIdx.x; i < PC_PATHS * A * B; i += blockDim.x) {
        int q = i / (A * B), rem = i - q * A * B, b = rem / A, a = rem - b * A;
        int path = q == 0 ? 0 : slot_path(q - 1);
        float sign = q == 0 ? 1.0f : slot_sign(q - 1);
        float2 w;
        if (ADJ) {
            float2 o = W[(adjoint_path(path) * A + a) * B + b];
            w = make_float2(o.x, -o.y);
        } else {
            w = W[(path * B + b) * A + a];
        }
        ws[i] = make_float2(sign * w.x, sign * w.y);
    }
}

template <int C>
__device__ __forceinline__ void load_channels(const float2 *f, int s, int k, int K, Cplx<float> h[C][3]) {
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int a = 0; a < C; a++) {
            float2 v = __ldg(f + (((size_t)s * 3 + c) * K + k) * C + a);
            h[a][c] = {v.x, v.y};
        }
}

// y = M h for every channel
template <int C>
__device__ __forceinline__ void transport(const Cplx<float> M[3][3], const Cplx<float> h[C][3], Cplx<float> y[C][3]) {
#pragma unroll
    for (int a = 0; a < C; a++)
#pragma unroll
        for (int r = 0; r < 3; r++) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                re = fmaf(M[r][c].re, h[a][c].re, fmaf(-M[r][c].im, h[a][c].im, re));
                im = fmaf(M[r][c].re, h[a][c].im, fmaf(M[r][c].im, h[a][c].re, im));
            }
            y[a][r] = {re, im};
        }
}

template <int A, int B>
__device__ __forceinline__ void mix(const float2 *ws, const Cplx<float> y[A][3], Cplx<float> acc[B][3]) {
#pragma unroll
    for (int b = 0; b < B; b++)
#pragma unroll
        for (int a = 0; a < A; a++) {
            float2 w = ws[b * A + a];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                acc[b][c].re = fmaf(w.x, y[a][c].re, fmaf(-w.y, y[a][c].im, acc[b][c].re));
                acc[b][c].im = fmaf(w.x, y[a][c].im, fmaf(w.y, y[a][c].re, acc[b][c].im));
            }
        }
}

// Calls f(q, u) for q = 0 (u = h at the site) and q = 1 + slot (u = L_slot h(neighbour)).
template <int A, int NR, typename F>
__device__ __forceinline__ void for_each_path(const PcLayerArgs &p, int s, int k, F &&f) {
    using FatC = LinkCodec<HISQ_FP32, 18>;
    using NaikC = LinkCodec<HISQ_FP32, NR>;
    const Geom &g = p.g;
    if (p.in_same) {
        Cplx<float> h[A][3];
        load_channels<A>(p.in_same, s, k, p.K, h);
        f(0, h);
    }
    if (!p.in_opp) return;
    const SiteCoord sc = decode_site(g, s, p.parity);
#pragma unroll
    for (int grp = 0; grp < FatC::GROUPS; grp++) {
        uint32_t u[FatC::WG * 4];
        FatC::load_group(p.fat, p.parity, g.Vh, s, grp, u);
#pragma unroll
        for (int l = 0; l < FatC::G; l++) {
            const int slot = grp * FatC::G + l;
            const int nb = neighbour(g, sc, s, slot >> 1, (slot & 1) ? -1 : 1);
            Cplx<float> M[3][3];
            FatC::decode(u, l, M);
            Cplx<float> h[A][3], y[A][3];
            load_channels<A>(p.in_opp, nb, k, p.K, h);
            transport<A>(M, h, y);
            f(1 + slot, y);
        }
    }
#pragma unroll
    for (int grp = 0; grp < NaikC::GROUPS; grp++) {
        uint32_t u[NaikC::WG * 4];
        NaikC::load_group(p.naik, p.parity, g.Vh, s, grp, u);
#pragma unroll
        for (int l = 0; l < NaikC::G; l++) {
            const int slot = grp * NaikC::G + l;
            const int nb = neighbour(g, sc, s, slot >> 1, (slot & 1) ? -3 : 3);
            Cplx<float> M[3][3];
            NaikC::decode(u, l, M);
            Cplx<float> h[A][3], y[A][3];
            load_channels<A>(p.in_opp, nb, k, p.K, h);
            transport<A>(M, h, y);
            f(9 + slot, y);
        }
    }
}

// one thread per (site, sample); K threads share a site's links
template <int A, int B, bool ADJ, int NR>
__global__ void __launch_bounds__(256) pc_layer_kernel(PcLayerArgs p) {
    __shared__ float2 ws[PC_PATHS * A * B];
    stage_weights<A, B, ADJ>(p.W, ws);
    __syncthreads();
    const int k = threadIdx.x % p.K, sl = threadIdx.x / p.K;
    for (int tile = blockIdx.x; (long)tile * p.spb < p.g.Vh; tile += gridDim.x) {
        const int s = tile * p.spb + sl;
        if (s >= p.g.Vh || sl >= p.spb) continue;
        Cplx<float> acc[B][3];
#pragma unroll
        for (int b = 0; b < B; b++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[b][c] = {0.f, 0.f};
        for_each_path<A, NR>(p, s, k, [&](int q, const Cplx<float>(&y)[A][3]) { mix<A, B>(ws + q * A * B, y, acc); });
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int b = 0; b < B; b++) p.out[(((size_t)s * 3 + c) * p.K + k) * B + b] = make_float2(acc[b][c].re, acc[b][c].im);
    }
}

// Weight gradient of a layer A -> B channels at one output parity:
//   gW[path][b][a] += sum_x sum_colour G_b(x) conj((T_path h_a)(x))   (summed over samples)
// G: [Vh][3][K][B] at the output parity.  Result: 17*B*A complex numbers (doubles) in dot_out,
// in the weight layout [path][b][a].  Deterministic: warp shuffles, fixed-order block and grid
// sums (last-block-done), FP64 above the warp.
struct PcGradArgs {
    PcLayerArgs L;       // in_same, in_opp: the layer input h; out unused
    const float2 *G;     // gradient w.r.t. the layer output at the output parity
    RedArgs red;
};

template <int A, int B, int NR>
__global__ void __launch_bounds__(256) pc_grad_kernel(PcGradArgs ga) {
    constexpr int ND = PC_PATHS * A * B * 2;  // doubles per partial
    extern __shared__ double red[];
    const PcLayerArgs &p = ga.L;
    const int k = threadIdx.x % p.K, sl = threadIdx.x / p.K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    // per-thread accumulators for all paths would not fit in registers: accumulate each path's
    // products across the thread's sites first (loop over sites inside the path loop is not
    // possible since paths are produced per site), so reduce per site visit into shared memory.
    for (int i = threadIdx.x; i < nwarps * ND; i += blockDim.x) red[i] = 0.0;
    __syncthreads();
    for (int tile = blockIdx.x; (long)tile * p.spb < p.g.Vh; tile += gridDim.x) {
        const int s = tile * p.spb + sl;
        const bool valid = s < p.g.Vh && sl < p.spb;
        Cplx<float> G[B][3];
        if (valid) {
            load_channels<B>(ga.G, s, k, p.K, G);
        } else {
#pragma unroll
            for (int b = 0; b < B; b++)
#pragma unroll
                for (int c = 0; c < 3; c++) G[b][c] = {0.f, 0.f};
        }
        auto body = [&](int q, const Cplx<float>(&y)[A][3]) {
            const int path = q == 0 ? 0 : slot_path(q - 1);
            const float sign = q == 0 ? 1.0f : slot_sign(q - 1);
#pragma unroll
            for (int b = 0; b < B; b++)
#pragma unroll
                for (int a = 0; a < A; a++) {
                    float re = 0.f, im = 0.f;
#pragma unroll
                    for (int c = 0; c < 3; c++) {  // G conj(y)
                        re += G[b][c].re * y[a][c].re + G[b][c].im * y[a][c].im;
                        im += G[b][c].im * y[a][c].re - G[b][c].re * y[a][c].im;
                    }
                    re *= sign;
                    im *= sign;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        re += __shfl_xor_sync(0xffffffffu, re, off);
                        im += __shfl_xor_sync(0xffffffffu, im, off);
                    }
                    if (lane == 0) {
                        double *d = red + warp * ND + ((path * B + b) * A + a) * 2;
                        d[0] += (double)re;
                        d[1] += (double)im;
                    }
                }
        };
        // every lane of a warp must reach the shuffles: invalid lanes contribute zeros
        if (valid) {
            for_each_path<A, NR>(p, s, k, body);
        } else {
            // mirror the path sequence of valid lanes with zero products
            Cplx<float> z[A][3];
#pragma unroll
            for (int a = 0; a < A; a++)
#pragma unroll
                for (int c = 0; c < 3; c++) z[a][c] = {0.f, 0.f};
            if (p.in_same) body(0, z);
            if (p.in_opp)
                for (int q = 1; q <= 16; q++) body(q, z);
        }
    }
    block_reduce_finish(red, nwarps, ND, 0, ga.red);
}

}  // namespace hisq
