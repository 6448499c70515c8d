// Context, errors, link packing, vector packing and the operator entry points
// hisq_dslash and hisq_aop.
#include <stdarg.h>
#include <string.h>
#include <math.h>
#include <algorithm>

#include "hisq_internal.cuh"
#include "dslash_launch.cuh"

namespace hisq {

static thread_local hisq_ctx *g_ctx = nullptr;
static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

hisq_ctx *current() { return g_ctx; }

int require_ctx(hisq_ctx **ctx) {
    if (!g_ctx) return set_error(HISQ_ERR_STATE, "no HISQ context on this thread (call hisq_init)");
    if (cudaSetDevice(g_ctx->device) != cudaSuccess)
        return set_error(HISQ_ERR_CUDA, "cudaSetDevice(%d) failed", g_ctx->device);
    *ctx = g_ctx;
    return HISQ_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int ensure_scratch(hisq_ctx *ctx, size_t partial_doubles, size_t tmp_bytes) {
    if (partial_doubles > ctx->partials_cap) {
        if (ctx->partials) cudaFree(ctx->partials);
        ctx->partials = nullptr;
        if (cudaMalloc(&ctx->partials, partial_doubles * sizeof(double)) != cudaSuccess) {
            ctx->partials_cap = 0;
            return set_error(HISQ_ERR_NOMEM, "cannot allocate %zu reduction partials", partial_doubles);
        }
        ctx->partials_cap = partial_doubles;
    }
    if (tmp_bytes > ctx->tmp_cap) {
        if (ctx->tmp) cudaFree(ctx->tmp);
        ctx->tmp = nullptr;
        if (cudaMalloc(&ctx->tmp, tmp_bytes) != cudaSuccess) {
            ctx->tmp_cap = 0;
            return set_error(HISQ_ERR_NOMEM, "cannot allocate %zu bytes of operator workspace", tmp_bytes);
        }
        ctx->tmp_cap = tmp_bytes;
    }
    return HISQ_OK;
}

// ------------------------------------------------------------------------------------------
// Link packing: canonical FP64 [4][V][3][3][2] -> per-parity gathered records.
// ------------------------------------------------------------------------------------------
struct C64 { double re, im; };

__device__ inline int lex_of_eo(const Geom &g, int s, int parity, int c[4]) {
    SiteCoord sc = decode_site(g, s, parity);
    for (int mu = 0; mu < 4; mu++) c[mu] = sc.c[mu];
    return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

__device__ inline int lex_shift(const Geom &g, const int c[4], int mu, int step) {
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] = ((d[mu] + step) % g.L[mu] + g.L[mu]) % g.L[mu];
    return d[0] + g.L[0] * (d[1] + g.L[1] * (d[2] + g.L[2] * d[3]));
}

// gathered link `slot` of the output site at lattice coordinates c (lexicographic index x):
// slot 2mu = U_{x,mu}; 2mu+1 = -U^dag_{x-hop mu,mu}
__device__ inline void gathered_link(const Geom &g, const double *U, const int c[4], int x, int slot, int hop,
                                     C64 M[3][3]) {
    int mu = slot >> 1;
    long V = 2L * g.Vh;
    if ((slot & 1) == 0) {
        const double *p = U + ((size_t)mu * V + x) * 18;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) M[a][b] = {p[6 * a + 2 * b], p[6 * a + 2 * b + 1]};
    } else {
        int y = lex_shift(g, c, mu, -hop);
        const double *p = U + ((size_t)mu * V + y) * 18;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) M[a][b] = {-p[6 * b + 2 * a], p[6 * b + 2 * a + 1]};
    }
}

template <int P>
__host__ __device__ constexpr int stored_real_bytes() {
    if constexpr (P == HISQ_DS) return 8;  // the (hi, lo) float pair
    else return Prec<P>::bytes;
}

template <int P>
__device__ inline void put_real(uint4 *words, int Vh, int W, int parity, int s, int e, double val) {
    constexpr int EB = stored_real_bytes<P>();
    int off = e * EB;
    int j = off / 16, b = off % 16;
    char *base = reinterpret_cast<char *>(words + ((size_t)parity * W + j) * Vh + s) + b;
    if constexpr (P == HISQ_FP64) *reinterpret_cast<double *>(base) = val;
    else if constexpr (P == HISQ_DS) {
        const float hi = __double2float_rn(val);
        reinterpret_cast<float *>(base)[0] = hi;
        reinterpret_cast<float *>(base)[1] = __double2float_rn(val - (double)hi);
    }
    else if constexpr (P == HISQ_FP32) *reinterpret_cast<float *>(base) = (float)val;
    else if constexpr (P == HISQ_FP16) *reinterpret_cast<__half *>(base) = __double2half(val);
    else *reinterpret_cast<__nv_bfloat16 *>(base) = __double2bfloat16(val);
}

// Records of the output sites of the storage lattice gs (the lattice itself, or one slab of it
// with ghost planes): storage site (x, y, z, ts) is the lattice site (x, y, z, (ts + t_off) mod Lt)
// and only planes ts in [t_lo, t_hi) are packed; t_off is even, so both agree on parity.
template <int P, int RECON>
__global__ void pack_links_kernel(Geom g, Geom gs, int t_off, int t_lo, int t_hi, const double *U, int hop,
                                  uint4 *words, float *scale, int W) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= 2L * gs.Vh) return;
    int parity = (int)(i / gs.Vh), s = (int)(i % gs.Vh);
    int c[4];
    lex_of_eo(gs, s, parity, c);
    if (c[3] < t_lo || c[3] >= t_hi) return;
    c[3] = (c[3] + t_off) % g.L[3];
    const int x = c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
    C64 M[8][3][3];
    for (int k = 0; k < 8; k++) gathered_link(g, U, c, x, k, hop, M[k]);
    double sc = 1.0;
    if (RECON == 18 && scale) {
        double m = 0.0;
        for (int k = 0; k < 8; k++)
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) m = fmax(m, fmax(fabs(M[k][a][b].re), fabs(M[k][a][b].im)));
        sc = m > 0.0 ? m : 1.0;
        scale[(size_t)parity * gs.Vh + s] = (float)sc;
    }
    for (int k = 0; k < 8; k++) {
        int o = k * RECON;
        if (RECON == 18) {
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    put_real<P>(words, gs.Vh, W, parity, s, o + 6 * a + 2 * b, M[k][a][b].re / sc);
                    put_real<P>(words, gs.Vh, W, parity, s, o + 6 * a + 2 * b + 1, M[k][a][b].im / sc);
                }
            continue;
        }
        // link = c W with W in SU(3): c = cube root of the (real) determinant
        C64(&A)[3][3] = M[k];
        auto mul = [](C64 x, C64 y) { return C64{x.re * y.re - x.im * y.im, x.re * y.im + x.im * y.re}; };
        auto sub = [](C64 x, C64 y) { return C64{x.re - y.re, x.im - y.im}; };
        C64 det = {0, 0};
        for (int b = 0; b < 3; b++) {
            C64 cof = sub(mul(A[1][(b + 1) % 3], A[2][(b + 2) % 3]), mul(A[1][(b + 2) % 3], A[2][(b + 1) % 3]));
            C64 t = mul(A[0][b], cof);
            det.re += t.re; det.im += t.im;
        }
        double c = cbrt(det.re);
        double ic = c != 0.0 ? 1.0 / c : 0.0;
        C64 Wm[3][3];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) Wm[a][b] = {A[a][b].re * ic, A[a][b].im * ic};
        if (RECON == 13) {
            for (int b = 0; b < 3; b++) {
                put_real<P>(words, gs.Vh, W, parity, s, o + 2 * b, Wm[0][b].re);
                put_real<P>(words, gs.Vh, W, parity, s, o + 2 * b + 1, Wm[0][b].im);
                put_real<P>(words, gs.Vh, W, parity, s, o + 6 + 2 * b, Wm[1][b].re);
                put_real<P>(words, gs.Vh, W, parity, s, o + 7 + 2 * b, Wm[1][b].im);
            }
            put_real<P>(words, gs.Vh, W, parity, s, o + 12, 24.0 * c);
        } else {
            put_real<P>(words, gs.Vh, W, parity, s, o + 0, atan2(Wm[0][0].im, Wm[0][0].re));
            put_real<P>(words, gs.Vh, W, parity, s, o + 1, atan2(Wm[2][0].im, Wm[2][0].re));
            put_real<P>(words, gs.Vh, W, parity, s, o + 2, Wm[0][1].re);
            put_real<P>(words, gs.Vh, W, parity, s, o + 3, Wm[0][1].im);
            put_real<P>(words, gs.Vh, W, parity, s, o + 4, Wm[0][2].re);
            put_real<P>(words, gs.Vh, W, parity, s, o + 5, Wm[0][2].im);
            put_real<P>(words, gs.Vh, W, parity, s, o + 6, Wm[1][0].re);
            put_real<P>(words, gs.Vh, W, parity, s, o + 7, Wm[1][0].im);
            put_real<P>(words, gs.Vh, W, parity, s, o + 8, 24.0 * c);
        }
    }
}

// decode every record back to FP64 gathered links: out [2][Vh][8][3][3][2]
template <int P, int RECON>
__global__ void export_links_kernel(Geom g, LinkField f, double *out) {
    using Codec = LinkCodec<P, RECON>;
    using real = typename Prec<P>::real;
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= 2L * g.Vh) return;
    int parity = (int)(i / g.Vh), s = (int)(i % g.Vh);
    real sc = (real)1;
    if (RECON == 18 && f.scale) sc = (real)f.scale[(size_t)parity * g.Vh + s];
    for (int grp = 0; grp < Codec::GROUPS; grp++) {
        uint32_t u[Codec::WG * 4];
        Codec::load_group(f, parity, g.Vh, s, grp, u);
        for (int l = 0; l < Codec::G; l++) {
            Cplx<real> M[3][3];
            Codec::decode(u, l, sc, M);
            int slot = grp * Codec::G + l;
            double *o = out + ((size_t)i * 8 + slot) * 18;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    o[6 * a + 2 * b] = (double)M[a][b].re;
                    o[6 * a + 2 * b + 1] = (double)M[a][b].im;
                }
        }
    }
}

template <int P>
static void launch_pack(int recon, const Geom &g, const Geom &gs, int t_off, int t_lo, int t_hi, const double *U,
                        int hop, uint4 *words, float *scale, int W, cudaStream_t st) {
    int threads = 128;
    int blocks = (int)((2L * gs.Vh + threads - 1) / threads);
    if (recon == 13)
        pack_links_kernel<P, 13><<<blocks, threads, 0, st>>>(g, gs, t_off, t_lo, t_hi, U, hop, words, scale, W);
    else if (recon == 9)
        pack_links_kernel<P, 9><<<blocks, threads, 0, st>>>(g, gs, t_off, t_lo, t_hi, U, hop, words, scale, W);
    else
        pack_links_kernel<P, 18><<<blocks, threads, 0, st>>>(g, gs, t_off, t_lo, t_hi, U, hop, words, scale, W);
}

template <int P>
static void launch_export(int recon, const Geom &g, LinkField f, double *out, cudaStream_t st) {
    int threads = 128;
    int blocks = (int)((2L * g.Vh + threads - 1) / threads);
    if (recon == 13) export_links_kernel<P, 13><<<blocks, threads, 0, st>>>(g, f, out);
    else if (recon == 9) export_links_kernel<P, 9><<<blocks, threads, 0, st>>>(g, f, out);
    else export_links_kernel<P, 18><<<blocks, threads, 0, st>>>(g, f, out);
}

void pack_links_into(int prec, int recon, const Geom &g, const Geom &gs, int t_off, int t_lo, int t_hi,
                     const double *U, int hop, uint4 *words, float *scale, int W, cudaStream_t st) {
    switch (prec) {
    case HISQ_DS: launch_pack<HISQ_DS>(18, g, gs, t_off, t_lo, t_hi, U, hop, words, scale, W, st); break;
    case HISQ_FP64: launch_pack<HISQ_FP64>(recon, g, gs, t_off, t_lo, t_hi, U, hop, words, scale, W, st); break;
    case HISQ_FP32: launch_pack<HISQ_FP32>(recon, g, gs, t_off, t_lo, t_hi, U, hop, words, scale, W, st); break;
    case HISQ_FP16: launch_pack<HISQ_FP16>(recon, g, gs, t_off, t_lo, t_hi, U, hop, words, scale, W, st); break;
    default: launch_pack<HISQ_BF16>(recon, g, gs, t_off, t_lo, t_hi, U, hop, words, scale, W, st); break;
    }
}

static void dispatch_pack(int prec, int recon, const Geom &g, const double *U, int hop, uint4 *words, float *scale,
                          int W, cudaStream_t st) {
    pack_links_into(prec, recon, g, g, 0, 0, g.L[3], U, hop, words, scale, W, st);
}

// ------------------------------------------------------------------------------------------
// Vector packing: canonical [n][Vh][3][2] doubles <-> internal bundle.
// ------------------------------------------------------------------------------------------
template <int P>
__global__ void pack_vec_kernel(int Vh, int n, const double *canon, void *internal) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)Vh * n) return;
    int s = (int)(i / n), r = (int)(i % n);
    const double *c = canon + ((size_t)r * Vh + s) * 6;
    Cplx<typename Prec<P>::real> w[3];
    for (int k = 0; k < 3; k++) w[k] = {(typename Prec<P>::real)c[2 * k], (typename Prec<P>::real)c[2 * k + 1]};
    VecView<P> v;
    v.data = internal;
    v.n = n;
    store_vec<P>(v, s, r, w);
}

template <int P>
__global__ void unpack_vec_kernel(int Vh, int n, const void *internal, double *canon) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)Vh * n) return;
    int s = (int)(i / n), r = (int)(i % n);
    VecView<P> v;
    v.data = const_cast<void *>(internal);
    v.n = n;
    Cplx<typename Prec<P>::real> w[3];
    load_vec<P>(v, s, r, w);
    double *c = canon + ((size_t)r * Vh + s) * 6;
    for (int k = 0; k < 3; k++) { c[2 * k] = (double)w[k].re; c[2 * k + 1] = (double)w[k].im; }
}

int pack_vectors(hisq_ctx *ctx, const double *canon_dev, void *internal, int n, int prec, cudaStream_t st) {
    int Vh = ctx->geom.Vh;
    int threads = 256;
    int blocks = (int)(((long)Vh * n + threads - 1) / threads);
    switch (prec) {
    case HISQ_FP64: pack_vec_kernel<HISQ_FP64><<<blocks, threads, 0, st>>>(Vh, n, canon_dev, internal); break;
    case HISQ_FP32: pack_vec_kernel<HISQ_FP32><<<blocks, threads, 0, st>>>(Vh, n, canon_dev, internal); break;
    case HISQ_FP16: pack_vec_kernel<HISQ_FP16><<<blocks, threads, 0, st>>>(Vh, n, canon_dev, internal); break;
    case HISQ_BF16: pack_vec_kernel<HISQ_BF16><<<blocks, threads, 0, st>>>(Vh, n, canon_dev, internal); break;
    default: return set_error(HISQ_ERR_ARG, "unknown precision %d", prec);
    }
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

int unpack_vectors(hisq_ctx *ctx, const void *internal, double *canon_dev, int n, int prec, cudaStream_t st) {
    int Vh = ctx->geom.Vh;
    int threads = 256;
    int blocks = (int)(((long)Vh * n + threads - 1) / threads);
    switch (prec) {
    case HISQ_FP64: unpack_vec_kernel<HISQ_FP64><<<blocks, threads, 0, st>>>(Vh, n, internal, canon_dev); break;
    case HISQ_FP32: unpack_vec_kernel<HISQ_FP32><<<blocks, threads, 0, st>>>(Vh, n, internal, canon_dev); break;
    case HISQ_FP16: unpack_vec_kernel<HISQ_FP16><<<blocks, threads, 0, st>>>(Vh, n, internal, canon_dev); break;
    case HISQ_BF16: unpack_vec_kernel<HISQ_BF16><<<blocks, threads, 0, st>>>(Vh, n, internal, canon_dev); break;
    default: return set_error(HISQ_ERR_ARG, "unknown precision %d", prec);
    }
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

// ------------------------------------------------------------------------------------------
// Dslash launch: shape selection and dispatch to the per-precision instantiations.
// ------------------------------------------------------------------------------------------
LaunchShape default_shape(int prec, int n) {
    // right-hand sides per thread: largest of 4, 2, 1 dividing n (8 for FP64 is too many registers)
    int R = 1;
    int maxR = prec == HISQ_FP64 ? 2 : prec == HISQ_DS ? 1 : 4;
    for (int c = maxR; c >= 1; c /= 2)
        if (n % c == 0) { R = c; break; }
    return {R, 256, 1};
}


int launch_dslash(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik, int copy, const DslashArgs &d,
                  const LaunchShape *shape, cudaStream_t stream, int *grid_out) {
    if (copy == LINKS_DS && !fat->residual_ds()) copy = LINKS_FP64;  // FP64 handles have no ds copy
    if (copy == LINKS_DS && (!fat->words_ds || !naik->words_ds))
        return set_error(HISQ_ERR_STATE, "links without their double-single copy");
    const bool ds = copy == LINKS_DS;
    int prec = copy_prec(fat, copy);
    int recon = copy != LINKS_INNER ? 18 : naik->recon;
    if (ds && d.epi == EPI_AOP) return set_error(HISQ_ERR_ARG, "double-single Dslash has no A-operator epilogue");
    if ((d.geom || d.fields) && (!d.geom || !d.fields || !shape))
        return set_error(HISQ_ERR_ARG, "a Dslash on another lattice needs its geometry, links and launch shape");
    const Geom &G = d.geom ? *d.geom : ctx->geom;
    LaunchShape sh = shape ? *shape : tuned_shape(ctx, fat, naik, d.n, copy);
    int R = sh.R;
    if (R != 1 && R != 2 && R != 4 && R != 8) R = 1;
    if (d.n % R != 0) R = 1;
    if (prec == HISQ_FP64 && R > 4) R = 4;  // FP64 kernels are built for up to four RHS per thread
    if (ds && R > 2) R = 2;                 // double-single kernels for up to two
    // lane splits exist for 18-real Naik records: two lanes up to four RHS per thread, four up to two
    int S = 1;
    if (!ds && recon == 18 && sh.S == 2 && R <= 4) S = 2;
    if (!ds && recon == 18 && sh.S == 4 && R <= 2) S = 4;
    const bool ranged = d.site_end > 0;  // the staged kernel covers whole parities only
    if (!ds && !ranged && recon == 18 && sh.S == 8 && R <= 2 && prec != HISQ_FP64 && d.epi != EPI_RESID) S = 8;
    if (!ds && ranged && recon == 18 && sh.S == 8 && R <= 2) S = 4;
    int t = (d.n + R - 1) / R;
    // reducing epilogues finish in one block that sums a partial per block: blocks of at least 128
    // threads keep both the partial count and that block's share of the sum small
    int spb, threads;
    if (S == 8) {
        // staged: threads = 4 t TS exactly (TS sites per tile), up to 512
        spb = std::max(1, std::min(sh.threads, 512) / (4 * t));
        threads = 4 * t * spb;
        if (threads % 32) return set_error(HISQ_ERR_ARG, "staged launch shape of %d threads is not whole warps", threads);
    } else {
        dslash_block_shape(d.n, R, S, sh.threads, d.epi != EPI_PLAIN, &spb, &threads);
        if (threads > 256) return set_error(HISQ_ERR_ARG, "launch shape of %d threads is too large", threads);
    }

    KArgs a;
    memset(&a, 0, sizeof(a));
    a.g = G;
    a.fat = ds ? fat->field_ds() : copy == LINKS_FP64 ? fat->field64() : fat->field();
    a.naik = ds ? naik->field_ds() : copy == LINKS_FP64 ? naik->field64() : naik->field();
    if (d.fields) {
        a.fat = d.fields[0];
        a.naik = d.fields[1];
    }
    a.in = d.in;
    a.out = d.out;
    a.n = d.n;
    a.t = t;
    a.spb = spb;
    a.parity = d.parity;
    a.mass2 = d.mass2;
    a.mass2v = d.mass2v;
    a.axpy = d.axpy_in;
    a.b = d.b;
    a.b_one = d.b_one;
    a.out_lo = d.out_lo;
    a.lo_prec = d.lo_prec;
    a.active = d.active;
    a.gate = d.gate;
    a.red.partials = d.partials;
    a.red.counter = d.counter;
    a.red.dot_out = d.dot_out;
    a.red.hook = d.hook;
    a.red.st = reinterpret_cast<SolverState *>(d.hook_state);
    a.red.partials_only = d.partials_only;
    a.err = ctx->dev_err;
    a.s0 = 0;
    a.s1 = G.Vh;
    if (ranged) {
        if (d.site_begin < 0 || d.site_end > G.Vh || d.site_begin >= d.site_end)
            return set_error(HISQ_ERR_ARG, "output site range [%d, %d) outside the parity", d.site_begin, d.site_end);
        a.s0 = d.site_begin;
        a.s1 = d.site_end;
    }

    size_t smem = 0;
    if (S == 8) {
        smem = staged_smem(a.fat.W + a.naik.W, spb, threads, d.n, d.epi != EPI_PLAIN);
        if (smem > 227 * 1024)
            return set_error(HISQ_ERR_ARG, "staged launch shape needs %zu bytes of shared memory", smem);
        if (d.epi != EPI_PLAIN && (!d.partials || !d.counter || (size_t)ctx->num_sms * 8 * d.n > d.partials_cap))
            return set_error(HISQ_ERR_ARG, "reduction scratch too small for the Dslash epilogue");
    } else if (d.epi != EPI_PLAIN) {
        size_t need = std::max((size_t)spb * d.n, (size_t)threads + 64);
        smem = need * sizeof(double);
        // the grid never exceeds one resident wave per SM times 64, nor the tile count
        if (!d.partials || !d.counter || dslash_partials_needed(a.s1 - a.s0, ctx->num_sms, spb, d.n) > d.partials_cap)
            return set_error(HISQ_ERR_ARG, "reduction scratch too small for the Dslash epilogue");
    }
    int grid = 0;
    cudaError_t e;
    switch (prec) {
    case HISQ_DS: e = launch_dslash_ds(a, d.epi, R, threads, smem, ctx->num_sms, stream, &grid); break;
    case HISQ_FP64: e = launch_dslash_prec<HISQ_FP64>(a, recon, d.epi, R, S, threads, smem, ctx->num_sms, stream, &grid); break;
    case HISQ_FP32: e = launch_dslash_prec<HISQ_FP32>(a, recon, d.epi, R, S, threads, smem, ctx->num_sms, stream, &grid); break;
    case HISQ_FP16: e = launch_dslash_prec<HISQ_FP16>(a, recon, d.epi, R, S, threads, smem, ctx->num_sms, stream, &grid); break;
    default: e = launch_dslash_prec<HISQ_BF16>(a, recon, d.epi, R, S, threads, smem, ctx->num_sms, stream, &grid); break;
    }
    if (e != cudaSuccess) return set_error(HISQ_ERR_CUDA, "Dslash launch failed: %s", cudaGetErrorString(e));
    if (grid_out) *grid_out = grid;
    return HISQ_OK;
}

static bool valid_prec(int p) { return p >= HISQ_FP64 && p <= HISQ_BF16; }

int check_pair(hisq_ctx *ctx, const hisq_links *fat, const hisq_links *naik) {
    if (!fat || !naik) return set_error(HISQ_ERR_ARG, "null links handle");
    if (fat->ctx != ctx || naik->ctx != ctx)
        return set_error(HISQ_ERR_STATE, "links handles belong to another context");
    if (fat->is_naik || !naik->is_naik) return set_error(HISQ_ERR_ARG, "expected (fat, naik) links handles");
    if (fat->prec != naik->prec) return set_error(HISQ_ERR_ARG, "fat and Naik links have different precisions");
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

const char *hisq_strerror(int status) {
    switch (status) {
    case HISQ_OK: return "success";
    case HISQ_ERR_ARG: return "invalid argument";
    case HISQ_ERR_CUDA: return "CUDA runtime error";
    case HISQ_ERR_NOMEM: return "out of memory";
    case HISQ_ERR_NOT_CONVERGED: return "solver did not converge within max_iter";
    case HISQ_ERR_BREAKDOWN: return "solver breakdown (non-finite value or non-positive <p,Ap>)";
    case HISQ_ERR_TIMEOUT: return "bounded device-side wait ran out";
    case HISQ_ERR_STATE: return "no context on this thread or handle of another context";
    default: return "unknown status";
    }
}

const char *hisq_last_error(void) { return g_err; }

void hisq_default_solver_params(hisq_solver_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->inner_prec = HISQ_FP32;
    p->delta = 0.0;  // by inner precision (default_delta)
    p->max_iter = 20000;
    p->bundle = 0;
    p->use_graph = 2;
    p->check_every = 1;
    p->pc = nullptr;
    p->stall_window = 50;
    p->stall_factor = 10.0;
    p->autotune = 1;
    p->time_kernels = 0;
    p->single_reduction = 1;
    p->l2_persist_links = 1;
}

int hisq_init(const int dims[4], int device, void *cuda_stream) {
    if (g_ctx) return set_error(HISQ_ERR_STATE, "this thread already has a HISQ context");
    if (!dims) return set_error(HISQ_ERR_ARG, "null dims");
    long V = 1;
    for (int mu = 0; mu < 4; mu++) {
        if (dims[mu] < 4 || dims[mu] % 2)
            return set_error(HISQ_ERR_ARG, "lattice extent %d in direction %d must be even and >= 4", dims[mu], mu);
        V *= dims[mu];
    }
    if (V / 2 > (1L << 30)) return set_error(HISQ_ERR_ARG, "lattice too large");
    int ndev = 0;
    HISQ_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return set_error(HISQ_ERR_ARG, "device %d out of range (%d devices)", device, ndev);
    HISQ_CUDA(cudaSetDevice(device));
    hisq_ctx *ctx = new (std::nothrow) hisq_ctx();
    if (!ctx) return set_error(HISQ_ERR_NOMEM, "context allocation failed");
    Geom &g = ctx->geom;
    for (int mu = 0; mu < 4; mu++) g.L[mu] = dims[mu];
    g.half = dims[0] / 2;
    g.Vh = (int)(V / 2);
    g.stride[0] = 1;
    g.stride[1] = g.half;
    g.stride[2] = g.half * dims[1];
    g.stride[3] = g.half * dims[1] * dims[2];
    g.plane_order = dims[3] < dims[2] ? 1 : 0;
    ctx->device = device;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return set_error(HISQ_ERR_CUDA, "cudaGetDeviceProperties failed");
    }
    ctx->num_sms = prop.multiProcessorCount;
    hisq_default_solver_params(&ctx->params);
    if (cudaMalloc(&ctx->counter, sizeof(unsigned int) * 4) != cudaSuccess ||
        cudaMalloc(&ctx->dot_out, sizeof(double) * HISQ_MAX_NRHS * 4) != cudaSuccess ||
        cudaMalloc(&ctx->dev_err, sizeof(int) * 4) != cudaSuccess) {
        if (ctx->counter) cudaFree(ctx->counter);
        if (ctx->dot_out) cudaFree(ctx->dot_out);
        delete ctx;
        return set_error(HISQ_ERR_NOMEM, "context scratch allocation failed");
    }
    cudaMemset(ctx->counter, 0, sizeof(unsigned int) * 4);
    cudaMemset(ctx->dev_err, 0, sizeof(int) * 4);
    g_ctx = ctx;
    return HISQ_OK;
}

int hisq_device_status(void) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    int flag = 0;
    HISQ_CUDA(cudaMemcpy(&flag, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        HISQ_CUDA(cudaMemset(ctx->dev_err, 0, sizeof(int)));
        return set_error(HISQ_ERR_TIMEOUT, "a bounded device wait (staged Dslash tile) ran out; its output is invalid");
    }
    return HISQ_OK;
}

int hisq_links_destroy(hisq_links *h) {
    if (!h) return HISQ_OK;
    if (h->words) cudaFree(h->words);
    if (h->scale) cudaFree(h->scale);
    if (h->words64) cudaFree(h->words64);
    if (h->words_ds) cudaFree(h->words_ds);
    hisq_ctx *ctx = h->ctx;
    if (ctx) {
        ctx->links.erase(std::remove(ctx->links.begin(), ctx->links.end(), h), ctx->links.end());
        // captured graphs hold the links' device pointers: a later handle may reuse this address
        ctx->tune_generation++;
    }
    delete h;
    return HISQ_OK;
}

int hisq_finalize(void) {
    hisq_ctx *ctx = g_ctx;
    if (!ctx) return set_error(HISQ_ERR_STATE, "no HISQ context on this thread");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    while (!ctx->links.empty()) hisq_links_destroy(ctx->links.back());
    while (!ctx->pcs.empty()) {
        hisq_pc *pc = ctx->pcs.back();
        ctx->pcs.pop_back();
        free_pc(pc);
    }
    free_workspace(ctx);
    free_multishift(ctx);
    if (ctx->l2_limit_saved) {  // give the context its L2 set-aside back as it was
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, ctx->l2_limit_old);
        cudaGetLastError();
    }
    if (ctx->partials) cudaFree(ctx->partials);
    if (ctx->tmp) cudaFree(ctx->tmp);
    if (ctx->counter) cudaFree(ctx->counter);
    if (ctx->dot_out) cudaFree(ctx->dot_out);
    if (ctx->dev_err) cudaFree(ctx->dev_err);
    delete ctx;
    g_ctx = nullptr;
    return HISQ_OK;
}

int hisq_links_create(hisq_links **out, const double *canon, int is_naik, int prec, int recon) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!out || !canon) return set_error(HISQ_ERR_ARG, "null argument");
    if (!valid_prec(prec)) return set_error(HISQ_ERR_ARG, "unknown precision %d", prec);
    if (recon != 18 && recon != 13 && recon != 9) return set_error(HISQ_ERR_ARG, "recon must be 18, 13 or 9");
    if (!is_naik && recon != 18) return set_error(HISQ_ERR_ARG, "fat links cannot be reconstructed (recon must be 18)");
    if (prec == HISQ_FP64 && recon != 18) return set_error(HISQ_ERR_ARG, "FP64 links are stored in full (recon 18)");
    const Geom &g = ctx->geom;
    size_t canon_bytes = (size_t)4 * 2 * g.Vh * 18 * sizeof(double);
    const double *U = canon;
    double *staged = nullptr;
    cudaStream_t st = ctx->stream;
    if (!is_device_ptr(canon)) {
        HISQ_CUDA(cudaMalloc(&staged, canon_bytes));
        if (cudaMemcpyAsync(staged, canon, canon_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaFree(staged);
            return set_error(HISQ_ERR_CUDA, "link upload failed");
        }
        U = staged;
    }
    hisq_links *h = new hisq_links();
    h->ctx = ctx;
    h->is_naik = is_naik ? 1 : 0;
    h->prec = prec;
    h->recon = recon;
    h->W = link_words(prec, recon);
    int hop = is_naik ? 3 : 1;
    int rc = HISQ_OK;
    size_t wbytes = (size_t)2 * h->W * g.Vh * sizeof(uint4);
    if (cudaMalloc(&h->words, wbytes) != cudaSuccess) rc = set_error(HISQ_ERR_NOMEM, "cannot allocate %zu link bytes", wbytes);
    if (rc == HISQ_OK && prec >= HISQ_FP16 && recon == 18 &&
        cudaMalloc(&h->scale, (size_t)2 * g.Vh * sizeof(float)) != cudaSuccess)
        rc = set_error(HISQ_ERR_NOMEM, "cannot allocate link scales");
    if (rc == HISQ_OK) dispatch_pack(prec, recon, g, U, hop, h->words, h->scale, h->W, st);
    if (rc == HISQ_OK && prec != HISQ_FP64) {
        // the FP64 copy (plain FP64 solves with these links) and the double-single copy (the
        // residual recomputations of mixed-precision solves)
        int W64 = link_words(HISQ_FP64, 18);
        size_t b64 = (size_t)2 * W64 * g.Vh * sizeof(uint4);
        if (cudaMalloc(&h->words64, b64) != cudaSuccess) rc = set_error(HISQ_ERR_NOMEM, "cannot allocate FP64 link copy");
        else dispatch_pack(HISQ_FP64, 18, g, U, hop, h->words64, nullptr, W64, st);
        if (rc == HISQ_OK) {
            if (cudaMalloc(&h->words_ds, b64) != cudaSuccess)
                rc = set_error(HISQ_ERR_NOMEM, "cannot allocate double-single link copy");
            else dispatch_pack(HISQ_DS, 18, g, U, hop, h->words_ds, nullptr, W64, st);
        }
    }
    if (rc == HISQ_OK) {
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "link packing failed: %s", cudaGetErrorString(e));
    }
    if (staged) cudaFree(staged);
    if (rc != HISQ_OK) {
        h->ctx = nullptr;
        hisq_links_destroy(h);
        return rc;
    }
    ctx->links.push_back(h);
    *out = h;
    return HISQ_OK;
}

int hisq_links_export(const hisq_links *h, double *out) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!h || !out) return set_error(HISQ_ERR_ARG, "null argument");
    if (h->ctx != ctx) return set_error(HISQ_ERR_STATE, "handle of another context");
    const Geom &g = ctx->geom;
    size_t bytes = (size_t)2 * g.Vh * 8 * 18 * sizeof(double);
    double *d;
    HISQ_CUDA(cudaMalloc(&d, bytes));
    LinkField f = h->field();
    switch (h->prec) {
    case HISQ_FP64: launch_export<HISQ_FP64>(h->recon, g, f, d, ctx->stream); break;
    case HISQ_FP32: launch_export<HISQ_FP32>(h->recon, g, f, d, ctx->stream); break;
    case HISQ_FP16: launch_export<HISQ_FP16>(h->recon, g, f, d, ctx->stream); break;
    default: launch_export<HISQ_BF16>(h->recon, g, f, d, ctx->stream); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess) return set_error(HISQ_ERR_CUDA, "link export failed: %s", cudaGetErrorString(e));
    return HISQ_OK;
}

size_t hisq_vector_bytes(int prec, int nrhs) {
    hisq_ctx *ctx = g_ctx;
    if (!ctx || !valid_prec(prec) || nrhs < 1) return 0;
    return vector_bytes(prec, ctx->geom.Vh, nrhs);
}

static int canon_io(hisq_ctx *ctx, const void *canon, size_t bytes, bool upload, double **dev, bool *staged) {
    *staged = false;
    if (is_device_ptr(canon)) {
        *dev = const_cast<double *>(reinterpret_cast<const double *>(canon));
        return HISQ_OK;
    }
    HISQ_CUDA(cudaMalloc(dev, bytes));
    *staged = true;
    if (upload) HISQ_CUDA(cudaMemcpyAsync(*dev, canon, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return HISQ_OK;
}

int hisq_pack(const double *canon, void *internal, int nrhs, int prec) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!canon || !internal) return set_error(HISQ_ERR_ARG, "null argument");
    if (!valid_prec(prec) || nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "bad precision or nrhs");
    size_t bytes = (size_t)nrhs * ctx->geom.Vh * 6 * sizeof(double);
    double *dev;
    bool staged;
    HISQ_CHECK(canon_io(ctx, canon, bytes, true, &dev, &staged));
    int rc = pack_vectors(ctx, dev, internal, nrhs, prec, ctx->stream);
    if (staged) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(dev);
    }
    return rc;
}

int hisq_unpack(const void *internal, double *canon, int nrhs, int prec) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!canon || !internal) return set_error(HISQ_ERR_ARG, "null argument");
    if (!valid_prec(prec) || nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "bad precision or nrhs");
    size_t bytes = (size_t)nrhs * ctx->geom.Vh * 6 * sizeof(double);
    double *dev;
    bool staged;
    HISQ_CHECK(canon_io(ctx, canon, bytes, false, &dev, &staged));
    int rc = unpack_vectors(ctx, internal, dev, nrhs, prec, ctx->stream);
    if (staged) {
        if (rc == HISQ_OK && cudaMemcpyAsync(canon, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
            rc = set_error(HISQ_ERR_CUDA, "download failed");
        cudaStreamSynchronize(ctx->stream);
        cudaFree(dev);
    }
    return rc;
}

int hisq_dslash(const hisq_links *fat, const hisq_links *naik, const void *in, void *out, int nrhs, int parity) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    HISQ_CHECK(check_pair(ctx, fat, naik));
    if (!in || !out) return set_error(HISQ_ERR_ARG, "null vector");
    if (in == out) return set_error(HISQ_ERR_ARG, "in and out must not overlap");
    if (nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_NRHS);
    if (parity != 0 && parity != 1) return set_error(HISQ_ERR_ARG, "parity must be 0 or 1");
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.in = in;
    d.out = out;
    d.n = nrhs;
    d.parity = parity;
    d.epi = EPI_PLAIN;
    return launch_dslash(ctx, fat, naik, false, d, nullptr, ctx->stream);
}

int hisq_dslash_full(const hisq_links *fat, const hisq_links *naik, const void *in, void *out, int nrhs) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    HISQ_CHECK(check_pair(ctx, fat, naik));
    if (!in || !out) return set_error(HISQ_ERR_ARG, "null vector");
    if (nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_NRHS);
    const size_t half = vector_bytes(fat->prec, ctx->geom.Vh, nrhs);
    const char *ib = static_cast<const char *>(in);
    char *ob = static_cast<char *>(out);
    if (ob < ib + 2 * half && ib < ob + 2 * half) return set_error(HISQ_ERR_ARG, "in and out must not overlap");
    for (int parity = 0; parity < 2; parity++) {  // output parity; the input is the other half
        DslashArgs d;
        memset(&d, 0, sizeof(d));
        d.in = ib + (size_t)(1 - parity) * half;
        d.out = ob + (size_t)parity * half;
        d.n = nrhs;
        d.parity = parity;
        d.epi = EPI_PLAIN;
        HISQ_CHECK(launch_dslash(ctx, fat, naik, false, d, nullptr, ctx->stream));
    }
    return HISQ_OK;
}

int hisq_aop(const hisq_links *fat, const hisq_links *naik, double mass, const void *in, void *out, int nrhs,
             double *pAp) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    HISQ_CHECK(check_pair(ctx, fat, naik));
    if (!in || !out) return set_error(HISQ_ERR_ARG, "null vector");
    if (in == out) return set_error(HISQ_ERR_ARG, "in and out must not overlap");
    if (nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_NRHS);
    size_t tmp_bytes = vector_bytes(fat->prec, ctx->geom.Vh, nrhs);
    size_t max_grid = (size_t)ctx->num_sms * 64;
    HISQ_CHECK(ensure_scratch(ctx, max_grid * HISQ_MAX_NRHS, tmp_bytes));
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.in = in;
    d.out = ctx->tmp;
    d.n = nrhs;
    d.parity = 1;
    d.epi = EPI_PLAIN;
    HISQ_CHECK(launch_dslash(ctx, fat, naik, false, d, nullptr, ctx->stream));
    d.in = ctx->tmp;
    d.out = out;
    d.parity = 0;
    d.epi = EPI_AOP;
    d.mass2 = mass * mass;
    d.axpy_in = in;
    d.partials = ctx->partials;
    d.partials_cap = ctx->partials_cap;
    d.counter = ctx->counter;
    d.dot_out = ctx->dot_out;
    HISQ_CHECK(launch_dslash(ctx, fat, naik, false, d, nullptr, ctx->stream));
    if (pAp) {
        HISQ_CUDA(cudaMemcpyAsync(pAp, ctx->dot_out, sizeof(double) * nrhs, cudaMemcpyDefault, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return HISQ_OK;
}

}  // extern "C"
