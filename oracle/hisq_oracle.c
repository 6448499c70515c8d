/*
 * Plain FP64 CPU oracle for the even-odd HISQ Dslash, the even-parity operator
 * A = m^2 - D_eo D_oe, conjugate gradient, multi-shift conjugate gradient, and the
 * gauge-covariant preconditioner network.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct statement of what the
 * CUDA library computes.  It shares no code, header, table or helper with the CUDA path;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Layouts (all double precision, complex numbers stored as (re, im) pairs):
 *   links   X, N : [4 mu][V lex][3 row][3 col][2]
 *   full vectors : [nrhs][V lex][3][2]
 *   eo vectors   : [nrhs][V/2][3][2], site of even-odd index i on parity p is the lex site
 *                  of parity p with lex/2 == i.
 * Lexicographic index i = x + Lx*(y + Ly*(z + Lz*t)); direction mu = 0..3 is x, y, z, t;
 * every extent is even; all index arithmetic is periodic (boundary signs live in the links).
 *
 * Built twice: plain (one thread) and with -fopenmp, where the site loops of the Dslash are
 * shared among the host's cores (the CPU baseline on all cores); both give identical results.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cplx;

static cplx c_add(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static cplx c_sub(cplx a, cplx b) { cplx r = {a.re - b.re, a.im - b.im}; return r; }
static cplx c_mul(cplx a, cplx b) { cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static cplx c_conj(cplx a) { cplx r = {a.re, -a.im}; return r; }
static cplx c_scale(double s, cplx a) { cplx r = {s * a.re, s * a.im}; return r; }

static long volume(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords_of(const int L[4], long i, int c[4]) {
    for (int mu = 0; mu < 4; mu++) { c[mu] = (int)(i % L[mu]); i /= L[mu]; }
}

static long lex_of(const int L[4], const int c[4]) {
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

static int parity_of(const int L[4], long i) {
    int c[4]; coords_of(L, i, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* lex index of the site reached from i by `step` hops in direction mu (periodic) */
static long hop(const int L[4], long i, int mu, int step) {
    int c[4]; coords_of(L, i, c);
    c[mu] = ((c[mu] + step) % L[mu] + L[mu]) % L[mu];
    return lex_of(L, c);
}

/* element (a, b) of the link U_{x,mu} */
static cplx link(const double *U, long V, int mu, long x, int a, int b) {
    const double *p = U + ((((long)mu * V + x) * 3 + a) * 3 + b) * 2;
    cplx r = {p[0], p[1]};
    return r;
}

static cplx vec(const double *v, long x, int a) {
    cplx r = {v[(x * 3 + a) * 2], v[(x * 3 + a) * 2 + 1]};
    return r;
}

static void put(double *v, long x, int a, cplx z) {
    v[(x * 3 + a) * 2] = z.re;
    v[(x * 3 + a) * 2 + 1] = z.im;
}

/*
 * Eq. (3): w_x = sum_{mu=0..3} [ X_{x,mu} v_{x+mu} - X^dag_{x-mu,mu} v_{x-mu}
 *                               + N_{x,mu} v_{x+3mu} - N^dag_{x-3mu,mu} v_{x-3mu} ].
 * `vin(y)` returns the colour vector at lex site y.  Result written to w[3].
 */
typedef cplx (*site_reader)(const void *ctx, long y, int a);

static void dslash_site(const int L[4], const double *X, const double *N, long x,
                        site_reader vin, const void *ctx, cplx w[3]) {
    long V = volume(L);
    for (int a = 0; a < 3; a++) { w[a].re = 0.0; w[a].im = 0.0; }
    for (int mu = 0; mu < 4; mu++) {
        long xp1 = hop(L, x, mu, +1), xm1 = hop(L, x, mu, -1);
        long xp3 = hop(L, x, mu, +3), xm3 = hop(L, x, mu, -3);
        for (int a = 0; a < 3; a++) {
            for (int b = 0; b < 3; b++) {
                /* forward one-hop: X_{x,mu} v_{x+mu} */
                w[a] = c_add(w[a], c_mul(link(X, V, mu, x, a, b), vin(ctx, xp1, b)));
                /* backward one-hop: (X^dag)_{ab} = conj(X_{ba}) of the link at x-mu */
                w[a] = c_sub(w[a], c_mul(c_conj(link(X, V, mu, xm1, b, a)), vin(ctx, xm1, b)));
                /* forward three-hop: N_{x,mu} v_{x+3mu} */
                w[a] = c_add(w[a], c_mul(link(N, V, mu, x, a, b), vin(ctx, xp3, b)));
                /* backward three-hop: N^dag of the link at x-3mu */
                w[a] = c_sub(w[a], c_mul(c_conj(link(N, V, mu, xm3, b, a)), vin(ctx, xm3, b)));
            }
        }
    }
}

static cplx read_full(const void *ctx, long y, int a) { return vec((const double *)ctx, y, a); }

/* even-odd vectors hold only the sites of the opposite parity; index y/2 */
static cplx read_eo(const void *ctx, long y, int a) { return vec((const double *)ctx, y / 2, a); }

/* Eq. (3) on the whole lattice for nrhs vectors: in/out [nrhs][V][3][2]. */
void oracle_dslash_full(const int L[4], const double *X, const double *N,
                        const double *in, double *out, int nrhs) {
    long V = volume(L);
    for (int r = 0; r < nrhs; r++) {
        const double *v = in + (long)r * V * 6;
        double *w = out + (long)r * V * 6;
        /* every site is computed on its own: with -fopenmp the sites are shared among threads and
           the result is the same to the bit */
        #pragma omp parallel for schedule(static)
        for (long x = 0; x < V; x++) {
            cplx s[3];
            dslash_site(L, X, N, x, read_full, v, s);
            for (int a = 0; a < 3; a++) put(w, x, a, s[a]);
        }
    }
}

/*
 * Eq. (3) restricted to output parity p (Eq. (4) for nrhs vectors): the input lives on parity
 * 1-p and the output on parity p, both in even-odd indexing [nrhs][V/2][3][2].
 * out_parity = 0 gives D_eo (odd -> even), out_parity = 1 gives D_oe (even -> odd).
 */
void oracle_dslash_eo(const int L[4], const double *X, const double *N,
                      const double *in, double *out, int nrhs, int out_parity) {
    long V = volume(L), Vh = V / 2;
    for (int r = 0; r < nrhs; r++) {
        const double *v = in + (long)r * Vh * 6;
        double *w = out + (long)r * Vh * 6;
        #pragma omp parallel for schedule(static)
        for (long x = 0; x < V; x++) {
            if (parity_of(L, x) != out_parity) continue;
            cplx s[3];
            dslash_site(L, X, N, x, read_eo, v, s);
            for (int a = 0; a < 3; a++) put(w, x / 2, a, s[a]);
        }
    }
}

/* A v = m^2 v - D_eo (D_oe v) on the even sites, [nrhs][V/2][3][2]. */
void oracle_aop(const int L[4], const double *X, const double *N, double mass,
                const double *in, double *out, int nrhs) {
    long Vh = volume(L) / 2;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)Vh * 6);
    for (int r = 0; r < nrhs; r++) {
        const double *v = in + (long)r * Vh * 6;
        double *w = out + (long)r * Vh * 6;
        oracle_dslash_eo(L, X, N, v, tmp, 1, 1);  /* tmp = D_oe v on odd sites */
        oracle_dslash_eo(L, X, N, tmp, w, 1, 0);  /* w = D_eo tmp on even sites */
        for (long i = 0; i < Vh * 6; i++) w[i] = mass * mass * v[i] - w[i];
    }
    free(tmp);
}

/* <u, v> = sum conj(u) v over n complex numbers */
static cplx dot(const double *u, const double *v, long n) {
    cplx s = {0.0, 0.0};
    for (long i = 0; i < n; i++) {
        cplx a = {u[2 * i], u[2 * i + 1]}, b = {v[2 * i], v[2 * i + 1]};
        s = c_add(s, c_mul(c_conj(a), b));
    }
    return s;
}

static double norm2(const double *u, long n) { return dot(u, u, n).re; }

/*
 * Textbook (Hestenes-Stiefel) conjugate gradient on A = m^2 - D_eo D_oe from x0 = 0, one
 * right-hand side: b, x are [V/2][3][2].  Once the recursive residual satisfies the relative
 * tolerance, the true residual |b - A x| / |b| is recomputed every iteration and the solve
 * stops when it meets tol.  Returns the iteration count, or -1 when max_iter is reached.
 * *true_rel receives the final true relative residual.
 */
int oracle_cg(const int L[4], const double *X, const double *N, double mass,
              const double *b, double *x, double tol, int max_iter, double *true_rel) {
    long Vh = volume(L) / 2, n = Vh * 3;
    double *r = (double *)malloc(sizeof(double) * n * 2);
    double *p = (double *)malloc(sizeof(double) * n * 2);
    double *Ap = (double *)malloc(sizeof(double) * n * 2);
    double bnorm = sqrt(norm2(b, n));
    memset(x, 0, sizeof(double) * n * 2);
    memcpy(r, b, sizeof(double) * n * 2);
    memcpy(p, b, sizeof(double) * n * 2);
    double rr = norm2(r, n);
    int iters = -1;
    *true_rel = 1.0;
    if (bnorm == 0.0) { *true_rel = 0.0; iters = 0; goto done; }
    for (int k = 1; k <= max_iter; k++) {
        oracle_aop(L, X, N, mass, p, Ap, 1);
        double alpha = rr / dot(p, Ap, n).re;
        for (long i = 0; i < 2 * n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; }
        double rr_new = norm2(r, n);
        if (sqrt(rr_new) <= tol * bnorm) {
            oracle_aop(L, X, N, mass, x, Ap, 1);
            for (long i = 0; i < 2 * n; i++) Ap[i] = b[i] - Ap[i];
            *true_rel = sqrt(norm2(Ap, n)) / bnorm;
            if (*true_rel <= tol) { iters = k; goto done; }
        }
        double beta = rr_new / rr;
        for (long i = 0; i < 2 * n; i++) p[i] = r[i] + beta * p[i];
        rr = rr_new;
    }
done:
    free(r); free(p); free(Ap);
    return iters;
}

/* ------------------------------------------------------------------------------------------
 * Gauge-covariant parallel-transport network (a linear preconditioner for A).
 *
 * Paths (17): 0 identity; 1+2mu : T^{+1}_mu h_x = X_{x,mu} h_{x+mu};
 *             2+2mu : T^{-1}_mu h_x = X^dag_{x-mu,mu} h_{x-mu};
 *             9+2mu : T^{+3}_mu h_x = N_{x,mu} h_{x+3mu};
 *             10+2mu: T^{-3}_mu h_x = N^dag_{x-3mu,mu} h_{x-3mu}.
 * A layer maps cin channels to cout channels of full-lattice colour fields:
 *   h'_{c}(x) = sum_{path} sum_{c'} W[path][c][c'] (T_path h_{c'})(x),  W complex.
 * The network has three layers, channels 1 -> 4 -> 4 -> 1.  Its input is an even-odd vector on
 * the even sites (zero on odd sites) and its output is the even-site part of the last layer.
 * Weights: layer l holds 17*cout*cin complex numbers, [path][cout][cin][2], layers concatenated.
 * ---------------------------------------------------------------------------------------- */

#define PC_PATHS 17

static void transport(const int L[4], const double *X, const double *N, int path,
                      const double *h, double *out) {
    long V = volume(L);
    for (long x = 0; x < V; x++) {
        cplx s[3];
        if (path == 0) {
            for (int a = 0; a < 3; a++) s[a] = vec(h, x, a);
        } else {
            int q = (path - 1) % 8, mu = q / 2, backward = q % 2;
            const double *U = (path <= 8) ? X : N;
            int step = (path <= 8) ? 1 : 3;
            for (int a = 0; a < 3; a++) { s[a].re = 0.0; s[a].im = 0.0; }
            if (!backward) {
                long y = hop(L, x, mu, step);
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++)
                        s[a] = c_add(s[a], c_mul(link(U, V, mu, x, a, b), vec(h, y, b)));
            } else {
                long y = hop(L, x, mu, -step);
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++)
                        s[a] = c_add(s[a], c_mul(c_conj(link(U, V, mu, y, b, a)), vec(h, y, b)));
            }
        }
        for (int a = 0; a < 3; a++) put(out, x, a, s[a]);
    }
}

/* path whose transport is the adjoint of `path` (T^{+k}_mu adjoint is T^{-k}_mu) */
static int adjoint_path(int path) {
    if (path == 0) return 0;
    int q = (path - 1) % 8;
    return (q % 2 == 0) ? path + 1 : path - 1;
}

/* one layer: in [cin][V][3][2] -> out [cout][V][3][2] */
void oracle_pc_layer(const int L[4], const double *X, const double *N, int cin, int cout,
                     const double *W, const double *in, double *out) {
    long V = volume(L), n = V * 3;
    double *t = (double *)malloc(sizeof(double) * n * 2);
    memset(out, 0, sizeof(double) * n * 2 * cout);
    for (int path = 0; path < PC_PATHS; path++) {
        for (int ci = 0; ci < cin; ci++) {
            transport(L, X, N, path, in + (long)ci * n * 2, t);
            for (int co = 0; co < cout; co++) {
                const double *w = W + (((long)path * cout + co) * cin + ci) * 2;
                cplx wc = {w[0], w[1]};
                double *o = out + (long)co * n * 2;
                for (long i = 0; i < n; i++) {
                    cplx z = c_mul(wc, (cplx){t[2 * i], t[2 * i + 1]});
                    o[2 * i] += z.re; o[2 * i + 1] += z.im;
                }
            }
        }
    }
    free(t);
}

static const int PC_CH[4] = {1, 4, 4, 1};

long oracle_pc_num_weights(void) {
    long s = 0;
    for (int l = 0; l < 3; l++) s += (long)PC_PATHS * PC_CH[l + 1] * PC_CH[l];
    return s;  /* complex weights */
}

static const double *layer_weights(const double *W, int layer) {
    long off = 0;
    for (int l = 0; l < layer; l++) off += (long)PC_PATHS * PC_CH[l + 1] * PC_CH[l];
    return W + off * 2;
}

/* network output y = even part of layer3(layer2(layer1(embed(r)))), r,y: [V/2][3][2] */
void oracle_pc_forward(const int L[4], const double *X, const double *N, const double *W,
                       const double *r, double *y) {
    long V = volume(L), n = V * 3;
    double *h0 = (double *)calloc((size_t)n * 2, sizeof(double));
    double *h1 = (double *)malloc(sizeof(double) * n * 2 * 4);
    double *h2 = (double *)malloc(sizeof(double) * n * 2 * 4);
    double *h3 = (double *)malloc(sizeof(double) * n * 2);
    for (long x = 0; x < V; x++)
        if (parity_of(L, x) == 0)
            for (int a = 0; a < 3; a++) put(h0, x, a, vec(r, x / 2, a));
    oracle_pc_layer(L, X, N, 1, 4, layer_weights(W, 0), h0, h1);
    oracle_pc_layer(L, X, N, 4, 4, layer_weights(W, 1), h1, h2);
    oracle_pc_layer(L, X, N, 4, 1, layer_weights(W, 2), h2, h3);
    for (long x = 0; x < V; x++)
        if (parity_of(L, x) == 0)
            for (int a = 0; a < 3; a++) put(y, x / 2, a, vec(h3, x, a));
    free(h0); free(h1); free(h2); free(h3);
}

/*
 * Backward of one layer.  g_out [cout][V][3][2] is the gradient of a real loss with respect to
 * the layer output in the form G = dL/dRe h' + i dL/dIm h'.  Accumulates
 *   gW[path][c][c'] += sum_x sum_a G_c(x,a) conj((T_path h_c')(x,a))
 * and, if g_in != NULL, writes g_in_{c'} = sum_path sum_c conj(W[path][c][c']) T_path^dag G_c.
 */
static void layer_backward(const int L[4], const double *X, const double *N, int cin, int cout,
                           const double *W, const double *in, const double *g_out,
                           double *gW, double *g_in) {
    long V = volume(L), n = V * 3;
    double *t = (double *)malloc(sizeof(double) * n * 2);
    for (int path = 0; path < PC_PATHS; path++) {
        for (int ci = 0; ci < cin; ci++) {
            transport(L, X, N, path, in + (long)ci * n * 2, t);
            for (int co = 0; co < cout; co++) {
                cplx s = dot(t, g_out + (long)co * n * 2, n);  /* sum conj(T h) G */
                double *g = gW + (((long)path * cout + co) * cin + ci) * 2;
                g[0] += s.re; g[1] += s.im;
            }
        }
    }
    if (g_in) {
        memset(g_in, 0, sizeof(double) * n * 2 * cin);
        for (int path = 0; path < PC_PATHS; path++) {
            for (int co = 0; co < cout; co++) {
                transport(L, X, N, adjoint_path(path), g_out + (long)co * n * 2, t);
                for (int ci = 0; ci < cin; ci++) {
                    const double *w = W + (((long)path * cout + co) * cin + ci) * 2;
                    cplx wc = {w[0], -w[1]};
                    double *o = g_in + (long)ci * n * 2;
                    for (long i = 0; i < n; i++) {
                        cplx z = c_mul(wc, (cplx){t[2 * i], t[2 * i + 1]});
                        o[2 * i] += z.re; o[2 * i + 1] += z.im;
                    }
                }
            }
        }
    }
    free(t);
}

/*
 * Weight gradient of a real loss through the network for one input r [V/2][3][2], given the
 * loss gradient with respect to the network output, gy = dL/dRe y + i dL/dIm y on the even sites
 * [V/2][3][2].  Accumulates into grad (layout of W) the chain rule of oracle_pc_loss_grad.
 */
void oracle_pc_backward(const int L[4], const double *X, const double *N, const double *W,
                        const double *r, const double *gy, double *grad) {
    long V = volume(L), n = V * 3;
    double *h0 = (double *)calloc((size_t)n * 2, sizeof(double));
    double *h1 = (double *)malloc(sizeof(double) * n * 2 * 4);
    double *h2 = (double *)malloc(sizeof(double) * n * 2 * 4);
    double *g3 = (double *)calloc((size_t)n * 2, sizeof(double));
    double *g2 = (double *)malloc(sizeof(double) * n * 2 * 4);
    double *g1 = (double *)malloc(sizeof(double) * n * 2 * 4);
    for (long x = 0; x < V; x++)
        if (parity_of(L, x) == 0)
            for (int a = 0; a < 3; a++) {
                put(h0, x, a, vec(r, x / 2, a));
                put(g3, x, a, vec(gy, x / 2, a));
            }
    oracle_pc_layer(L, X, N, 1, 4, layer_weights(W, 0), h0, h1);
    oracle_pc_layer(L, X, N, 4, 4, layer_weights(W, 1), h1, h2);
    layer_backward(L, X, N, 4, 1, layer_weights(W, 2), h2, g3, grad + (layer_weights(W, 2) - W), g2);
    layer_backward(L, X, N, 4, 4, layer_weights(W, 1), h1, g2, grad + (layer_weights(W, 1) - W), g1);
    layer_backward(L, X, N, 1, 4, layer_weights(W, 0), h0, g1, grad + (layer_weights(W, 0) - W), NULL);
    free(h0); free(h1); free(h2); free(g3); free(g2); free(g1);
}

/*
 * Training loss and gradient over K pairs (r_k, e_k), each [V/2][3][2] with A e_k = r_k: the
 * error of the network's correction measured in the residual norm,
 *   loss = (1/K) sum_k |A (M r_k - e_k)|^2 / |r_k|^2,
 * so that lambda p(lambda) ~ 1 is fitted over the whole spectrum of A (what CG needs).
 * grad receives dloss/dRe W + i dloss/dIm W for every complex weight (same layout as W).
 * The output gradient is gy_k = 2 A (A (y_k - e_k)) / (K |r_k|^2) (A is Hermitian).
 */
double oracle_pc_loss_grad(const int L[4], const double *X, const double *N, double mass, const double *W,
                           int K, const double *r, const double *e, double *grad) {
    long Vh = volume(L) / 2, m = Vh * 3;
    long nw = oracle_pc_num_weights();
    double *y = (double *)malloc(sizeof(double) * m * 2);
    double *d = (double *)malloc(sizeof(double) * m * 2);
    double *gy = (double *)malloc(sizeof(double) * m * 2);
    double loss = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * nw * 2);
    for (int k = 0; k < K; k++) {
        const double *rk = r + (long)k * Vh * 6, *ek = e + (long)k * Vh * 6;
        oracle_pc_forward(L, X, N, W, rk, y);
        for (long i = 0; i < 2 * m; i++) y[i] -= ek[i];
        oracle_aop(L, X, N, mass, y, d, 1);                 /* d = A (y - e) */
        double rnorm2 = norm2(rk, m);
        loss += norm2(d, m) / rnorm2 / K;
        if (!grad) continue;
        oracle_aop(L, X, N, mass, d, gy, 1);                /* gy = A d */
        for (long i = 0; i < 2 * m; i++) gy[i] *= 2.0 / (K * rnorm2);
        oracle_pc_backward(L, X, N, W, rk, gy, grad);
    }
    free(y); free(d); free(gy);
    return loss;
}

/*
 * Adjoint of one layer: g_in_{c'} = sum_path sum_c conj(W[path][c][c']) T_path^dag g_out_c, with
 * T_path^dag the transport of the reverse hop (adjoint_path).  g_out [cout][V][3][2] ->
 * g_in [cin][V][3][2].
 */
static void layer_adjoint(const int L[4], const double *X, const double *N, int cin, int cout,
                          const double *W, const double *g_out, double *g_in) {
    long V = volume(L), n = V * 3;
    double *t = (double *)malloc(sizeof(double) * n * 2);
    memset(g_in, 0, sizeof(double) * n * 2 * cin);
    for (int path = 0; path < PC_PATHS; path++) {
        for (int co = 0; co < cout; co++) {
            transport(L, X, N, adjoint_path(path), g_out + (long)co * n * 2, t);
            for (int ci = 0; ci < cin; ci++) {
                const double *w = W + (((long)path * cout + co) * cin + ci) * 2;
                cplx wc = c_conj((cplx){w[0], w[1]});
                double *o = g_in + (long)ci * n * 2;
                for (long i = 0; i < n; i++) {
                    cplx z = c_mul(wc, (cplx){t[2 * i], t[2 * i + 1]});
                    o[2 * i] += z.re; o[2 * i + 1] += z.im;
                }
            }
        }
    }
    free(t);
}

/* y = M^dag u: the adjoint of the network map r -> oracle_pc_forward(r) on even sites,
 * layer1^dag layer2^dag layer3^dag applied to u embedded on the even sites, even part kept. */
void oracle_pc_adjoint(const int L[4], const double *X, const double *N, const double *W,
                       const double *u, double *y) {
    long V = volume(L), n = V * 3;
    double *g3 = (double *)calloc((size_t)n * 2, sizeof(double));
    double *g2 = (double *)malloc(sizeof(double) * n * 2 * 4);
    double *g1 = (double *)malloc(sizeof(double) * n * 2 * 4);
    double *g0 = (double *)malloc(sizeof(double) * n * 2);
    for (long x = 0; x < V; x++)
        if (parity_of(L, x) == 0)
            for (int a = 0; a < 3; a++) put(g3, x, a, vec(u, x / 2, a));
    layer_adjoint(L, X, N, 4, 1, layer_weights(W, 2), g3, g2);
    layer_adjoint(L, X, N, 4, 4, layer_weights(W, 1), g2, g1);
    layer_adjoint(L, X, N, 1, 4, layer_weights(W, 0), g1, g0);
    for (long x = 0; x < V; x++)
        if (parity_of(L, x) == 0)
            for (int a = 0; a < 3; a++) put(y, x / 2, a, vec(g0, x, a));
    free(g3); free(g2); free(g1); free(g0);
}

/*
 * The same training loss for the normal form of the network, M = N^dag N (Hermitian and
 * positive semi-definite for any weights, so preconditioned CG keeps its short recurrence):
 *   loss = (1/K) sum_k |A (N^dag N r_k - e_k)|^2 / |r_k|^2.
 * With h = N r, y = N^dag h and gy = 2 A A (y - e) / (K |r|^2), the weights enter twice:
 * through N^dag (dloss = Re <h, dN gy>: the backward of N at input gy with output gradient h)
 * and through N (dloss = Re <N gy, dN r>: the backward of N at input r with output gradient
 * N gy).
 */
double oracle_pc_loss_grad_normal(const int L[4], const double *X, const double *N, double mass, const double *W,
                                  int K, const double *r, const double *e, double *grad) {
    long Vh = volume(L) / 2, m = Vh * 3;
    long nw = oracle_pc_num_weights();
    double *h = (double *)malloc(sizeof(double) * m * 2);
    double *y = (double *)malloc(sizeof(double) * m * 2);
    double *d = (double *)malloc(sizeof(double) * m * 2);
    double *gy = (double *)malloc(sizeof(double) * m * 2);
    double *ngy = (double *)malloc(sizeof(double) * m * 2);
    double loss = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * nw * 2);
    for (int k = 0; k < K; k++) {
        const double *rk = r + (long)k * Vh * 6, *ek = e + (long)k * Vh * 6;
        oracle_pc_forward(L, X, N, W, rk, h);
        oracle_pc_adjoint(L, X, N, W, h, y);
        for (long i = 0; i < 2 * m; i++) y[i] -= ek[i];
        oracle_aop(L, X, N, mass, y, d, 1);                 /* d = A (y - e) */
        double rnorm2 = norm2(rk, m);
        loss += norm2(d, m) / rnorm2 / K;
        if (!grad) continue;
        oracle_aop(L, X, N, mass, d, gy, 1);                /* gy = A d */
        for (long i = 0; i < 2 * m; i++) gy[i] *= 2.0 / (K * rnorm2);
        oracle_pc_backward(L, X, N, W, gy, h, grad);        /* through N^dag */
        oracle_pc_forward(L, X, N, W, gy, ngy);
        oracle_pc_backward(L, X, N, W, rk, ngy, grad);      /* through N */
    }
    free(h); free(y); free(d); free(gy); free(ngy);
    return loss;
}

/*
 * One Adam step (Kingma & Ba 2014) on n real parameters, t = step number starting at 1:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 */
void oracle_adam_step(long n, double *theta, const double *g, double *m, double *v, int t,
                      double lr, double b1, double b2, double eps) {
    for (long i = 0; i < n; i++) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mhat = m[i] / (1.0 - pow(b1, t));
        double vhat = v[i] / (1.0 - pow(b2, t));
        theta[i] -= lr * mhat / (sqrt(vhat) + eps);
    }
}

/*
 * Flexible conjugate gradient (Notay 2000) with the network as a variable preconditioner,
 * truncated to one previous direction (Polak-Ribiere form), for complex Hermitian A:
 *   z_k = P r_k;  beta_k = <r_k - r_{k-1}, z_k> / <r_{k-1}, p_{k-1}>;  p_k = z_k + beta_k p_{k-1};
 *   alpha_k = <p_k, r_k> / <p_k, A p_k>;  x += alpha_k p_k;  r -= alpha_k A p_k,
 * with <u, v> = sum conj(u) v (alpha and beta are complex when P is not Hermitian).  This beta
 * makes p_k A-orthogonal to p_{k-1} and this alpha makes r_{k+1} orthogonal to p_k, for any P.
 * The preconditioner P is the network M itself (form 0), its normal form M^dag M (form 1), or
 * its Hermitian part (M + M^dag) / 2 (form 2), M^dag being the adjoint network.
 * Stops when the true relative residual meets tol (checked as in oracle_cg).  Returns the
 * iteration count or -1; x holds the iterate reached either way.
 */
int oracle_fcg(const int L[4], const double *X, const double *N, double mass, const double *W,
               const double *b, double *x, double tol, int max_iter, double *true_rel, int form) {
    long Vh = volume(L) / 2, n = Vh * 3;
    double *r = (double *)malloc(sizeof(double) * n * 2);
    double *r_old = (double *)malloc(sizeof(double) * n * 2);
    double *z = (double *)malloc(sizeof(double) * n * 2);
    double *p = (double *)calloc((size_t)n * 2, sizeof(double));
    double *Ap = (double *)malloc(sizeof(double) * n * 2);
    double bnorm = sqrt(norm2(b, n));
    cplx rp_old = {1.0, 0.0};
    int iters = -1;
    memset(x, 0, sizeof(double) * n * 2);
    memcpy(r, b, sizeof(double) * n * 2);
    *true_rel = 1.0;
    if (bnorm == 0.0) { *true_rel = 0.0; iters = 0; goto done; }
    for (int k = 1; k <= max_iter; k++) {
        if (form == 1) {                      /* z = M^dag (M r) */
            oracle_pc_forward(L, X, N, W, r, Ap);
            oracle_pc_adjoint(L, X, N, W, Ap, z);
        } else if (form == 2) {               /* z = (M r + M^dag r) / 2 */
            oracle_pc_forward(L, X, N, W, r, z);
            oracle_pc_adjoint(L, X, N, W, r, Ap);
            for (long i = 0; i < 2 * n; i++) z[i] = 0.5 * (z[i] + Ap[i]);
        } else {                              /* z = M r */
            oracle_pc_forward(L, X, N, W, r, z);
        }
        cplx beta = {0.0, 0.0};
        if (k > 1) {
            for (long i = 0; i < 2 * n; i++) Ap[i] = r[i] - r_old[i];
            cplx num = dot(Ap, z, n);
            double den = rp_old.re * rp_old.re + rp_old.im * rp_old.im;
            /* num / rp_old = num * conj(rp_old) / |rp_old|^2 */
            beta = c_scale(1.0 / den, c_mul(num, c_conj(rp_old)));
        }
        for (long i = 0; i < n; i++) {
            cplx pi = {p[2 * i], p[2 * i + 1]}, zi = {z[2 * i], z[2 * i + 1]};
            cplx q = c_add(zi, c_mul(beta, pi));
            p[2 * i] = q.re; p[2 * i + 1] = q.im;
        }
        oracle_aop(L, X, N, mass, p, Ap, 1);
        cplx pr = dot(p, r, n);
        double pAp = dot(p, Ap, n).re;
        cplx alpha = c_scale(1.0 / pAp, pr);
        rp_old = c_conj(pr);  /* <r_k, p_k> */
        memcpy(r_old, r, sizeof(double) * n * 2);
        for (long i = 0; i < n; i++) {
            cplx pi = {p[2 * i], p[2 * i + 1]}, api = {Ap[2 * i], Ap[2 * i + 1]};
            cplx dx = c_mul(alpha, pi), dr = c_mul(alpha, api);
            x[2 * i] += dx.re; x[2 * i + 1] += dx.im;
            r[2 * i] -= dr.re; r[2 * i + 1] -= dr.im;
        }
        if (sqrt(norm2(r, n)) <= tol * bnorm) {
            oracle_aop(L, X, N, mass, x, Ap, 1);
            for (long i = 0; i < 2 * n; i++) Ap[i] = b[i] - Ap[i];
            *true_rel = sqrt(norm2(Ap, n)) / bnorm;
            if (*true_rel <= tol) { iters = k; goto done; }
        }
    }
done:
    free(r); free(r_old); free(z); free(p); free(Ap);
    return iters;
}

/*
 * Multi-shift conjugate gradient (Jegerlehner 1996, hep-lat/9612014; the shifted-system solver
 * of rational-approximation workflows, not part of the paper): x_j = (A + sigma_j)^{-1} b for
 * nshift shifts sigma_j > -m^2, all from the Krylov space of one Hestenes-Stiefel CG on the
 * base system A + sigma_base, sigma_base = min_j sigma_j.  Every shifted residual is a multiple
 * of the base residual, r_j = zeta_j r; with s_j = sigma_j - sigma_base, alpha, beta the base
 * coefficients of this and (alpha_prev, beta_prev) the previous iteration:
 *   zeta_j^new = zeta_j zeta_j^old alpha_prev
 *                / (zeta_j^old alpha_prev (1 + s_j alpha) + alpha beta_prev (zeta_j^old - zeta_j)),
 *   alpha_j = alpha zeta_j^new / zeta_j,   x_j += alpha_j p_j,
 *   beta_j = beta (zeta_j^new / zeta_j)^2,   p_j = zeta_j^new r^new + beta_j p_j,
 * starting from zeta = zeta^old = 1, alpha_prev = 1, beta_prev = 0, p_j = b, x_j = 0.  Shift j
 * stops (x_j frozen) once |zeta_j| |r| <= tol |b| and its true residual |b - (A + sigma_j) x_j|
 * recomputed in FP64 confirms tol; the base iterates until every shift has stopped.
 * b: [V/2][3][2]; x: [nshift][V/2][3][2]; iters[j]: the iteration at which shift j stopped
 * (-1 if it never did); true_rel[j]: its final true relative residual.  Returns the number of
 * base iterations, or -1 when max_iter was reached first.
 */
int oracle_cg_multishift(const int L[4], const double *X, const double *N, double mass, const double *b,
                         int nshift, const double *shifts, double *x, double tol, int max_iter, int *iters,
                         double *true_rel) {
    long Vh = volume(L) / 2, n = Vh * 3;
    double *r = (double *)malloc(sizeof(double) * n * 2);
    double *p = (double *)malloc(sizeof(double) * n * 2);
    double *Ap = (double *)malloc(sizeof(double) * n * 2);
    double *ps = (double *)malloc(sizeof(double) * n * 2 * nshift);
    double *zeta = (double *)malloc(sizeof(double) * nshift * 3);
    double *zeta_old = zeta + nshift, *zeta_new = zeta + 2 * nshift;
    int *live = (int *)malloc(sizeof(int) * nshift);
    double sigma_base = shifts[0];
    for (int j = 1; j < nshift; j++)
        if (shifts[j] < sigma_base) sigma_base = shifts[j];
    const double mass_base = sqrt(mass * mass + sigma_base);
    double bnorm = sqrt(norm2(b, n));
    memcpy(r, b, sizeof(double) * n * 2);
    memcpy(p, b, sizeof(double) * n * 2);
    for (int j = 0; j < nshift; j++) {
        memcpy(ps + (long)j * n * 2, b, sizeof(double) * n * 2);
        memset(x + (long)j * n * 2, 0, sizeof(double) * n * 2);
        zeta[j] = zeta_old[j] = 1.0;
        live[j] = 1;
        iters[j] = -1;
        true_rel[j] = 1.0;
    }
    int result = -1, remaining = nshift;
    if (bnorm == 0.0) {
        for (int j = 0; j < nshift; j++) { iters[j] = 0; true_rel[j] = 0.0; }
        result = 0;
        remaining = 0;
    }
    double rr = norm2(r, n), alpha_prev = 1.0, beta_prev = 0.0;
    for (int k = 1; k <= max_iter && remaining > 0; k++) {
        oracle_aop(L, X, N, mass_base, p, Ap, 1);
        double alpha = rr / dot(p, Ap, n).re;
        for (int j = 0; j < nshift; j++) {
            if (!live[j]) continue;
            double s = shifts[j] - sigma_base;
            zeta_new[j] = zeta[j] * zeta_old[j] * alpha_prev /
                          (zeta_old[j] * alpha_prev * (1.0 + s * alpha) + alpha * beta_prev * (zeta_old[j] - zeta[j]));
            double alpha_j = alpha * zeta_new[j] / zeta[j];
            double *xj = x + (long)j * n * 2, *pj = ps + (long)j * n * 2;
            for (long i = 0; i < 2 * n; i++) xj[i] += alpha_j * pj[i];
        }
        for (long i = 0; i < 2 * n; i++) r[i] -= alpha * Ap[i];
        double rr_new = norm2(r, n);
        double beta_base = rr_new / rr;
        for (int j = 0; j < nshift; j++) {
            if (!live[j]) continue;
            double ratio = zeta_new[j] / zeta[j];
            double beta_j = beta_base * ratio * ratio;
            double *pj = ps + (long)j * n * 2;
            for (long i = 0; i < 2 * n; i++) pj[i] = zeta_new[j] * r[i] + beta_j * pj[i];
            zeta_old[j] = zeta[j];
            zeta[j] = zeta_new[j];
            if (fabs(zeta[j]) * sqrt(rr_new) <= tol * bnorm) {
                double *xj = x + (long)j * n * 2;
                oracle_aop(L, X, N, sqrt(mass * mass + shifts[j]), xj, Ap, 1);
                for (long i = 0; i < 2 * n; i++) Ap[i] = b[i] - Ap[i];
                true_rel[j] = sqrt(norm2(Ap, n)) / bnorm;
                if (true_rel[j] <= tol) {
                    live[j] = 0;
                    iters[j] = k;
                    remaining--;
                }
            }
        }
        for (long i = 0; i < 2 * n; i++) p[i] = r[i] + beta_base * p[i];
        rr = rr_new;
        alpha_prev = alpha;
        beta_prev = beta_base;
        if (remaining == 0) result = k;
    }
    free(r); free(p); free(Ap); free(ps); free(zeta); free(live);
    return result;
}

/*
 * Z2 noise for the stochastic trace estimates of Eq. (2).  The generator is splitmix64 (Steele,
 * Lea & Flood 2014): the state advances by gamma = 0x9E3779B97F4A7C15 per output and each output
 * is the state passed through the published mixing function.  oracle_splitmix64(seed, i) is the
 * i-th output (i = 0, 1, ...) of the generator started from `seed`.
 */
unsigned long long oracle_splitmix64(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ULL) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* n noise vectors [n][V/2][3][2] on the even sites: vector k (k = first, first + 1, ...), colour
 * component e = 3 s + c takes the real value -1 if the top bit of output (3 V/2) k + e of the
 * generator is set, else +1; imaginary parts are 0. */
void oracle_z2_noise(const int L[4], unsigned long long seed, unsigned long long first, int n, double *out) {
    long Vh = volume(L) / 2, per = 3 * Vh;
    for (int k = 0; k < n; k++)
        for (long e = 0; e < per; e++) {
            unsigned long long z = oracle_splitmix64(seed, (first + (unsigned long long)k) * (unsigned long long)per + e);
            out[((long)k * per + e) * 2] = (z >> 63) ? -1.0 : 1.0;
            out[((long)k * per + e) * 2 + 1] = 0.0;
        }
}

/*
 * Stochastic estimate of Tr A^{-1} over the even sites, Eq. (2) without derivative factors:
 * (1/N) sum_k eta_k^dag A^{-1} eta_k with eta_k = noise vector k of `seed`, each A^{-1} eta_k from
 * oracle_cg to tol.  samples[k] (may be NULL) receives Re eta_k^dag A^{-1} eta_k.  Returns the
 * mean, or NaN if a solve missed tol.  (For the staggered matrix M = m + D of Eq. (3), whose even
 * block of M^{-1} is m A^{-1} and whose odd block has the same trace, Tr M^{-1} = 2 m Tr A^{-1}.)
 */
double oracle_trace_inverse(const int L[4], const double *X, const double *N, double mass, int nnoise,
                            unsigned long long seed, double tol, double *samples) {
    long Vh = volume(L) / 2, n = Vh * 3;
    double *eta = (double *)malloc(sizeof(double) * n * 2);
    double *x = (double *)malloc(sizeof(double) * n * 2);
    double sum = 0.0;
    int ok = 1;
    for (int k = 0; k < nnoise; k++) {
        double rel;
        oracle_z2_noise(L, seed, (unsigned long long)k, 1, eta);
        if (oracle_cg(L, X, N, mass, eta, x, tol, 100000, &rel) < 0) ok = 0;
        double v = dot(eta, x, n).re;
        if (samples) samples[k] = v;
        sum += v;
    }
    free(eta); free(x);
    return ok ? sum / nnoise : NAN;
}
