/*
 * hisq.h - C ABI of the GB300 (sm_103a) multi-right-hand-side even-odd HISQ Dslash and the
 * conjugate-gradient solvers built on it.
 *
 * Operator (Eq. (3), HISQ Dslash in terms of fat links X and Naik links N):
 *   w_x = sum_{mu=0..3} [ X_{x,mu} v_{x+mu} - X^dag_{x-mu,mu} v_{x-mu}
 *                        + N_{x,mu} v_{x+3mu} - N^dag_{x-3mu,mu} v_{x-3mu} ]
 * applied to bundles of n right-hand sides that share one read of the links (Eq. (4)).
 * Hops of 1 and 3 flip the site parity, so D = [[0, D_eo], [D_oe, 0]]; the solvers work on the
 * even sites with the Hermitian positive definite A = m^2 - D_eo D_oe.
 *
 * Geometry and canonical (exchange) layouts:
 *   lattice (Lx, Ly, Lz, Lt), every extent even and >= 4; V = Lx Ly Lz Lt.
 *   lexicographic site index i = x + Lx (y + Ly (z + Lz t)); parity (x+y+z+t) mod 2;
 *   even-odd index of a site within its parity = i / 2.
 *   canonical links:   double [4 mu][V][3 row][3 col][2 re/im]
 *   canonical vectors: double [nrhs][V/2][3 colour][2 re/im], sites of one parity in
 *                      even-odd order.
 * Staggered phases and boundary signs are part of the links; the library applies Eq. (3) to
 * whatever X and N it is given, with periodic index arithmetic.
 *
 * Internal vector layout (what hisq_dslash, hisq_aop and the preconditioner read and write):
 *   site-major with the right-hand sides of a site adjacent:
 *     HISQ_FP64 / HISQ_FP32 / HISQ_BF16: element (s, c, r) is the complex number at index
 *                (s*3 + c)*n + r, stored as double2 / float2 / __nv_bfloat162 (BF16 unscaled);
 *     HISQ_FP16: one 16-byte record per (site, rhs) at index s*n + r: the three colour
 *                components as __half2 followed by a float scale; value = half * scale, and
 *                the scale is the largest |real or imaginary part| of the three components.
 *   hisq_vector_bytes() gives the size of one such bundle.
 *
 * Threads and contexts: hisq_init() creates a context bound to the calling host thread (one
 * lattice, one device, one stream).  Every other call uses the calling thread's context.
 *
 * Pointers: arguments named "device" must be device memory of the context's device; arguments
 * named "host or device" may be either (the library detects which).  Ownership of every buffer
 * passed in stays with the caller.  Handles (hisq_links, hisq_pc) and the solver workspace are
 * owned by the library and freed by the matching *_destroy call or by hisq_finalize().
 *
 * Errors: every function returns HISQ_OK (0) or a negative hisq_status.  Nothing aborts, traps or
 * waits without bound.  hisq_last_error() gives a one-line description of the last failure in
 * the calling thread.
 */
#ifndef HISQ_H
#define HISQ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HISQ_OK = 0,
    HISQ_ERR_ARG = -1,            /* invalid argument (null pointer, size, precision, parity) */
    HISQ_ERR_CUDA = -2,           /* a CUDA runtime call failed */
    HISQ_ERR_NOMEM = -3,          /* device or host allocation failed */
    HISQ_ERR_NOT_CONVERGED = -4,  /* a solve missed its tolerance within max_iter */
    HISQ_ERR_BREAKDOWN = -5,      /* NaN/Inf or a non-positive <p, A p> in a solve */
    HISQ_ERR_TIMEOUT = -6,        /* a bounded device-side wait ran out */
    HISQ_ERR_STATE = -7           /* no context on this thread, or handles of another context */
} hisq_status;

typedef enum { HISQ_FP64 = 0, HISQ_FP32 = 1, HISQ_FP16 = 2, HISQ_BF16 = 3 } hisq_prec;

#define HISQ_MAX_BUNDLE 16   /* right-hand sides per solver bundle */
#define HISQ_MAX_NRHS 64     /* right-hand sides per hisq_dslash / hisq_aop call */
#define HISQ_PC_WEIGHTS 408  /* complex weights of the preconditioner network */
#define HISQ_MAX_SHIFTS 16   /* shifts per multi-shift solve */

typedef struct hisq_links hisq_links;
typedef struct hisq_pc hisq_pc;

/* ---- context ------------------------------------------------------------------------------ */

/* Create the calling thread's context: lattice dims[4] = (Lx, Ly, Lz, Lt) (even, >= 4), CUDA
 * device ordinal, and the cudaStream_t all work is issued on (NULL = the legacy default
 * stream).  Fails with HISQ_ERR_STATE if the thread already has a context. */
int hisq_init(const int dims[4], int device, void *cuda_stream);

/* Destroy the calling thread's context and everything it owns (links, preconditioners,
 * workspace, captured graphs). */
int hisq_finalize(void);

/* Synchronise the context's stream and report whether a bounded device-side wait ran out since
 * the last call (HISQ_ERR_TIMEOUT; the output of that launch is invalid and the flag is
 * cleared), else HISQ_OK.  The staged Dslash waits for its tiles' bulk copies with such a
 * bound, so a lost transfer ends the kernel instead of hanging it. */
int hisq_device_status(void);

/* Measured dense FMA throughput of the context's device in TFLOP/s (an FMA counted as two
 * flops): chains of independent FP32 and FP64 fused multiply-adds on every SM, timed with CUDA
 * events (about 0.1 s).  The denominators of the FP32- and FP64-bound rooflines; the paper has
 * no counterpart. */
int hisq_measure_fma_peaks(double *fp32_tflops, double *fp64_tflops);

const char *hisq_strerror(int status);
const char *hisq_last_error(void);

/* ---- links (packed once per gauge field) -------------------------------------------------- */

/* Pack one kind of link field for the Dslash.  canon: host or device, canonical layout
 * double[4][V][3][3][2], the fat links X (is_naik = 0, hop 1) or the Naik links N (is_naik = 1,
 * hop 3).  prec: storage precision of the copy the Dslash reads.  recon: 18 (full matrix),
 * or, for Naik links only, 13 (two rows of W plus c, where N = c W, W in SU(3)) or 9 (eight
 * SU(3) parameters plus c); 13 and 9 are exact only for links of that form (Sec. 2: Naik links
 * can be rebuilt from 9 or 13/14 reals; fat links cannot).  16-bit 18-real links carry one
 * float scale per site.  When prec != HISQ_FP64 the handle also keeps an FP64 copy, used by the
 * solvers' FP64 residual recomputation.  The input is not retained. */
int hisq_links_create(hisq_links **h, const double *canon, int is_naik, int prec, int recon);
int hisq_links_destroy(hisq_links *h);

/* Decode the packed copy back to FP64 (the links as the Dslash sees them) for checking:
 * out (host) double[2 parity][V/2][8 slot][3][3][2], slot 2mu = U_{x,mu} and slot 2mu+1 =
 * -U^dag_{x-k mu,mu} (k = 1 fat, 3 Naik) for the site x of the given parity and even-odd index. */
int hisq_links_export(const hisq_links *h, double *out);

/* ---- vectors ------------------------------------------------------------------------------ */

/* Bytes of one internal even-odd bundle of nrhs vectors in precision prec. */
size_t hisq_vector_bytes(int prec, int nrhs);

/* canonical (host or device, double[nrhs][V/2][3][2]) <-> internal (device) layout. */
int hisq_pack(const double *canon, void *internal, int nrhs, int prec);
int hisq_unpack(const void *internal, double *canon, int nrhs, int prec);

/* ---- operators ---------------------------------------------------------------------------- */

/* w = D_{p,1-p} v for nrhs (1..HISQ_MAX_NRHS) right-hand sides, Eq. (3)-(4): the input lives on
 * parity 1-parity and the output on `parity` (0: D_eo, odd -> even; 1: D_oe, even -> odd).
 * in, out: device, internal layout in the links' precision; they must not overlap.  fat and
 * naik must share the context and the precision.  Allocates nothing. */
int hisq_dslash(const hisq_links *fat, const hisq_links *naik, const void *in, void *out,
                int nrhs, int parity);

/* w = D v on the whole lattice, Eq. (3) as printed (both parities): in and out are each two
 * internal bundles of nrhs vectors back to back, the even-site bundle first, then the odd-site
 * one (hisq_vector_bytes(prec, nrhs) bytes each); out_even = D_eo in_odd, out_odd = D_oe in_even.
 * Same requirements as hisq_dslash; allocates nothing. */
int hisq_dslash_full(const hisq_links *fat, const hisq_links *naik, const void *in, void *out,
                     int nrhs);

/* A-operator with fused dot product: out = m^2 in - D_eo (D_oe in) on the even sites, and
 * pAp[r] = Re <in_r, out_r> accumulated in FP64.  in, out: device, internal layout in the links'
 * precision; pAp: host or device, nrhs doubles (may be NULL).  The odd-parity intermediate lives
 * in the context's workspace, which grows on demand (cudaMalloc). */
int hisq_aop(const hisq_links *fat, const hisq_links *naik, double mass, const void *in,
             void *out, int nrhs, double *pAp);

/* FP64-accurate residual r_k = rhs_k - A x_k, A = mass^2 - D_eo D_oe on the even sites (the
 * operator of Sec. 1's inversions, Eq. (3) restricted to the two parities), for k < nrhs, in the
 * arithmetic the solvers' reliable updates use for these links: for FP32/FP16/BF16 handles the
 * double-single form of the links (every FP64 real as a pair of floats, 48-bit significand) with
 * exact products (Dekker 1971, by fused multiply-add) and error-free sums (Knuth's two-sum,
 * Ogita-Rump-Oishi cascaded summation) on the FP32 pipe, then b - m^2 x + D t in FP64; for FP64
 * handles native FP64.  rhs, x, r: host or device canonical double[nrhs][V/2][3][2] (r may alias
 * neither); res2: host or device double[nrhs] receiving |r_k|^2 (may be NULL).  Allocates its
 * scratch (cudaMalloc) for the call and synchronises the context's stream. */
int hisq_residual(const hisq_links *fat, const hisq_links *naik, double mass, const double *rhs,
                  const double *x, double *r, int nrhs, double *res2);

/* ---- domain decomposition along t (the lattice split over accelerators) ------------------- */

#define HISQ_MAX_SLABS 8

typedef struct hisq_slabs hisq_slabs;

/* Cut the context's lattice along t into nslab slabs of Lt / nslab time planes (an even number,
 * at least 4) held on this GPU as a multi-GPU run would hold them on several: each slab keeps the
 * gathered link records of its own output sites in precision prec (18 reals per link; the
 * backward links at its lower end come from the neighbouring slab at pack time) and its own
 * vectors with three ghost time planes at either end, the reach of the Naik term (Eq. (3):
 * hops of 1 and 3).  fat, naik: device canonical double[4][V][3][3][2] (as hisq_links_create).
 * Allocates the slabs' storage. */
int hisq_slabs_create(hisq_slabs **h, const double *fat, const double *naik, int prec, int nslab);
int hisq_slabs_destroy(hisq_slabs *h);

/* out = D_{parity, 1-parity} in (Eq. (3)-(4), nrhs right-hand sides) through the decomposition:
 * the input is scattered into the slabs; each slab packs its three outgoing planes at either end
 * (face-pack kernel); the faces are copied into the neighbours' ghost planes on a second stream
 * (cudaMemcpyAsync) while the interior kernel computes the output planes whose +-3 neighbours are
 * the slab's own; the boundary kernels then compute the three planes at either end; the outputs
 * are gathered.  in, out: device canonical double[nrhs][V/2][3][2] (in on parity 1 - parity).
 * ms (host, may be NULL) receives four CUDA-event times in milliseconds: face packing, the
 * interior kernels, the halo copies, and the decomposed Dslash from face packing to the last
 * boundary kernel. */
int hisq_slabs_dslash(hisq_slabs *h, const double *in, double *out, int nrhs, int parity, double *ms);

/* ---- A-operator without allocation -------------------------------------------------------- */

/* Size of the static device scratch behind hisq_aop_noalloc (per device, held until exit). */
#define HISQ_AOP_NOALLOC_SCRATCH_BYTES (16u << 20)

/* hisq_aop without any device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc -- code whose device memory is owned by another
 * allocator (a framework's caching pool or a fixed budget that must not be exceeded behind its
 * back), code on a latency-critical path that cannot afford cudaMalloc's implicit device-wide
 * synchronisation, and code that must not fail with an out-of-memory error in the middle of a
 * run.  It computes the same out and pAp as hisq_aop (same kernels, a fixed launch shape instead
 * of the autotuned one), but its scratch -- the odd-parity intermediate, the reduction partials and
 * the block counter -- lives in one file-scope static __device__ array of
 * HISQ_AOP_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU which loads the library holds until the
 * process exits.  The caller still passes in and out (device, internal layout in the links'
 * precision) and pAp (host or device, nrhs doubles, may be NULL).
 * Limits: the odd-parity intermediate (hisq_vector_bytes(prec, nrhs)) must fit in the scratch
 * less 1 MiB of reduction space, e.g. FP32 32^3x8 up to nrhs = 4; larger requests return
 * HISQ_ERR_ARG with a message naming the limit, and nothing is launched.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The address is kept for
 * the life of the process: it stays valid until the device is reset (cudaDeviceReset tears down
 * the context that holds the array; do not call this entry point after one).  Every call shares the
 * one array and leaves its contents behind (the block counter is cleared at the start of each
 * call): calls that overlap on the GPU, from several streams or host threads, race. */
int hisq_aop_noalloc(const hisq_links *fat, const hisq_links *naik, double mass, const void *in,
                     void *out, int nrhs, double *pAp);

/* ---- solvers ------------------------------------------------------------------------------ */

typedef struct {
    int inner_prec;       /* HISQ_FP64: plain FP64 CG; FP32/FP16/BF16: mixed precision with FP64
                             reliable updates (needs links packed in that precision) */
    double delta;         /* reliable update when |r| < delta * |r at the last update|; 0
                             (default) = by inner precision: FP32 0.01, FP16 0.03, BF16 0.1 (the
                             iterated residual follows the operator of the stored links, so a
                             coarser storage needs updates at smaller drops); else in (0, 1) */
    int max_iter;         /* per right-hand side (default 20000) */
    int bundle;           /* right-hand sides per bundle, 1..HISQ_MAX_BUNDLE; 0 (default) = the
                             autotuner's choice among 1, 2, 4, 8, 12, 16 and min(nrhs, 16): the
                             split of nrhs into bundles with the least summed tuned Dslash time
                             (min(nrhs, 16) when autotune is 0) */
    int use_graph;        /* driver of a bundle: 0 host-driven iterations; 1 one captured CUDA
                             graph with device-side control flow (WHILE/IF conditional nodes);
                             2 (default) one persistent cooperative kernel for the whole solve,
                             with bounded grid barriers (plain CG, 18-real Naik links; otherwise,
                             or if the grid cannot be co-resident, the graph driver) */
    int check_every;      /* host-driven mode: iterations between residual read-backs (1) */
    const hisq_pc *pc;    /* learned preconditioner for flexible CG; NULL = plain CG */
    int stall_window;     /* flexible CG: fall back to plain CG if the residual does not drop */
    double stall_factor;  /* by stall_factor within stall_window iterations (10, 50) */
    int autotune;         /* 1: time the Dslash launch shapes on first use of a shape */
    int time_kernels;     /* 1: record CUDA events around every Dslash launch (host-driven) or
                             around each persistent solve kernel, with its phase times (stats) */
    int debug_barrier_timeout; /* test hook for failure detection: 1 makes every grid barrier of
                             the persistent solve wait for one block more than it launches, so the
                             bounded waits run out and the solve returns HISQ_ERR_TIMEOUT */
    int persistent_threads; /* block size of the persistent solve kernel: 0 = 512; otherwise a
                             multiple of 32 up to 1024 (one right-hand side per thread) or 512;
                             the grid is every block that fits on the GPU at once */
    int single_reduction; /* persistent driver: 1 (default) Hestenes-Stiefel CG with one
                             reduction per iteration (<p, A p>, |A p|^2 and the update phase's
                             |r|^2 together; beta from |r - alpha A p|^2 = alpha^2 |A p|^2 - |r|^2),
                             three grid barriers an iteration; 0 the two-reduction form of the
                             other drivers, four barriers */
    double multishift_tol; /* hisq_cg_multishift with inner_prec != FP64: relative residual to
                             which the shared low-precision iteration runs before the per-shift
                             FP64 refinement; 0 (default) = 1e-7 for FP32, 1e-4 for FP16/BF16 */
    int l2_persist_links; /* persistent driver: 1 (default) keeps the inner-precision Naik links
                             resident in L2 during the solve when they fit the device's persisting
                             set-aside (stream access-policy window over them, released after the
                             solve, the set-aside restored by hisq_finalize); 0 = plain caching */
} hisq_solver_params;

void hisq_default_solver_params(hisq_solver_params *p);
int hisq_set_solver_params(const hisq_solver_params *p);
int hisq_get_solver_params(hisq_solver_params *p);

/* Solve A x_k = rhs_k (A = mass^2 - D_eo D_oe, even sites) for k < nrhs to the relative true
 * residual |b - A x| / |b| <= tol, checked in FP64 on the GPU.  A right-hand side counts as
 * converged once the library's FP64 true residual is at most 0.95 tol, so that the caller's own
 * FP64 recomputation (another summation order) also finds it within tol.  rhs[k], x[k]: host or device,
 * canonical double[V/2][3][2] each; x is output only (initial guess 0).  The right-hand sides
 * are solved in bundles that share every link read; converged ones are masked out.
 * Returns HISQ_ERR_NOT_CONVERGED (stats filled, x holds the last iterate) if any right-hand
 * side misses tol within max_iter. */
int hisq_cg_solve(const hisq_links *fat, const hisq_links *naik, const double *const rhs[],
                  double *x[], int nrhs, double mass, double tol);

/* Multi-shift CG (Jegerlehner, hep-lat/9612014; the shifted solves of rational approximations,
 * which the paper does not treat): x_j = (A + shifts[j])^{-1} rhs for j < nshift
 * (1..HISQ_MAX_SHIFTS), every shift to the relative FP64 true residual
 * |b - (A + shifts[j]) x_j| / |b| <= tol.  One CG iteration on the smallest shift (one A p) serves
 * all shifts: their residuals stay multiples of its residual.  With inner_prec FP64 the iteration
 * runs in FP64 until every shift meets tol.  Otherwise it runs in the inner precision (links
 * packed in it) until every shift's recursive residual meets max(tol, multishift_tol), and the
 * shifts are then refined by defect correction: their FP64 residuals are solved together as one
 * bundle of shifted systems (right-hand side j with mass^2 + shifts[j]) by the mixed-precision
 * persistent CG and the corrections added, until every FP64 true residual meets tol (as in
 * hisq_cg_solve, at most 0.95 tol in the library's own FP64 check).  rhs, x[j]: host or device
 * canonical double[V/2][3][2]; shifts: host
 * double[nshift], each > -mass^2, any order.  hisq_last_stats then reports per shift:
 * iterations[j] = shared iterations until shift j met its recursive residual plus its
 * refinement iterations, and true_residual[j].  Errors as hisq_cg_solve. */
int hisq_cg_multishift(const hisq_links *fat, const hisq_links *naik, const double *rhs, double *x[],
                       int nshift, const double *shifts, double mass, double tol);

/* ---- stochastic traces (Eq. (2)) ----------------------------------------------------------- */

/* Z2 noise vectors for the stochastic trace estimates of Eq. (2): out (device, canonical
 * double[n][V/2][3][2]) receives vectors first .. first + n - 1 of the stream `seed`.  Component
 * e = 3 s + c of vector k is -1 if the top bit of output (3 V/2) k + e of splitmix64 started from
 * seed is set, else +1 (imaginary parts 0); splitmix64 (Steele, Lea & Flood 2014): state + i
 * times 0x9E3779B97F4A7C15, then its mixing function, so every vector is generated independently
 * on the device. */
int hisq_z2_noise(double *out, int n, unsigned long long seed, unsigned long long first);

/* Stochastic estimate of Tr A^{-1} over the even sites (Eq. (2) with no derivative factors):
 * (1/N) sum_k Re eta_k^dag A^{-1} eta_k over the N = nnoise noise vectors 0 .. N-1 of `seed`
 * (hisq_z2_noise), each solve by hisq_cg_solve's solver with the current parameters (precision,
 * bundles) to tol, the products eta^dag x in FP64.  estimate, std_error (sample standard deviation
 * over sqrt(N), 0 for N = 1; may be NULL) and samples (double[N], the per-noise products; may be
 * NULL): host.  For the staggered matrix M = m + D, Tr M^{-1} = 2 m Tr A^{-1}.  hisq_last_stats
 * then reports the solves (one entry per noise vector).  Allocates two chunks of up to 64
 * canonical vectors for the duration of the call.  Errors as hisq_cg_solve. */
int hisq_trace_inverse(const hisq_links *fat, const hisq_links *naik, double mass, int nnoise,
                       unsigned long long seed, double tol, double *estimate, double *std_error,
                       double *samples);

typedef struct {
    int nrhs;
    int converged;            /* right-hand sides that met tol */
    int bundles;              /* bundles solved */
    int bundle_size;          /* right-hand sides per bundle used */
    int max_iterations;       /* largest per-right-hand-side iteration count */
    long total_iterations;    /* sum over right-hand sides */
    long bundle_iterations;   /* sum over bundles of the iterations each bundle ran */
    int reliable_updates;     /* FP64 residual recomputations, summed over right-hand sides */
    int fallbacks;            /* flexible-CG stalls that switched to plain CG */
    double seconds;           /* wall time of the hisq_cg_solve call */
    double dslash_ms;         /* summed inner-precision Dslash kernel time (time_kernels = 1,
                                 host-driven mode only) */
    int dslash_launches;      /* inner-precision Dslash launches timed */
    double dslash64_ms;       /* summed FP64 (residual recomputation) Dslash kernel time */
    int dslash64_launches;
    double flops;             /* useful flops: (2*1146 + 72) per even site, RHS and iteration */
    long kernel_launches;     /* kernels of this library launched by the solve */
    double solve_kernel_ms;   /* summed duration of the persistent solve kernels (use_graph = 2,
                                 time_kernels = 1; CUDA events on the solve's stream) */
    int solve_kernel_launches;
    double phase_ms[5];       /* inside those kernels, block 0's time from one grid barrier to the
                                 next, summed per phase (each with its scalar step): [0] D_oe p,
                                 [1] A p = m^2 p - D_eo t with <p, A p>, [2] the p, x, r update
                                 with |r|^2, [3] FP64 residual recomputations, [4] unused (0: the
                                 direction p = r + beta p is formed inside phases 0-2) */
    int shared_iterations;    /* hisq_cg_multishift: iterations of the shared multi-shift CG */
    long refine_iterations;   /* hisq_cg_multishift: CG iterations of the per-shift refinements */
    double shared_seconds;    /* hisq_cg_multishift: wall time of the shared iteration */
    long recompute_passes;    /* bundle iterations that ran a residual recomputation (each pass
                                 reads the FP64-accurate links once for the right-hand sides due) */
} hisq_solve_stats;

/* Statistics of the calling thread's last hisq_cg_solve or hisq_cg_multishift.  iterations
 * (int[nrhs]) and true_residual (double[nrhs], FP64 |b - A x| / |b| per right-hand side, or per
 * shift) are host arrays or NULL. */
int hisq_last_stats(hisq_solve_stats *s, int *iterations, double *true_residual);

/* Pick and cache the fastest Dslash launch shape for nrhs right-hand sides in the links'
 * precision, timing every candidate with CUDA events after an L2 flush.  Writes the
 * chosen right-hand sides per thread, threads per block and lanes per site (1; 2 when the fat
 * and Naik halves of a site run on two lanes; 4 when each lane takes two directions of one kind;
 * 8 for that split with staged link records, see hisq_set_launch_shape) if the pointers are not
 * NULL.  Allocates its
 * timing buffers. */
int hisq_autotune(const hisq_links *fat, const hisq_links *naik, int nrhs, int *rhs_per_thread,
                  int *block_threads, int *lanes_per_site);

/* Pin the Dslash launch shape used for nrhs right-hand sides with links of (prec, recon):
 * rhs_per_thread in {1, 2, 4, 8} dividing nrhs (FP64: 1, 2, 4), block_threads in 32..256,
 * lanes_per_site 1, 2 (18-real Naik links, rhs_per_thread <= 4) or 4 (18-real Naik links,
 * rhs_per_thread <= 2), or 8: the four-lane split with each tile's link records staged in shared
 * memory by the bulk-copy engine (18-real Naik, FP32/FP16/BF16, rhs_per_thread <= 2; tiles of
 * block_threads / (4 nrhs / rhs_per_thread) sites, block_threads up to 512).
 * Overrides the autotuner's choice for that key. */
int hisq_set_launch_shape(int prec, int recon, int nrhs, int rhs_per_thread, int block_threads,
                          int lanes_per_site);

/* ---- learned preconditioner --------------------------------------------------------------- */

/* A gauge-covariant parallel-transport network, channels 1 -> 4 -> 4 -> 1, 17 paths per layer
 * (identity, T^{+-1}_mu through X, T^{+-3}_mu through N), complex weights stored as
 * double[HISQ_PC_WEIGHTS][2]: layer 1 [17][4][1], layer 2 [17][4][4], layer 3 [17][1][4]
 * ([path][out channel][in channel]); path 0 identity, 1+2mu / 2+2mu the +/- one-hop through X,
 * 9+2mu / 10+2mu the +/- three-hop through N.  Acts on FP32 internal vectors of the even sites
 * (zero on odd sites); the output is the even-site part. */
int hisq_pc_create(hisq_pc **pc, const double *weights /* host, NULL = identity network */);
int hisq_pc_destroy(hisq_pc *pc);
int hisq_pc_set_weights(hisq_pc *pc, const double *weights /* host */);
int hisq_pc_get_weights(const hisq_pc *pc, double *weights /* host */);

/* out = M(in) for nrhs (1..HISQ_MAX_BUNDLE) FP32 internal even-site vectors (device). */
int hisq_pc_apply(const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik,
                  const void *in, void *out, int nrhs);

/* out = M^dag(in): the adjoint network (the adjoint layers in reverse order). */
int hisq_pc_apply_adjoint(const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik,
                          const void *in, void *out, int nrhs);

/* out = M_H(in), M_H = (M + M^dag) / 2, the Hermitian part of the network. */
int hisq_pc_apply_hermitian(const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik,
                            const void *in, void *out, int nrhs);

/* out = M^dag M (in), the normal form of the network: Hermitian and positive semi-definite for
 * any weights. */
int hisq_pc_apply_normal(const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik,
                         const void *in, void *out, int nrhs);

/* Which operator of the network the handle stands for, in training (hisq_pc_loss_grad,
 * hisq_pc_train) and as the preconditioner of hisq_cg_solve's flexible CG.  A trained M is not
 * Hermitian, and flexible CG truncated to one previous direction then loses conjugacy; both
 * forms keep the short recurrence of preconditioned CG:
 *   HISQ_PC_NORMAL (default)  P = M^dag M, positive semi-definite by construction;
 *   HISQ_PC_HERMITIAN_PART    P = (M + M^dag) / 2, trained as M itself. */
#define HISQ_PC_NORMAL 1
#define HISQ_PC_HERMITIAN_PART 0
int hisq_pc_set_form(hisq_pc *pc, int form);

/* Training loss over K pairs (r_k, e_k) with A e_k = r_k (residual and error of a CG iterate):
 *   loss = (1/K) sum_k |A (P r_k - e_k)|^2 / |r_k|^2,  A = mass^2 - D_eo D_oe,
 * with P = M^dag M (HISQ_PC_NORMAL) or P = M (HISQ_PC_HERMITIAN_PART), i.e. the error of the
 * preconditioner's correction measured in the residual norm, and its gradient
 * dL/dRe W + i dL/dIm W (host or device double[HISQ_PC_WEIGHTS][2]); r, e: device FP32 internal
 * bundles of K (1..HISQ_MAX_BUNDLE) vectors each. */
int hisq_pc_loss_grad(const hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, double mass,
                      const void *r, const void *e, int K, double *loss, double *grad);

/* One Adam step (Kingma & Ba) on the real and imaginary parts of the weights, on the GPU:
 * grad host or device double[HISQ_PC_WEIGHTS][2]; step counts from 1. */
int hisq_pc_adam_step(hisq_pc *pc, const double *grad, int step, double lr, double beta1,
                      double beta2, double eps);

/* Train on K pairs (device FP32 internal, stored as ceil(K/16) consecutive bundles of 16
 * vectors, the last one padded) for `epochs` passes of minibatches of `batch` (<= 16) pairs
 * with Adam at learning rate lr, on the loss of hisq_pc_loss_grad.  loss_history (host, epochs
 * doubles, may be NULL) receives the mean loss of each epoch.  Consecutive calls continue one
 * Adam run (moments and step count kept in the handle; hisq_pc_set_weights starts a new one),
 * so training can be interleaved with validation solves. */
int hisq_pc_train(hisq_pc *pc, const hisq_links *fat, const hisq_links *naik, double mass,
                  const void *r, const void *e, int K, int batch, int epochs, double lr,
                  double *loss_history);

#ifdef __cplusplus
}
#endif

#endif /* HISQ_H */
