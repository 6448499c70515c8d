// Domain decomposition of the even-odd Dslash (Eq. (3)-(4)) along t, as a lattice split over
// several accelerators would run it, with every slab held on this one GPU.
//
// The lattice is cut into nslab slabs of Lt / nslab time planes.  A slab stores its sites in a
// slab lattice of Lt / nslab + 8 planes: its own planes at ts = 4 .. Lt/nslab + 3, and three ghost
// planes on either side (ts = 1..3 and Lt/nslab + 4 .. Lt/nslab + 6) for the depth-3 reach of the
// Naik term; four planes of margin keep the slab lattice's parity that of the full lattice.  Each
// slab has the gathered link records of its own output sites only (the backward links of its first
// planes come from the neighbouring slab's sites at pack time, so the record layout is unchanged)
// and its own input, output and send buffers: nothing reads another slab's memory except the
// halo copies.
//
// One Dslash of output parity p: (1) every slab packs the three outgoing planes of its input at
// either end into a send buffer (the face-pack kernel: in the even-odd layout a time plane of one
// parity is a contiguous run of Lx Ly Lz / 2 sites); (2) on a second stream the send buffers are
// copied into the neighbours' ghost planes (plain cudaMemcpyAsync, the copies a NVLink peer or a
// network transfer would make); (3) meanwhile the interior kernel computes the output sites whose
// +-3 neighbours in t are the slab's own; (4) once the halo has arrived, the boundary kernels
// compute the three planes at either end.  Interior and boundary are the library's Dslash kernel
// restricted to a range of output sites of the slab lattice.
#include <string.h>
#include <algorithm>

#include "hisq_internal.cuh"

struct hisq_slabs {
    hisq_ctx *ctx;
    int nslab, prec, Lts;   // slabs, storage precision, own planes per slab
    int phv;                // sites of one parity in one time plane (Lx Ly Lz / 2)
    hisq::Geom g;           // the slab lattice (Lx, Ly, Lz, Lts + 8)
    struct Slab {
        uint4 *fat = nullptr, *naik = nullptr;
        float *fat_scale = nullptr, *naik_scale = nullptr;
        void *in = nullptr, *out = nullptr, *send = nullptr;
    } s[HISQ_MAX_SLABS];
    int cap_n;              // right-hand sides the vector buffers hold
    hisq_links fat_h, naik_h;  // precision and encoding for the launch dispatch (no storage)
    cudaStream_t halo;
    cudaEvent_t ev[8];      // packed, halo arrived, and timing marks
};

namespace hisq {

// canonical [n][V/2][3][2] (lattice g, parity q) -> slab k's internal bundle, own planes only
template <int P>
__global__ void slab_scatter_kernel(Geom g, Geom gs, int t0, int q, const double *canon, void *internal, int n,
                                    int s_begin, int count) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)count * n) return;
    const int ss = s_begin + (int)(i / n), r = (int)(i % n);
    const SiteCoord sc = decode_site(gs, ss, q);
    const int t = sc.c[3] - 4 + t0;
    const long lex = sc.c[0] + (long)g.L[0] * (sc.c[1] + (long)g.L[1] * (sc.c[2] + (long)g.L[2] * t));
    const double *c = canon + ((size_t)r * g.Vh + lex / 2) * 6;
    Cplx<typename Prec<P>::real> w[3];
    for (int k = 0; k < 3; k++) w[k] = {(typename Prec<P>::real)c[2 * k], (typename Prec<P>::real)c[2 * k + 1]};
    store_vec<P>(VecView<P>{internal, n}, ss, r, w);
}

// slab k's internal output bundle (own planes) -> canonical [n][V/2][3][2] of the lattice
template <int P>
__global__ void slab_gather_kernel(Geom g, Geom gs, int t0, int p, const void *internal, double *canon, int n,
                                   int s_begin, int count) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)count * n) return;
    const int ss = s_begin + (int)(i / n), r = (int)(i % n);
    const SiteCoord sc = decode_site(gs, ss, p);
    const int t = sc.c[3] - 4 + t0;
    const long lex = sc.c[0] + (long)g.L[0] * (sc.c[1] + (long)g.L[1] * (sc.c[2] + (long)g.L[2] * t));
    Cplx<typename Prec<P>::real> w[3];
    load_vec<P>(VecView<P>{const_cast<void *>(internal), n}, ss, r, w);
    double *c = canon + ((size_t)r * g.Vh + lex / 2) * 6;
    for (int k = 0; k < 3; k++) {
        c[2 * k] = (double)w[k].re;
        c[2 * k + 1] = (double)w[k].im;
    }
}

// The face-pack kernel: the three outgoing planes at the low end (ts = 4..6, from word low_word)
// and at the high end (ts = Lts + 1 .. Lts + 3, from word high_word) of the input bundle into the
// send buffer [low face][high face], each face `face_words` 16-byte words long (3 planes of one
// parity, every right-hand side).
__global__ void slab_pack_faces_kernel(const uint4 *in, uint4 *send, long low_word, long high_word, long face_words) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 2 * face_words; i += (long)gridDim.x * blockDim.x)
        send[i] = in[(i < face_words ? low_word : high_word - face_words) + i];
}

template <int P>
static void scatter(const hisq_slabs *h, int k, int q, const double *canon, int n, cudaStream_t st) {
    const int count = h->Lts * h->phv, threads = 256;
    const long items = (long)count * n;
    slab_scatter_kernel<P><<<(int)((items + threads - 1) / threads), threads, 0, st>>>(
        h->ctx->geom, h->g, k * h->Lts, q, canon, h->s[k].in, n, 4 * h->phv, count);
}

template <int P>
static void gather(const hisq_slabs *h, int k, int p, double *canon, int n, cudaStream_t st) {
    const int count = h->Lts * h->phv, threads = 256;
    const long items = (long)count * n;
    slab_gather_kernel<P><<<(int)((items + threads - 1) / threads), threads, 0, st>>>(
        h->ctx->geom, h->g, k * h->Lts, p, h->s[k].out, canon, n, 4 * h->phv, count);
}

static void free_slabs(hisq_slabs *h) {
    for (int k = 0; k < HISQ_MAX_SLABS; k++) {
        void *b[] = {h->s[k].fat, h->s[k].naik, h->s[k].fat_scale, h->s[k].naik_scale, h->s[k].in, h->s[k].out,
                     h->s[k].send};
        for (void *p : b)
            if (p) cudaFree(p);
        h->s[k] = hisq_slabs::Slab();
    }
}

static int ensure_vectors(hisq_slabs *h, int n) {
    if (n <= h->cap_n) return HISQ_OK;
    const size_t vb = vector_bytes(h->prec, h->g.Vh, n);
    const size_t face = vector_bytes(h->prec, 3 * h->phv, n);
    for (int k = 0; k < h->nslab; k++) {
        for (void **p : {&h->s[k].in, &h->s[k].out, &h->s[k].send}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
        if (cudaMalloc(&h->s[k].in, vb) != cudaSuccess || cudaMalloc(&h->s[k].out, vb) != cudaSuccess ||
            cudaMalloc(&h->s[k].send, 2 * face) != cudaSuccess) {
            h->cap_n = 0;
            return set_error(HISQ_ERR_NOMEM, "cannot allocate slab vectors for %d right-hand sides", n);
        }
        // ghost planes of a slab hold copies only; start them (and the unused margin) at zero
        HISQ_CUDA(cudaMemsetAsync(h->s[k].in, 0, vb, h->ctx->stream));
    }
    h->cap_n = n;
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" {

int hisq_slabs_create(hisq_slabs **out, const double *fat, const double *naik, int prec, int nslab) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!out || !fat || !naik) return set_error(HISQ_ERR_ARG, "null argument");
    if (prec < HISQ_FP64 || prec > HISQ_BF16) return set_error(HISQ_ERR_ARG, "unknown precision %d", prec);
    const Geom &G = ctx->geom;
    if (nslab < 2 || nslab > HISQ_MAX_SLABS || G.L[3] % nslab || (G.L[3] / nslab) % 2 || G.L[3] / nslab < 4)
        return set_error(HISQ_ERR_ARG, "%d slabs of Lt = %d: each slab needs an even number (>= 4) of time planes",
                         nslab, G.L[3]);
    if (!is_device_ptr(fat) || !is_device_ptr(naik)) return set_error(HISQ_ERR_ARG, "links must be device pointers");
    hisq_slabs *h = new hisq_slabs();
    h->ctx = ctx;
    h->nslab = nslab;
    h->prec = prec;
    h->Lts = G.L[3] / nslab;
    h->phv = G.half * G.L[1] * G.L[2];
    Geom &g = h->g;
    g = G;
    g.L[3] = h->Lts + 8;
    g.Vh = h->phv * g.L[3];
    g.plane_order = 0;  // slab passes cover ranges of time planes in index order
    h->cap_n = 0;
    h->fat_h.ctx = h->naik_h.ctx = ctx;
    h->fat_h.prec = h->naik_h.prec = prec;
    h->fat_h.recon = h->naik_h.recon = 18;
    h->naik_h.is_naik = 1;
    h->fat_h.W = h->naik_h.W = link_words(prec, 18);
    const int W = link_words(prec, 18);
    const size_t wbytes = (size_t)2 * W * g.Vh * sizeof(uint4);
    const bool scaled = prec >= HISQ_FP16;
    int rc = HISQ_OK;
    cudaStream_t st = ctx->stream;
    for (int k = 0; k < nslab && rc == HISQ_OK; k++) {
        if (cudaMalloc(&h->s[k].fat, wbytes) != cudaSuccess || cudaMalloc(&h->s[k].naik, wbytes) != cudaSuccess ||
            (scaled && (cudaMalloc(&h->s[k].fat_scale, 2 * g.Vh * sizeof(float)) != cudaSuccess ||
                        cudaMalloc(&h->s[k].naik_scale, 2 * g.Vh * sizeof(float)) != cudaSuccess))) {
            rc = set_error(HISQ_ERR_NOMEM, "cannot allocate the links of slab %d", k);
            break;
        }
        cudaMemsetAsync(h->s[k].fat, 0, wbytes, st);
        cudaMemsetAsync(h->s[k].naik, 0, wbytes, st);
        // own planes ts = 4 .. Lts + 3 are lattice planes t = k Lts .. (k + 1) Lts - 1
        const int t_off = k * h->Lts - 4;
        pack_links_into(prec, 18, G, g, t_off, 4, 4 + h->Lts, fat, 1, h->s[k].fat, h->s[k].fat_scale, W, st);
        pack_links_into(prec, 18, G, g, t_off, 4, 4 + h->Lts, naik, 3, h->s[k].naik, h->s[k].naik_scale, W, st);
    }
    if (rc == HISQ_OK && cudaStreamCreateWithFlags(&h->halo, cudaStreamNonBlocking) != cudaSuccess)
        rc = set_error(HISQ_ERR_CUDA, "cannot create the halo stream");
    for (int i = 0; i < 8 && rc == HISQ_OK; i++)
        if (cudaEventCreate(&h->ev[i]) != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "cannot create events");
    if (rc == HISQ_OK) {
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = set_error(HISQ_ERR_CUDA, "slab link packing failed: %s", cudaGetErrorString(e));
    }
    if (rc != HISQ_OK) {
        free_slabs(h);
        delete h;
        return rc;
    }
    *out = h;
    return HISQ_OK;
}

int hisq_slabs_destroy(hisq_slabs *h) {
    if (!h) return HISQ_OK;
    cudaStreamSynchronize(h->ctx->stream);
    if (h->halo) {
        cudaStreamSynchronize(h->halo);
        cudaStreamDestroy(h->halo);
    }
    for (int i = 0; i < 8; i++)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    free_slabs(h);
    delete h;
    return HISQ_OK;
}

int hisq_slabs_dslash(hisq_slabs *h, const double *in, double *out, int nrhs, int parity, double *ms) {
    hisq_ctx *ctx;
    HISQ_CHECK(require_ctx(&ctx));
    if (!h || !in || !out) return set_error(HISQ_ERR_ARG, "null argument");
    if (h->ctx != ctx) return set_error(HISQ_ERR_STATE, "slabs of another context");
    if (nrhs < 1 || nrhs > HISQ_MAX_NRHS) return set_error(HISQ_ERR_ARG, "nrhs must be in 1..%d", HISQ_MAX_NRHS);
    if (parity != 0 && parity != 1) return set_error(HISQ_ERR_ARG, "parity must be 0 or 1");
    if (!is_device_ptr(in) || !is_device_ptr(out)) return set_error(HISQ_ERR_ARG, "in and out must be device pointers");
    HISQ_CHECK(ensure_vectors(h, nrhs));
    cudaStream_t st = ctx->stream;
    const int q = 1 - parity, phv = h->phv, Lts = h->Lts, P = h->prec;
    for (int k = 0; k < h->nslab; k++) {
        switch (P) {
        case HISQ_FP64: scatter<HISQ_FP64>(h, k, q, in, nrhs, st); break;
        case HISQ_FP32: scatter<HISQ_FP32>(h, k, q, in, nrhs, st); break;
        case HISQ_FP16: scatter<HISQ_FP16>(h, k, q, in, nrhs, st); break;
        default: scatter<HISQ_BF16>(h, k, q, in, nrhs, st); break;
        }
    }
    HISQ_CUDA(cudaGetLastError());
    // launch shape: the tuned one of the full lattice for this precision and bundle, else the default
    LaunchShape shape = default_shape(P, nrhs);
    auto it = ctx->tuned.find(TuneKey{P, 18, nrhs, 0});
    if (it != ctx->tuned.end()) shape = it->second;
    // words of one site (all right-hand sides) and of one face (three planes)
    const size_t site_bytes = vector_bytes(P, 1, nrhs);
    const long plane_words = (long)(site_bytes * phv / 16);
    const long face_words = 3 * plane_words;
    HISQ_CUDA(cudaEventRecord(h->ev[2], st));  // start
    // (1) faces of every slab
    for (int k = 0; k < h->nslab; k++) {
        const int blocks = (int)std::min<long>((2 * face_words + 255) / 256, (long)ctx->num_sms * 8);
        slab_pack_faces_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const uint4 *>(h->s[k].in),
                                                       reinterpret_cast<uint4 *>(h->s[k].send), 4 * plane_words,
                                                       (long)(Lts + 1) * plane_words, face_words);
    }
    HISQ_CUDA(cudaGetLastError());
    HISQ_CUDA(cudaEventRecord(h->ev[0], st));
    // (2) halo copies on the second stream: slab k's low face -> slab k-1's high ghosts, its high
    // face -> slab k+1's low ghosts (periodic in t)
    HISQ_CUDA(cudaStreamWaitEvent(h->halo, h->ev[0], 0));
    for (int k = 0; k < h->nslab; k++) {
        const int lo = (k + h->nslab - 1) % h->nslab, hi = (k + 1) % h->nslab;
        const uint4 *send = reinterpret_cast<const uint4 *>(h->s[k].send);
        HISQ_CUDA(cudaMemcpyAsync(reinterpret_cast<uint4 *>(h->s[lo].in) + (long)(Lts + 4) * plane_words, send,
                                  face_words * 16, cudaMemcpyDeviceToDevice, h->halo));
        HISQ_CUDA(cudaMemcpyAsync(reinterpret_cast<uint4 *>(h->s[hi].in) + 1L * plane_words, send + face_words,
                                  face_words * 16, cudaMemcpyDeviceToDevice, h->halo));
    }
    HISQ_CUDA(cudaEventRecord(h->ev[1], h->halo));
    // (3) interior output planes ts = 7 .. Lts: their +-3 neighbours are the slab's own
    DslashArgs d;
    memset(&d, 0, sizeof(d));
    d.n = nrhs;
    d.parity = parity;
    d.epi = EPI_PLAIN;
    d.geom = &h->g;
    const int ilo = 7, ihi = Lts + 1;
    HISQ_CUDA(cudaEventRecord(h->ev[3], st));
    if (ihi > ilo) {
        for (int k = 0; k < h->nslab; k++) {
            const LinkField f[2] = {{h->s[k].fat, h->s[k].fat_scale, link_words(P, 18)},
                                    {h->s[k].naik, h->s[k].naik_scale, link_words(P, 18)}};
            d.fields = f;
            d.in = h->s[k].in;
            d.out = h->s[k].out;
            d.site_begin = ilo * phv;
            d.site_end = ihi * phv;
            HISQ_CHECK(launch_dslash(ctx, &h->fat_h, &h->naik_h, LINKS_INNER, d, &shape, st));
        }
    }
    HISQ_CUDA(cudaEventRecord(h->ev[4], st));
    // (4) boundary planes once the halo is in: ts = 4..6 and Lts + 1 .. Lts + 3 (all own planes
    // when the slab is too thin for an interior)
    HISQ_CUDA(cudaStreamWaitEvent(st, h->ev[1], 0));
    for (int k = 0; k < h->nslab; k++) {
        const LinkField f[2] = {{h->s[k].fat, h->s[k].fat_scale, link_words(P, 18)},
                                {h->s[k].naik, h->s[k].naik_scale, link_words(P, 18)}};
        d.fields = f;
        d.in = h->s[k].in;
        d.out = h->s[k].out;
        if (ihi > ilo) {
            d.site_begin = 4 * phv;
            d.site_end = ilo * phv;
            HISQ_CHECK(launch_dslash(ctx, &h->fat_h, &h->naik_h, LINKS_INNER, d, &shape, st));
            d.site_begin = ihi * phv;
            d.site_end = (Lts + 4) * phv;
            HISQ_CHECK(launch_dslash(ctx, &h->fat_h, &h->naik_h, LINKS_INNER, d, &shape, st));
        } else {
            d.site_begin = 4 * phv;
            d.site_end = (Lts + 4) * phv;
            HISQ_CHECK(launch_dslash(ctx, &h->fat_h, &h->naik_h, LINKS_INNER, d, &shape, st));
        }
    }
    HISQ_CUDA(cudaEventRecord(h->ev[5], st));
    for (int k = 0; k < h->nslab; k++) {
        switch (P) {
        case HISQ_FP64: gather<HISQ_FP64>(h, k, parity, out, nrhs, st); break;
        case HISQ_FP32: gather<HISQ_FP32>(h, k, parity, out, nrhs, st); break;
        case HISQ_FP16: gather<HISQ_FP16>(h, k, parity, out, nrhs, st); break;
        default: gather<HISQ_BF16>(h, k, parity, out, nrhs, st); break;
        }
    }
    HISQ_CUDA(cudaGetLastError());
    if (ms) {
        // [0] face packing, [1] interior, [2] halo copies (second stream), [3] start to end of the
        // boundary kernels (the decomposed Dslash without the scatter and gather)
        HISQ_CUDA(cudaEventSynchronize(h->ev[5]));
        float a = 0, b = 0, c = 0, e = 0;
        cudaEventElapsedTime(&a, h->ev[2], h->ev[0]);
        cudaEventElapsedTime(&b, h->ev[3], h->ev[4]);
        cudaEventElapsedTime(&c, h->ev[0], h->ev[1]);
        cudaEventElapsedTime(&e, h->ev[2], h->ev[5]);
        ms[0] = a;
        ms[1] = b;
        ms[2] = c;
        ms[3] = e;
    }
    return HISQ_OK;
}

}  // extern "C"
