// kx_api.cu -- host side of the C ABI declared in include/kx.h.
#include <math.h>
#include <string.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "kx_internal.cuh"

#define KX_PI_H 3.14159265358979323846

int kx_set_error(kx_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return code;
}

bool kx_fault(const char *what) {
    const char *e = getenv("KX_FAULT");
    if (!e || !*e) return false;
    const size_t L = strlen(what);
    for (const char *p = e;;) {
        const char *q = strchr(p, ',');
        const size_t len = q ? (size_t)(q - p) : strlen(p);
        if (len == L && strncmp(p, what, L) == 0) return true;
        if (!q) return false;
        p = q + 1;
    }
}

extern "C" const char *kx_strerror(int code) {
    switch (code) {
    case KX_OK: return "ok";
    case KX_PENDING: return "pending";
    case KX_EINVAL: return "invalid argument";
    case KX_ENOMEM: return "out of memory";
    case KX_EADMIT: return "admission refused (footprint above budget)";
    case KX_ENEG: return "negative distribution in a fixed step";
    case KX_ENONFINITE: return "non-finite value";
    case KX_ESINGULAR: return "singular projection system";
    case KX_ENOCONV: return "no convergence within max_attempts";
    case KX_ETIMEOUT: return "bounded wait expired";
    case KX_ECUDA: return "CUDA error";
    case KX_ENOTSUP: return "not supported";
    default: return "unknown status";
    }
}

extern "C" const char *kx_last_error(const kx_ctx *ctx) {
    return ctx ? ctx->last_error.c_str() : "no context";
}

// ------------------------------------------------------------------ context
extern "C" int kx_create(kx_ctx **out, int device, void *cuda_stream) {
    if (!out) return KX_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
        return KX_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return KX_ECUDA;
    kx_ctx *c = new (std::nothrow) kx_ctx();
    if (!c) return KX_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->d_arena = nullptr;
    c->arena_bytes = 0;
    c->h_pinned = nullptr;
    c->pinned_bytes = 0;
    c->launches = 0;
    if (kx_contract_prepare() != cudaSuccess) {
        delete c;
        return KX_ECUDA;
    }
    kx_batch_prepare();
    *out = c;
    return KX_OK;
}

extern "C" void kx_destroy(kx_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->d_arena) cudaFree(ctx->d_arena);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    delete ctx;
}

extern "C" int kx_set_stream(kx_ctx *ctx, void *cuda_stream) {
    if (!ctx) return KX_EINVAL;
    ctx->stream = (cudaStream_t)cuda_stream;
    return KX_OK;
}

static int kx_arena_reserve(kx_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->arena_bytes) return KX_OK;
    if (kx_fault("alloc")) return kx_set_error(ctx, KX_ENOMEM, "arena allocation failed (KX_FAULT=alloc)");
    KX_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->d_arena) cudaFree(ctx->d_arena);
    ctx->d_arena = nullptr;
    ctx->arena_bytes = 0;
    size_t want = std::max(bytes, (size_t)1 << 20);
    if (cudaMalloc(&ctx->d_arena, want) != cudaSuccess) {
        cudaGetLastError();
        return kx_set_error(ctx, KX_ENOMEM, "arena allocation failed");
    }
    ctx->arena_bytes = want;
    return KX_OK;
}

static int kx_pinned_reserve(kx_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->pinned_bytes) return KX_OK;
    KX_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    ctx->h_pinned = nullptr;
    ctx->pinned_bytes = 0;
    size_t want = std::max(bytes, (size_t)1 << 16);
    if (cudaMallocHost(&ctx->h_pinned, want) != cudaSuccess) {
        cudaGetLastError();
        return kx_set_error(ctx, KX_ENOMEM, "pinned allocation failed");
    }
    ctx->pinned_bytes = want;
    return KX_OK;
}

static size_t kx_align(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch views of one batched evaluation, carved from a base pointer.
// Bytes of one row partial: (hi, lo) floats on the FP32 path, (G, L) doubles else.
static size_t kx_partial_bytes(const kx_kernel *k) {
    return k->precision == KX_FP32 ? sizeof(float2) : sizeof(double2);
}

// Partials per instance: the FP32 path's task slots, else rows x chunks.
static size_t kx_partial_slots(const kx_kernel *k) {
    return k->precision == KX_FP32 ? (size_t)k->tslots : (size_t)k->n * kx_chunks_per_row(k);
}

size_t kx_views_bytes(const kx_kernel *k, int B) {
    const size_t n = k->n, chunks = kx_chunks_per_row(k);
    size_t s = 0;
    s += kx_align(sizeof(double) * B);               // fmax
    s += kx_align(sizeof(double) * B * n);           // lf64
    s += kx_align(sizeof(float2) * B * (n + 4));     // tl
    s += kx_align(sizeof(float2) * B * n);           // td
    s += kx_align(kx_partial_bytes(k) * B * kx_partial_slots(k)); // partial
    s += kx_align(sizeof(double) * B);               // rfmax
    s += kx_align(sizeof(double) * B);               // fsc
    s += kx_align(sizeof(float) * B * 5 * KX_FIT_W); // fitp
    s += kx_align(sizeof(float4) * B);               // fit
    s += kx_align(sizeof(int) * B);                  // flags
    s += kx_align(sizeof(double) * B);               // M2
    s += kx_align(sizeof(kx_diag) * B);              // diag
    s += kx_align(sizeof(int));                      // err
    if (k->precision == KX_FP32 && k->stats) {
        s += kx_align(sizeof(float4) * B * n);       // tq
        s += kx_align(sizeof(float) * B * n);        // tlam
    }
    if (k->precision == KX_SPLIT_TF32) {
        const size_t Bpad = ((B + 127) / 128) * 128;
        s += kx_align(sizeof(float) * Bpad * n);                             // fT
        s += kx_align(sizeof(float) * Bpad * (size_t)k->gsk * k->nis);       // Gs
        if (k->cheb_K) {
            s += kx_align(sizeof(float) * Bpad * (size_t)k->KBL * 16 * 2);   // yt
            s += kx_align(sizeof(float) * Bpad * (size_t)k->lsk * k->nis);   // Lp
            s += kx_align(sizeof(int) * B);                                   // cflag
        }
        if (k->stats) s += kx_align(sizeof(double) * B * n);                  // qsum
    }
    return s;
}

void kx_carve_views(const kx_kernel *k, int B, void *base, kx_batch_views *v) {
    const size_t n = k->n;
    const int chunks = kx_chunks_per_row(k);
    char *p = (char *)base;
    v->fmax = (double *)p; p += kx_align(sizeof(double) * B);
    v->lf64 = (double *)p; p += kx_align(sizeof(double) * B * n);
    v->tl = (float2 *)p; p += kx_align(sizeof(float2) * B * (n + 4));
    v->td = (float2 *)p; p += kx_align(sizeof(float2) * B * n);
    v->partial = (double2 *)p; p += kx_align(kx_partial_bytes(k) * B * kx_partial_slots(k));
    v->rfmax = (double *)p; p += kx_align(sizeof(double) * B);
    v->fsc = (double *)p; p += kx_align(sizeof(double) * B);
    v->fitp = (float *)p; p += kx_align(sizeof(float) * B * 5 * KX_FIT_W);
    v->fit = (float4 *)p; p += kx_align(sizeof(float4) * B);
    v->flags = (int *)p; p += kx_align(sizeof(int) * B);
    v->M2 = (double *)p; p += kx_align(sizeof(double) * B);
    v->diag = (kx_diag *)p; p += kx_align(sizeof(kx_diag) * B);
    v->err = (int *)p; p += kx_align(sizeof(int));
    v->chunks = chunks;
    v->rtask = k->d_rtask;
    v->fT = v->Gs = nullptr;
    v->yt = v->Lp = nullptr;
    v->cflag = nullptr;
    v->qsum = nullptr;
    v->cheb_K = k->cheb_K;
    v->KBL = k->KBL;
    v->gsk = k->gsk;
    v->lsk = k->lsk;
    v->nis = k->nis;
    v->tq = nullptr;
    v->tlam = nullptr;
    v->eta = k->stats;
    v->grid_div = 1;
    v->tune_tag = 0;
    if (k->precision == KX_FP32 && k->stats) {
        v->tq = (float4 *)p; p += kx_align(sizeof(float4) * B * n);
        v->tlam = (float *)p; p += kx_align(sizeof(float) * B * n);
    }
    v->B = B;
    v->Bpad = ((B + 127) / 128) * 128;
    if (k->precision == KX_SPLIT_TF32) {
        const size_t Bpad = v->Bpad;
        v->fT = (float *)p; p += kx_align(sizeof(float) * Bpad * n);
        v->Gs = (float *)p; p += kx_align(sizeof(float) * Bpad * (size_t)k->gsk * k->nis);
        if (k->cheb_K) {
            v->yt = (float *)p; p += kx_align(sizeof(float) * Bpad * (size_t)k->KBL * 16 * 2);
            v->Lp = (float *)p; p += kx_align(sizeof(float) * Bpad * (size_t)k->lsk * k->nis);
            v->cflag = (int *)p; p += kx_align(sizeof(int) * B);
        }
        if (k->stats) {
            v->qsum = (double *)p;
            p += kx_align(sizeof(double) * B * n);
        }
    }
}

cudaError_t kx_views_clear(const kx_kernel *, int, const kx_batch_views &v, cudaStream_t s) {
    return cudaMemsetAsync(v.err, 0, sizeof(int), s);
}

// ----------------------------------------------------------------- kernel
// Gauss-Legendre nodes on [-1, 1] (ascending): Newton's method on P_n started
// from the Tricomi-type estimate cos(pi (4k - 1)/(4n + 2)); P_n, P_n' from the
// Bonnet recurrence; w_k = 2 / ((1 - x_k^2) P_n'(x_k)^2).
static void kx_gauss_legendre(int n, kx_gl_nodes *gl) {
    for (int k = 1; k <= n; ++k) {
        double x = cos(KX_PI_H * (4.0 * k - 1.0) / (4.0 * n + 2.0));
        double dp = 1.0;
        for (int it = 0; it < 64; ++it) {
            double pkm1 = 1.0, pk = x;
            for (int j = 2; j <= n; ++j) {
                double pn = ((2.0 * j - 1.0) * x * pk - (j - 1.0) * pkm1) / j;
                pkm1 = pk;
                pk = pn;
            }
            if (n == 1) { pk = x; pkm1 = 1.0; }
            dp = n * (x * pk - pkm1) / (x * x - 1.0);
            double dx = pk / dp;
            x -= dx;
            if (fabs(dx) <= 1e-17) break;
        }
        double pkm1 = 1.0, pk = x;
        for (int j = 2; j <= n; ++j) {
            double pn = ((2.0 * j - 1.0) * x * pk - (j - 1.0) * pkm1) / j;
            pkm1 = pk;
            pk = pn;
        }
        if (n == 1) { pk = x; pkm1 = 1.0; }
        dp = n * (x * pk - pkm1) / (x * x - 1.0);
        gl->x[n - k] = x;
        gl->w[n - k] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

static void kx_free_kernel(kx_kernel *k) {
    if (!k) return;
    cudaSetDevice(k->device);
    void *ptrs[] = {k->d_p, k->d_E, k->d_dp, k->d_dE, k->d_h, k->d_pair, k->d_W64,
                    k->d_om64, k->d_jl, k->d_vt, k->d_W32, k->d_pk, k->d_roff, k->d_rtask,
                    k->d_task, k->d_bins, k->d_Sg, k->d_lel, k->d_lnm, k->d_lseg, k->d_lsw,
                    k->d_lorder, k->d_Mtile, k->d_vt_all, k->d_pos};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete k;
}

template <typename T>
static int kx_dev_alloc(kx_ctx *ctx, T **p, size_t count, long long *bytes) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (kx_fault("alloc")) return kx_set_error(ctx, KX_ENOMEM, "kernel table allocation failed (KX_FAULT=alloc)");
    if (cudaMalloc((void **)p, sizeof(T) * count) != cudaSuccess) {
        cudaGetLastError();
        return kx_set_error(ctx, KX_ENOMEM, "kernel table allocation failed");
    }
    *bytes += (long long)(sizeof(T) * count);
    return KX_OK;
}

// Grid of Appendix A at scale factor a (host, FP64, no FMA): p = q/a,
// E = sqrt(p^2 + m^2), trapezoid widths Dq, Dp = Dq/a, dE = p Dp/E, h = p^2 Dp.
static void kx_grid_host(kx_kernel *k, const double *q, double a, double mass) {
    const int n = k->n;
    k->p.resize(n); k->E.resize(n); k->dp.resize(n); k->dE.resize(n); k->h.resize(n);
    for (int i = 0; i < n; ++i) {
        double dq;
        if (i == 0) dq = (q[1] - q[0]) / 2.0;
        else if (i == n - 1) dq = (q[n - 1] - q[n - 2]) / 2.0;
        else dq = (q[i + 1] - q[i - 1]) / 2.0;
        k->p[i] = q[i] / a;
        k->E[i] = sqrt(k->p[i] * k->p[i] + mass * mass);
        k->dp[i] = dq / a;
        k->dE[i] = k->p[i] * k->dp[i] / k->E[i];
        k->h[i] = k->p[i] * k->p[i] * k->dp[i];
    }
}

static int kx_build_kernel_ex(kx_ctx *ctx, const kx_grid_desc *d, kx_kernel **out, bool rescalable);

extern "C" int kx_build_kernel(kx_ctx *ctx, const kx_grid_desc *d, kx_kernel **out) {
    return kx_build_kernel_ex(ctx, d, out, false);
}

// rescalable: a kernel rebuilt in place at other scale factors (kx_kernel_rescale)
static int kx_build_kernel_ex(kx_ctx *ctx, const kx_grid_desc *d, kx_kernel **out, bool rescalable) {
    kx_nvtx range_("kx_build_kernel");
    if (!ctx || !d || !out) return KX_EINVAL;
    *out = nullptr;
    const int n = d->n;
    if (n < 4 || n > KX_MAX_N || !d->q) return kx_set_error(ctx, KX_EINVAL, "n must be in [4, 512]");
    if (!(d->a > 0) || !(d->mass > 0)) return kx_set_error(ctx, KX_EINVAL, "a and mass must be > 0");
    if (d->n_mu < 0 || d->n_mu > KX_MAX_NMU)
        return kx_set_error(ctx, KX_EINVAL, "n_mu in [1, 64], or 0 for the exact angular kernel");
    if (d->measure != KX_MEASURE_ENERGY && d->measure != KX_MEASURE_LITERAL)
        return kx_set_error(ctx, KX_EINVAL, "unknown measure");
    if (d->stats < -1 || d->stats > 1) return kx_set_error(ctx, KX_EINVAL, "stats in {-1, 0, +1}");
    if (d->stats != 0 && d->precision == KX_SPLIT_TF32 && d->loss_terms != 0)
        return kx_set_error(ctx, KX_ENOTSUP, "quantum statistics on the split path: exact loss only");
    if (d->loss_terms != 0 && d->precision != KX_SPLIT_TF32)
        return kx_set_error(ctx, KX_ENOTSUP, "the Chebyshev loss GEMM: KX_SPLIT_TF32 path only");
    if (d->loss_terms != 0 && d->loss_terms != 8 && d->loss_terms != 16 && d->loss_terms != 32)
        return kx_set_error(ctx, KX_EINVAL, "loss_terms must be 0, 8, 16 or 32");
    if (d->precision != KX_FP64 && d->precision != KX_FP32 && d->precision != KX_SPLIT_TF32)
        return kx_set_error(ctx, KX_ENOTSUP, "precision not available in this library");
    for (int i = 0; i < n; ++i) {
        if (!(d->q[i] > 0) || !isfinite(d->q[i]))
            return kx_set_error(ctx, KX_EINVAL, "q must be finite and > 0");
        if (i && !(d->q[i] > d->q[i - 1]))
            return kx_set_error(ctx, KX_EINVAL, "q must be strictly ascending");
    }
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    kx_kernel *k = new (std::nothrow) kx_kernel();
    if (!k) return KX_ENOMEM;
    k->refcount = 1;
    k->device = ctx->device;
    k->n = n;
    k->n_mu = d->n_mu;
    k->stats = d->stats;
    k->measure = d->measure;
    k->precision = d->precision;
    k->cheb_K = d->precision == KX_SPLIT_TF32 ? d->loss_terms : 0;
    k->a = d->a;
    k->mass = d->mass;
    k->P = (long long)n * (n + 1) / 2;
    k->bytes = 0;
    k->rescalable = rescalable;
    // grid (Appendix A; trapezoid widths in q)
    k->q.assign(d->q, d->q + n);
    kx_grid_host(k, d->q, d->a, d->mass);
    std::vector<uint32_t> pair;
    pair.reserve(k->P);
    for (int a = 0; a < n; ++a)
        for (int b = a; b < n; ++b) pair.push_back((uint32_t)a | ((uint32_t)b << 16));
    std::vector<uint32_t> vt;
    for (int a = 0; a < n; ++a)
        for (int m0 = a; m0 < n; m0 += 4) vt.push_back((uint32_t)a | ((uint32_t)m0 << 16));
    k->V = (int)vt.size();

    int rc = KX_OK;
    long long *by = &k->bytes;
    cudaStream_t s = ctx->stream;
#define KX_ALLOC(ptr, cnt)                                 \
    if ((rc = kx_dev_alloc(ctx, &ptr, cnt, by)) != KX_OK) { \
        kx_free_kernel(k);                                  \
        return rc;                                          \
    }
    KX_ALLOC(k->d_p, n); KX_ALLOC(k->d_E, n); KX_ALLOC(k->d_dp, n); KX_ALLOC(k->d_dE, n);
    KX_ALLOC(k->d_h, n);
    KX_ALLOC(k->d_pair, k->P);
    KX_ALLOC(k->d_W64, (size_t)n * k->P);
    KX_ALLOC(k->d_om64, (size_t)n * k->P);
    KX_ALLOC(k->d_jl, (size_t)n * k->P);
    uint32_t *d_vt_all = nullptr;   // FP32 build only: global vector list and row positions
    int *d_pos = nullptr, *d_rcnt = nullptr;
    if (k->precision == KX_FP32) {
        long long tmp = 0;
        if ((rc = kx_dev_alloc(ctx, &d_vt_all, k->V, &tmp)) != KX_OK ||
            (rc = kx_dev_alloc(ctx, &d_pos, (size_t)n * k->V, &tmp)) != KX_OK ||
            (rc = kx_dev_alloc(ctx, &d_rcnt, n, &tmp)) != KX_OK) {
            cudaFree(d_vt_all);
            cudaFree(d_pos);
            kx_free_kernel(k);
            return rc;
        }
    }
#undef KX_ALLOC
    unsigned long long *d_cnt = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto fail = [&](const char *what, cudaError_t e) {
        if (d_cnt) cudaFree(d_cnt);
        cudaFree(d_vt_all);
        cudaFree(d_pos);
        cudaFree(d_rcnt);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        kx_free_kernel(k);
        return kx_set_error(ctx, KX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
#define KX_CHK(what, expr) \
    if ((e = (expr)) != cudaSuccess) return fail(what, e);
    KX_CHK("upload grid", cudaMemcpyAsync(k->d_p, k->p.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    KX_CHK("upload grid", cudaMemcpyAsync(k->d_E, k->E.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    KX_CHK("upload grid", cudaMemcpyAsync(k->d_dp, k->dp.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    KX_CHK("upload grid", cudaMemcpyAsync(k->d_dE, k->dE.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    KX_CHK("upload grid", cudaMemcpyAsync(k->d_h, k->h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    KX_CHK("upload pairs", cudaMemcpyAsync(k->d_pair, pair.data(), sizeof(uint32_t) * k->P, cudaMemcpyHostToDevice, s));
    if (d_vt_all)
        KX_CHK("upload vectors", cudaMemcpyAsync(d_vt_all, vt.data(), sizeof(uint32_t) * k->V, cudaMemcpyHostToDevice, s));
    kx_gl_nodes &gl = k->gl;
    memset(&gl, 0, sizeof(gl));
    if (k->n_mu > 0) kx_gauss_legendre(k->n_mu, &gl);
    KX_CHK("event", cudaEventCreate(&e0));
    KX_CHK("event", cudaEventCreate(&e1));
    KX_CHK("malloc", cudaMalloc(&d_cnt, sizeof(unsigned long long)));
    KX_CHK("memset", cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), s));
    KX_CHK("event", cudaEventRecord(e0, s));
    KX_CHK("build", kx_launch_build_fp64(k, gl, s));
    if (k->precision == KX_FP32) {
        // rows compacted to the vectors inside the kinematic support
        KX_CHK("support", kx_launch_keep_scan(k, d_vt_all, k->V, d_pos, d_rcnt, s, rescalable));
        std::vector<int> rcnt(n);
        KX_CHK("copy", cudaMemcpyAsync(rcnt.data(), d_rcnt, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
        KX_CHK("sync", cudaStreamSynchronize(s));
        // streaming work: units of 32 x vpl vectors of a row (64 on grids up to
        // 160 points, 128 above); rows padded to whole units (zero weights), so
        // every unit is a full, 16-byte aligned block of each table.  The units
        // of all rows, in order, are cut into KX_BINS bins of equal size (fixed
        // per kernel, so the split does not depend on the device or the batch);
        // a bin's units within one row form one task with its own partial slot.
        k->vpl = n <= 160 ? 2 : 4;
        const int unit = 32 * k->vpl;
        std::vector<int> roff(n + 1, 0);
        for (int i = 0; i < n; ++i) roff[i + 1] = roff[i] + (rcnt[i] + unit - 1) / unit * unit;
        k->Vt = roff[n];
        std::vector<long long> uoff(n + 1, 0);   // first global unit of each row
        for (int i = 0; i < n; ++i) uoff[i + 1] = uoff[i] + (roff[i + 1] - roff[i]) / unit;
        const long long units = uoff[n];
        std::vector<int> bins(KX_BINS + 1, 0);
        std::vector<int4> task;
        std::vector<int> row_tasks(n, 0);
        int row = 0;
        for (int b = 0; b < KX_BINS; ++b) {
            bins[b] = (int)task.size();
            long long u0 = units * b / KX_BINS, u1 = units * (b + 1) / KX_BINS;
            while (u0 < u1) {
                while (uoff[row + 1] <= u0) ++row;
                const long long e = std::min(u1, uoff[row + 1]);
                task.push_back(make_int4(row, (int)(u0 - uoff[row]), (int)(e - uoff[row]), row_tasks[row]));
                ++row_tasks[row];
                u0 = e;
            }
        }
        bins[KX_BINS] = (int)task.size();
        k->bin_units = 0;
        for (int b = 0; b < KX_BINS; ++b) {
            int nu = 0;
            for (int t = bins[b]; t < bins[b + 1]; ++t) nu += task[t].z - task[t].y;
            k->bin_units = std::max(k->bin_units, nu);
        }
        // partial slots: MT per row (the largest task count, rounded up to
        // even), slot k of row i at k n + i: a row's slots sit at a fixed
        // stride and the rows of one slot index are adjacent (coalesced reads
        // in the row combine)
        int MT = 2;
        for (int i = 0; i < n; ++i) MT = std::max(MT, (row_tasks[i] + 1) & ~1);
        std::vector<int2> rtask(n);
        for (int i = 0; i < n; ++i) rtask[i] = make_int2(i, row_tasks[i]);
        for (auto &t : task) t.w = t.w * n + t.x;   // slot = index in the row x n + row
        k->ntask = (int)task.size();
        k->tslots = n * MT;
        long long *by2 = &k->bytes;
        if ((rc = kx_dev_alloc(ctx, &k->d_vt, k->Vt, by2)) != KX_OK ||
            (rc = kx_dev_alloc(ctx, &k->d_W32, (size_t)k->Vt * 4, by2)) != KX_OK ||
            (rc = kx_dev_alloc(ctx, &k->d_pk, (size_t)k->Vt * 4, by2)) != KX_OK ||
            (rc = kx_dev_alloc(ctx, &k->d_roff, n + 1, by2)) != KX_OK ||
            (rc = kx_dev_alloc(ctx, &k->d_rtask, n, by2)) != KX_OK ||
            (rc = kx_dev_alloc(ctx, &k->d_task, task.size(), by2)) != KX_OK ||
            (rc = kx_dev_alloc(ctx, &k->d_bins, KX_BINS + 1, by2)) != KX_OK) {
            cudaFree(d_cnt);
            cudaFree(d_vt_all);
            cudaFree(d_pos);
            cudaFree(d_rcnt);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            kx_free_kernel(k);
            return rc;
        }
        // padding vectors stay zero: (n, m0) = (0, 0), W = 0, pk = 0
        KX_CHK("clear", cudaMemsetAsync(k->d_vt, 0, sizeof(uint32_t) * k->Vt, s));
        KX_CHK("clear", cudaMemsetAsync(k->d_W32, 0, sizeof(float) * k->Vt * 4, s));
        KX_CHK("clear", cudaMemsetAsync(k->d_pk, 0, sizeof(uint32_t) * k->Vt * 4, s));
        KX_CHK("upload rows", cudaMemcpyAsync(k->d_roff, roff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
        KX_CHK("upload rows", cudaMemcpyAsync(k->d_rtask, rtask.data(), sizeof(int2) * n, cudaMemcpyHostToDevice, s));
        if (!task.empty())
            KX_CHK("upload tasks", cudaMemcpyAsync(k->d_task, task.data(), sizeof(int4) * task.size(), cudaMemcpyHostToDevice, s));
        KX_CHK("upload bins", cudaMemcpyAsync(k->d_bins, bins.data(), sizeof(int) * (KX_BINS + 1), cudaMemcpyHostToDevice, s));
        KX_CHK("pack", kx_launch_pack_fp32(k, d_vt_all, k->V, d_pos, s));
        ctx->launches += 1;
    }
    KX_CHK("event", cudaEventRecord(e1, s));
    KX_CHK("count", kx_launch_count_nnz(k, d_cnt, s));
    ctx->launches += k->precision == KX_FP32 ? 3 : 2;
    unsigned long long cnt = 0;
    KX_CHK("copy", cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    KX_CHK("sync", cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    k->build_ms = ms;
    k->nnz = (long long)cnt;
    cudaFree(d_cnt);
    if (rescalable) {   // kept for the rebuilds at other scale factors
        k->d_vt_all = d_vt_all;
        k->d_pos = d_pos;
    } else {
        cudaFree(d_vt_all);
        cudaFree(d_pos);
    }
    cudaFree(d_rcnt);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
#undef KX_CHK
    if (k->precision == KX_SPLIT_TF32) {
        int rc2 = kx_batch_build_tables(ctx, k);
        if (rc2) {
            kx_free_kernel(k);
            return rc2;
        }
    }
    if (k->precision == KX_FP32)
        k->stream_bytes = k->Vt * 36 + (long long)k->ntask * 16 + (long long)(n + 1) * 4 + (KX_BINS + 1) * 4;
    else if (k->precision == KX_FP64)
        k->stream_bytes = (long long)n * k->P * 18 + k->P * 4;
    else
        k->stream_bytes = (long long)((k->nis + 255) / 256) * std::min(4, k->nsubI) * 1024 * 8 *
                              (k->KBG + (k->cheb_K ? k->KBL : 0)) +
                          (k->cheb_K ? 0 : k->nlel * 8 + k->nseg * 8);
    if (k->precision != KX_FP64 && !rescalable) {
        // the FP32 and batched paths read only their own tables
        cudaFree(k->d_W64); k->d_W64 = nullptr;
        cudaFree(k->d_om64); k->d_om64 = nullptr;
        cudaFree(k->d_jl); k->d_jl = nullptr;
        k->bytes -= (long long)n * k->P * (8 + 8 + 2);
    }
    *out = k;
    return KX_OK;
}

extern "C" void kx_kernel_retain(kx_kernel *k) {
    if (k) __atomic_add_fetch(&k->refcount, 1, __ATOMIC_SEQ_CST);
}

extern "C" void kx_kernel_release(kx_kernel *k) {
    if (!k) return;
    if (__atomic_sub_fetch(&k->refcount, 1, __ATOMIC_SEQ_CST) == 0) kx_free_kernel(k);
}

extern "C" int kx_kernel_get_info(const kx_kernel *k, kx_kernel_info *info) {
    if (!k || !info) return KX_EINVAL;
    info->n = k->n;
    info->n_mu = k->n_mu;
    info->measure = k->measure;
    info->precision = k->precision;
    info->unique_elements = (long long)k->n * k->P;
    info->nonzero_elements = k->nnz;
    info->tensor_bytes = k->bytes;
    info->build_ms = k->build_ms;
    info->stream_bytes = k->stream_bytes;
    return KX_OK;
}

extern "C" int kx_kernel_grid(const kx_kernel *k, double *p, double *E, double *dp, double *dE,
                              double *h) {
    if (!k) return KX_EINVAL;
    size_t b = sizeof(double) * k->n;
    if (p) memcpy(p, k->p.data(), b);
    if (E) memcpy(E, k->E.data(), b);
    if (dp) memcpy(dp, k->dp.data(), b);
    if (dE) memcpy(dE, k->dE.data(), b);
    if (h) memcpy(h, k->h.data(), b);
    return KX_OK;
}

extern "C" int kx_kernel_row(const kx_kernel *k, int i, double *W, int *jL, double *omega) {
    if (!k || i < 0 || i >= k->n) return KX_EINVAL;
    if (!k->d_W64) return KX_ENOTSUP;
    if (cudaSetDevice(k->device) != cudaSuccess) return KX_ECUDA;
    const size_t P = k->P;
    if (W && cudaMemcpy(W, k->d_W64 + i * P, sizeof(double) * P, cudaMemcpyDeviceToHost) != cudaSuccess)
        return KX_ECUDA;
    if (omega && cudaMemcpy(omega, k->d_om64 + i * P, sizeof(double) * P, cudaMemcpyDeviceToHost) != cudaSuccess)
        return KX_ECUDA;
    if (jL) {
        std::vector<uint16_t> t(P);
        if (cudaMemcpy(t.data(), k->d_jl + i * P, sizeof(uint16_t) * P, cudaMemcpyDeviceToHost) != cudaSuccess)
            return KX_ECUDA;
        for (size_t e = 0; e < P; ++e) jL[e] = t[e];
    }
    return KX_OK;
}

// -------------------------------------------------------------- collision
static double kx_M2(double mass, double sigma) { return 64.0 * KX_PI_H * mass * mass * sigma; }

static int kx_check_batch(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma) {
    if (!ctx || !k || B < 1 || !sigma) return kx_set_error(ctx, KX_EINVAL, "bad batch arguments");
    if (k->device != ctx->device) return kx_set_error(ctx, KX_EINVAL, "kernel on another device");
    for (int b = 0; b < B; ++b)
        if (!(sigma[b] > 0) || !isfinite(sigma[b]))
            return kx_set_error(ctx, KX_EINVAL, "sigma must be finite and > 0");
    return KX_OK;
}

static int kx_collision_impl(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma,
                             const double *f_dev, double *C_dev, int project, kx_diag *diag,
                             size_t extra_offset) {
    cudaStream_t s = ctx->stream;
    kx_batch_views v;
    kx_carve_views(k, B, (char *)ctx->d_arena + extra_offset, &v);
    std::vector<double> M2(B);
    for (int b = 0; b < B; ++b) M2[b] = kx_M2(k->mass, sigma[b]);
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(v.M2, M2.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
    KX_CUDA_TRY(ctx, kx_views_clear(k, B, v, s));
    KX_CUDA_TRY(ctx, kx_launch_prep(k, B, f_dev, v, nullptr, s));
    if (kx_tune_contraction(k, B, f_dev, v, nullptr, s, &ctx->launches))
        return kx_set_error(ctx, KX_ECUDA, "contraction autotuning failed");
    KX_CUDA_TRY(ctx, kx_launch_contract(k, B, f_dev, v, nullptr, 1, s));
    // KX_FAULT=deverr: the flag a contraction sets when one of its bounded device
    // waits expires is set from the host instead (no wait is made to expire)
    if (kx_fault("deverr")) KX_CUDA_TRY(ctx, cudaMemsetAsync(v.err, 0x01, 1, s));
    KX_CUDA_TRY(ctx, kx_launch_finalize(k, B, f_dev, v, C_dev, project, diag != nullptr, s));
    ctx->launches += 3;
    if (diag) {
        KX_CUDA_TRY(ctx, cudaMemcpyAsync(diag, v.diag, sizeof(kx_diag) * B, cudaMemcpyDeviceToHost, s));
        KX_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        for (int b = 0; b < B; ++b)
            if (diag[b].status == KX_ETIMEOUT) return kx_set_error(ctx, KX_ETIMEOUT, "a bounded device wait of the contraction expired");
        for (int b = 0; b < B; ++b)
            if (diag[b].status != KX_OK) return KX_ENONFINITE;
    }
    return KX_OK;
}

extern "C" int kx_collision(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma,
                            const double *f_dev, double *C_dev, int project, kx_diag *diag) {
    kx_nvtx range_("kx_collision");
    int rc = kx_check_batch(ctx, k, B, sigma);
    if (rc) return rc;
    if (!f_dev || !C_dev) return kx_set_error(ctx, KX_EINVAL, "null device pointer");
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if ((rc = kx_arena_reserve(ctx, kx_views_bytes(k, B))) != KX_OK) return rc;
    return kx_collision_impl(ctx, k, B, sigma, f_dev, C_dev, project, diag, 0);
}

extern "C" int kx_collision_host(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma,
                                 const double *f_host, double *C_host, int project, kx_diag *diag) {
    kx_nvtx range_("kx_collision_host");
    int rc = kx_check_batch(ctx, k, B, sigma);
    if (rc) return rc;
    if (!f_host || !C_host) return kx_set_error(ctx, KX_EINVAL, "null host pointer");
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const size_t fb = kx_align(sizeof(double) * B * k->n);
    if ((rc = kx_arena_reserve(ctx, 2 * fb + kx_views_bytes(k, B))) != KX_OK) return rc;
    double *d_f = (double *)ctx->d_arena;
    double *d_C = (double *)((char *)ctx->d_arena + fb);
    cudaStream_t s = ctx->stream;
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(d_f, f_host, sizeof(double) * B * k->n, cudaMemcpyHostToDevice, s));
    if (kx_fault("nan")) KX_CUDA_TRY(ctx, cudaMemsetAsync(d_f, 0xff, sizeof(double), s));   // f[0][0] = NaN
    rc = kx_collision_impl(ctx, k, B, sigma, d_f, d_C, project, diag, 2 * fb);
    if (rc && rc != KX_ENONFINITE) return rc;
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(C_host, d_C, sizeof(double) * B * k->n, cudaMemcpyDeviceToHost, s));
    KX_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return rc;
}

// ------------------------------------------------------------ integration
struct kx_solve_layout {
    size_t views, f, k1, fp, st, src, shapes, mb, total;
};

static kx_solve_layout kx_layout_solve(const kx_kernel *k, int B, int n_shape_rows, bool own_f) {
    kx_solve_layout L;
    size_t o = 0;
    L.views = o; o += kx_align(kx_views_bytes(k, B));
    L.f = o; o += own_f ? kx_align(sizeof(double) * B * k->n) : 0;
    L.k1 = o; o += kx_align(sizeof(double) * B * k->n);
    L.fp = o; o += kx_align(sizeof(double) * B * k->n);
    L.st = o; o += kx_align(sizeof(kx_inst_state) * B);
    L.src = o; o += kx_align(sizeof(kx_src_dev) * B);
    L.shapes = o; o += kx_align(sizeof(double) * std::max(1, n_shape_rows) * k->n);
    L.mb = o; o += kx_align(sizeof(double) * 3 * B);
    L.total = o;
    return L;
}

static int kx_check_params(kx_ctx *ctx, const kx_solve_params *p) {
    if (!p) return kx_set_error(ctx, KX_EINVAL, "null params");
    if (!(p->rtol >= 0) || !(p->atol >= 0) || !(p->rtol + p->atol > 0))
        return kx_set_error(ctx, KX_EINVAL, "rtol/atol must be >= 0, not both 0");
    if (!(p->h0 > 0)) return kx_set_error(ctx, KX_EINVAL, "h0 must be > 0");
    if (p->max_attempts < 1) return kx_set_error(ctx, KX_EINVAL, "max_attempts must be >= 1");
    if (p->chains < 0 || p->chains > 2) return kx_set_error(ctx, KX_EINVAL, "chains must be 0, 1 or 2");
    return KX_OK;
}

// Normalised source shapes and per-instance source descriptors.
// hw: the weights that normalise the shapes (sum_j hw_j shape_j = 1); the
// kernel's h when null (the expanding universe passes the comoving q^2 Dq).
static int kx_sources_host(kx_ctx *ctx, const kx_kernel *k, int B, const kx_source *src, int nsets,
                           std::vector<kx_src_dev> &sd, std::vector<double> &shapes,
                           const double *hw = nullptr) {
    sd.assign(B, kx_src_dev());
    shapes.clear();
    const int n = k->n;
    if (src && nsets != 1 && nsets != B)
        return kx_set_error(ctx, KX_EINVAL, "n_src_sets must be 1 or batch");
    std::vector<long long> set_off;
    for (int s = 0; src && s < nsets; ++s) {
        const kx_source &S = src[s];
        if (S.n_src < 0 || S.n_src > KX_MAX_SRC)
            return kx_set_error(ctx, KX_EINVAL, "n_src must be in [0, 4]");
        if (S.n_src && (!S.shape || !S.rate || !S.tau || !S.t_on))
            return kx_set_error(ctx, KX_EINVAL, "null source array");
        set_off.push_back((long long)shapes.size());
        for (int r = 0; r < S.n_src; ++r) {
            double norm = 0.0;
            for (int j = 0; j < n; ++j) {
                double v = S.shape[(size_t)r * n + j];
                if (!(v >= 0) || !isfinite(v)) return kx_set_error(ctx, KX_EINVAL, "source shape must be >= 0");
                norm += (hw ? hw[j] : k->h[j]) * v;
            }
            if (!(norm > 0) || !(S.tau[r] > 0))
                return kx_set_error(ctx, KX_EINVAL, "source shape must have positive weight, tau > 0");
            for (int j = 0; j < n; ++j) shapes.push_back(S.shape[(size_t)r * n + j] / norm);
        }
    }
    for (int b = 0; b < B; ++b) {
        kx_src_dev &d = sd[b];
        d.t_off = -INFINITY;
        if (!src) continue;
        const int s = nsets == 1 ? 0 : b;
        const kx_source &S = src[s];
        d.n_src = S.n_src;
        d.shape_off = set_off[s];
        for (int r = 0; r < S.n_src; ++r) {
            d.rate[r] = S.rate[r];
            d.tau[r] = S.tau[r];
            d.t_on[r] = S.t_on[r];
            d.t_off = std::max(d.t_off, S.t_on[r] + S.tau[r] * log(1e12));
        }
    }
    if (shapes.empty()) shapes.push_back(0.0);
    return KX_OK;
}

struct kx_run {
    kx_batch_views v;
    kx_step_views sv;
    double *mb;
};

// offset: the run's place in the context arena (several runs side by side:
// the grouped solve); the arena must already hold offset + the run's bytes
// when offset > 0.
static int kx_setup_run(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma,
                        const kx_source *src, int nsets, const kx_solve_params *par,
                        const double *t0, const double *h0, double *f_dev, bool own_f,
                        kx_run *run, double **f_used, const double *src_weights = nullptr,
                        size_t offset = 0) {
    std::vector<kx_src_dev> sd;
    std::vector<double> shapes;
    int rc = kx_sources_host(ctx, k, B, src, nsets, sd, shapes, src_weights);
    if (rc) return rc;
    kx_solve_layout L = kx_layout_solve(k, B, (int)(shapes.size() / k->n) + 1, own_f);
    if (offset == 0 && (rc = kx_arena_reserve(ctx, L.total)) != KX_OK) return rc;
    if (offset + L.total > ctx->arena_bytes) return kx_set_error(ctx, KX_ENOMEM, "arena too small for the run");
    char *base = (char *)ctx->d_arena + offset;
    kx_carve_views(k, B, base + L.views, &run->v);
    kx_step_views &sv = run->sv;
    sv.f = own_f ? (double *)(base + L.f) : f_dev;
    sv.k1 = (double *)(base + L.k1);
    sv.fp = (double *)(base + L.fp);
    sv.st = (kx_inst_state *)(base + L.st);
    sv.src = (const kx_src_dev *)(base + L.src);
    sv.shapes = (const double *)(base + L.shapes);
    sv.rtol = par->rtol;
    sv.atol = par->atol;
    sv.h_min = par->h_min;
    sv.h_max = par->h_max > 0 ? par->h_max : INFINITY;
    sv.l1_tol = par->l1_tol;
    sv.max_attempts = par->max_attempts;
    sv.fixed = par->fixed_step;
    sv.check_every = par->check_every;
    sv.project = par->project;
    sv.hscale = 1.0;
    run->mb = (double *)(base + L.mb);
    *f_used = sv.f;
    std::vector<kx_inst_state> st(B);
    std::vector<double> M2(B);
    for (int b = 0; b < B; ++b) {
        memset(&st[b], 0, sizeof(kx_inst_state));
        st[b].t = t0 ? t0[b] : par->t0;
        st[b].h = h0 ? h0[b] : par->h0;
        st[b].t_end = par->t_end;
        st[b].l1 = INFINITY;
        st[b].done = !(st[b].t < st[b].t_end);
        M2[b] = kx_M2(k->mass, sigma[b]);
    }
    cudaStream_t s = ctx->stream;
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(sv.st, st.data(), sizeof(kx_inst_state) * B, cudaMemcpyHostToDevice, s));
    KX_CUDA_TRY(ctx, cudaMemcpyAsync((void *)sv.src, sd.data(), sizeof(kx_src_dev) * B, cudaMemcpyHostToDevice, s));
    KX_CUDA_TRY(ctx, cudaMemcpyAsync((void *)sv.shapes, shapes.data(), sizeof(double) * shapes.size(), cudaMemcpyHostToDevice, s));
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(run->v.M2, M2.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
    KX_CUDA_TRY(ctx, kx_views_clear(k, B, run->v, s));
    return KX_OK;
}

// One Heun attempt: contraction, stage 1, contraction, stage 2.  Inside a
// sequence (first = false for all but its first attempt) every launch may start
// early (programmatic dependent launch): each kernel waits for its predecessor
// before it reads the predecessor's outputs.
static cudaError_t kx_enqueue_attempt(const kx_kernel *k, int B, const kx_run &r, cudaStream_t s,
                                      bool first = true) {
    cudaError_t e;
    if ((e = kx_launch_contract(k, B, r.sv.f, r.v, r.sv.st, 1, s, !first)) != cudaSuccess) return e;
    if ((e = kx_launch_stage(k, B, r.v, r.sv, 1, s, true)) != cudaSuccess) return e;
    if ((e = kx_launch_contract(k, B, r.sv.fp, r.v, r.sv.st, 2, s, true)) != cudaSuccess) return e;
    return kx_launch_stage(k, B, r.v, r.sv, 2, s, true);
}

static int kx_collect(kx_ctx *ctx, const kx_kernel *k, int B, const kx_run &r, kx_result *res,
                      double *t_out, double *h_out, double latency) {
    cudaStream_t s = ctx->stream;
    std::vector<kx_inst_state> st(B);
    std::vector<double> mb(3 * B);
    KX_CUDA_TRY(ctx, kx_launch_mbfit(k, B, r.sv.f, r.mb, s, r.sv.st, nullptr));
    ctx->launches += 1;
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(st.data(), r.sv.st, sizeof(kx_inst_state) * B, cudaMemcpyDeviceToHost, s));
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(mb.data(), r.mb, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, s));
    KX_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    int worst = KX_OK;
    for (int b = 0; b < B; ++b) {
        if (t_out) t_out[b] = st[b].t;
        if (h_out) h_out[b] = st[b].h;
        if (res) {
            kx_result &o = res[b];
            o.t = st[b].t;
            o.h = st[b].h;
            o.T_mb = mb[3 * b];
            o.ln_z_mb = mb[3 * b + 1];
            o.l1_to_mb = mb[3 * b + 2];
            o.steps = st[b].steps;
            o.rejects = st[b].rejects;
            o.evals = st[b].evals;
            o.status = st[b].status;
            o.converged = st[b].converged;
            o.latency_s = latency;
        }
        if (st[b].status != KX_OK && worst == KX_OK) worst = st[b].status;
    }
    return worst;
}

extern "C" int kx_step(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma,
                       const kx_source *src, int nsets, const kx_solve_params *par, double *t_host,
                       double *h_host, double *f_dev, kx_result *res) {
    kx_nvtx range_("kx_step");
    int rc = kx_check_batch(ctx, k, B, sigma);
    if (rc) return rc;
    if ((rc = kx_check_params(ctx, par)) != KX_OK) return rc;
    if (!t_host || !h_host || !f_dev) return kx_set_error(ctx, KX_EINVAL, "null t/h/f");
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    kx_run r;
    double *f = nullptr;
    if ((rc = kx_setup_run(ctx, k, B, sigma, src, nsets, par, t_host, h_host, f_dev, false, &r, &f)))
        return rc;
    (void)f;
    r.sv.max_attempts = (long long)1 << 62;
    cudaStream_t s = ctx->stream;
    KX_CUDA_TRY(ctx, kx_launch_prep(k, B, r.sv.f, r.v, r.sv.st, s));
    KX_CUDA_TRY(ctx, kx_enqueue_attempt(k, B, r, s));
    ctx->launches += 5;
    return kx_collect(ctx, k, B, r, res, t_host, h_host, 0.0);
}

// Device-resident integration: G attempts per captured graph; the host keeps
// one graph in flight ahead of the status word it reads (bounded wall time).
// A captured graph of G attempts of run r.
static cudaError_t kx_capture_attempts(const kx_kernel *k, int B, const kx_run &r, int G, cudaGraph_t *gr,
                                       cudaGraphExec_t *ex) {
    cudaStream_t cap = nullptr;
    cudaError_t x = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (x == cudaSuccess) x = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (x == cudaSuccess) {
        for (int a = 0; a < G && x == cudaSuccess; ++a) x = kx_enqueue_attempt(k, B, r, cap, a == 0);
        cudaError_t x2 = cudaStreamEndCapture(cap, gr);
        if (x == cudaSuccess) x = x2;
    }
    if (x == cudaSuccess) x = cudaGraphInstantiate(ex, *gr, 0);
    if (cap) cudaStreamDestroy(cap);
    return x;
}

// Prepares a run's graph of G attempts on stream s: f's tables, the FP32
// streaming variant (tuned in place when the size has no choice yet, unless
// tune is false), the split path's launch choices, then the capture (not when
// capture is false: the caller captures).  *launched: graph replays the tuning
// made (real attempts of this run).
static int kx_run_prepare(kx_ctx *ctx, const kx_kernel *k, int B, const kx_run &r, cudaStream_t s, int G,
                          cudaGraph_t *graph_out, cudaGraphExec_t *exec_out, long long *launched,
                          bool tune = true, bool capture_graph = true) {
    KX_CUDA_TRY(ctx, kx_launch_prep(k, B, r.sv.f, r.v, r.sv.st, s));
    ctx->launches += 1;
    // The FP32 path's streaming variant: tuned here, on this solve's own
    // attempt graphs (one captured per candidate, replayed in turn on real
    // attempts, the fastest kept), when the size has no choice yet.  The
    // variants give the same bits, so the trajectory does not depend on the
    // order of the replays.  A stand-in predecessor does not rank them the way
    // the stages between contractions do.
    int cand[8], nc = 0;
    if (tune && !kx_stream_is_tuned(k, B, r.v.grid_div, r.v.tune_tag))
        nc = kx_stream_candidate_list(k, B, r.v.grid_div, cand);
    if (tune && nc <= 1 && kx_tune_contraction(k, B, r.sv.f, r.v, r.sv.st, s, &ctx->launches))
        return kx_set_error(ctx, KX_ECUDA, "contraction autotuning failed");
    if (k->precision == KX_SPLIT_TF32) {
        // one contraction outside the capture: the split path tunes its launch
        // choices on first use (the graph's first attempt recomputes it)
        KX_CUDA_TRY(ctx, kx_launch_contract(k, B, r.sv.f, r.v, r.sv.st, 1, s, false));
        ctx->launches += 3;
    }
    if (kx_fault("deverr")) KX_CUDA_TRY(ctx, cudaMemsetAsync(r.v.err, 0x01, 1, s));   // as in kx_collision
    if (!capture_graph) return KX_OK;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto capture = [&](cudaGraph_t *gr, cudaGraphExec_t *ex) { return kx_capture_attempts(k, B, r, G, gr, ex); };
    cudaError_t e = cudaSuccess;
    if (nc > 1) {
        cudaGraph_t gs[8] = {};
        cudaGraphExec_t xs[8] = {};
        const int rounds = 3;   // the first replays warm the graphs up (not timed)
        cudaEvent_t te[3][8][2] = {};
        for (int c = 0; c < nc && e == cudaSuccess; ++c) {
            kx_stream_pin(k, B, r.v.grid_div, r.v.tune_tag, cand[c]);
            e = capture(&gs[c], &xs[c]);
        }
        for (int rd = 0; rd < rounds && e == cudaSuccess; ++rd)
            for (int c = 0; c < nc && e == cudaSuccess; ++c) {
                if (rd > 0) {
                    e = cudaEventCreate(&te[rd][c][0]);
                    if (e == cudaSuccess) e = cudaEventCreate(&te[rd][c][1]);
                    if (e == cudaSuccess) e = cudaEventRecord(te[rd][c][0], s);
                }
                if (e == cudaSuccess) e = cudaGraphLaunch(xs[c], s);
                if (e == cudaSuccess && rd > 0) e = cudaEventRecord(te[rd][c][1], s);
                ++*launched;
                ctx->launches += 4LL * G;
            }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        int best = 0;
        float best_ms = 0.f;
        for (int c = 0; c < nc && e == cudaSuccess; ++c) {
            float ms = 0.f;
            for (int rd = 1; rd < rounds && e == cudaSuccess; ++rd) {
                float t = 0.f;
                e = cudaEventElapsedTime(&t, te[rd][c][0], te[rd][c][1]);
                if (rd == 1 || t < ms) ms = t;
            }
            if (e == cudaSuccess && (c == 0 || ms < best_ms)) {
                best_ms = ms;
                best = c;
            }
        }
        for (int rd = 0; rd < rounds; ++rd)
            for (int c = 0; c < nc; ++c)
                for (int q = 0; q < 2; ++q)
                    if (te[rd][c][q]) cudaEventDestroy(te[rd][c][q]);
        kx_stream_pin(k, B, r.v.grid_div, r.v.tune_tag, cand[best]);
        for (int c = 0; c < nc; ++c) {
            if (c == best) continue;
            if (xs[c]) cudaGraphExecDestroy(xs[c]);
            if (gs[c]) cudaGraphDestroy(gs[c]);
        }
        graph = gs[best];
        exec = xs[best];
    } else {
        e = capture(&graph, &exec);
    }
    if (e != cudaSuccess) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        return kx_set_error(ctx, KX_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    *graph_out = graph;
    *exec_out = exec;
    return KX_OK;
}

static int kx_solve_run(kx_ctx *ctx, const kx_kernel *k, int B, const kx_run &r,
                        const kx_solve_params *par, kx_result *res) {
    cudaStream_t s = ctx->stream;
    const auto t_start = std::chrono::steady_clock::now();
    const int G = 16;
    int rc = KX_OK;
    if ((rc = kx_pinned_reserve(ctx, 2 * sizeof(kx_inst_state) * (size_t)B)) != KX_OK) return rc;
    kx_inst_state *h_st = (kx_inst_state *)ctx->h_pinned;
    long long launched = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if ((rc = kx_run_prepare(ctx, k, B, r, s, G, &graph, &exec, &launched)) != KX_OK) return rc;
    cudaError_t e = cudaSuccess;
    // two status buffers / events: graph g+1 runs while the host reads graph g's status
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
    const long long max_launch = (long long)par->max_attempts / G + 2;
    const double wall_limit = 600.0;
    const bool fault_timeout = kx_fault("timeout");
    auto launch_one = [&](int slot) -> cudaError_t {
        cudaError_t x = cudaGraphLaunch(exec, s);
        if (x == cudaSuccess)
            x = cudaMemcpyAsync(h_st + (size_t)slot * B, r.sv.st, sizeof(kx_inst_state) * B,
                                cudaMemcpyDeviceToHost, s);
        if (x == cudaSuccess) x = cudaEventRecord(ev[slot], s);
        ++launched;
        ctx->launches += 4LL * G;
        return x;
    };
    e = launch_one(0);
    if (e == cudaSuccess && launched < max_launch) e = launch_one(1);
    for (long long g = 0; e == cudaSuccess; ++g) {
        const int slot = (int)(g & 1);
        for (;;) {  // bounded wait on the status copy of graph g
            if (fault_timeout) { rc = KX_ETIMEOUT; break; }
            cudaError_t q = cudaEventQuery(ev[slot]);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) { e = q; break; }
            double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            if (el > wall_limit) { rc = KX_ETIMEOUT; break; }
            std::this_thread::yield();
        }
        if (e != cudaSuccess || rc) break;
        bool all_done = true;
        for (int b = 0; b < B; ++b) all_done &= h_st[(size_t)slot * B + b].done != 0;
        if (all_done || launched >= max_launch) break;
        e = launch_one(slot);
    }
    cudaStreamSynchronize(s);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return kx_set_error(ctx, KX_ECUDA, std::string("solve loop: ") + cudaGetErrorString(e));
    const double latency = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    int worst = kx_collect(ctx, k, B, r, res, nullptr, nullptr, latency);
    if (rc) return rc;
    return worst;
}

// Whether kx_solve runs a batch as concurrent per-instance chains (the
// chains field of kx_solve_params).
#define KX_CHAINS_MAX 8
static bool kx_use_chains(const kx_kernel *k, int B, const kx_solve_params *par) {
    if (par->chains == 1 || B < 2) return false;
    if (par->chains == 2) return B <= KX_CHAINS_MAX;
    return k->precision == KX_FP32 && B <= 4;
}

// A small batch as concurrent chains: every instance its own run (arena
// region, state, captured graph of G attempts) on its own stream, each graph
// relaunched as its chain's status arrives (two in flight per chain).  The
// chains' kernels fill one another's dependency gaps: at N = 128 an attempt
// of a batch is a chain of four latency-bound kernels.  An instance's
// arithmetic does not depend on the batch it is launched with, so the results
// are those of the single-batch solve bit for bit.  f_dev: device [B][n] (in
// place); arena_base: the arena offset of the first chain's region.
static int kx_solve_chains(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma, const kx_source *src,
                           int nsets, const kx_solve_params *par, double *f_dev, kx_result *res,
                           size_t arena_base = 0) {
    const auto t_start = std::chrono::steady_clock::now();
    const int n = k->n, G = 16;
    int rc = KX_OK;
    const size_t per = kx_align(kx_layout_solve(k, 1, KX_MAX_SRC + 1, false).total);
    if ((rc = kx_arena_reserve(ctx, arena_base + per * B)) != KX_OK) return rc;
    std::vector<kx_run> runs(B);
    for (int b = 0; b < B; ++b) {
        double *f = nullptr;
        const kx_source *sb = src ? src + (nsets == B ? b : 0) : nullptr;
        // (the arena is reserved above: the region at offset 0 does not move it)
        if ((rc = kx_setup_run(ctx, k, 1, sigma + b, sb, sb ? 1 : 0, par, nullptr, nullptr, f_dev + (size_t)b * n,
                               false, &runs[b], &f, nullptr, arena_base + per * b)))
            return rc;
    }
    if ((rc = kx_pinned_reserve(ctx, 2 * sizeof(kx_inst_state) * (size_t)B)) != KX_OK) return rc;
    kx_inst_state *h_st = (kx_inst_state *)ctx->h_pinned;
    std::vector<cudaStream_t> cs(B, nullptr);
    std::vector<cudaGraph_t> graph(B, nullptr);
    std::vector<cudaGraphExec_t> exec(B, nullptr);
    std::vector<cudaEvent_t> ev(2 * B, nullptr);
    std::vector<long long> launched(B, 0), g(B, 0);
    std::vector<int> done(B, 0);
    std::vector<double> lat(B, 0.0);
    cudaEvent_t fork = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(fork, ctx->stream);   // after the runs' uploads
    for (int b = 0; b < B && e == cudaSuccess; ++b) {
        e = cudaStreamCreateWithFlags(&cs[b], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs[b], fork, 0);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[2 * b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[2 * b + 1], cudaEventDisableTiming);
    }
    // The streaming variant of chain launches has its own tuning key (the
    // chains share the GPU): when it has no choice yet, every candidate's
    // graphs of all chains are replayed together, in turn, and timed from the
    // first chain's start to the last chain's end; the fastest candidate's
    // graphs are kept.
    for (int b = 0; b < B; ++b) runs[b].v.tune_tag = B;
    int cand[8], nc = 0;
    if (!kx_stream_is_tuned(k, 1, 1, B)) nc = kx_stream_candidate_list(k, 1, 1, cand);
    for (int b = 0; b < B && e == cudaSuccess && rc == KX_OK; ++b)
        rc = kx_run_prepare(ctx, k, 1, runs[b], cs[b], G, &graph[b], &exec[b], &launched[b], nc <= 1, nc <= 1);
    if (nc > 1 && e == cudaSuccess && rc == KX_OK) {
        std::vector<cudaGraph_t> gx((size_t)nc * B, nullptr);
        std::vector<cudaGraphExec_t> xx((size_t)nc * B, nullptr);
        for (int c = 0; c < nc && e == cudaSuccess; ++c) {
            kx_stream_pin(k, 1, 1, B, cand[c]);
            for (int b = 0; b < B && e == cudaSuccess; ++b)
                e = kx_capture_attempts(k, 1, runs[b], G, &gx[(size_t)c * B + b], &xx[(size_t)c * B + b]);
        }
        const int rounds = 3;   // (the first round warms the graphs up: not timed)
        std::vector<cudaEvent_t> t0((size_t)rounds * nc, nullptr), t1((size_t)rounds * nc, nullptr);
        cudaEvent_t done_b = nullptr;
        cudaStream_t ts = nullptr;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done_b, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
        for (size_t j = 0; j < t0.size() && e == cudaSuccess; ++j) {
            e = cudaEventCreate(&t0[j]);
            if (e == cudaSuccess) e = cudaEventCreate(&t1[j]);
        }
        for (int b = 0; b < B && e == cudaSuccess; ++b) {   // after every chain's preparation
            e = cudaEventRecord(done_b, cs[b]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ts, done_b, 0);
        }
        for (int rd = 0; rd < rounds && e == cudaSuccess; ++rd)
            for (int c = 0; c < nc && e == cudaSuccess; ++c) {
                const size_t j = (size_t)rd * nc + c;
                e = cudaEventRecord(t0[j], ts);
                for (int b = 0; b < B && e == cudaSuccess; ++b) {
                    e = cudaStreamWaitEvent(cs[b], t0[j], 0);
                    if (e == cudaSuccess) e = cudaGraphLaunch(xx[(size_t)c * B + b], cs[b]);
                    if (e == cudaSuccess) e = cudaEventRecord(done_b, cs[b]);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(ts, done_b, 0);
                    ++launched[b];
                    ctx->launches += 4LL * G;
                }
                if (e == cudaSuccess) e = cudaEventRecord(t1[j], ts);
            }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ts);
        int best = 0;
        float best_ms = 0.f;
        for (int c = 0; c < nc && e == cudaSuccess; ++c) {
            float ms = 0.f;
            for (int rd = 1; rd < rounds && e == cudaSuccess; ++rd) {
                float t = 0.f;
                e = cudaEventElapsedTime(&t, t0[(size_t)rd * nc + c], t1[(size_t)rd * nc + c]);
                if (rd == 1 || t < ms) ms = t;
            }
            if (e == cudaSuccess && (c == 0 || ms < best_ms)) {
                best_ms = ms;
                best = c;
            }
        }
        for (size_t j = 0; j < t0.size(); ++j) {
            if (t0[j]) cudaEventDestroy(t0[j]);
            if (t1[j]) cudaEventDestroy(t1[j]);
        }
        if (done_b) cudaEventDestroy(done_b);
        if (ts) cudaStreamDestroy(ts);
        if (e == cudaSuccess) kx_stream_pin(k, 1, 1, B, cand[best]);
        for (int c = 0; c < nc; ++c)
            for (int b = 0; b < B; ++b) {
                const size_t j = (size_t)c * B + b;
                if (c == best && e == cudaSuccess) {
                    graph[b] = gx[j];
                    exec[b] = xx[j];
                } else {
                    if (xx[j]) cudaGraphExecDestroy(xx[j]);
                    if (gx[j]) cudaGraphDestroy(gx[j]);
                }
            }
    }
    const long long max_launch = (long long)par->max_attempts / G + 2;
    const double wall_limit = 600.0;
    const bool fault_timeout = kx_fault("timeout");
    auto launch_one = [&](int b, int slot) -> cudaError_t {
        cudaError_t x = cudaGraphLaunch(exec[b], cs[b]);
        if (x == cudaSuccess)
            x = cudaMemcpyAsync(h_st + 2 * (size_t)b + slot, runs[b].sv.st, sizeof(kx_inst_state),
                                cudaMemcpyDeviceToHost, cs[b]);
        if (x == cudaSuccess) x = cudaEventRecord(ev[2 * b + slot], cs[b]);
        ++launched[b];
        ctx->launches += 4LL * G;
        return x;
    };
    for (int b = 0; b < B && e == cudaSuccess && rc == KX_OK; ++b) {
        e = launch_one(b, 0);
        if (e == cudaSuccess && launched[b] < max_launch) e = launch_one(b, 1);
    }
    int remaining = B;
    while (remaining > 0 && e == cudaSuccess && rc == KX_OK) {
        bool progressed = false;
        for (int b = 0; b < B && e == cudaSuccess; ++b) {
            if (done[b]) continue;
            const int slot = (int)(g[b] & 1);
            const cudaError_t q = cudaEventQuery(ev[2 * b + slot]);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                e = q;
                break;
            }
            progressed = true;
            if (h_st[2 * (size_t)b + slot].done || launched[b] >= max_launch) {
                done[b] = 1;
                --remaining;
                lat[b] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
                continue;
            }
            e = launch_one(b, slot);
            ++g[b];
        }
        if (!progressed && e == cudaSuccess) {
            if (fault_timeout) rc = KX_ETIMEOUT;
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            if (el > wall_limit) rc = KX_ETIMEOUT;
            std::this_thread::yield();
        }
    }
    for (int b = 0; b < B; ++b)
        if (cs[b]) cudaStreamSynchronize(cs[b]);
    for (int b = 0; b < B; ++b) {
        if (exec[b]) cudaGraphExecDestroy(exec[b]);
        if (graph[b]) cudaGraphDestroy(graph[b]);
        if (cs[b]) cudaStreamDestroy(cs[b]);
    }
    for (auto x : ev)
        if (x) cudaEventDestroy(x);
    if (fork) cudaEventDestroy(fork);
    if (rc != KX_OK && rc != KX_ETIMEOUT) return rc;
    if (e != cudaSuccess) return kx_set_error(ctx, KX_ECUDA, std::string("solve chains: ") + cudaGetErrorString(e));
    int worst = KX_OK;
    for (int b = 0; b < B; ++b) {
        const int w = kx_collect(ctx, k, 1, runs[b], res ? res + b : nullptr, nullptr, nullptr,
                                 lat[b] > 0.0 ? lat[b]
                                              : std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
        if (w != KX_OK && worst == KX_OK) worst = w;
    }
    if (rc) return rc;
    return worst;
}

extern "C" int kx_solve(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma,
                        const kx_source *src, int nsets, const kx_solve_params *par, double *f_dev,
                        kx_result *res) {
    kx_nvtx range_("kx_solve");
    int rc = kx_check_batch(ctx, k, B, sigma);
    if (rc) return rc;
    if ((rc = kx_check_params(ctx, par)) != KX_OK) return rc;
    if (!f_dev) return kx_set_error(ctx, KX_EINVAL, "null f");
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (kx_use_chains(k, B, par)) return kx_solve_chains(ctx, k, B, sigma, src, nsets, par, f_dev, res);
    kx_run r;
    double *f = nullptr;
    if ((rc = kx_setup_run(ctx, k, B, sigma, src, nsets, par, nullptr, nullptr, f_dev, false, &r, &f)))
        return rc;
    return kx_solve_run(ctx, k, B, r, par, res);
}

extern "C" int kx_profile_attempts(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma,
                                   const kx_source *src, int nsets, const kx_solve_params *par, double *f_dev,
                                   int attempts, double *us) {
    kx_nvtx range_("kx_profile_attempts");
    int rc = kx_check_batch(ctx, k, B, sigma);
    if (rc) return rc;
    if ((rc = kx_check_params(ctx, par)) != KX_OK) return rc;
    if (!f_dev || !us || attempts < 1 || attempts > 100000)
        return kx_set_error(ctx, KX_EINVAL, "bad arguments");
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    kx_run r;
    double *f = nullptr;
    if ((rc = kx_setup_run(ctx, k, B, sigma, src, nsets, par, nullptr, nullptr, f_dev, false, &r, &f)))
        return rc;
    cudaStream_t s = ctx->stream;
    KX_CUDA_TRY(ctx, kx_launch_prep(k, B, r.sv.f, r.v, r.sv.st, s));
    ctx->launches += 1;
    // events between the attempts' four kernels, each launched in plain stream
    // order (no programmatic overlap): event j..j+1 brackets one kernel
    std::vector<cudaEvent_t> ev((size_t)attempts * 4 + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t j = 0; j < ev.size() && e == cudaSuccess; ++j) e = cudaEventCreate(&ev[j]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    for (int a = 0; a < attempts && e == cudaSuccess; ++a) {
        cudaEvent_t *q = ev.data() + (size_t)a * 4;
        e = kx_launch_contract(k, B, r.sv.f, r.v, r.sv.st, 1, s, false);
        if (e == cudaSuccess) e = cudaEventRecord(q[1], s);
        if (e == cudaSuccess) e = kx_launch_stage(k, B, r.v, r.sv, 1, s, false);
        if (e == cudaSuccess) e = cudaEventRecord(q[2], s);
        if (e == cudaSuccess) e = kx_launch_contract(k, B, r.sv.fp, r.v, r.sv.st, 2, s, false);
        if (e == cudaSuccess) e = cudaEventRecord(q[3], s);
        if (e == cudaSuccess) e = kx_launch_stage(k, B, r.v, r.sv, 2, s, false);
        if (e == cudaSuccess) e = cudaEventRecord(q[4], s);
        ctx->launches += 4;
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev.back());
    double sum[4] = {0.0, 0.0, 0.0, 0.0};
    for (int a = 0; a < attempts && e == cudaSuccess; ++a)
        for (int j = 0; j < 4 && e == cudaSuccess; ++j) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[(size_t)a * 4 + j], ev[(size_t)a * 4 + j + 1]);
            sum[j] += ms;
        }
    for (auto x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return kx_set_error(ctx, KX_ECUDA, std::string("profile: ") + cudaGetErrorString(e));
    for (int j = 0; j < 4; ++j) us[j] = 1e3 * sum[j] / attempts;
    return KX_OK;
}

extern "C" int kx_check_status(kx_ctx *ctx, int reset, int *checked, long long *failures, int *first_site,
                               long long *first_index) {
    if (!ctx || !checked || !failures || !first_site || !first_index) return KX_EINVAL;
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    KX_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    unsigned int a[3] = {0u, 0u, 0u}, b[3] = {0u, 0u, 0u};
    if (kx_chk_read_contract(a, reset != 0) || kx_chk_read_batch(b, reset != 0))
        return kx_set_error(ctx, KX_ECUDA, "check record");
    *checked = KX_CHECKED;
    *failures = (long long)a[0] + (long long)b[0];
    const unsigned int *first = a[0] ? a : b;
    *first_site = (int)first[1];
    *first_index = (long long)(int)first[2];
    return KX_OK;
}

extern "C" int kx_check_probe(kx_ctx *ctx, int index, int limit, int *result) {
    if (!ctx || !result || limit < 0) return KX_EINVAL;
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int *d = nullptr;
    KX_CUDA_TRY(ctx, cudaMalloc(&d, sizeof(int)));
    cudaError_t e = kx_launch_chk_probe(index, limit, d, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(result, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    ctx->launches += 1;
    if (e != cudaSuccess) return kx_set_error(ctx, KX_ECUDA, std::string("check probe: ") + cudaGetErrorString(e));
    return KX_OK;
}

extern "C" int kx_solve_host(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma,
                             const kx_source *src, int nsets, const kx_solve_params *par,
                             double *f_host, kx_result *res) {
    kx_nvtx range_("kx_solve_host");
    int rc = kx_check_batch(ctx, k, B, sigma);
    if (rc) return rc;
    if ((rc = kx_check_params(ctx, par)) != KX_OK) return rc;
    if (!f_host) return kx_set_error(ctx, KX_EINVAL, "null f");
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (kx_use_chains(k, B, par)) {
        // f at the start of the arena, the chains' regions after it
        const size_t fb = kx_align(sizeof(double) * B * k->n);
        const size_t per = kx_align(kx_layout_solve(k, 1, KX_MAX_SRC + 1, false).total);
        if ((rc = kx_arena_reserve(ctx, fb + per * B)) != KX_OK) return rc;
        double *f = (double *)ctx->d_arena;
        cudaStream_t s = ctx->stream;
        KX_CUDA_TRY(ctx, cudaMemcpyAsync(f, f_host, sizeof(double) * B * k->n, cudaMemcpyHostToDevice, s));
        if (kx_fault("nan")) KX_CUDA_TRY(ctx, cudaMemsetAsync(f, 0xff, sizeof(double), s));   // f[0][0] = NaN
        int rc2 = kx_solve_chains(ctx, k, B, sigma, src, nsets, par, f, res, fb);
        if (rc2 == KX_ECUDA || rc2 == KX_ETIMEOUT || rc2 == KX_ENOMEM || rc2 == KX_EINVAL) return rc2;
        KX_CUDA_TRY(ctx, cudaMemcpyAsync(f_host, f, sizeof(double) * B * k->n, cudaMemcpyDeviceToHost, s));
        KX_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        return rc2;
    }
    kx_run r;
    double *f = nullptr;
    if ((rc = kx_setup_run(ctx, k, B, sigma, src, nsets, par, nullptr, nullptr, nullptr, true, &r, &f)))
        return rc;
    cudaStream_t s = ctx->stream;
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(f, f_host, sizeof(double) * B * k->n, cudaMemcpyHostToDevice, s));
    if (kx_fault("nan")) KX_CUDA_TRY(ctx, cudaMemsetAsync(f, 0xff, sizeof(double), s));   // f[0][0] = NaN
    int rc2 = kx_solve_run(ctx, k, B, r, par, res);
    if (rc2 == KX_ECUDA || rc2 == KX_ETIMEOUT) return rc2;
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(f_host, f, sizeof(double) * B * k->n, cudaMemcpyDeviceToHost, s));
    KX_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return rc2;
}

// ------------------------------------------------------ uneven batch
// Device-resident integration of G batches on different grids (split-TF32
// kernels) as one sequence of grouped launches: per Heun stage one gain-GEMM
// launch and one loss-GEMM launch over the work items of all G kernels, the
// exact loss per kernel (Chebyshev path: the flagged instances only), and one
// stage launch over all instances; A attempts per captured graph.
extern "C" int kx_solve_grouped(kx_ctx *ctx, int G, const kx_kernel *const *ks, const int *B,
                                const double *const *sigma, const kx_solve_params *par, double *const *f_dev,
                                kx_result *const *res) {
    kx_nvtx range_("kx_solve_grouped");
    if (!ctx || G < 1 || G > 8 || !ks || !B || !sigma || !f_dev) return kx_set_error(ctx, KX_EINVAL, "bad arguments");
    int rc = kx_check_params(ctx, par);
    if (rc) return rc;
    if (par->fixed_step) return kx_set_error(ctx, KX_ENOTSUP, "grouped solve: adaptive steps only");
    for (int g = 0; g < G; ++g) {
        if ((rc = kx_check_batch(ctx, ks[g], B[g], sigma[g])) != KX_OK) return rc;
        if (!f_dev[g]) return kx_set_error(ctx, KX_EINVAL, "null f");
        if (ks[g]->precision != KX_SPLIT_TF32)
            return kx_set_error(ctx, KX_ENOTSUP, "grouped solve: KX_SPLIT_TF32 kernels");
    }
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    // one arena region per group
    std::vector<size_t> off(G + 1, 0);
    for (int g = 0; g < G; ++g) off[g + 1] = off[g] + kx_align(kx_layout_solve(ks[g], B[g], 1, false).total);
    if ((rc = kx_arena_reserve(ctx, off[G])) != KX_OK) return rc;
    std::vector<kx_run> runs(G);
    for (int g = 0; g < G; ++g) {
        double *f = nullptr;
        // (the first region sits at offset 0: reserved above, so no reallocation)
        if ((rc = kx_setup_run(ctx, ks[g], B[g], sigma[g], nullptr, 0, par, nullptr, nullptr, f_dev[g], false,
                               &runs[g], &f, nullptr, off[g])))
            return rc;
    }
    cudaStream_t s = ctx->stream;
    std::vector<const kx_batch_views *> vs(G);
    std::vector<const kx_step_views *> svs(G);
    std::vector<const kx_inst_state *> sts(G);
    for (int g = 0; g < G; ++g) {
        vs[g] = &runs[g].v;
        svs[g] = &runs[g].sv;
        sts[g] = runs[g].sv.st;
        KX_CUDA_TRY(ctx, kx_launch_prep(ks[g], B[g], runs[g].sv.f, runs[g].v, runs[g].sv.st, s));
        ctx->launches += 1;
    }
    // one timeout flag for the grouped launches, seen by every group's stage
    int *d_err = runs[0].v.err;
    for (int g = 1; g < G; ++g) runs[g].v.err = d_err;
    // side streams and events: the grids' exact loss kernels run side by side
    // (forked and joined inside the captured graph)
    struct side_t {
        std::vector<cudaStream_t> st;
        std::vector<cudaEvent_t> ev;
        ~side_t() {
            for (auto x : st)
                if (x) cudaStreamDestroy(x);
            for (auto x : ev)
                if (x) cudaEventDestroy(x);
        }
    } side;
    if (G > 1) {
        side.st.assign(G, nullptr);
        side.ev.assign(G + 1, nullptr);
        for (int g = 0; g < G; ++g) KX_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&side.st[g], cudaStreamNonBlocking));
        for (int g = 0; g <= G; ++g) KX_CUDA_TRY(ctx, cudaEventCreateWithFlags(&side.ev[g], cudaEventDisableTiming));
    }
    auto attempt = [&](cudaStream_t cs) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int stage = 1; stage <= 2 && e == cudaSuccess; ++stage) {
            // the contraction's input: f (stage 1) or the predictor f_p (stage 2),
            // prepared by the previous stage kernel
            e = kx_launch_batch_contract_grouped(G, ks, B, vs.data(), sts.data(), stage, d_err, cs,
                                                 G > 1 ? side.st.data() : nullptr, G > 1 ? side.ev.data() : nullptr);
            if (e == cudaSuccess) e = kx_launch_stage_grouped(G, ks, B, vs.data(), svs.data(), stage, cs);
        }
        return e;
    };
    const int A = 8;   // attempts per graph
    // one contraction outside the capture: the split path tunes its launch
    // choices on first use (the graph's first attempt recomputes it)
    KX_CUDA_TRY(ctx, kx_launch_batch_contract_grouped(G, ks, B, vs.data(), sts.data(), 1, d_err, s));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int a = 0; a < A && e == cudaSuccess; ++a) e = attempt(cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return kx_set_error(ctx, KX_ECUDA, std::string("grouped graph capture: ") + cudaGetErrorString(e));
    }
    int Btot = 0;
    for (int g = 0; g < G; ++g) Btot += B[g];
    if ((rc = kx_pinned_reserve(ctx, sizeof(kx_inst_state) * (size_t)Btot)) != KX_OK) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return rc;
    }
    kx_inst_state *h_st = (kx_inst_state *)ctx->h_pinned;
    const auto t_start = std::chrono::steady_clock::now();
    const long long max_launch = (long long)par->max_attempts / A + 2;
    for (long long launched = 0; e == cudaSuccess && launched < max_launch;) {
        e = cudaGraphLaunch(exec, s);
        ++launched;
        ctx->launches += (long long)A * (2 * (2 + G) + 2);
        for (int g = 0, o = 0; g < G && e == cudaSuccess; o += B[g], ++g)
            e = cudaMemcpyAsync(h_st + o, runs[g].sv.st, sizeof(kx_inst_state) * B[g], cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        bool all = true;
        for (int b = 0; b < Btot; ++b) all &= h_st[b].done != 0;
        if (all) break;
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() > 3600.0) {
            rc = KX_ETIMEOUT;
            break;
        }
    }
    cudaStreamSynchronize(s);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return kx_set_error(ctx, KX_ECUDA, std::string("grouped solve: ") + cudaGetErrorString(e));
    const double latency = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    int worst = KX_OK;
    for (int g = 0; g < G; ++g) {
        int w = kx_collect(ctx, ks[g], B[g], runs[g], res ? res[g] : nullptr, nullptr, nullptr, latency);
        if (w != KX_OK && worst == KX_OK) worst = w;
    }
    if (rc) return kx_set_error(ctx, rc, "grouped solve: wall-clock limit");
    return worst;
}

// ------------------------------------------------------ expanding universe
// Rebuilds a rescalable kernel in place at scale factor a (stream ordered):
// host grid, upload, FP64 tables, and for the FP32 path the uncompacted FP32
// tables (every vector kept, so the layout does not depend on the support).
static int kx_kernel_rescale(kx_ctx *ctx, kx_kernel *k, double a) {
    cudaStream_t s = ctx->stream;
    const int n = k->n;
    kx_grid_host(k, k->q.data(), a, k->mass);
    k->a = a;
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(k->d_p, k->p.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(k->d_E, k->E.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(k->d_dp, k->dp.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(k->d_dE, k->dE.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(k->d_h, k->h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    KX_CUDA_TRY(ctx, kx_launch_build_fp64(k, k->gl, s));
    ctx->launches += 1;
    if (k->precision == KX_FP32) {
        KX_CUDA_TRY(ctx, kx_launch_pack_fp32(k, k->d_vt_all, k->V, k->d_pos, s));
        ctx->launches += 1;
    }
    return KX_OK;
}

// H(u) = exp of the piecewise-linear interpolation of ln H (linear
// extrapolation beyond the table; constant for a single point)
static double kx_hubble(const kx_expansion *ex, double u) {
    if (ex->n_h == 1) return exp(ex->ln_H[0]);
    int k = 0;
    while (k + 2 < ex->n_h && u > ex->u[k + 1]) ++k;
    const double sl = (ex->ln_H[k + 1] - ex->ln_H[k]) / (ex->u[k + 1] - ex->u[k]);
    return exp(ex->ln_H[k] + sl * (u - ex->u[k]));
}

extern "C" int kx_solve_expanding(kx_ctx *ctx, const kx_grid_desc *grid, double sigma, const kx_source *src,
                                  const kx_expansion *ex, const kx_solve_params *par, double *f_dev,
                                  kx_expansion_result *res) {
    kx_nvtx range_("kx_solve_expanding");
    if (!ctx || !grid || !ex || !f_dev) return kx_set_error(ctx, KX_EINVAL, "null argument");
    int rc = kx_check_params(ctx, par);
    if (rc) return rc;
    if (grid->precision != KX_FP64 && grid->precision != KX_FP32)
        return kx_set_error(ctx, KX_ENOTSUP, "expanding universe: FP64 and FP32 paths");
    if (grid->stats != 0 || grid->loss_terms != 0)
        return kx_set_error(ctx, KX_ENOTSUP, "expanding universe: dilute statistics, exact loss");
    if (ex->n_h < 1 || !ex->ln_H || (ex->n_h > 1 && !ex->u) || !(ex->du_rk4 > 0) || ex->check_every < 1 ||
        !(ex->eps_switch >= 0) || !(ex->u_end >= ex->u0) || !isfinite(ex->u0) || !isfinite(ex->u_end))
        return kx_set_error(ctx, KX_EINVAL, "bad expansion description");
    for (int j = 0; j < ex->n_h; ++j) {
        if (!isfinite(ex->ln_H[j])) return kx_set_error(ctx, KX_EINVAL, "ln H must be finite");
        if (j && !(ex->u[j] > ex->u[j - 1])) return kx_set_error(ctx, KX_EINVAL, "u table must ascend");
    }
    if (!(sigma > 0) || !isfinite(sigma)) return kx_set_error(ctx, KX_EINVAL, "sigma must be finite and > 0");
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    kx_grid_desc d = *grid;
    d.a = exp(ex->u0);
    kx_kernel *k = nullptr;
    if ((rc = kx_build_kernel_ex(ctx, &d, &k, true)) != KX_OK) return rc;
    struct Guard {
        kx_kernel *k;
        double *nu;
        ~Guard() {
            if (nu) cudaFree(nu);
            kx_kernel_release(k);
        }
    } guard{k, nullptr};
    const int n = k->n;
    // comoving weights q^2 Dq (the h of a = 1) normalise the source shapes
    std::vector<double> hc(n);
    for (int i = 0; i < n; ++i) {
        const double dq = i == 0 ? (grid->q[1] - grid->q[0]) / 2.0
                                 : (i == n - 1 ? (grid->q[n - 1] - grid->q[n - 2]) / 2.0
                                               : (grid->q[i + 1] - grid->q[i - 1]) / 2.0);
        hc[i] = grid->q[i] * grid->q[i] * dq;
    }
    kx_solve_params pp = *par;
    pp.t0 = ex->u0;
    pp.t_end = ex->u_end;
    pp.fixed_step = 0;
    pp.l1_tol = 0.0;
    pp.check_every = 0;
    pp.project = 1;
    kx_run r;
    double *f = nullptr;
    if ((rc = kx_setup_run(ctx, k, 1, &sigma, src, src ? 1 : 0, &pp, nullptr, nullptr, f_dev, false, &r, &f,
                           hc.data())))
        return rc;
    if (cudaMalloc(&guard.nu, sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        return kx_set_error(ctx, KX_ENOMEM, "expanding universe: scratch allocation failed");
    }
    cudaStream_t s = ctx->stream;
    const double M2 = kx_M2(k->mass, sigma);
    std::vector<double> nu(n), fh(n);
    long long rk4 = 0, checks = 0;
    double gh = 0.0, u_switch = NAN;
    // Gamma_2->2 / H at u: the number-weighted loss rate of the operator at a(u)
    auto gamma_over_H = [&](double u, bool *over) -> int {
        int e = kx_kernel_rescale(ctx, k, exp(u));
        if (e) return e;
        KX_CUDA_TRY(ctx, kx_launch_loss_rate64(k, f, guard.nu, s));
        ctx->launches += 1;
        KX_CUDA_TRY(ctx, cudaMemcpyAsync(nu.data(), guard.nu, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        KX_CUDA_TRY(ctx, cudaMemcpyAsync(fh.data(), f, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        KX_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        double num = 0.0, den = 0.0;
        for (int i = 0; i < n; ++i) {
            num += k->h[i] * fh[i] * nu[i];
            den += k->h[i] * fh[i];
        }
        gh = den > 0.0 ? M2 * num / den / kx_hubble(ex, u) : 0.0;
        ++checks;
        *over = gh > ex->eps_switch;
        return KX_OK;
    };
    // regime 1: the sources alone, RK4 on fixed intervals of u
    double u = ex->u0;
    bool sw = false;
    if ((rc = gamma_over_H(u, &sw))) return rc;
    if (sw) u_switch = u;
    while (!sw && u < ex->u_end) {
        // step k spans [u0 + k du, u0 + (k + 1) du], the last one clipped at u_end
        double dd = ex->du_rk4;
        u = ex->u0 + (double)rk4 * ex->du_rk4;
        if (u + dd >= ex->u_end) dd = ex->u_end - u;
        const double u1 = u + 0.5 * dd, u2 = u + dd;
        KX_CUDA_TRY(ctx, kx_launch_rk4_sources(k, f, r.sv.src, r.sv.shapes, u, dd, 1.0 / kx_hubble(ex, u),
                                               1.0 / kx_hubble(ex, u1), 1.0 / kx_hubble(ex, u2), s));
        ctx->launches += 1;
        u = (u + dd >= ex->u_end) ? ex->u_end : u + dd;
        ++rk4;
        if (rk4 % ex->check_every == 0) {
            if ((rc = gamma_over_H(u, &sw))) return rc;
            if (sw) u_switch = u;
        }
    }
    // regime 2: adaptive Heun in u with the collisions, the kernel rebuilt at
    // the scale factor of each evaluation
    kx_inst_state st;
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(&st, r.sv.st, sizeof(st), cudaMemcpyDeviceToHost, s));
    KX_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    st.t = u;
    st.done = !(sw && u < ex->u_end);
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(r.sv.st, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    const double h_max = par->h_max > 0 ? par->h_max : INFINITY;
    const auto t_start = std::chrono::steady_clock::now();
    while (!st.done) {
        double htry = st.h;
        if (htry > h_max) htry = h_max;
        if (htry < par->h_min) htry = par->h_min;
        if (st.t + htry >= st.t_end) htry = st.t_end - st.t;
        const double u1 = st.t, u2 = st.t + htry;
        for (int stage = 1; stage <= 2; ++stage) {
            const double us = stage == 1 ? u1 : u2;
            if ((rc = kx_kernel_rescale(ctx, k, exp(us)))) return rc;
            double *fin = stage == 1 ? r.sv.f : r.sv.fp;
            KX_CUDA_TRY(ctx, kx_launch_prep(k, 1, fin, r.v, r.sv.st, s));
            KX_CUDA_TRY(ctx, kx_launch_contract(k, 1, fin, r.v, r.sv.st, stage, s));
            r.sv.hscale = 1.0 / kx_hubble(ex, us);
            KX_CUDA_TRY(ctx, kx_launch_stage(k, 1, r.v, r.sv, stage, s));
            ctx->launches += 3;
        }
        KX_CUDA_TRY(ctx, cudaMemcpyAsync(&st, r.sv.st, sizeof(st), cudaMemcpyDeviceToHost, s));
        KX_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() > 3600.0)
            return kx_set_error(ctx, KX_ETIMEOUT, "expanding universe: wall-clock limit");
    }
    kx_result out;
    int worst = kx_collect(ctx, k, 1, r, &out, nullptr, nullptr, 0.0);
    if (res) {
        res->r = out;
        res->r.t = st.t > u ? st.t : u;
        res->u_switch = u_switch;
        res->gamma_over_H = gh;
        res->rk4_steps = rk4;
        res->checks = checks;
    }
    return worst;
}

extern "C" int kx_mb_fit(kx_ctx *ctx, const kx_kernel *k, int B, const double *f_dev, double *out) {
    if (!ctx || !k || B < 1 || !f_dev || !out) return KX_EINVAL;
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int rc = kx_arena_reserve(ctx, kx_align(sizeof(double) * 3 * B));
    if (rc) return rc;
    double *d = (double *)ctx->d_arena;
    KX_CUDA_TRY(ctx, kx_launch_mbfit(k, B, f_dev, d, ctx->stream));
    ctx->launches += 1;
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(out, d, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, ctx->stream));
    KX_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return KX_OK;
}

extern "C" int kx_wait_check(kx_ctx *ctx, long long cycles, int *expired_host) {
    if (!ctx || !expired_host || cycles < 1 || cycles > KX_WAIT_CYCLES_MAX)
        return kx_set_error(ctx, KX_EINVAL, "cycles must be in [1, 2^32]");
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int rc = kx_arena_reserve(ctx, kx_align(sizeof(int)));
    if (rc) return rc;
    int *d = (int *)ctx->d_arena;
    KX_CUDA_TRY(ctx, kx_launch_wait_check(cycles, d, ctx->stream));
    ctx->launches += 1;
    KX_CUDA_TRY(ctx, cudaMemcpyAsync(expired_host, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    KX_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return KX_OK;
}

// ---------------------------------------------------------------- profiling
extern "C" long long kx_launch_count(const kx_ctx *ctx) { return ctx ? ctx->launches : 0; }

extern "C" int kx_time_contraction(kx_ctx *ctx, const kx_kernel *k, int B, const double *f_dev,
                                   int iters, long long flush_bytes, double *avg_ms) {
    if (!ctx || !k || B < 1 || !f_dev || iters < 1 || !avg_ms || flush_bytes < 0) return KX_EINVAL;
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int rc = kx_arena_reserve(ctx, kx_views_bytes(k, B));
    if (rc) return rc;
    cudaStream_t s = ctx->stream;
    kx_batch_views v;
    kx_carve_views(k, B, ctx->d_arena, &v);
    void *flush = nullptr;
    if (flush_bytes > 0 && cudaMalloc(&flush, (size_t)flush_bytes) != cudaSuccess) {
        cudaGetLastError();
        return kx_set_error(ctx, KX_ENOMEM, "flush buffer");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = kx_views_clear(k, B, v, s);
    if (e == cudaSuccess) e = kx_launch_prep(k, B, f_dev, v, nullptr, s);
    ctx->launches += 1;
    if (e == cudaSuccess && kx_tune_contraction(k, B, f_dev, v, nullptr, s, &ctx->launches)) e = cudaErrorUnknown;
    double total = 0.0;
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        if (flush) e = cudaMemsetAsync(flush, it & 0xff, (size_t)flush_bytes, s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = kx_launch_contract(k, B, f_dev, v, nullptr, 1, s);
        ctx->launches += 1;
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        total += ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (flush) cudaFree(flush);
    if (e != cudaSuccess) return kx_set_error(ctx, KX_ECUDA, std::string("time contraction: ") + cudaGetErrorString(e));
    *avg_ms = total / iters;
    return KX_OK;
}

extern "C" int kx_time_collision(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma,
                                 const double *f_dev, double *C_dev, int project, int iters,
                                 double *avg_ms) {
    int rc = kx_check_batch(ctx, k, B, sigma);
    if (rc) return rc;
    if (!f_dev || !C_dev || iters < 1 || !avg_ms) return kx_set_error(ctx, KX_EINVAL, "bad arguments");
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if ((rc = kx_arena_reserve(ctx, kx_views_bytes(k, B))) != KX_OK) return rc;
    // one plain evaluation (uploads |M|^2, tunes the contraction), then the
    // same three launches captured once and replayed
    if ((rc = kx_collision_impl(ctx, k, B, sigma, f_dev, C_dev, project, nullptr, 0)) != KX_OK) return rc;
    cudaStream_t s = ctx->stream;
    KX_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    kx_batch_views v;
    kx_carve_views(k, B, ctx->d_arena, &v);
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = kx_launch_prep(k, B, f_dev, v, nullptr, cap);
        if (e == cudaSuccess) e = kx_launch_contract(k, B, f_dev, v, nullptr, 1, cap);
        if (e == cudaSuccess) e = kx_launch_finalize(k, B, f_dev, v, C_dev, project, 0, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);   // warm
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int it = 0; it < iters && e == cudaSuccess; ++it) e = cudaGraphLaunch(exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    ctx->launches += 3LL * (iters + 1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess)
        return kx_set_error(ctx, KX_ECUDA, std::string("time collision: ") + cudaGetErrorString(e));
    *avg_ms = (double)ms / iters;
    return KX_OK;
}

extern "C" int kx_time_contractions(kx_ctx *ctx, int nk, const kx_kernel *const *ks, int B,
                                    const double *f_dev, int iters, int pdl, double *avg_ms) {
    if (!ctx || nk < 1 || !ks || B < 1 || !f_dev || iters < 1 || !avg_ms) return KX_EINVAL;
    for (int i = 0; i < nk; ++i)
        if (!ks[i] || ks[i]->n != ks[0]->n) return KX_EINVAL;
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    std::vector<size_t> off(nk + 1, 0);
    for (int i = 0; i < nk; ++i) off[i + 1] = off[i] + kx_align(kx_views_bytes(ks[i], B));
    int rc = kx_arena_reserve(ctx, off[nk]);
    if (rc) return rc;
    cudaStream_t s = ctx->stream;
    std::vector<kx_batch_views> v(nk);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nk && e == cudaSuccess; ++i) {
        kx_carve_views(ks[i], B, (char *)ctx->d_arena + off[i], &v[i]);
        e = kx_views_clear(ks[i], B, v[i], s);
        if (e == cudaSuccess) e = kx_launch_prep(ks[i], B, f_dev, v[i], nullptr, s);
        ctx->launches += 1;
        if (e == cudaSuccess && kx_tune_contraction(ks[i], B, f_dev, v[i], nullptr, s, &ctx->launches))
            e = cudaErrorUnknown;
    }
    // one untimed pass, then iters passes over the kernels back to back
    for (int i = 0; i < nk && e == cudaSuccess; ++i, ++ctx->launches)
        e = kx_launch_contract(ks[i], B, f_dev, v[i], nullptr, 1, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int it = 0; it < iters && e == cudaSuccess; ++it)
        for (int i = 0; i < nk && e == cudaSuccess; ++i, ++ctx->launches)
            e = kx_launch_contract(ks[i], B, f_dev, v[i], nullptr, 1, s, pdl != 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess)
        return kx_set_error(ctx, KX_ECUDA, std::string("time contractions: ") + cudaGetErrorString(e));
    *avg_ms = (double)ms / ((double)iters * nk);
    return KX_OK;
}
