// kx_noalloc.cu -- kx_collision_noalloc: the collision term without any
// device or host allocation inside the call.
//
// Some callers cannot allocate GPU memory at the moment they need the
// collision term: code running inside an allocator callback or a memory-pool
// hook, a host that has pre-reserved all device memory for itself, or an
// embedding runtime that forbids cudaMalloc after start-up.  kx_collision draws
// its scratch from a context arena that may grow with cudaMalloc; this entry
// point instead uses one fixed scratch array compiled into the library.
//
// The scratch array lives in device global memory, one copy per GPU that
// loads the library, and stays resident until the process exits.  Host code
// must not pass the array's name to a kernel (on the host that name is only a
// stand-in, not a device address); its device address is looked up once per
// device with cudaGetSymbolAddress, on the first call made on that device.
#include <math.h>

#include <mutex>
#include <string>
#include <vector>

#include "kx_internal.cuh"

// Maximum scratch of one call: 8 MiB.  A call needs the same scratch as
// kx_collision's arena (per instance: partial row sums plus the prepared
// distribution tables); this covers, e.g., 64 instances at n = 512 on the FP32
// path, or 15 instances at n = 512 on the FP64 path.
#define KX_NOALLOC_SCRATCH_BYTES (8u << 20)
#define KX_NOALLOC_MAX_BATCH 64
#define KX_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char kx_noalloc_scratch[KX_NOALLOC_SCRATCH_BYTES];

struct kx_noalloc_m2 {
    double m2[KX_NOALLOC_MAX_BATCH];
};

// Stores the per-instance |M|^2 into the scratch array's M2 slots (device code
// can name the array directly; the offset is relative to its start).
__global__ void k_noalloc_store_m2(kx_noalloc_m2 vals, int B, size_t m2_offset) {
    int b = threadIdx.x;
    if (b < B) reinterpret_cast<double *>(kx_noalloc_scratch + m2_offset)[b] = vals.m2[b];
}

static std::mutex kx_noalloc_mutex;
static void *kx_noalloc_addr[KX_NOALLOC_MAX_DEVICES];

// Device address of the scratch array on `device` (which must be current).
static int kx_noalloc_base(kx_ctx *ctx, int device, void **out) {
    if (device < 0 || device >= KX_NOALLOC_MAX_DEVICES)
        return kx_set_error(ctx, KX_EINVAL, "device index out of range for the fixed scratch");
    std::lock_guard<std::mutex> lock(kx_noalloc_mutex);
    if (!kx_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, kx_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return kx_set_error(ctx, KX_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") +
                                                   cudaGetErrorString(e));
        kx_noalloc_addr[device] = p;
    }
    *out = kx_noalloc_addr[device];
    return KX_OK;
}

extern "C" int kx_collision_noalloc(kx_ctx *ctx, const kx_kernel *k, int B,
                                    const double *sigma_host, const double *f_dev,
                                    double *C_dev, int project) {
    if (!ctx || !k || !sigma_host || !f_dev || !C_dev || B < 1)
        return kx_set_error(ctx, KX_EINVAL, "bad arguments");
    if (k->device != ctx->device) return kx_set_error(ctx, KX_EINVAL, "kernel on another device");
    if (B > KX_NOALLOC_MAX_BATCH)
        return kx_set_error(ctx, KX_EINVAL, "batch above the fixed-scratch limit of 64 instances");
    for (int b = 0; b < B; ++b)
        if (!(sigma_host[b] > 0) || !isfinite(sigma_host[b]))
            return kx_set_error(ctx, KX_EINVAL, "sigma must be finite and > 0");
    const size_t need = kx_views_bytes(k, B);
    if (need > KX_NOALLOC_SCRATCH_BYTES)
        return kx_set_error(ctx, KX_EINVAL,
                            "scratch of " + std::to_string(need) +
                                " bytes needed, above the fixed 8 MiB of kx_collision_noalloc; "
                                "use fewer instances per call");
    KX_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    void *base = nullptr;
    int rc = kx_noalloc_base(ctx, ctx->device, &base);
    if (rc) return rc;
    // Every scratch word a call reads is written earlier in the same call (the
    // prepared tables by the prep kernel, every partial by the contraction,
    // M2 below), except the flag a contraction sets when one of its bounded
    // device waits expires: that one is cleared here (a memset allocates
    // nothing), so that an expiry in one call is not reported by the next.
    kx_batch_views v;
    kx_carve_views(k, B, base, &v);
    KX_CUDA_TRY(ctx, cudaMemsetAsync(v.err, 0, sizeof(int), ctx->stream));
    kx_noalloc_m2 m2;
    for (int b = 0; b < KX_NOALLOC_MAX_BATCH; ++b)
        m2.m2[b] = b < B ? 64.0 * 3.14159265358979323846 * k->mass * k->mass * sigma_host[b] : 0.0;
    cudaStream_t s = ctx->stream;
    k_noalloc_store_m2<<<1, KX_NOALLOC_MAX_BATCH, 0, s>>>(m2, B,
                                                          (size_t)((char *)v.M2 - (char *)base));
    KX_CUDA_TRY(ctx, cudaGetLastError());
    KX_CUDA_TRY(ctx, kx_launch_prep(k, B, f_dev, v, nullptr, s));
    KX_CUDA_TRY(ctx, kx_launch_contract(k, B, f_dev, v, nullptr, 1, s));
    KX_CUDA_TRY(ctx, kx_launch_finalize(k, B, f_dev, v, C_dev, project, 0, s));
    ctx->launches += 4;
    return KX_OK;
}
