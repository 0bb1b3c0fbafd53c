// kx_batch.cu -- collision term for many distributions sharing one kernel.
//
// C_ib = G_ib - f_ib L_ib (Sec. 4.1, dilute), with
//   gain  G_ib = sum_{n,m} W_inm f_nb f_mb = sum_n f_nb T_(i n) b,  T = W_full F,
//   loss  L_ib = sum_{n<=m} S_inm f_t b (eq. app_log_interp),
// where W_full[(i n)][m] is the n <-> m symmetrised kernel as an (N^2 x N)
// matrix and F[m][b] the distributions.  T is a dense GEMM on the tcgen05
// tensor cores: TF32 operands split into hi + lo parts (hi*hi + hi*lo + lo*hi,
// relative error ~2^-21), FP32 accumulation in tensor memory.  The loss is not
// a GEMM (f_t is a log-interpolation, nonlinear in f): it is evaluated exactly
// with one exp2 per element and instance.  Both are scaled by f_max (per
// instance) and combined in FP64 by the row-combine/projection kernel.
#include <algorithm>
#include <numeric>
#include <cstring>
#include <vector>

#include "kx_internal.cuh"

#define KX_MMA_NT 64               // instances per MMA tile (the MMA's N)
#define KX_ATILE 4096              // floats per A tile: 128 rows x 32 k
#define KX_BTILE 2048              // floats per B tile: 64 rows x 32 k
#define KX_GEMM_SMEM (65536 + 32768 + 64)
#define KX_LOSS_WARPS 16           // warps per loss block (one shared instance table)

#include "kx_ptx.cuh"

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading-dimension
// byte offset >> 4 (16-29), stride-dimension byte offset >> 4 (32-45), the
// fixed 0b001 at bits 46-48, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t kx_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t kx_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void kx_mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void kx_mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void kx_tmem_ld16(uint32_t taddr, float *r) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) r[k] = __uint_as_float(v[k]);
}

__device__ __forceinline__ float kx_ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float kx_omega(uint32_t w) {
    return __uint_as_float(0x3f800000u | (w & 0x7fffffu)) - 1.0f;
}

// --------------------------------------------------------- gain GEMM (T)
// One CTA (4 warps) per (128-row M tile, 64-instance N tile).  Thread 0 stages
// the hi/lo operand tiles of each 32-wide k block with bulk copies into a
// two-stage ring (mbarrier transaction counts), issues the 3 x 4 MMAs of the
// block (M = 128, N = 64, K = 8 each) and commits them to the stage's
// completion barrier.  The accumulator (128 lanes x 64 FP32 columns of tensor
// memory) is read back by all four warps (warp w owns lanes 32w..32w+31).
__global__ void __launch_bounds__(128)
    k_gain_mma(const float *__restrict__ A, const float *__restrict__ Bt, float *__restrict__ T,
               int KB, int ldT, int *err) {
    extern __shared__ __align__(1024) unsigned char kx_gsm[];
    float *sA = reinterpret_cast<float *>(kx_gsm);                  // [2 stages][hi, lo][4096]
    float *sB = reinterpret_cast<float *>(kx_gsm + 65536);          // [2 stages][hi, lo][2048]
    uint64_t *bars = reinterpret_cast<uint64_t *>(kx_gsm + 98304);  // full[2], done[2]
    uint32_t *slot = reinterpret_cast<uint32_t *>(kx_gsm + 98304 + 32);
    int *okf = reinterpret_cast<int *>(kx_gsm + 98304 + 40);
    const int nt = blockIdx.x, mt = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float *Ab = A + (size_t)mt * KB * 2 * KX_ATILE;
    const float *Bb = Bt + (size_t)nt * KB * 2 * KX_BTILE;
    const uint32_t full0 = kx_smem_u32(&bars[0]), done0 = kx_smem_u32(&bars[2]);
    if (tid == 0) {
        for (int k = 0; k < 4; ++k) kx_mbar_init(kx_smem_u32(&bars[k]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *okf = 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
                         kx_smem_u32(slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    if (tid == 0) {
        constexpr uint32_t idesc = kx_idesc_tf32(128, KX_MMA_NT);
        int ok = 1;
        int issued = 0;   // k blocks whose copies were issued
        auto load = [&](int kb, int s) {
            const uint32_t bar = full0 + 8 * s;
            kx_mbar_expect_tx(bar, 2 * KX_ATILE * 4 + 2 * KX_BTILE * 4);
            kx_bulk_g2s(kx_smem_u32(sA + (2 * s) * KX_ATILE), Ab + (size_t)(2 * kb) * KX_ATILE,
                        KX_ATILE * 4, bar);
            kx_bulk_g2s(kx_smem_u32(sA + (2 * s + 1) * KX_ATILE),
                        Ab + (size_t)(2 * kb + 1) * KX_ATILE, KX_ATILE * 4, bar);
            kx_bulk_g2s(kx_smem_u32(sB + (2 * s) * KX_BTILE), Bb + (size_t)(2 * kb) * KX_BTILE,
                        KX_BTILE * 4, bar);
            kx_bulk_g2s(kx_smem_u32(sB + (2 * s + 1) * KX_BTILE),
                        Bb + (size_t)(2 * kb + 1) * KX_BTILE, KX_BTILE * 4, bar);
            issued = kb + 1;
        };
        load(0, 0);
        int committed = 0;  // k blocks whose MMAs were committed
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb & 1;
            if (kb + 1 < KB) {
                // the stage about to be refilled was read by the MMAs of block kb - 1
                if (kb >= 1 && !kx_mbar_wait(done0 + 8 * (s ^ 1), ((kb - 1) >> 1) & 1)) {
                    ok = 0;
                    break;
                }
                load(kb + 1, s ^ 1);
            }
            if (!kx_mbar_wait(full0 + 8 * s, (kb >> 1) & 1)) {
                ok = 0;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aH = kx_smem_u32(sA + (2 * s) * KX_ATILE);
            const uint32_t aL = kx_smem_u32(sA + (2 * s + 1) * KX_ATILE);
            const uint32_t bH = kx_smem_u32(sB + (2 * s) * KX_BTILE);
            const uint32_t bL = kx_smem_u32(sB + (2 * s + 1) * KX_BTILE);
#pragma unroll
            for (int step = 0; step < 4; ++step) {
                const uint32_t o = 256u * step;   // 8 TF32 = two 16-byte core-matrix columns
                kx_mma_tf32(tmem, kx_desc(aH + o, 128, 1024), kx_desc(bH + o, 128, 1024), idesc,
                            (kb | step) ? 1u : 0u);
                kx_mma_tf32(tmem, kx_desc(aH + o, 128, 1024), kx_desc(bL + o, 128, 1024), idesc, 1u);
                kx_mma_tf32(tmem, kx_desc(aL + o, 128, 1024), kx_desc(bH + o, 128, 1024), idesc, 1u);
            }
            kx_mma_commit(done0 + 8 * s);
            committed = kb + 1;
        }
        if (ok && !kx_mbar_wait(done0 + 8 * ((KB - 1) & 1), ((KB - 1) >> 1) & 1)) ok = 0;
        if (!ok) {
            // give outstanding copies and MMAs a bounded chance to land before the
            // shared memory and tensor memory are released
            for (int kb = committed; kb < issued; ++kb) kx_mbar_wait(full0 + 8 * (kb & 1), (kb >> 1) & 1);
            if (committed > 0)
                kx_mbar_wait(done0 + 8 * ((committed - 1) & 1), ((committed - 1) >> 1) & 1);
            *okf = 0;
            atomicExch(err, 1);
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (*okf) {
        const int row = mt * 128 + warp * 32 + lane;
        float *Tr = T + (size_t)row * ldT + (size_t)nt * KX_MMA_NT;
#pragma unroll
        for (int c = 0; c < KX_MMA_NT; c += 16) {
            float r[16];
            kx_tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
#pragma unroll
            for (int q = 0; q < 16; q += 4)
                *reinterpret_cast<float4 *>(Tr + c + q) = make_float4(r[q], r[q + 1], r[q + 2], r[q + 3]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------- exact loss
// One block per (row i, group of 32 instances); lane = instance.  The row's
// nonzero elements, sorted by bracket j_L, are split into 16 contiguous ranges
// (one per warp); each element's (S, j_L, omega) is warp-uniform.  A warp walks
// its range group by group (all elements of a group share j_L, so the lane's
// (l2_j, l2_{j+1} - l2_j) is read once per group) with a branch-free loop of
// four independent accumulators.  Per element and instance: one FMA for the
// interpolated exponent, one ex2, one FMA; group sums are added in FP64.  The
// block also forms the gain G_ib = sum_n f'_nb T_(i n) b from the GEMM output.
__global__ void __launch_bounds__(KX_LOSS_WARPS * 32)
    k_batch_loss(int n, int B, int Bpad, const uint2 *__restrict__ lel,
                 const int *__restrict__ lrow, const int *__restrict__ lgrp,
                 const float2 *__restrict__ td,
                 const float *__restrict__ fT, const float *__restrict__ T,
                 const double *__restrict__ fmax, double2 *__restrict__ partial,
                 const kx_inst_state *__restrict__ st, int stage) {
    extern __shared__ float2 kx_ltab[];   // [n][32]
    __shared__ double red[2][KX_LOSS_WARPS][32];
    const int i = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * 32 + lane;
    const bool act = b < B && !(st && (st[b].done || (stage == 2 && st[b].skip2)));
    if (!__syncthreads_or(act)) return;
    for (int j = warp; j < n; j += KX_LOSS_WARPS)
        kx_ltab[j * 32 + lane] = act ? td[(long long)b * n + j] : make_float2(-2000.f, 0.f);
    __syncthreads();
    const int e0 = lrow[i], e1 = lrow[i + 1];
    const int per = (e1 - e0 + KX_LOSS_WARPS - 1) / KX_LOSS_WARPS;
    const int ea = e0 + warp * per, eb = min(e1, ea + per);
    const int *gs = lgrp + (size_t)i * (n + 1);   // first element of each bracket group j
    double accd = 0.0;
    int e = ea;
    while (e < eb) {
        // one bracket group: (l2_j, l2_{j+1} - l2_j) of this lane's instance is fixed
        const int j = __ldg(&lel[e].y) >> 23;
        const int gend = min(eb, __ldg(gs + j + 1));
        const float2 t = kx_ltab[j * 32 + lane];
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (; e + 8 <= gend; e += 8) {
            uint2 x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = __ldg(lel + e + q);
#pragma unroll
            for (int q = 0; q < 8; q += 4) {
                a0 = fmaf(__uint_as_float(x[q].x), kx_ex2f(fmaf(kx_omega(x[q].y), t.y, t.x)), a0);
                a1 = fmaf(__uint_as_float(x[q + 1].x), kx_ex2f(fmaf(kx_omega(x[q + 1].y), t.y, t.x)), a1);
                a2 = fmaf(__uint_as_float(x[q + 2].x), kx_ex2f(fmaf(kx_omega(x[q + 2].y), t.y, t.x)), a2);
                a3 = fmaf(__uint_as_float(x[q + 3].x), kx_ex2f(fmaf(kx_omega(x[q + 3].y), t.y, t.x)), a3);
            }
        }
        for (; e < gend; ++e) {
            const uint2 x0 = __ldg(lel + e);
            a0 = fmaf(__uint_as_float(x0.x), kx_ex2f(fmaf(kx_omega(x0.y), t.y, t.x)), a0);
        }
        accd += (double)((a0 + a1) + (a2 + a3));
    }
    float g = 0.f;
    for (int nn = warp; nn < n; nn += KX_LOSS_WARPS)
        g = fmaf(fT[(size_t)nn * Bpad + b], T[((size_t)i * n + nn) * Bpad + b], g);
    red[0][warp][lane] = accd;
    red[1][warp][lane] = g;
    __syncthreads();
    if (warp == 0 && act) {
        double L = 0.0, G = 0.0;
#pragma unroll
        for (int w = 0; w < KX_LOSS_WARPS; ++w) {
            L += red[0][w][lane];
            G += red[1][w][lane];
        }
        const double fm = fmax[b];
        partial[(size_t)b * n + i] = make_double2(fm * fm * G, fm * L);
    }
}

void kx_batch_prepare() {
    cudaFuncSetAttribute(k_gain_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, KX_GEMM_SMEM);
    cudaFuncSetAttribute(k_batch_loss, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         KX_MAX_N * 32 * (int)sizeof(float2));
    cudaGetLastError();
}

cudaError_t kx_launch_batch_contract(const kx_kernel *k, int B, const kx_batch_views &v,
                                     const kx_inst_state *st, int stage, int *d_err,
                                     cudaStream_t s) {
    const int KB = k->Kpad / 32, MT = k->Mpad / 128, NT = v.Bpad / KX_MMA_NT;
    dim3 g1(NT, MT);
    k_gain_mma<<<g1, 128, KX_GEMM_SMEM, s>>>(k->d_Atile, v.bt, v.T, KB, v.Bpad, d_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g2((B + 31) / 32, k->n);
    k_batch_loss<<<g2, KX_LOSS_WARPS * 32, (size_t)k->n * 32 * sizeof(float2), s>>>(
        k->n, B, v.Bpad, k->d_lel, k->d_lrow, k->d_lgrp, v.td, v.fT, v.T, v.fmax, v.partial, st,
        stage);
    return cudaGetLastError();
}

// ------------------------------------------------------ host table build
// From the device FP64 tables (symmetrised S over n <= m, j_L, omega):
//  A tiles: W_full[(i n)][m] = S_inm / 2 (n != m), S_inn (n = m), TF32 hi/lo
//           (hi rounded to nearest TF32, lo = W - hi), in MMA operand tiles;
//  loss list: per row, the nonzero S with packed (j_L, omega) sorted by j_L
//           (omega rounding to 1 stored as (j_L + 1, 0), as in the FP32 path).
static float kx_tf32_round(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u += 0x1000u;            // round to nearest, ties away from zero, on the 13 dropped bits
    u &= 0xffffe000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

int kx_batch_build_tables(kx_ctx *ctx, kx_kernel *k) {
    const int n = k->n;
    const long long P = k->P;
    std::vector<double> W((size_t)n * P), om((size_t)n * P);
    std::vector<uint16_t> jl((size_t)n * P);
    if (cudaMemcpy(W.data(), k->d_W64, sizeof(double) * W.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(om.data(), k->d_om64, sizeof(double) * om.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(jl.data(), k->d_jl, sizeof(uint16_t) * jl.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return kx_set_error(ctx, KX_ECUDA, "batched build: table download failed");
    k->Mpad = ((n * n + 127) / 128) * 128;
    k->Kpad = ((n + 31) / 32) * 32;
    const int MT = k->Mpad / 128, KB = k->Kpad / 32;
    std::vector<float> At((size_t)MT * KB * 2 * KX_ATILE, 0.f);
    std::vector<uint2> lel;
    std::vector<int> lrow(n + 1, 0);
    std::vector<int> lgrp((size_t)n * (n + 1), 0);
    std::vector<long long> base(n);
    for (int a = 0; a < n; ++a) base[a] = (long long)a * n - (long long)a * (a - 1) / 2;
    std::vector<std::pair<uint32_t, uint32_t>> row;
    for (int i = 0; i < n; ++i) {
        row.clear();
        for (int a = 0; a < n; ++a) {
            for (int b = 0; b < n; ++b) {
                const int lo = a < b ? a : b, hi = a < b ? b : a;
                const size_t e = (size_t)i * P + base[lo] + (hi - lo);
                const double wf = lo == hi ? W[e] : 0.5 * W[e];
                const float w = (float)wf;
                const float wh = kx_tf32_round(w);
                const float wl = w - wh;
                const int r = i * n + a;
                const int mt = r / 128, rl = r % 128, kb = b / 32, kk = b % 32;
                const size_t t = ((size_t)mt * KB + kb) * 2;
                At[t * KX_ATILE + kx_tile_offset(rl, kk)] = wh;
                At[(t + 1) * KX_ATILE + kx_tile_offset(rl, kk)] = wl;
                if (a <= b && W[e] != 0.0) {
                    uint32_t j = jl[e];
                    double q = rint(om[e] * 8388608.0);
                    if (q >= 8388608.0) {
                        j += 1;
                        q = 0.0;
                    }
                    const float ws = (float)W[e];
                    uint32_t wb;
                    memcpy(&wb, &ws, 4);
                    row.push_back({wb, (j << 23) | (uint32_t)q});
                }
            }
        }
        std::stable_sort(row.begin(), row.end(), [](const std::pair<uint32_t, uint32_t> &x,
                                                    const std::pair<uint32_t, uint32_t> &y) {
            return (x.second >> 23) < (y.second >> 23);
        });
        const int row0 = (int)lel.size();
        size_t pos = 0;
        for (int j = 0; j <= n; ++j) {
            while (pos < row.size() && (int)(row[pos].second >> 23) < j) ++pos;
            lgrp[(size_t)i * (n + 1) + j] = row0 + (int)pos;
        }
        for (auto &p : row) lel.push_back(make_uint2(p.first, p.second));
        lrow[i + 1] = (int)lel.size();
    }
    if (lel.empty()) lel.push_back(make_uint2(0u, 0u));
    if (cudaMalloc(&k->d_Atile, sizeof(float) * At.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lel, sizeof(uint2) * lel.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lrow, sizeof(int) * lrow.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lgrp, sizeof(int) * lgrp.size()) != cudaSuccess) {
        cudaGetLastError();
        return kx_set_error(ctx, KX_ENOMEM, "batched build: allocation failed");
    }
    k->bytes += (long long)(sizeof(float) * At.size() + sizeof(uint2) * lel.size() +
                            sizeof(int) * (lrow.size() + lgrp.size()));
    if (cudaMemcpy(k->d_Atile, At.data(), sizeof(float) * At.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lel, lel.data(), sizeof(uint2) * lel.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lrow, lrow.data(), sizeof(int) * lrow.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lgrp, lgrp.data(), sizeof(int) * lgrp.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return kx_set_error(ctx, KX_ECUDA, "batched build: table upload failed");
    return KX_OK;
}
