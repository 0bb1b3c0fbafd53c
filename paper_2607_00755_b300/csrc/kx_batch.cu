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

#define KX_ATILE (128 * KX_TILE_K)   // floats per A tile: 128 rows x 16 k
#define KX_BTILE (64 * KX_TILE_K)    // floats per B tile: 64 rows x 16 k
#define KX_SEG 64                  // elements per loss segment at most (one j_L)

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
// Packed pairs of FP32 values (.f32x2): the per-lane arithmetic is that of the
// scalar fma (round to nearest, no flush), two values per instruction.
__device__ __forceinline__ unsigned long long kx_pk2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 kx_upk2(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long kx_fma2(unsigned long long a, unsigned long long b,
                                                      unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// --------------------------------------------------------- gain GEMM (fused)
// One CTA (4 warps) per (128-row M tile of W_full, N tile of up to 256
// instances), two CTAs per SM.  Thread 0 stages the hi/lo operand tiles of each
// 16-wide k block with bulk copies into a two-stage ring (mbarrier transaction
// counts: the A tile and up to four 64-instance B tiles, which form one 256-row
// K-major operand), issues the 3 x 2 MMAs of the block (M = 128, N = NTc,
// K = 8 each) and commits them to the stage's completion barrier.  The accumulator
// (128 lanes x NTc FP32 columns of tensor memory) holds T = W_full F for the
// tile's rows (i, a); the epilogue forms the gain directly: each thread
// multiplies its row's T by f'_a (instance-minor f/f_max) into a shared-memory
// product matrix (128 instance columns at a time), and each column is summed
// over the rows of every grid point i the tile touches, giving one FP32 partial
// per (tile, i, instance):
//   Gp[(mt * segmax + i - i_first(mt)) * Bpad + b] = sum_{a in tile} f'_ab T_(i a) b,
// i_first(mt) = floor(128 mt / n).  T itself never reaches global memory.
#define KX_GN 256
#define KX_GSTAGE (2 * KX_ATILE * 4 + 2 * 4 * KX_BTILE * 4)   // A hi/lo 16 KB + B hi/lo 32 KB
#define KX_GAIN_SMEM(S) ((S) * KX_GSTAGE + 128)
#define KX_GP_LD 129                                          // product matrix: [128 cols][128 rows + 1]
static_assert(128 * KX_GP_LD * 4 <= 2 * KX_GSTAGE, "product matrix must fit in the stage buffers");

__host__ __device__ __forceinline__ int kx_gain_segmax(int n) { return 128 / n + 2; }

// S: stages of the copy ring.  Two stages and two CTAs per SM (one CTA's
// epilogue and copy waits overlap the other's MMAs) measured faster than four
// stages and one CTA per SM (0.273 vs 0.300 ms for the N = 192, B = 512
// contraction).
template <int S>
__global__ void __launch_bounds__(128, S == 2 ? 2 : 1)
    k_gain_fused(const float *__restrict__ A, const float *__restrict__ Bt,
                 const float *__restrict__ fT, float *__restrict__ Gp, int KB, int n, int Bpad,
                 int *err) {
    extern __shared__ __align__(1024) unsigned char kx_gsm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(kx_gsm + S * KX_GSTAGE);   // full[S], done[S]
    uint32_t *slot = reinterpret_cast<uint32_t *>(kx_gsm + S * KX_GSTAGE + 16 * S);
    int *okf = reinterpret_cast<int *>(kx_gsm + S * KX_GSTAGE + 16 * S + 8);
    const int nt = blockIdx.x, mt = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NTc = min(KX_GN, Bpad - nt * KX_GN);   // 64, 128, 192 or 256
    const int nsub = NTc >> 6;
    const float *Ab = A + (size_t)mt * KB * 2 * KX_ATILE;
    const uint32_t full0 = kx_smem_u32(&bars[0]), done0 = kx_smem_u32(&bars[S]);
    if (tid == 0) {
        for (int k = 0; k < 2 * S; ++k) kx_mbar_init(kx_smem_u32(&bars[k]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *okf = 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                         kx_smem_u32(slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    if (tid == 0) {
        const uint32_t idesc = kx_idesc_tf32(128, NTc);
        int ok = 1;
        int issued = 0;   // k blocks whose copies were issued
        auto stage_a = [&](int s) { return kx_gsm + (size_t)s * KX_GSTAGE; };
        auto stage_b = [&](int s) { return kx_gsm + (size_t)s * KX_GSTAGE + 2 * KX_ATILE * 4; };
        auto load = [&](int kb, int s) {
            const uint32_t bar = full0 + 8 * s;
            kx_mbar_expect_tx(bar, 2 * KX_ATILE * 4 + 2 * nsub * KX_BTILE * 4);
            unsigned char *a = stage_a(s), *bsm = stage_b(s);
            kx_bulk_g2s(kx_smem_u32(a), Ab + (size_t)(2 * kb) * KX_ATILE, KX_ATILE * 4, bar);
            kx_bulk_g2s(kx_smem_u32(a + KX_ATILE * 4), Ab + (size_t)(2 * kb + 1) * KX_ATILE, KX_ATILE * 4, bar);
            for (int j = 0; j < nsub; ++j) {
                const float *src = Bt + ((size_t)(nt * 4 + j) * KB + kb) * 2 * KX_BTILE;
                kx_bulk_g2s(kx_smem_u32(bsm + j * KX_BTILE * 4), src, KX_BTILE * 4, bar);
                kx_bulk_g2s(kx_smem_u32(bsm + 4 * KX_BTILE * 4 + j * KX_BTILE * 4), src + KX_BTILE,
                            KX_BTILE * 4, bar);
            }
            issued = kb + 1;
        };
        // blocks 0 .. S - 2 in flight before the first MMA; iteration kb refills
        // the stage of block kb - 1 with block kb + S - 1
        for (int kb = 0; kb < S - 1 && kb < KB; ++kb) load(kb, kb);
        int committed = 0;  // k blocks whose MMAs were committed
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb % S;
            if (kb + S - 1 < KB) {
                const int sr = (kb + S - 1) % S;
                // the stage about to be refilled was read by the MMAs of block kb - 1
                if (kb >= 1 && !kx_mbar_wait(done0 + 8 * sr, ((kb - 1) / S) & 1)) {
                    ok = 0;
                    break;
                }
                load(kb + S - 1, sr);
            }
            if (!kx_mbar_wait(full0 + 8 * s, (kb / S) & 1)) {
                ok = 0;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aH = kx_smem_u32(stage_a(s)), aL = aH + KX_ATILE * 4;
            const uint32_t bH = kx_smem_u32(stage_b(s)), bL = bH + 4 * KX_BTILE * 4;
#pragma unroll
            for (int step = 0; step < KX_TILE_K / 8; ++step) {
                const uint32_t o = 256u * step;   // 8 TF32 = two 16-byte core-matrix columns
                kx_mma_tf32(tmem, kx_desc(aH + o, 128, 512), kx_desc(bH + o, 128, 512), idesc,
                            (kb | step) ? 1u : 0u);
                kx_mma_tf32(tmem, kx_desc(aH + o, 128, 512), kx_desc(bL + o, 128, 512), idesc, 1u);
                kx_mma_tf32(tmem, kx_desc(aL + o, 128, 512), kx_desc(bH + o, 128, 512), idesc, 1u);
            }
            kx_mma_commit(done0 + 8 * s);
            committed = kb + 1;
        }
        if (ok && !kx_mbar_wait(done0 + 8 * ((KB - 1) % S), ((KB - 1) / S) & 1)) ok = 0;
        if (!ok) {
            // give outstanding copies and MMAs a bounded chance to land before the
            // shared memory and tensor memory are released
            for (int kb = committed; kb < issued; ++kb) kx_mbar_wait(full0 + 8 * (kb % S), (kb / S) & 1);
            if (committed > 0)
                kx_mbar_wait(done0 + 8 * ((committed - 1) % S), ((committed - 1) / S) & 1);
            *okf = 0;
            atomicExch(err, 1);
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = *okf != 0;
    const int nrows = n * n;
    const int rl = warp * 32 + lane, r = mt * 128 + rl;
    const bool rin = r < nrows;
    const float *frow = fT + (size_t)(rin ? r % n : 0) * Bpad + (size_t)nt * KX_GN;
    float *sP = reinterpret_cast<float *>(kx_gsm);   // free: every copy landed, every MMA completed
    const int segmax = kx_gain_segmax(n), i_first = (mt * 128) / n;
    for (int h0 = 0; h0 < NTc; h0 += 128) {
        const int hw = min(128, NTc - h0);
        if (ok) {
            // products f'_ab T_(i a) b of columns h0 .. h0 + hw - 1 into sP[col][row]
            for (int c = 0; c < hw; c += 16) {
                float t[16];
                kx_tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h0 + c), t);
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    const float4 f4 = rin ? __ldg(reinterpret_cast<const float4 *>(frow + h0 + c + q))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                    sP[(c + q) * KX_GP_LD + rl] = t[q] * f4.x;
                    sP[(c + q + 1) * KX_GP_LD + rl] = t[q + 1] * f4.y;
                    sP[(c + q + 2) * KX_GP_LD + rl] = t[q + 2] * f4.z;
                    sP[(c + q + 3) * KX_GP_LD + rl] = t[q + 3] * f4.w;
                }
            }
        }
        __syncthreads();
        // column sums over the rows of each grid point i in the tile (four
        // interleaved FP32 partial sums, combined pairwise)
        if (ok && tid < hw) {
            const float *pc = sP + tid * KX_GP_LD;
            for (int sg = 0; sg < segmax; ++sg) {
                const int i = i_first + sg;
                if (i >= n) break;
                const int r0 = max(mt * 128, i * n) - mt * 128, r1 = min(mt * 128 + 128, (i + 1) * n) - mt * 128;
                if (r0 >= r1) break;
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
                int rr = r0;
                for (; rr + 4 <= r1; rr += 4) {
                    a0 += pc[rr];
                    a1 += pc[rr + 1];
                    a2 += pc[rr + 2];
                    a3 += pc[rr + 3];
                }
                for (; rr < r1; ++rr) a0 += pc[rr];
                Gp[(size_t)(mt * segmax + sg) * Bpad + (size_t)nt * KX_GN + h0 + tid] = (a0 + a1) + (a2 + a3);
            }
        }
        __syncthreads();   // sP is refilled by the next half
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------- Chebyshev loss GEMM
// L'_ib = sum_c Lp[c][i][b],  Lp[c][i][b] = sum_{(j,k) in chunk c} M_k[i][j] Y'_k[j][b]
// (Y' = Y / f_max): the loss rate of the Chebyshev expansion of f_t as one
// split-TF32 GEMM, A = M (rows i, 128-row tiles), B = Y' (rows b, 64-row
// tiles), K = the flattened (j, k) index in 16-wide blocks, cut into lsk
// chunks of KC blocks (fixed by the kernel, so an instance's sums do not
// depend on the batch).  A work item is (row tile, instance tile of up to 256,
// chunk); the CTAs take work items round robin (persistent, one CTA per SM).
// Warp-specialised: warp 0 (one lane) stages the hi/lo tiles of each k block
// with bulk copies into an S-stage ring (full/empty mbarriers), warp 1 (one
// lane) issues the 3 x 2 MMAs of each block (hi*hi + hi*lo + lo*hi, K = 8 per
// MMA) into one of two tensor-memory accumulators and commits the block to the
// stage's empty barrier and the item to the accumulator's full barrier; warps
// 2-5 read the accumulator of the previous item (lane quarter = warp % 4) and
// store it as FP32 partials while the next item's MMAs run.  Every wait is
// bounded: on expiry the CTA sets *err, every role stops, copies and MMAs in
// flight get a bounded wait, and tensor memory is freed.
#define KX_LG_STAGES 4
#define KX_LG_SMEM (KX_LG_STAGES * KX_GSTAGE + 256)

// A bounded mbarrier wait that also gives up when another role of the CTA has
// given up (abort != 0); on its own expiry it raises abort and *err.
__device__ __forceinline__ bool kx_wait_role(uint32_t bar, uint32_t parity, volatile int *abort, int *err) {
    const long long t0 = clock64();
    for (;;) {
        if (kx_mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > KX_WAIT_CYCLES) {
            *abort = 1;
            atomicExch(err, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void kx_mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(192, 1)
    k_loss_gemm(const float *__restrict__ A, const float *__restrict__ Bt, float *__restrict__ Lp,
                int KB, int KC, int lsk, int MT, int NT, int Bpad, int n, int ncols, int *err) {
    constexpr int S = KX_LG_STAGES;
    extern __shared__ __align__(1024) unsigned char kx_lsm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(kx_lsm + S * KX_GSTAGE);   // full[S] empty[S] accf[2] acce[2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * S + 4);
    volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
    int *issued = reinterpret_cast<int *>(tslot + 2);          // [S] last round issued per stage (+1)
    int *seen = issued + S;                                     // [S] last round consumed per stage (+1)
    int *lastc = seen + S;                                      // rounds committed by the MMA thread
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t full0 = kx_smem_u32(&bars[0]), empty0 = kx_smem_u32(&bars[S]);
    const uint32_t accf0 = kx_smem_u32(&bars[2 * S]), acce0 = kx_smem_u32(&bars[2 * S + 2]);
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            kx_mbar_init(full0 + 8 * q, 1);
            kx_mbar_init(empty0 + 8 * q, 1);
            issued[q] = 0;
            seen[q] = 0;
        }
        for (int q = 0; q < 2; ++q) {
            kx_mbar_init(accf0 + 8 * q, 1);
            kx_mbar_init(acce0 + 8 * q, 4);   // one arrival per epilogue warp
        }
        *lastc = 0;
        *abort = 0;
        kx_fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(kx_smem_u32(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const int items = MT * NT * lsk;
    const int half = ncols >> 1;   // columns of one accumulator
    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            for (int w = blockIdx.x; w < items && !*abort; w += gridDim.x) {
                const int c = w % lsk, nt = (w / lsk) % NT, mt = w / (lsk * NT);
                const int kb0 = c * KC, kb1 = min(KB, kb0 + KC);
                const int nsub = min(KX_GN, Bpad - nt * KX_GN) >> 6;
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int q = it % S, round = it / S;
                    if (round > 0 && !kx_wait_role(empty0 + 8 * q, (round - 1) & 1, abort, err)) break;
                    const uint32_t bar = full0 + 8 * q;
                    kx_mbar_expect_tx(bar, 2 * KX_ATILE * 4 + 2 * nsub * KX_BTILE * 4);
                    unsigned char *sa = kx_lsm + (size_t)q * KX_GSTAGE, *sb = sa + 2 * KX_ATILE * 4;
                    const float *a = A + ((size_t)mt * KB + kb) * 2 * KX_ATILE;
                    kx_bulk_g2s(kx_smem_u32(sa), a, KX_ATILE * 4, bar);
                    kx_bulk_g2s(kx_smem_u32(sa + KX_ATILE * 4), a + KX_ATILE, KX_ATILE * 4, bar);
                    for (int j = 0; j < nsub; ++j) {
                        const float *src = Bt + ((size_t)(nt * 4 + j) * KB + kb) * 2 * KX_BTILE;
                        kx_bulk_g2s(kx_smem_u32(sb + j * KX_BTILE * 4), src, KX_BTILE * 4, bar);
                        kx_bulk_g2s(kx_smem_u32(sb + 4 * KX_BTILE * 4 + j * KX_BTILE * 4), src + KX_BTILE,
                                    KX_BTILE * 4, bar);
                    }
                    issued[q] = round + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, li = 0;
            for (int w = blockIdx.x; w < items && !*abort; w += gridDim.x, ++li) {
                const int c = w % lsk, nt = (w / lsk) % NT;
                const int kb0 = c * KC, kb1 = min(KB, kb0 + KC);
                const int NTc = min(KX_GN, Bpad - nt * KX_GN);
                const int buf = li & 1, use = li >> 1;
                if (use > 0 && !kx_wait_role(acce0 + 8 * buf, (use - 1) & 1, abort, err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(buf * half);
                const uint32_t idesc = kx_idesc_tf32(128, NTc);
                bool ok = true;
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int q = it % S, round = it / S;
                    if (!kx_wait_role(full0 + 8 * q, round & 1, abort, err)) {
                        ok = false;
                        break;
                    }
                    seen[q] = round + 1;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t aH = kx_smem_u32(kx_lsm + (size_t)q * KX_GSTAGE), aL = aH + KX_ATILE * 4;
                    const uint32_t bH = aH + 2 * KX_ATILE * 4, bL = bH + 4 * KX_BTILE * 4;
#pragma unroll
                    for (int step = 0; step < KX_TILE_K / 8; ++step) {
                        const uint32_t o = 256u * step;
                        kx_mma_tf32(d, kx_desc(aH + o, 128, 512), kx_desc(bH + o, 128, 512), idesc,
                                    (kb > kb0 || step) ? 1u : 0u);
                        kx_mma_tf32(d, kx_desc(aH + o, 128, 512), kx_desc(bL + o, 128, 512), idesc, 1u);
                        kx_mma_tf32(d, kx_desc(aL + o, 128, 512), kx_desc(bH + o, 128, 512), idesc, 1u);
                    }
                    kx_mma_commit(empty0 + 8 * q);
                    *lastc = it + 1;
                }
                if (!ok) break;
                kx_mma_commit(accf0 + 8 * buf);
            }
        }
    } else {
        const int qtr = warp & 3;   // tensor-memory lane quarter this warp may read
        int li = 0;
        for (int w = blockIdx.x; w < items; w += gridDim.x, ++li) {
            const int c = w % lsk, nt = (w / lsk) % NT, mt = w / (lsk * NT);
            const int NTc = min(KX_GN, Bpad - nt * KX_GN);
            const int buf = li & 1, use = li >> 1;
            bool ok = true;
            if (lane == 0) ok = kx_wait_role(accf0 + 8 * buf, use & 1, abort, err);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = mt * 128 + qtr * 32 + lane;
            float *dst = Lp + ((size_t)c * MT * 128 + row) * Bpad + (size_t)nt * KX_GN;
            for (int c0 = 0; c0 < NTc; c0 += 16) {
                float t[16];
                kx_tmem_ld16(tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(buf * half + c0), t);
                if (row < n) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4 *>(dst + c0 + q) = make_float4(t[q], t[q + 1], t[q + 2], t[q + 3]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) kx_mbar_arrive(acce0 + 8 * buf);
        }
    }
    __syncthreads();
    if (*abort && tid == 0) {
        // bounded waits for the copies and MMAs still in flight before the shared
        // and tensor memory are released
        for (int q = 0; q < S; ++q)
            if (issued[q] > seen[q]) kx_mbar_wait(full0 + 8 * q, (issued[q] - 1) & 1, 1ll << 24);
        if (*lastc > 0) {
            const int it = *lastc - 1;
            kx_mbar_wait(empty0 + 8 * (it % S), (it / S) & 1, 1ll << 24);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ------------------------------------------------------------- exact loss
// A row's nonzero elements are sorted by bracket j_L and cut into segments of at
// most 64 elements with one j_L each, zero-padded to a multiple of 4 (host
// build); an element is (S_inm, omega) as two floats.  One block per (group of 32 IPL instances, row); lane l holds
// instances l, l + 32, ... of the group.  The block loads its instances'
// (l2_j, D_j) tables once (IPL float2 per lane and j, read coalesced from the
// instance-minor td); the row's segments are dealt to the warps by the host,
// balanced by element count.  A warp
// loads a segment's elements with one coalesced load (the next segment's are in
// flight meanwhile) into its shared-memory slot, reads its (l2_j, D_j) once,
// and then per element and instance spends one FMA (interpolated exponent), one
// ex2 and one FMA (weight): the element's own decode is a broadcast read of two
// floats shared by the IPL instances.  The FP32 sums (four per instance) go
// into a double-float accumulator (exact TwoSum) after every 64 or more
// elements, FP64 across warps.  The block also
// adds up the gain G_ib from the fused GEMM's per-tile partials.  Rows are
// taken longest first (lorder) so that the short ones fill the tail.
__device__ __forceinline__ void kx_two_sum_f(float a, float b, float &s, float &e) {
    s = a + b;
    const float bv = s - a;
    e = (a - (s - bv)) + (b - bv);
}

template <int IPL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, (WARPS <= 16 && IPL <= 2) ? 2 : 1)
    k_batch_loss(int n, int B, int tds, int Bpad, const float2 *__restrict__ lel,
                 const int2 *__restrict__ lseg, const int *__restrict__ lsw,
                 const int *__restrict__ lorder, const float2 *__restrict__ td,
                 const float *__restrict__ Gp, const double *__restrict__ fmax,
                 double2 *__restrict__ partial,
                 const kx_inst_state *__restrict__ st, int stage,
                 const float *__restrict__ Lp, const int *__restrict__ cflag, int lsk, int MTL) {
    // [n][32][IPL] (l2_j, D_j) table; after the loss loop the same space holds
    // the cross-warp reduction [2][WARPS][32 IPL] doubles
    extern __shared__ __align__(16) float2 kx_ltab[];
    __shared__ __align__(16) float2 s_el[WARPS][KX_SEG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int b[IPL];
    bool act[IPL];
    bool any = false;
#pragma unroll
    for (int s = 0; s < IPL; ++s) {
        b[s] = blockIdx.x * (32 * IPL) + s * 32 + lane;
        act[s] = b[s] < B && !(st && (st[b[s]].done || (stage == 2 && st[b[s]].skip2)));
        any |= act[s];
    }
    if (!__syncthreads_or(any)) return;
    const int i = lorder[blockIdx.y];
    // Chebyshev loss (Lp non-null): the loss comes from the GEMM partials; the
    // exact loop runs only for a block holding an instance whose truncation
    // bound was exceeded (cflag), and only that instance takes its result
    bool exact = true;
    if (Lp) {
        bool fl = false;
#pragma unroll
        for (int s = 0; s < IPL; ++s) fl |= act[s] && cflag[b[s]] != 0;
        exact = __syncthreads_or(fl) != 0;
    }
    float hi[IPL], lo[IPL];
#pragma unroll
    for (int s = 0; s < IPL; ++s) hi[s] = lo[s] = 0.f;
    if (exact) {
        // layout: IPL = 1: float2 at [j][lane]; else float4 (two instances) at
        // [j][IPL / 2][lane], so that each table read is one conflict-free LDS.128
        for (int j = warp; j < n; j += WARPS) {
            float2 v[IPL];
#pragma unroll
            for (int s = 0; s < IPL; ++s) v[s] = act[s] ? td[(size_t)j * tds + b[s]] : make_float2(-2000.f, 0.f);
            if constexpr (IPL == 1) {
                kx_ltab[j * 32 + lane] = v[0];
            } else {
#pragma unroll
                for (int h = 0; h < IPL / 2; ++h)
                    reinterpret_cast<float4 *>(kx_ltab)[(j * (IPL / 2) + h) * 32 + lane] =
                        make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y);
            }
        }
        __syncthreads();
        // this warp's segments of row i (balanced across the warps by the host)
        const int gend = lsw[i * WARPS + warp + 1];
        int g = lsw[i * WARPS + warp];
        float a[IPL][4];   // FP32 sums of elements 0..3 of each four
#pragma unroll
        for (int s = 0; s < IPL; ++s) a[s][0] = a[s][1] = a[s][2] = a[s][3] = 0.f;
        int na = 0;   // elements in the FP32 sums since the last flush
        // descriptors run two segments ahead of the compute, elements one
        int2 dsc = make_int2(0, 0), dn = dsc;
        float2 el0 = make_float2(0.f, 0.f), el1 = el0;
        if (g < gend) {
            dsc = __ldg(lseg + g);
            const int c = dsc.y & 255;
            if (lane < c) el0 = __ldg(lel + dsc.x + lane);
            if (lane + 32 < c) el1 = __ldg(lel + dsc.x + 32 + lane);
        }
        if (g + 1 < gend) dn = __ldg(lseg + g + 1);
        for (; g < gend; ++g) {
            int2 dnn = dn;
            if (g + 2 < gend) dnn = __ldg(lseg + g + 2);
            float2 en0 = make_float2(0.f, 0.f), en1 = en0;
            if (g + 1 < gend) {
                const int c = dn.y & 255;
                if (lane < c) en0 = __ldg(lel + dn.x + lane);
                if (lane + 32 < c) en1 = __ldg(lel + dn.x + 32 + lane);
            }
            s_el[warp][lane] = el0;
            s_el[warp][32 + lane] = el1;
            __syncwarp();
            const int j = dsc.y >> 8, c4 = dsc.y & 255;   // count, a multiple of 4
            float2 t[IPL];
            if constexpr (IPL == 1) {
                t[0] = kx_ltab[j * 32 + lane];
            } else {
#pragma unroll
                for (int h = 0; h < IPL / 2; ++h) {
                    const float4 q = reinterpret_cast<const float4 *>(kx_ltab)[(j * (IPL / 2) + h) * 32 + lane];
                    t[2 * h] = make_float2(q.x, q.y);
                    t[2 * h + 1] = make_float2(q.z, q.w);
                }
            }
            // a pair of elements per float4, stored (S_0, S_1, omega_0, omega_1); per
            // pair and instance one packed FMA for the two exponents, two ex2 and two
            // FMAs for the weights (scalar: the ex2 results need no repacking).  A
            // running pointer keeps the loop's address arithmetic to one add per four
            // elements.
            unsigned long long tD[IPL], tL[IPL];
#pragma unroll
            for (int s = 0; s < IPL; ++s) {
                tD[s] = kx_pk2(t[s].y, t[s].y);
                tL[s] = kx_pk2(t[s].x, t[s].x);
            }
            const float4 *pe = reinterpret_cast<const float4 *>(s_el[warp]);
            const float4 *const pend = pe + (c4 >> 1);
#pragma unroll 4
            for (; pe < pend; pe += 2) {
                const float4 x01 = pe[0], x23 = pe[1];
                const unsigned long long w01 = kx_pk2(x01.z, x01.w), w23 = kx_pk2(x23.z, x23.w);
#pragma unroll
                for (int s = 0; s < IPL; ++s) {
                    const float2 e01 = kx_upk2(kx_fma2(w01, tD[s], tL[s]));
                    const float2 e23 = kx_upk2(kx_fma2(w23, tD[s], tL[s]));
                    a[s][0] = fmaf(x01.x, kx_ex2f(e01.x), a[s][0]);
                    a[s][1] = fmaf(x01.y, kx_ex2f(e01.y), a[s][1]);
                    a[s][2] = fmaf(x23.x, kx_ex2f(e23.x), a[s][2]);
                    a[s][3] = fmaf(x23.y, kx_ex2f(e23.y), a[s][3]);
                }
            }
            // the FP32 sums go into the double-float accumulator once they hold at
            // least 64 elements (short segments share a flush), and at the end
            na += c4;
            if (na >= KX_SEG) {
#pragma unroll
                for (int s = 0; s < IPL; ++s) {
                    float sm, er;
                    kx_two_sum_f(hi[s], (a[s][0] + a[s][1]) + (a[s][2] + a[s][3]), sm, er);
                    hi[s] = sm;
                    lo[s] += er;
                    a[s][0] = a[s][1] = a[s][2] = a[s][3] = 0.f;
                }
                na = 0;
            }
            __syncwarp();   // the slot is refilled next segment
            dsc = dn;
            dn = dnn;
            el0 = en0;
            el1 = en1;
        }
#pragma unroll
        for (int s = 0; s < IPL; ++s) {
            float sm, er;
            kx_two_sum_f(hi[s], (a[s][0] + a[s][1]) + (a[s][2] + a[s][3]), sm, er);
            hi[s] = sm;
            lo[s] += er;
        }
    }   // exact
    __syncthreads();   // every warp is done with the table
    double *red = reinterpret_cast<double *>(kx_ltab);   // [WARPS][32 IPL]
#pragma unroll
    for (int s = 0; s < IPL; ++s) red[warp * 32 * IPL + s * 32 + lane] = (double)hi[s] + (double)lo[s];
    __syncthreads();
    if (warp < IPL) {
        const int s = warp;   // warp s finishes instance slot s
        const int bb = blockIdx.x * (32 * IPL) + s * 32 + lane;
        if (bb < B && !(st && (st[bb].done || (stage == 2 && st[bb].skip2)))) {
            double L = 0.0, G = 0.0;
            if (Lp && cflag[bb] == 0) {
                // the GEMM's k chunks in order
                for (int c = 0; c < lsk; ++c) L += (double)Lp[((size_t)c * MTL * 128 + i) * Bpad + bb];
            } else {
#pragma unroll
                for (int w = 0; w < WARPS; ++w) L += red[w * 32 * IPL + s * 32 + lane];
            }
            // the gain of row i: the GEMM tiles' partials over the rows (i, a)
            const int segmax = 128 / n + 2;
            for (int mt = (i * n) / 128; mt <= (i * n + n - 1) / 128; ++mt)
                G += (double)Gp[(size_t)(mt * segmax + i - (mt * 128) / n) * Bpad + bb];
            const double fm = fmax[bb];
            partial[(size_t)bb * n + i] = make_double2(fm * fm * G, fm * L);
        }
    }
}

// Loss-kernel shape for an n-point grid: two instances per lane while the
// table (n x 32 x 2 float2) leaves room for two 16-warp blocks per SM or, up to
// n = 400, for one 32-warp block; one instance per lane (32 warps) above that.
// (Four instances per lane, one 16-warp block per SM, measured slower at
// n = 192: the occupancy is worth more than the shared element reads.)
struct kx_loss_shape {
    int ipl, warps;
};
static kx_loss_shape kx_loss_shape_for(int n) {
    if (n <= 200) return {2, 16};
    if (n <= 400) return {2, 32};
    return {1, 32};
}
// dynamic shared memory: the table, or the reduction if that is larger
static size_t kx_loss_smem(int n, kx_loss_shape sh) {
    return std::max((size_t)n, (size_t)sh.warps) * 32 * sh.ipl * sizeof(float2);
}

void kx_batch_prepare() {
    cudaFuncSetAttribute(k_gain_fused<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, KX_GAIN_SMEM(2));
    cudaFuncSetAttribute(k_loss_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, KX_LG_SMEM);
    cudaFuncSetAttribute(k_batch_loss<2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_smem(200, {2, 16}));
    cudaFuncSetAttribute(k_batch_loss<2, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_smem(400, {2, 32}));
    cudaFuncSetAttribute(k_batch_loss<1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_smem(KX_MAX_N, {1, 32}));
    cudaGetLastError();
}

cudaError_t kx_launch_batch_contract(const kx_kernel *k, int B, const kx_batch_views &v,
                                     const kx_inst_state *st, int stage, int *d_err,
                                     cudaStream_t s) {
    const int KB = k->Kpad / KX_TILE_K, MT = k->Mpad / 128, NT = (v.Bpad + KX_GN - 1) / KX_GN;
    dim3 g1(NT, MT);
    k_gain_fused<2><<<g1, 128, KX_GAIN_SMEM(2), s>>>(k->d_Atile, v.bt, v.fT, v.Gp, KB, k->n, v.Bpad, d_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float *Lp = nullptr;
    if (k->cheb_K) {
        // the Chebyshev loss GEMM: one CTA per SM over the work items
        const int MT = k->MTL, NTl = (v.Bpad + KX_GN - 1) / KX_GN;
        const int items = MT * NTl * k->lsk;
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int maxc = std::min(KX_GN, v.Bpad);
        int ncols = 32;
        while (ncols < 2 * maxc) ncols <<= 1;
        k_loss_gemm<<<std::min(items, sms), 192, KX_LG_SMEM, s>>>(k->d_Mtile, v.yt, v.Lp, k->KBL, 8, k->lsk,
                                                                  MT, NTl, v.Bpad, k->n, ncols, d_err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        Lp = v.Lp;
    }
    const kx_loss_shape sh = kx_loss_shape_for(k->n);
    const int per = 32 * sh.ipl;
    dim3 g2((B + per - 1) / per, k->n);
    const size_t smem = kx_loss_smem(k->n, sh);
    if (sh.ipl == 2 && sh.warps == 16)
        k_batch_loss<2, 16><<<g2, 512, smem, s>>>(k->n, B, v.B, v.Bpad, k->d_lel, k->d_lseg, k->d_lsw,
                                                  k->d_lorder, v.td, v.Gp, v.fmax, v.partial, st, stage,
                                                  Lp, v.cflag, k->lsk, k->MTL);
    else if (sh.ipl == 2)
        k_batch_loss<2, 32><<<g2, 1024, smem, s>>>(k->n, B, v.B, v.Bpad, k->d_lel, k->d_lseg, k->d_lsw,
                                                   k->d_lorder, v.td, v.Gp, v.fmax, v.partial, st, stage,
                                                   Lp, v.cflag, k->lsk, k->MTL);
    else
        k_batch_loss<1, 32><<<g2, 1024, smem, s>>>(k->n, B, v.B, v.Bpad, k->d_lel, k->d_lseg, k->d_lsw,
                                                   k->d_lorder, v.td, v.Gp, v.fmax, v.partial, st, stage,
                                                   Lp, v.cflag, k->lsk, k->MTL);
    return cudaGetLastError();
}

// ------------------------------------------------------ host table build
// From the device FP64 tables (symmetrised S over n <= m, j_L, omega):
//  A tiles: W_full[(i n)][m] = S_inm / 2 (n != m), S_inn (n = m), TF32 hi/lo
//           (hi rounded to nearest TF32, lo = W - hi), in MMA operand tiles;
//  loss list: per row, the nonzero (S, omega) as floats sorted by j_L, cut into
//           segments of at most KX_SEG elements of one j_L, each zero-padded to
//           a multiple of 4: (first element, j_L << 8 | padded count) per
//           segment; each row's segments are dealt to the loss kernel's warps
//           (longest first, to the least loaded), stored warp by warp with the
//           first segment of every (row, warp); the rows ordered by element
//           count, longest first.
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
    const int MT = k->Mpad / 128, KB = k->Kpad / KX_TILE_K;
    std::vector<float> At((size_t)MT * KB * 2 * KX_ATILE, 0.f);
    std::vector<float2> lel;
    std::vector<int2> lseg;
    const int WARPS = kx_loss_shape_for(n).warps;
    std::vector<int> lsw((size_t)n * WARPS + 1, 0), rlen(n, 0);
    std::vector<long long> base(n);
    for (int a = 0; a < n; ++a) base[a] = (long long)a * n - (long long)a * (a - 1) / 2;
    struct El {
        int j;
        float w, om;
    };
    std::vector<El> row;
    std::vector<std::pair<size_t, size_t>> seg;
    std::vector<size_t> ord;
    std::vector<int> owner;
    std::vector<long long> load;
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
                const int mt = r / 128, rl = r % 128, kb = b / KX_TILE_K, kk = b % KX_TILE_K;
                const size_t t = ((size_t)mt * KB + kb) * 2;
                At[t * KX_ATILE + kx_tile_offset(rl, kk)] = wh;
                At[(t + 1) * KX_ATILE + kx_tile_offset(rl, kk)] = wl;
                if (a <= b && W[e] != 0.0) row.push_back({(int)jl[e], (float)W[e], (float)om[e]});
            }
        }
        std::stable_sort(row.begin(), row.end(), [](const El &x, const El &y) { return x.j < y.j; });
        // segments (first element in row, end), then longest-first assignment to
        // the least loaded warp (cost: padded count + a fixed per-segment share)
        seg.clear();
        for (size_t p0 = 0; p0 < row.size();) {
            size_t p1 = p0;
            while (p1 < row.size() && row[p1].j == row[p0].j && p1 - p0 < KX_SEG) ++p1;
            seg.push_back({p0, p1});
            p0 = p1;
        }
        const auto cost = [&](size_t q) { return (long long)((seg[q].second - seg[q].first + 3) & ~(size_t)3) + 16; };
        ord.resize(seg.size());
        std::iota(ord.begin(), ord.end(), (size_t)0);
        std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return cost(x) > cost(y); });
        owner.assign(seg.size(), 0);
        load.assign(WARPS, 0);
        for (size_t q : ord) {
            const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            owner[q] = w;
            load[w] += cost(q);
        }
        for (int w = 0; w < WARPS; ++w) {
            lsw[(size_t)i * WARPS + w] = (int)lseg.size();
            for (size_t q = 0; q < seg.size(); ++q) {
                if (owner[q] != w) continue;
                const size_t p0 = seg[q].first, p1 = seg[q].second;
                const int c4 = (int)((p1 - p0 + 3) & ~(size_t)3);
                lseg.push_back(make_int2((int)lel.size(), (row[p0].j << 8) | c4));
                // element pairs as (S_0, S_1), (omega_0, omega_1); zero padding
                for (size_t e = 0; e < (size_t)c4; e += 2) {
                    const bool v0 = p0 + e < p1, v1 = p0 + e + 1 < p1;
                    lel.push_back(make_float2(v0 ? row[p0 + e].w : 0.f, v1 ? row[p0 + e + 1].w : 0.f));
                    lel.push_back(make_float2(v0 ? row[p0 + e].om : 0.f, v1 ? row[p0 + e + 1].om : 0.f));
                }
            }
        }
        rlen[i] = (int)row.size();
    }
    lsw[(size_t)n * WARPS] = (int)lseg.size();
    // Chebyshev loss (loss_terms = K): M_k[i][j] = sum_{n<=m: j_L = j} S_inm T_k(2 omega - 1)
    // in FP64 (T_k by the three-term recurrence), as TF32 hi/lo tiles of 128 rows i
    // x 16 columns of the flattened (j, k) index j K + k
    std::vector<float> Mt;
    if (k->cheb_K) {
        const int K = k->cheb_K;
        k->MTL = (n + 127) / 128;
        k->KBL = ((n - 1) * K + 15) / 16;
        k->lsk = (k->KBL + 7) / 8;   // GEMM work items of about eight k blocks
        std::vector<double> M((size_t)n * (n - 1) * K, 0.0);
        for (int i = 0; i < n; ++i) {
            for (long long e = 0; e < P; ++e) {
                const size_t x = (size_t)i * P + e;
                if (W[x] == 0.0) continue;
                const double t = 2.0 * om[x] - 1.0;
                double *Mi = &M[((size_t)i * (n - 1) + jl[x]) * K];
                double T0 = 1.0, T1 = t;
                Mi[0] += W[x];
                if (K > 1) Mi[1] += W[x] * t;
                for (int kk = 2; kk < K; ++kk) {
                    const double T2 = 2.0 * t * T1 - T0;
                    Mi[kk] += W[x] * T2;
                    T0 = T1;
                    T1 = T2;
                }
            }
        }
        Mt.assign((size_t)k->MTL * k->KBL * 2 * KX_ATILE, 0.f);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j + 1 < n; ++j)
                for (int kk = 0; kk < K; ++kk) {
                    const float w = (float)M[((size_t)i * (n - 1) + j) * K + kk];
                    const float wh = kx_tf32_round(w), wl = w - wh;
                    const int c = j * K + kk, mt = i / 128, r = i % 128, kb = c / KX_TILE_K;
                    const size_t t = ((size_t)mt * k->KBL + kb) * 2;
                    Mt[t * KX_ATILE + kx_tile_offset(r, c % KX_TILE_K)] = wh;
                    Mt[(t + 1) * KX_ATILE + kx_tile_offset(r, c % KX_TILE_K)] = wl;
                }
        if (cudaMalloc(&k->d_Mtile, sizeof(float) * Mt.size()) != cudaSuccess) {
            cudaGetLastError();
            return kx_set_error(ctx, KX_ENOMEM, "batched build: allocation failed");
        }
        k->bytes += (long long)(sizeof(float) * Mt.size());
        if (cudaMemcpy(k->d_Mtile, Mt.data(), sizeof(float) * Mt.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return kx_set_error(ctx, KX_ECUDA, "batched build: table upload failed");
    }
    std::vector<int> lorder(n);
    std::iota(lorder.begin(), lorder.end(), 0);
    std::stable_sort(lorder.begin(), lorder.end(), [&](int x, int y) { return rlen[x] > rlen[y]; });
    if (lel.empty()) lel.push_back(make_float2(0.f, 0.f));
    if (lseg.empty()) lseg.push_back(make_int2(0, 0));
    if (cudaMalloc(&k->d_Atile, sizeof(float) * At.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lel, sizeof(float2) * lel.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lseg, sizeof(int2) * lseg.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lsw, sizeof(int) * lsw.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lorder, sizeof(int) * lorder.size()) != cudaSuccess) {
        cudaGetLastError();
        return kx_set_error(ctx, KX_ENOMEM, "batched build: allocation failed");
    }
    k->nseg = (long long)lsw[(size_t)n * WARPS];
    k->nlel = (long long)lel.size();
    k->bytes += (long long)(sizeof(float) * At.size() + sizeof(float2) * lel.size() +
                            sizeof(int2) * lseg.size() + sizeof(int) * (lsw.size() + lorder.size()));
    if (cudaMemcpy(k->d_Atile, At.data(), sizeof(float) * At.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lel, lel.data(), sizeof(float2) * lel.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lseg, lseg.data(), sizeof(int2) * lseg.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lsw, lsw.data(), sizeof(int) * lsw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lorder, lorder.data(), sizeof(int) * lorder.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return kx_set_error(ctx, KX_ECUDA, "batched build: table upload failed");
    return KX_OK;
}
