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

#include <map>
#include <mutex>
#include <tuple>
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
// The same MMA with the A operand (M rows x 8 TF32 of k, row m in lane m, k in
// consecutive columns) read from tensor memory at column address ta.
__device__ __forceinline__ void kx_mma_tf32_at(uint32_t tmem, uint32_t ta, uint64_t b, uint32_t idesc,
                                               uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem),
        "r"(ta), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// C (4 or 8) consecutive 32-bit columns of this thread's lane (the warp's lane
// quarter) from registers; completion is awaited with tcgen05.wait::st.
template <int C>
__device__ __forceinline__ void kx_tmem_st(uint32_t taddr, const uint32_t *v) {
    static_assert(C == 4 || C == 8, "4 or 8 columns");
    if constexpr (C == 8)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                     "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                     : "memory");
    else
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(v[0]),
                     "r"(v[1]), "r"(v[2]), "r"(v[3])
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
// ------------------------------------------------ split-TF32 GEMMs (tcgen05)
// Both contractions of the batched path are GEMMs with the instances as the M
// dimension (128-row tiles) and the grid points i as the N dimension (tiles of
// up to 256), FP32 partials per k chunk:
//   gain (GEN): out[c][b][i] = sum_{p in chunk c} (f'_n f'_m)_{b p} S_{i p},
//               p = (n <= m) pairs, S the n <-> m symmetrised kernel (2 U B
//               useful MACs, eq. discrete_collision_operator's gain);
//   loss:       out[c][b][i] = sum_{(j,k) in chunk c} Y'_{b (j k)} M_{i (j k)}
//               (the Chebyshev expansion of f_t, eq. app_log_interp).
// f' = f / f_max.  The B operand (S or M: rows i, K-major) is a kernel table
// in 64-row TF32 hi/lo tiles, staged by bulk copies; the A operand is the
// per-call coefficient tiles (loss, bulk copies) or is generated by the
// generating warps from the staged f' block and their pair lists (gain:
// f'_n f'_m in FP32, split into TF32 hi + lo) and stored into tensor memory
// (tcgen05.st; the MMAs read A from there) or into the stage's shared memory.
// Products hi*hi + hi*lo + lo*hi (K = 8 per MMA) accumulate in FP32 in tensor
// memory.  The k chunks are fixed by the
// kernel (not by the batch), so an instance's sums do not depend on the batch.
// A work item is (instance tile, i tile, chunk); the CTAs take them round
// robin (persistent, one CTA per SM).  Roles (G = KX_SG_GW): warps 0 .. G-1
// generate the gain's A operand of each stage of an S-stage ring (G/4 warps
// per 32 instance rows, 16/(G/4) pairs each), warp G lane 0 issues the MMAs
// into one of two accumulators (one where the tensor-memory columns do not
// hold two and the A stages), warps G+1 .. G+4 read the previous item's
// accumulator (tensor-memory lane quarter = warp % 4) and store its partials
// while the next item's MMAs run, warp G+5 (one lane) issues the bulk copies
// of each stage (full barrier: the copy bytes plus one arrival per generating
// warp; empty barrier: the MMAs' commit).  Operand tiles of one (i tile, k block) are
// contiguous per hi/lo part, so a stage takes two (gain) or four (loss) copies.  Every wait is bounded: on
// expiry the CTA sets *err and every role stops; copies and MMAs in flight get
// a bounded wait before shared and tensor memory are released.
#define KX_GN 256                                             // i columns per tile
#define KX_SG_GW 8                        // generating warps (gain), a multiple of 4 dividing 64
#define KX_SG_PPW (64 / KX_SG_GW)         // pairs of a k block per generating warp
#define KX_SG_MMAW KX_SG_GW               // the MMA warp
#define KX_SG_EPIW (KX_SG_GW + 1)         // the first of the four epilogue warps
#define KX_SG_CPYW (KX_SG_GW + 5)         // the bulk-copy warp
#define KX_SG_THREADS ((KX_SG_GW + 6) * 32)
#define KX_GAIN_KC 32   // k blocks per chunk of the gain GEMM (a work item; at most 32: one per lane)
static_assert(KX_GAIN_KC <= 32, "a generating warp builds its pair list with one lane per k block");
static_assert(KX_SG_GW % 4 == 0 && 64 % KX_SG_GW == 0 && KX_SG_PPW % 4 == 0,
              "generating warps: whole lane quarters, pairs per warp a multiple of 4");
#define KX_LOSS_KC 8    // k blocks per chunk of the loss GEMM

// A bounded mbarrier wait that also gives up when another role of the CTA has
// given up (abort != 0); on its own expiry it raises abort and *err.
// nap_ns > 0: sleep that long between tests (for roles whose waits are long
// and not on the critical path, so that they leave the issue slots to the
// generating and MMA warps).
__device__ __forceinline__ bool kx_wait_role(uint32_t bar, uint32_t parity, volatile int *abort, int *err,
                                             unsigned nap_ns = 0u) {
    const long long t0 = clock64();
    for (;;) {
        if (kx_mbar_try_wait(bar, parity)) return true;
        if (nap_ns) __nanosleep(nap_ns);
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

// One GEMM of a (grouped) launch: its operands, output and shape; its work
// items are item0 .. item0 + MTb NTi chunks - 1 of the launch.
#define KX_MAX_GROUPS 8
struct kx_sg_problem {
    const float *At, *Bt;
    float *out;
    const float *fT;
    long long P;
    int n, KB, KC, chunks, MTb, NTi, nsubI, Bpad, nis, item0;
};
struct kx_sg_list {
    kx_sg_problem p[KX_MAX_GROUPS];
    int np, items;
};
__device__ __forceinline__ int kx_sg_find(const kx_sg_list &L, int w) {
    int g = 0;
    while (g + 1 < L.np && w >= L.p[g + 1].item0) ++g;
    return g;
}

// Shared- and tensor-memory plan of a split GEMM.  Shared memory: S stages of
// B (hi, lo: 2 x nsb x 4 KB, nsb = 64-row i tiles of the widest i tile), plus A
// (hi, lo: 2 x 8 KB) unless A sits in tensor memory; for the gain with n <= 256
// also the f' block of the item's 128 instances (fs[n][128], one bulk copy)
// that the generating warps read instead of global memory.  Tensor memory
// (ncols columns): nbuf accumulators of up to `half` columns at columns
// 0 and half, and with atm (the gain only) the S stages of the generated A
// operand, 32 columns each (16 k of hi, 16 of lo; lane = instance row), stage
// q at column a0 + (q / 2) a2 + (q % 2) 32.
// The epilogue's staging rows (ew = 32 or 16 columns, 0: none): each epilogue
// warp passes its 32 rows x ew accumulator columns through shared memory
// (rows padded to ew + 4 floats) so that its global stores are whole row
// segments of ew floats, eight or four lanes per row, instead of one 16-byte
// piece per lane in 32 rows.
struct kx_sg_plan {
    int S, nsb, stage, aoff, fs, pt, eb, ew, smem, atm, ncols, half, nbuf, a0, a2;
};
__host__ __device__ __forceinline__ int kx_sg_acol(const kx_sg_plan &pl, int q) {
    return pl.a0 + (q >> 1) * pl.a2 + (q & 1) * 32;
}
// wmax: the widest i tile (columns of an accumulator); req_S: the ring depth
// wanted (0: as many stages as fit, at most 4); use_fs: stage the f' block when
// it fits (0: the generating warps read global memory); req_atm: the gain's A
// operand in tensor memory (1, the default) or in shared memory (0).  None of
// them changes a result: the k chunks, their order and the MMAs are fixed.
__host__ __device__ inline kx_sg_plan kx_sg_plan_for(bool gen, int n, int nsubI, int wmax, int req_S = 0,
                                                     int use_fs = 1, int req_atm = 1) {
    kx_sg_plan pl;
    pl.atm = gen && req_atm ? 1 : 0;
    pl.nsb = nsubI < 4 ? nsubI : 4;
    pl.aoff = pl.atm ? 0 : 2 * KX_ATILE * 4;
    pl.stage = pl.aoff + 2 * pl.nsb * KX_BTILE * 4;
    pl.fs = (gen && n <= 256 && use_fs) ? 128 * n * 4 : 0;   // (n, nsubI: the largest of a grouped launch)
    pl.pt = gen ? KX_SG_GW * KX_GAIN_KC * KX_SG_PPW * 4 : 0;    // the generating warps' pair lists
    const int budget = 227 * 1024 - 256 - pl.pt;
    int sfull = (budget - pl.fs) / pl.stage;
    if (sfull > 4) sfull = 4;
    // the widest epilogue staging that keeps min(sfull, 3) stages
    pl.eb = 0;
    pl.ew = 0;
    for (int w = 32; w >= 16; w -= 16) {
        const int eb = 4 * 32 * (w + 4) * 4;
        const int need = sfull < 3 ? sfull : 3;
        if ((budget - pl.fs - eb) / pl.stage >= need) {
            pl.eb = eb;
            pl.ew = w;
            break;
        }
    }
    pl.S = (budget - pl.fs - pl.eb) / pl.stage;
    if (pl.S > 4) pl.S = 4;
    if (req_S > 0 && req_S < pl.S) pl.S = req_S;
    pl.smem = pl.S * pl.stage + pl.fs + pl.pt + pl.eb + 256;
    pl.a0 = 0;
    pl.a2 = 64;
    int p2 = 32;   // accumulator width: the widest i tile, rounded up to a power of two
    while (p2 < wmax) p2 <<= 1;
    pl.nbuf = 2;
    pl.half = p2;
    if (!pl.atm) {
        pl.ncols = 2 * p2;
    } else if (2 * p2 + 32 * pl.S <= 512) {
        // two accumulators, then the A stages
        pl.a0 = 2 * p2;
        pl.ncols = 32;
        while (pl.ncols < 2 * p2 + 32 * pl.S) pl.ncols <<= 1;
    } else if (wmax <= 192) {
        // accumulators at 0 and 256; the A stages in the 64 columns after each
        pl.ncols = 512;
        pl.half = 256;
        pl.a0 = 192;
        pl.a2 = 256;
    } else {
        // one accumulator of 256 columns (its epilogue does not overlap the next
        // item's MMAs), the A stages after it
        pl.ncols = 512;
        pl.nbuf = 1;
        pl.half = 256;
        pl.a0 = 256;
    }
    return pl;
}

// GEN: the gain (A generated from f' and the packed pairs n <= m); else the
// loss (A = the coefficient tiles At [Bpad/128][KB][hi, lo][2048]).  Bt:
// [NTi][KB][hi, lo][nsb x 1024] (nsb = min(4, nsubI) 64-row tiles of i per i
// tile, zero padded).  out: [chunks][Bpad][nis].  fT: [Bpad/128][n][128] (GEN).
// Packed pair p = base(n) + m - n, base(n) = n (2N - n + 1) / 2.
__device__ __forceinline__ long long kx_pair_base(int n, int N) { return (long long)n * (2 * N - n + 1) / 2; }
__device__ __forceinline__ void kx_pair_decode(long long p, int N, int &n, int &m) {
    const float b = 2.f * N + 1.f;
    int x = (int)floorf(0.5f * (b - sqrtf(fmaxf(b * b - 8.f * (float)p, 0.f))));
    x = max(0, min(x, N - 1));
    if (x + 1 < N && kx_pair_base(x + 1, N) <= p) ++x;   // FP32 rounding: at most one step either way
    if (kx_pair_base(x, N) > p) --x;
    n = x;
    m = x + (int)(p - kx_pair_base(x, N));
}
template <bool GEN>
__global__ void __launch_bounds__(KX_SG_THREADS, 1)
    k_split_gemm(const kx_sg_list L, const kx_sg_plan pl, int *err) {
    extern __shared__ __align__(1024) unsigned char kx_gsm[];
    const int S = pl.S;
    float *fs = reinterpret_cast<float *>(kx_gsm + S * pl.stage);   // f' block (GEN, n <= 256)
    // the generating warps' pair lists (GEN): warp w's (n | m << 16) of its PPW
    // pairs of each k block of the current item
    uint32_t *ptab = reinterpret_cast<uint32_t *>(kx_gsm + S * pl.stage + pl.fs);
    float *ebuf = reinterpret_cast<float *>(kx_gsm + S * pl.stage + pl.fs + pl.pt);   // epilogue staging rows
    uint64_t *bars = reinterpret_cast<uint64_t *>(kx_gsm + S * pl.stage + pl.fs + pl.pt + pl.eb);
    // bars: full[4] empty[4] accf[2] acce[2] fbar fsfree
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 14);
    volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
    int *issued = reinterpret_cast<int *>(tslot + 2);   // [4] rounds issued per stage
    int *seen = issued + 4;                             // [4] rounds consumed per stage
    int *lastc = seen + 4;                              // k blocks committed by the MMA thread
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t full0 = kx_smem_u32(&bars[0]), empty0 = kx_smem_u32(&bars[4]);
    const uint32_t accf0 = kx_smem_u32(&bars[8]), acce0 = kx_smem_u32(&bars[10]);
    const uint32_t fbar = kx_smem_u32(&bars[12]), fsfree = kx_smem_u32(&bars[13]);
    const bool fsm = GEN && pl.fs > 0;
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            kx_mbar_init(full0 + 8 * q, GEN ? 1 + KX_SG_GW : 1);   // GEN: the copy arrival + the generating warps
            kx_mbar_init(empty0 + 8 * q, 1);
            issued[q] = 0;
            seen[q] = 0;
        }
        for (int q = 0; q < 2; ++q) {
            kx_mbar_init(accf0 + 8 * q, 1);
            kx_mbar_init(acce0 + 8 * q, 4);   // one arrival per epilogue warp
        }
        kx_mbar_init(fbar, 1);
        kx_mbar_init(fsfree, KX_SG_GW);   // one arrival per generating warp
        *lastc = 0;
        *abort = 0;
        kx_fence_mbar_init();
    }
    if (warp == KX_SG_MMAW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(kx_smem_u32(tslot)),
                     "r"(pl.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const int items = L.items;
    const int half = pl.half, nbuf = pl.nbuf;   // accumulator columns, accumulators
    const bool atm = GEN && pl.atm;               // the generated A operand in tensor memory
    int fissued = 0;               // f' blocks requested (tid 0) / waited for (producers)
    if (warp == KX_SG_CPYW) {
        // ---- bulk copies: B (hi, lo) and, for the loss, A (hi, lo) of each stage
        if (lane == 0) {
            int it = 0;
            for (int w = blockIdx.x; w < items && !*abort; w += gridDim.x) {
                const kx_sg_problem &pb = L.p[kx_sg_find(L, w)];
                const int wl = w - pb.item0, KB = pb.KB;
                const int c = wl % pb.chunks, nt = (wl / pb.chunks) % pb.NTi, mt = wl / (pb.chunks * pb.NTi);
                const int kb0 = c * pb.KC, kb1 = min(KB, kb0 + pb.KC);
                const int nsbp = min(4, pb.nsubI);   // the problem's 64-row i tiles per i tile
                const uint32_t bbytes = (uint32_t)(nsbp * KX_BTILE * 4);
                bool ok = true;
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int q = it % S, round = it / S;
                    if (round > 0 && !kx_wait_role(empty0 + 8 * q, (round - 1) & 1, abort, err, 64u)) {
                        ok = false;
                        break;
                    }
                    unsigned char *sa = kx_gsm + (size_t)q * pl.stage, *sb = sa + pl.aoff;
                    const uint32_t bar = full0 + 8 * q;
                    kx_mbar_expect_tx(bar, (GEN ? 0u : 2u * KX_ATILE * 4) + 2 * bbytes);
                    const float *bsrc = pb.Bt + ((size_t)nt * KB + kb) * 2 * nsbp * KX_BTILE;
                    kx_bulk_g2s(kx_smem_u32(sb), bsrc, bbytes, bar);
                    kx_bulk_g2s(kx_smem_u32(sb + pl.nsb * KX_BTILE * 4), bsrc + nsbp * KX_BTILE, bbytes, bar);
                    if (!GEN) {
                        const float *asrc = pb.At + ((size_t)mt * KB + kb) * 2 * KX_ATILE;
                        kx_bulk_g2s(kx_smem_u32(sa), asrc, KX_ATILE * 4, bar);
                        kx_bulk_g2s(kx_smem_u32(sa + KX_ATILE * 4), asrc + KX_ATILE, KX_ATILE * 4, bar);
                    }
                    issued[q] = round + 1;
                }
                if (!ok) break;
            }
        }
    } else if (warp < KX_SG_GW) {
        // ---- the gain's A operand: row r = f'_n f'_m of instance b for the 16
        // pairs of each k block (warp w: rows 32 (w % 4) .., pairs PPW (w / 4) ..)
        if (GEN) {
            int it = 0;
            const int row = tid & 127, ph = (tid >> 7) * KX_SG_PPW;   // instance row in the tile, first pair
            for (int w = blockIdx.x; w < items && !*abort; w += gridDim.x) {
                const kx_sg_problem &pb = L.p[kx_sg_find(L, w)];
                const int wl = w - pb.item0, n = pb.n;
                const long long P = pb.P;
                const int c = wl % pb.chunks, mt = wl / (pb.chunks * pb.NTi);
                const int kb0 = c * pb.KC, kb1 = min(pb.KB, kb0 + pb.KC);
                const float *fblk = pb.fT + (size_t)mt * n * 128;   // this instance tile's f' [n][128]
                bool ok = true;
                if (fsm) {
                    // the item's f' block, once every generating warp is done with
                    // the previous one (fsfree: one arrival per warp)
                    int r = 1;
                    if (tid == 0) {
                        if (fissued > 0) r = kx_wait_role(fsfree, (fissued - 1) & 1, abort, err);
                        if (r) {
                            kx_mbar_expect_tx(fbar, (uint32_t)(n * 512));
                            kx_bulk_g2s(kx_smem_u32(fs), fblk, (uint32_t)(n * 512), fbar);
                        }
                    }
                    if (lane == 0 && r) r = kx_wait_role(fbar, fissued & 1, abort, err);
                    r = __shfl_sync(0xffffffffu, r, 0);
                    ++fissued;
                    if (!r) break;
                }
                // this warp's pair list of the item: lane j decodes the first of the
                // warp's PPW pairs of k block kb0 + j and steps on to the others
                // (row a holds the pairs m = a .. N - 1; after (a, N - 1) comes
                // (a + 1, a + 1)); padding pairs past P are 0xffff
                uint32_t *wpt = ptab + warp * (KX_GAIN_KC * KX_SG_PPW);
                if (lane < kb1 - kb0) {
                    const long long p0 = (long long)(kb0 + lane) * 16 + ph;
                    int a = n - 1, c = n;
                    if (p0 < P) kx_pair_decode(p0, n, a, c);
#pragma unroll
                    for (int e = 0; e < KX_SG_PPW; ++e) {
                        wpt[lane * KX_SG_PPW + e] = p0 + e < P ? (uint32_t)a | ((uint32_t)c << 16) : 0xffffu;
                        if (++c == n) c = ++a;
                    }
                }
                __syncwarp();
                // y = f'_n f'_m of this lane's row for the warp's PPW pairs of k block
                // kb (the pairs are the same in every lane; padding pairs give 0)
                auto gen_y = [&](int kb, float *y) {
                    int nn[KX_SG_PPW], mm[KX_SG_PPW];
                    const uint4 *wq = reinterpret_cast<const uint4 *>(wpt + (kb - kb0) * KX_SG_PPW);
#pragma unroll
                    for (int e4 = 0; e4 < KX_SG_PPW / 4; ++e4) {
                        const uint4 w4 = wq[e4];
                        const uint32_t wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const bool in = wv[e] != 0xffffu;
                            nn[4 * e4 + e] = in ? KX_IDX((int)(wv[e] & 0xffffu), n, KX_SITE_GAIN_PAIR) : -1;
                            mm[4 * e4 + e] = in ? KX_IDX((int)(wv[e] >> 16), n, KX_SITE_GAIN_PAIR) : 0;
                        }
                    }
                    // (the source is chosen outside the unrolled loops, so that the
                    // loads are issued back to back)
                    if (fsm) {
#pragma unroll
                        for (int e = 0; e < KX_SG_PPW; ++e) {
                            const float v = fs[max(nn[e], 0) * 128 + row] * fs[mm[e] * 128 + row];
                            y[e] = nn[e] >= 0 ? v : 0.f;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < KX_SG_PPW; ++e) {
                            const float v = __ldg(fblk + (size_t)max(nn[e], 0) * 128 + row) *
                                            __ldg(fblk + (size_t)mm[e] * 128 + row);
                            y[e] = nn[e] >= 0 ? v : 0.f;
                        }
                    }
                };
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int q = it % S, round = it / S;
                    if (round > 0) {
                        int r = 1;
                        if (lane == 0) r = kx_wait_role(empty0 + 8 * q, (round - 1) & 1, abort, err);
                        r = __shfl_sync(0xffffffffu, r, 0);
                        if (!r) {
                            ok = false;
                            break;
                        }
                        // the MMAs that read this stage are complete (their commit)
                        if (atm) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    }
                    float *ah = reinterpret_cast<float *>(kx_gsm + (size_t)q * pl.stage), *al = ah + KX_ATILE;
                    float y[KX_SG_PPW];
                    gen_y(kb, y);
                    if (atm) {
                        // this lane's row of the stage: columns ph .. ph + PPW - 1 (hi)
                        // and 16 + ph .. (lo) of the warp's lane quarter
                        uint32_t h[KX_SG_PPW], l[KX_SG_PPW];
#pragma unroll
                        for (int e = 0; e < KX_SG_PPW; ++e) {
                            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h[e]) : "f"(y[e]));
                            l[e] = __float_as_uint(y[e] - __uint_as_float(h[e]));
                        }
                        const uint32_t ta = tmem + ((uint32_t)(row & ~31) << 16) + (uint32_t)(kx_sg_acol(pl, q) + ph);
                        kx_tmem_st<KX_SG_PPW>(ta, h);
                        kx_tmem_st<KX_SG_PPW>(ta + 16u, l);
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    } else {
#pragma unroll
                        for (int q4 = 0; q4 < KX_SG_PPW; q4 += 4) {
                            float h[4], l[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                uint32_t hb;
                                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(y[q4 + e]));
                                h[e] = __uint_as_float(hb);
                                l[e] = y[q4 + e] - h[e];
                            }
                            const int off = kx_tile_offset(row, ph + q4);
                            *reinterpret_cast<float4 *>(ah + off) = make_float4(h[0], h[1], h[2], h[3]);
                            *reinterpret_cast<float4 *>(al + off) = make_float4(l[0], l[1], l[2], l[3]);
                        }
                        // generic-proxy writes become visible to the tensor core (async proxy)
                        kx_fence_proxy_async();
                    }
                    __syncwarp();
                    if (lane == 0) kx_mbar_arrive(full0 + 8 * q);
                }
                if (!ok) break;
                if (fsm) {
                    // this warp's reads of the f' block are done (its last A tile written)
                    __syncwarp();
                    if (lane == 0) kx_mbar_arrive(fsfree);
                }
            }
        }
    } else if (warp == KX_SG_MMAW) {
        // ---- MMA issue
        if (lane == 0) {
            int it = 0, li = 0;
            for (int w = blockIdx.x; w < items && !*abort; w += gridDim.x, ++li) {
                const kx_sg_problem &pb = L.p[kx_sg_find(L, w)];
                const int wl = w - pb.item0;
                const int c = wl % pb.chunks, nt = (wl / pb.chunks) % pb.NTi;
                const int kb0 = c * pb.KC, kb1 = min(pb.KB, kb0 + pb.KC);
                const int Ni = min(KX_GN, pb.nis - nt * KX_GN);
                const int buf = li % nbuf, use = li / nbuf;
                if (use > 0 && !kx_wait_role(acce0 + 8 * buf, (use - 1) & 1, abort, err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(buf * half);
                const uint32_t idesc = kx_idesc_tf32(128, Ni);
                bool ok = true;
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int q = it % S, round = it / S;
                    if (!kx_wait_role(full0 + 8 * q, round & 1, abort, err)) {
                        ok = false;
                        break;
                    }
                    seen[q] = round + 1;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t aH = kx_smem_u32(kx_gsm + (size_t)q * pl.stage), aL = aH + KX_ATILE * 4;
                    const uint32_t bH = aH + pl.aoff, bL = bH + pl.nsb * KX_BTILE * 4;
                    if (atm) {
                        const uint32_t tH = tmem + (uint32_t)kx_sg_acol(pl, q), tL = tH + 16u;
#pragma unroll
                        for (int step = 0; step < KX_TILE_K / 8; ++step) {
                            const uint32_t o = 256u * step, c = 8u * step;   // 8 TF32 of k
                            kx_mma_tf32_at(d, tH + c, kx_desc(bH + o, 128, 512), idesc, (kb > kb0 || step) ? 1u : 0u);
                            kx_mma_tf32_at(d, tH + c, kx_desc(bL + o, 128, 512), idesc, 1u);
                            kx_mma_tf32_at(d, tL + c, kx_desc(bH + o, 128, 512), idesc, 1u);
                        }
                    } else {
#pragma unroll
                        for (int step = 0; step < KX_TILE_K / 8; ++step) {
                            const uint32_t o = 256u * step;   // 8 TF32 = two 16-byte core-matrix columns
                            kx_mma_tf32(d, kx_desc(aH + o, 128, 512), kx_desc(bH + o, 128, 512), idesc,
                                        (kb > kb0 || step) ? 1u : 0u);
                            kx_mma_tf32(d, kx_desc(aH + o, 128, 512), kx_desc(bL + o, 128, 512), idesc, 1u);
                            kx_mma_tf32(d, kx_desc(aL + o, 128, 512), kx_desc(bH + o, 128, 512), idesc, 1u);
                        }
                    }
                    kx_mma_commit(empty0 + 8 * q);
                    *lastc = it + 1;
                }
                if (!ok) break;
                kx_mma_commit(accf0 + 8 * buf);
            }
        }
    } else {
        // ---- epilogue: FP32 partials out[c][b][i]
        const int qtr = warp & 3;   // tensor-memory lane quarter this warp may read
        int li = 0;
        for (int w = blockIdx.x; w < items; w += gridDim.x, ++li) {
            const kx_sg_problem &pb = L.p[kx_sg_find(L, w)];
            const int wl = w - pb.item0, nis = pb.nis;
            const int c = wl % pb.chunks, nt = (wl / pb.chunks) % pb.NTi, mt = wl / (pb.chunks * pb.NTi);
            const int Ni = min(KX_GN, nis - nt * KX_GN);
            const int buf = li % nbuf, use = li / nbuf;
            int ok = 1;
            if (lane == 0) ok = kx_wait_role(accf0 + 8 * buf, use & 1, abort, err, 256u);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int b = mt * 128 + qtr * 32 + lane;
            const uint32_t tl = tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(buf * half);
            const int ew = pl.ew;
            if (ew) {
                // lane l: row l's ew columns into its staging row (columns up to
                // Ni rounded up to ew, all inside the accumulator); then lanes
                // (l / k, l % k), k = ew / 4 lanes per row, store float4 pieces of
                // 32 / k rows per instruction (rows are whole ew-float segments)
                float *wb = ebuf + (warp - KX_SG_EPIW) * 32 * (ew + 4);
                const int k = ew >> 2, rpi = 32 / k, rr = lane / k, pp = lane % k;
                float *dst0 = pb.out + ((size_t)c * pb.Bpad + (size_t)mt * 128 + qtr * 32) * nis + (size_t)nt * KX_GN;
                for (int c0 = 0; c0 < Ni; c0 += ew) {
                    float t[16];
                    for (int h = 0; h < ew; h += 16) {
                        kx_tmem_ld16(tl + (uint32_t)(c0 + h), t);
#pragma unroll
                        for (int q = 0; q < 16; q += 4)
                            *reinterpret_cast<float4 *>(wb + lane * (ew + 4) + h + q) =
                                make_float4(t[q], t[q + 1], t[q + 2], t[q + 3]);
                    }
                    __syncwarp();
                    for (int r0 = 0; r0 < 32; r0 += rpi) {
                        const int r = r0 + rr;
                        const float4 x = *reinterpret_cast<const float4 *>(wb + r * (ew + 4) + 4 * pp);
                        // (Ni is a multiple of 16: a piece lies wholly inside the tile or
                        // wholly past it; the columns past Ni are read, not stored)
                        if (mt * 128 + qtr * 32 + r < pb.Bpad && c0 + 4 * pp < Ni)
                            *reinterpret_cast<float4 *>(dst0 + (size_t)r * nis + c0 + 4 * pp) = x;
                    }
                    __syncwarp();
                }
            } else {
                float *dst = pb.out + ((size_t)c * pb.Bpad + b) * nis + (size_t)nt * KX_GN;
                for (int c0 = 0; c0 < Ni; c0 += 16) {
                    float t[16];
                    kx_tmem_ld16(tl + (uint32_t)c0, t);
                    if (b < pb.Bpad) {
#pragma unroll
                        for (int q = 0; q < 16; q += 4)
                            *reinterpret_cast<float4 *>(dst + c0 + q) = make_float4(t[q], t[q + 1], t[q + 2], t[q + 3]);
                    }
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
        if (fsm && fissued > 0) kx_mbar_wait(fbar, (fissued - 1) & 1, 1ll << 24);
        if (*lastc > 0) {
            const int it = *lastc - 1;
            kx_mbar_wait(empty0 + 8 * (it % S), (it / S) & 1, 1ll << 24);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == KX_SG_MMAW)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(pl.ncols) : "memory");
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
    k_batch_loss(int n, int B, int tds, const float2 *__restrict__ lel,
                 const int2 *__restrict__ lseg, const int *__restrict__ lsw,
                 const int *__restrict__ lorder, const float2 *__restrict__ td,
                 const double *__restrict__ fmax, double2 *__restrict__ partial,
                 const kx_inst_state *__restrict__ st, int stage, const int *__restrict__ cflag, int nel) {
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
        // Chebyshev loss (cflag non-null): only the instances whose truncation
        // bound was exceeded take the exact loss
        if (cflag && act[s]) act[s] = cflag[b[s]] != 0;
        any |= act[s];
    }
    if (!__syncthreads_or(any)) return;
    const int i = KX_IDX(lorder[blockIdx.y], n, KX_SITE_LOSS_ROW);
    float hi[IPL], lo[IPL];
    (void)nel;
#pragma unroll
    for (int s = 0; s < IPL; ++s) hi[s] = lo[s] = 0.f;
    {
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
            if (lane < c) el0 = __ldg(lel + KX_IDX(dsc.x + lane, nel, KX_SITE_LOSS_ELEM));
            if (lane + 32 < c) el1 = __ldg(lel + KX_IDX(dsc.x + 32 + lane, nel, KX_SITE_LOSS_ELEM));
        }
        if (g + 1 < gend) dn = __ldg(lseg + g + 1);
        for (; g < gend; ++g) {
            int2 dnn = dn;
            if (g + 2 < gend) dnn = __ldg(lseg + g + 2);
            float2 en0 = make_float2(0.f, 0.f), en1 = en0;
            if (g + 1 < gend) {
                const int c = dn.y & 255;
                if (lane < c) en0 = __ldg(lel + KX_IDX(dn.x + lane, nel, KX_SITE_LOSS_ELEM));
                if (lane + 32 < c) en1 = __ldg(lel + KX_IDX(dn.x + 32 + lane, nel, KX_SITE_LOSS_ELEM));
            }
            s_el[warp][lane] = el0;
            s_el[warp][32 + lane] = el1;
            __syncwarp();
            const int j = KX_IDX(dsc.y >> 8, n, KX_SITE_LOSS_BRACKET), c4 = dsc.y & 255;   // count, a multiple of 4
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
    }
    __syncthreads();   // every warp is done with the table
    double *red = reinterpret_cast<double *>(kx_ltab);   // [WARPS][32 IPL]
#pragma unroll
    for (int s = 0; s < IPL; ++s) red[warp * 32 * IPL + s * 32 + lane] = (double)hi[s] + (double)lo[s];
    __syncthreads();
    if (warp < IPL) {
        const int s = warp;   // warp s finishes instance slot s
        const int bb = blockIdx.x * (32 * IPL) + s * 32 + lane;
        if (bb < B && !(st && (st[bb].done || (stage == 2 && st[bb].skip2))) && !(cflag && cflag[bb] == 0)) {
            double L = 0.0;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) L += red[w * 32 * IPL + s * 32 + lane];
            partial[(size_t)bb * n + i] = make_double2(0.0, fmax[bb] * L);   // the gain: the GEMM's partials
        }
    }
}

// The exact loss with quantum statistics (eq. Lambda_quantum).  With
// eta = +1 (BE) or -1 (FD) an element's factor
//   f_n f_m (1 + eta f_i)(1 + eta f~) - f_i f~ (1 + eta f_n)(1 + eta f_m)
// sums over a row to (1 + eta f_i) G_i - f_i L_i - eta f_i P_i + eta Q_i
// (eta^2 = 1), with G_i = sum S f_n f_m (the gain GEMM), L_i = sum S f~,
// P_i = sum S f~ (f_n + f_m) and Q_i = sum S f~ f_n f_m.  This kernel makes
// L, P and Q of each (instance, row): the dilute kernel's segments and
// per-element exponent, and per element the pair's f'_n, f'_m (f' = f / f_max,
// from the gain's f' block) read from a shared-memory table by the pair
// indices of the element (d_lnm).  One instance per lane, WARPS warps (the
// loss list's warp split); the FP32 sums flush into double-float accumulators
// every 64 or more elements, FP64 across warps.  Output: partial[b][i] =
// (f_max^2 P', f_max L'), qsum[b][i] = f_max^3 Q' (primes: f' units).
template <int IPL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1)
    k_batch_loss_q(int n, int B, int tds, const float2 *__restrict__ lel, const uint32_t *__restrict__ lnm,
                   const int2 *__restrict__ lseg, const int *__restrict__ lsw, const int *__restrict__ lorder,
                   const float2 *__restrict__ td, const float *__restrict__ fT, const double *__restrict__ fmax,
                   double2 *__restrict__ partial, double *__restrict__ qsum,
                   const kx_inst_state *__restrict__ st, int stage, int nel) {
    // IPL = 1: [n][32] (l2_j, D_j) and [n][32] f'_j; IPL = 2 (two instances per
    // lane, packed f32x2 arithmetic): [n][32] (l2, l2', D, D') and [n][32] (f', f'').
    // After the loop the same space holds the reduction [3][WARPS][32 IPL] doubles.
    extern __shared__ __align__(16) float2 kx_ltab[];
    float *ftab = reinterpret_cast<float *>(kx_ltab + (size_t)n * 32 * IPL);
    __shared__ __align__(16) float2 s_el[WARPS][KX_SEG];
    __shared__ __align__(16) uint32_t s_nm[WARPS][KX_SEG];
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
    const int i = KX_IDX(lorder[blockIdx.y], n, KX_SITE_LOSS_ROW);
    for (int j = warp; j < n; j += WARPS) {
        float2 t[IPL];
        float fv[IPL];
#pragma unroll
        for (int s = 0; s < IPL; ++s) {
            t[s] = act[s] ? td[(size_t)j * tds + b[s]] : make_float2(-2000.f, 0.f);
            fv[s] = act[s] ? fT[((size_t)(b[s] >> 7) * n + j) * 128 + (b[s] & 127)] : 0.f;
        }
        if constexpr (IPL == 1) {
            kx_ltab[j * 32 + lane] = t[0];
            ftab[j * 32 + lane] = fv[0];
        } else {
            reinterpret_cast<float4 *>(kx_ltab)[j * 32 + lane] = make_float4(t[0].x, t[1].x, t[0].y, t[1].y);
            reinterpret_cast<float2 *>(ftab)[j * 32 + lane] = make_float2(fv[0], fv[1]);
        }
    }
    __syncthreads();
    // per instance slot: double-float accumulators of L, P and Q
    float hl[IPL], ll[IPL], hp[IPL], lp[IPL], hq[IPL], lq[IPL];
#pragma unroll
    for (int s = 0; s < IPL; ++s) hl[s] = ll[s] = hp[s] = lp[s] = hq[s] = lq[s] = 0.f;
    {
        const int gend = lsw[i * WARPS + warp + 1];
        int g = lsw[i * WARPS + warp];
        // FP32 sums of elements 0..3 of each four, per slot (IPL = 2: packed pairs)
        unsigned long long aL[4], aP[4], aQ[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) aL[u] = aP[u] = aQ[u] = 0ull;
        int na = 0;
        for (; g < gend; ++g) {
            const int2 dsc = __ldg(lseg + g);
            const int c = dsc.y & 255;
            float2 el0 = make_float2(0.f, 0.f), el1 = el0;
            uint32_t nm0 = 0u, nm1 = 0u;
            if (lane < c) {
                const int x = KX_IDX(dsc.x + lane, nel, KX_SITE_LOSS_ELEM);
                el0 = __ldg(lel + x);
                nm0 = __ldg(lnm + x);
            }
            if (lane + 32 < c) {
                const int x = KX_IDX(dsc.x + 32 + lane, nel, KX_SITE_LOSS_ELEM);
                el1 = __ldg(lel + x);
                nm1 = __ldg(lnm + x);
            }
            s_el[warp][lane] = el0;
            s_el[warp][32 + lane] = el1;
            s_nm[warp][lane] = nm0;
            s_nm[warp][32 + lane] = nm1;
            __syncwarp();
            const int j = KX_IDX(dsc.y >> 8, n, KX_SITE_LOSS_BRACKET), c4 = c;   // a multiple of 4
            // (l2, D) of the slots: scalar (IPL = 1) or packed pairs (IPL = 2)
            unsigned long long tL, tD;
            if constexpr (IPL == 1) {
                const float2 t = kx_ltab[j * 32 + lane];
                tL = kx_pk2(t.x, 0.f);
                tD = kx_pk2(t.y, 0.f);
            } else {
                const float4 t = reinterpret_cast<const float4 *>(kx_ltab)[j * 32 + lane];
                tL = kx_pk2(t.x, t.y);
                tD = kx_pk2(t.z, t.w);
            }
            const float4 *pe = reinterpret_cast<const float4 *>(s_el[warp]);
            const uint4 *pn = reinterpret_cast<const uint4 *>(s_nm[warp]);
            for (int e4 = 0; e4 < c4; e4 += 4, pe += 2, ++pn) {
                // elements e4 .. e4 + 3: (S_0, S_1, omega_0, omega_1), (S_2, S_3, omega_2, omega_3)
                const float4 x01 = pe[0], x23 = pe[1];
                const uint4 w4 = *pn;
                const float S[4] = {x01.x, x01.y, x23.x, x23.y}, om[4] = {x01.z, x01.w, x23.z, x23.w};
                const uint32_t nm[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int a = KX_IDX((int)(nm[u] & 0xffffu), n, KX_SITE_LOSS_PAIR);
                    const int m = KX_IDX((int)(nm[u] >> 16), n, KX_SITE_LOSS_PAIR);
                    if constexpr (IPL == 1) {
                        const float ft = kx_ex2f(fmaf(om[u], kx_upk2(tD).x, kx_upk2(tL).x));
                        const float fn = ftab[a * 32 + lane], fm = ftab[m * 32 + lane];
                        const float w = S[u] * ft;
                        const float2 A = kx_upk2(aL[u]), Pq = kx_upk2(aP[u]), Qq = kx_upk2(aQ[u]);
                        aL[u] = kx_pk2(fmaf(S[u], ft, A.x), 0.f);
                        aP[u] = kx_pk2(fmaf(w, fn + fm, Pq.x), 0.f);
                        aQ[u] = kx_pk2(fmaf(w, fn * fm, Qq.x), 0.f);
                    } else {
                        // both slots at once: per lane the scalar operations (round to
                        // nearest, no flush) of the IPL = 1 form
                        const float2 e = kx_upk2(kx_fma2(kx_pk2(om[u], om[u]), tD, tL));
                        const unsigned long long ft = kx_pk2(kx_ex2f(e.x), kx_ex2f(e.y));
                        const unsigned long long S2 = kx_pk2(S[u], S[u]), z = 0ull;
                        const unsigned long long fn = reinterpret_cast<const unsigned long long *>(ftab)[a * 32 + lane];
                        const unsigned long long fm = reinterpret_cast<const unsigned long long *>(ftab)[m * 32 + lane];
                        const unsigned long long w = kx_fma2(S2, ft, z);                   // S f~
                        const unsigned long long sum = kx_fma2(fn, kx_pk2(1.f, 1.f), fm);  // f_n + f_m
                        const unsigned long long prd = kx_fma2(fn, fm, z);                 // f_n f_m
                        aL[u] = kx_fma2(S2, ft, aL[u]);
                        aP[u] = kx_fma2(w, sum, aP[u]);
                        aQ[u] = kx_fma2(w, prd, aQ[u]);
                    }
                }
            }
            na += c4;
            const bool flush = na >= KX_SEG;
            if (flush) {
                const float2 L0 = kx_upk2(aL[0]), L1 = kx_upk2(aL[1]), L2 = kx_upk2(aL[2]), L3 = kx_upk2(aL[3]);
                const float2 P0 = kx_upk2(aP[0]), P1 = kx_upk2(aP[1]), P2 = kx_upk2(aP[2]), P3 = kx_upk2(aP[3]);
                const float2 Q0 = kx_upk2(aQ[0]), Q1 = kx_upk2(aQ[1]), Q2 = kx_upk2(aQ[2]), Q3 = kx_upk2(aQ[3]);
                const float sL[2] = {(L0.x + L1.x) + (L2.x + L3.x), (L0.y + L1.y) + (L2.y + L3.y)};
                const float sP[2] = {(P0.x + P1.x) + (P2.x + P3.x), (P0.y + P1.y) + (P2.y + P3.y)};
                const float sQ[2] = {(Q0.x + Q1.x) + (Q2.x + Q3.x), (Q0.y + Q1.y) + (Q2.y + Q3.y)};
#pragma unroll
                for (int s = 0; s < IPL; ++s) {
                    float sm, er;
                    kx_two_sum_f(hl[s], sL[s], sm, er);
                    hl[s] = sm;
                    ll[s] += er;
                    kx_two_sum_f(hp[s], sP[s], sm, er);
                    hp[s] = sm;
                    lp[s] += er;
                    kx_two_sum_f(hq[s], sQ[s], sm, er);
                    hq[s] = sm;
                    lq[s] += er;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) aL[u] = aP[u] = aQ[u] = 0ull;
                na = 0;
            }
            __syncwarp();   // the slots are refilled next segment
        }
        {
            const float2 L0 = kx_upk2(aL[0]), L1 = kx_upk2(aL[1]), L2 = kx_upk2(aL[2]), L3 = kx_upk2(aL[3]);
            const float2 P0 = kx_upk2(aP[0]), P1 = kx_upk2(aP[1]), P2 = kx_upk2(aP[2]), P3 = kx_upk2(aP[3]);
            const float2 Q0 = kx_upk2(aQ[0]), Q1 = kx_upk2(aQ[1]), Q2 = kx_upk2(aQ[2]), Q3 = kx_upk2(aQ[3]);
            const float sL[2] = {(L0.x + L1.x) + (L2.x + L3.x), (L0.y + L1.y) + (L2.y + L3.y)};
            const float sP[2] = {(P0.x + P1.x) + (P2.x + P3.x), (P0.y + P1.y) + (P2.y + P3.y)};
            const float sQ[2] = {(Q0.x + Q1.x) + (Q2.x + Q3.x), (Q0.y + Q1.y) + (Q2.y + Q3.y)};
#pragma unroll
            for (int s = 0; s < IPL; ++s) {
                float sm, er;
                kx_two_sum_f(hl[s], sL[s], sm, er);
                hl[s] = sm;
                ll[s] += er;
                kx_two_sum_f(hp[s], sP[s], sm, er);
                hp[s] = sm;
                lp[s] += er;
                kx_two_sum_f(hq[s], sQ[s], sm, er);
                hq[s] = sm;
                lq[s] += er;
            }
        }
    }
    __syncthreads();   // every warp is done with the tables
    double *red = reinterpret_cast<double *>(kx_ltab);   // [3][WARPS][32 IPL]
#pragma unroll
    for (int s = 0; s < IPL; ++s) {
        red[((0 * WARPS + warp) * IPL + s) * 32 + lane] = (double)hl[s] + (double)ll[s];
        red[((1 * WARPS + warp) * IPL + s) * 32 + lane] = (double)hp[s] + (double)lp[s];
        red[((2 * WARPS + warp) * IPL + s) * 32 + lane] = (double)hq[s] + (double)lq[s];
    }
    __syncthreads();
    if (warp < IPL) {
        const int s = warp;   // warp s finishes instance slot s
        const int bb = blockIdx.x * (32 * IPL) + s * 32 + lane;
        if (bb < B && !(st && (st[bb].done || (stage == 2 && st[bb].skip2)))) {
            double L = 0.0, P = 0.0, Q = 0.0;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) {
                L += red[((0 * WARPS + w) * IPL + s) * 32 + lane];
                P += red[((1 * WARPS + w) * IPL + s) * 32 + lane];
                Q += red[((2 * WARPS + w) * IPL + s) * 32 + lane];
            }
            const double fm = fmax[bb];
            partial[(size_t)bb * n + i] = make_double2(fm * fm * P, fm * L);
            qsum[(size_t)bb * n + i] = fm * fm * fm * Q;
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
// (the warps per block fix the kernel's segment tables; the instances per lane
// can be tuned: an instance's sums do not depend on them)
// dynamic shared memory: the table, or the reduction if that is larger
static size_t kx_loss_smem(int n, kx_loss_shape sh) {
    return std::max((size_t)n, (size_t)sh.warps) * 32 * sh.ipl * sizeof(float2);
}
// quantum statistics: the (l2, D) and f' tables, or the three reductions; two
// instances per lane while the tables fit (n <= 256), else one
static int kx_loss_q_ipl(int n) { return n <= 256 ? 2 : 1; }
static size_t kx_loss_q_smem(int n, int warps, int ipl) {
    return std::max((size_t)n * 32 * ipl * (sizeof(float2) + sizeof(float)),
                    (size_t)3 * warps * 32 * ipl * sizeof(double));
}

void kx_batch_prepare() {
    cudaFuncSetAttribute(k_split_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_split_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_batch_loss<2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_smem(200, {2, 16}));
    cudaFuncSetAttribute(k_batch_loss<2, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_smem(400, {2, 32}));
    cudaFuncSetAttribute(k_batch_loss<1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_smem(KX_MAX_N, {1, 32}));
    cudaFuncSetAttribute(k_batch_loss<1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_smem(200, {1, 16}));
    cudaFuncSetAttribute(k_batch_loss_q<1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_q_smem(KX_MAX_N, 16, 1));
    cudaFuncSetAttribute(k_batch_loss_q<1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_q_smem(KX_MAX_N, 32, 1));
    cudaFuncSetAttribute(k_batch_loss_q<2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_q_smem(256, 16, 2));
    cudaFuncSetAttribute(k_batch_loss_q<2, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kx_loss_q_smem(256, 32, 2));
    cudaGetLastError();
}

// ------------------------------------------------------------ MMA issue rate
// One thread per CTA (one CTA per SM) issues R MMAs of M = 128, N = n, K = 8
// (kind::tf32) or 16 (kind::f16, bf16 operands) from zero tiles in shared memory
// (the GEMMs' no-swizzle K-major layout) into a tensor-memory accumulator, commits
// and waits (bounded); cycles of CTA 0 go to out[0], whether the wait completed to
// out[1].
template <int KIND>
__global__ void __launch_bounds__(128, 1) k_mma_rate(int n, int R, long long *out) {
    __shared__ __align__(1024) unsigned char sm[128 * 64 + 256 * 64];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (int)sizeof(sm) / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(sm)[i] = 0u;
    if (tid == 0) {
        kx_mbar_init(kx_smem_u32(&bar), 1);
        kx_fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(kx_smem_u32(&tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    kx_fence_proxy_async();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tslot;
    if (tid == 0) {
        const uint32_t a = kx_smem_u32(sm), b = kx_smem_u32(sm + 128 * 64);
        // D F32; A, B tf32 (2, kind::tf32) or bf16 (1, kind::f16); K-major; N >> 3, M >> 4
        const uint32_t fmt = KIND == 0 ? 2u : 1u;
        const uint32_t id = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | (8u << 24);
        const long long t0 = clock64();
        for (int r = 0; r < R; ++r) {
            const uint32_t acc = r > 0 ? 1u : 0u;
            if (KIND == 0)
                kx_mma_tf32(tmem, kx_desc(a, 128, 512), kx_desc(b, 128, 512), id, acc);
            else
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                             "l"(kx_desc(a, 128, 512)), "l"(kx_desc(b, 128, 512)), "r"(id), "r"(acc)
                             : "memory");
        }
        kx_mma_commit(kx_smem_u32(&bar));
        const bool ok = kx_mbar_wait(kx_smem_u32(&bar), 0);
        const long long t1 = clock64();
        if (blockIdx.x == 0) {
            out[0] = t1 - t0;
            out[1] = ok ? 1 : 0;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

extern "C" int kx_measure_mma_rate(kx_ctx *ctx, int kind, int n, double *flop_per_clk_sm, double *cycles_per_mma) {
    if (!ctx || (kind != 0 && kind != 1) || n < 16 || n > 256 || n % 16 || !flop_per_clk_sm || !cycles_per_mma)
        return KX_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return KX_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    long long *d = nullptr, h[2] = {0, 0};
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) return KX_ENOMEM;
    const int R = 4096;
    if (kind == 0) k_mma_rate<0><<<sms > 0 ? sms : 148, 128, 0, ctx->stream>>>(n, R, d);
    else k_mma_rate<1><<<sms > 0 ? sms : 148, 128, 0, ctx->stream>>>(n, R, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    ctx->launches += 1;
    if (e != cudaSuccess || !h[1] || h[0] <= 0) return KX_ECUDA;
    *cycles_per_mma = (double)h[0] / R;
    *flop_per_clk_sm = 2.0 * 128 * n * (kind == 0 ? 8 : 16) / *cycles_per_mma;
    return KX_OK;
}

// ------------------------------------------------------------ split tuner
// The split path's result-neutral launch choices: the GEMM ring depth and the
// f' staging (per launch shape: gain or loss, the widest grid, its i tiles,
// the work items), and the exact loss kernel's instances per lane (per grid
// and batch).  Each is timed on the launch's own operands the first time the
// shape is launched outside a stream capture (the GEMMs and the loss kernel
// rewrite their partials with the same values, so the repeats are harmless)
// and kept for the process; under capture the default rule is used.
struct kx_sg_choice {
    int S, fs, atm;
};
static std::mutex g_sg_mu;
static std::map<std::tuple<int, int, int, int, int>, kx_sg_choice> g_sg_tuned;   // (dev, gen, n, nsubI, items)
static std::map<std::tuple<int, int, int>, int> g_loss_tuned;                     // (dev, n, B) -> ipl
static bool g_split_tuning = true;
static int g_gain_operand = 0;   // 0: either (timed; default tensor memory), 1: shared memory, 2: tensor memory

static bool kx_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// best (min over 3 repeats after one warm launch) of the candidates; launch(c)
// enqueues candidate c on s.  Candidate 0 is the rule's choice: another one is
// taken only when it is at least 5 % faster.  The candidates of a shape are often
// within a few per cent, where the noise would pick at random, and the repeats
// run with the operands warm in L2, which flatters the choices that read them
// from L2 (f' unstaged) against the calls' cold first touch.
template <typename F>
static int kx_time_candidates(int nc, cudaStream_t s, F launch) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return 0;
    }
    int best = 0;
    float best_ms = 0.f, rule_ms = 0.f;
    for (int c = 0; c < nc; ++c) {
        float ms_c = 0.f;
        cudaError_t e = launch(c);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            float ms = 0.f;
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch(c);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (r == 0 || ms < ms_c)) ms_c = ms;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (c == 0) rule_ms = ms_c;
        if (best_ms <= 0.f || ms_c < best_ms) {   // (the first candidate that ran)
            best_ms = ms_c;
            best = c;
        }
    }
    if (best != 0 && rule_ms > 0.f && best_ms > 0.95f * rule_ms) best = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

extern "C" int kx_set_split_tuning(int enabled) {
    std::lock_guard<std::mutex> lock(g_sg_mu);
    g_split_tuning = enabled != 0;
    if (!g_split_tuning) {
        g_sg_tuned.clear();
        g_loss_tuned.clear();
    }
    return KX_OK;
}

extern "C" int kx_set_gain_operand(int where) {
    if (where < 0 || where > 2) return KX_EINVAL;
    std::lock_guard<std::mutex> lock(g_sg_mu);
    if (where != g_gain_operand) g_sg_tuned.clear();
    g_gain_operand = where;
    return KX_OK;
}

extern "C" int kx_get_split_tuning(const kx_kernel *k, int B, int *gain_S, int *gain_fs, int *loss_S,
                                   int *loss_ipl, int *tuned, int *gain_atm) {
    if (!k || B < 1 || !gain_S || !gain_fs || !loss_S || !loss_ipl || !tuned || !gain_atm) return KX_EINVAL;
    if (k->precision != KX_SPLIT_TF32) return KX_ENOTSUP;
    int dev = 0;
    cudaGetDevice(&dev);
    const int Bpad = (B + 127) / 128 * 128;
    const int NTi = (k->nis + KX_GN - 1) / KX_GN;
    const int ig = Bpad / 128 * NTi * k->gsk, il = Bpad / 128 * NTi * k->lsk;
    const int wmax = std::min(KX_GN, k->nis);
    std::lock_guard<std::mutex> lock(g_sg_mu);
    *tuned = 0;
    const kx_sg_plan dg = kx_sg_plan_for(true, k->n, k->nsubI, wmax, 0, 1, g_gain_operand != 1),
                     dl = kx_sg_plan_for(false, k->n, k->nsubI, wmax);
    *gain_S = dg.S;
    *gain_fs = dg.fs > 0;
    *gain_atm = dg.atm;
    *loss_S = k->cheb_K ? dl.S : 0;
    *loss_ipl = kx_loss_shape_for(k->n).ipl;
    auto ig_it = g_sg_tuned.find(std::make_tuple(dev, 1, k->n, k->nsubI, ig));
    if (ig_it != g_sg_tuned.end()) {
        const kx_sg_choice &c = ig_it->second;
        const kx_sg_plan p = kx_sg_plan_for(true, k->n, k->nsubI, wmax, c.S, c.fs, c.atm);
        *gain_S = p.S;
        *gain_fs = p.fs > 0;
        *gain_atm = p.atm;
        *tuned |= 1;
    }
    auto il_it = g_sg_tuned.find(std::make_tuple(dev, 0, k->n, k->nsubI, il));
    if (k->cheb_K && il_it != g_sg_tuned.end()) {
        *loss_S = kx_sg_plan_for(false, k->n, k->nsubI, wmax, il_it->second.S, 0).S;
        *tuned |= 2;
    }
    auto lo_it = g_loss_tuned.find(std::make_tuple(dev, k->n, B));
    if (lo_it != g_loss_tuned.end()) {
        *loss_ipl = lo_it->second;
        *tuned |= 4;
    }
    return KX_OK;
}

// Persistent grid of a split GEMM: one CTA per SM, at most one per work item.
static int kx_sg_grid(int items) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 148;
    }
    return std::max(1, std::min(items, sms));
}

// The gain (GEN) or Chebyshev-loss GEMM problem of one kernel and batch.
static kx_sg_problem kx_sg_problem_for(bool gen, const kx_kernel *k, const kx_batch_views &v, int item0) {
    kx_sg_problem pb;
    pb.At = gen ? nullptr : v.yt;
    pb.Bt = gen ? k->d_Sg : k->d_Mtile;
    pb.out = gen ? v.Gs : v.Lp;
    pb.fT = v.fT;
    pb.P = k->P;
    pb.n = k->n;
    pb.KB = gen ? k->KBG : k->KBL;
    pb.KC = gen ? KX_GAIN_KC : KX_LOSS_KC;
    pb.chunks = gen ? k->gsk : k->lsk;
    pb.MTb = v.Bpad / 128;
    pb.NTi = (k->nis + KX_GN - 1) / KX_GN;
    pb.nsubI = k->nsubI;
    pb.Bpad = v.Bpad;
    pb.nis = k->nis;
    pb.item0 = item0;
    return pb;
}

// One launch of the gain (GEN) or loss GEMM over the problems of G kernels.
static cudaError_t kx_launch_split_gemm(bool gen, int G, const kx_kernel *const *ks, const kx_batch_views *const *vs,
                                        int *d_err, cudaStream_t s) {
    kx_sg_list L;
    L.np = 0;
    int items = 0, nmax = 0, nsmax = 0, wmax = 0;
    for (int g = 0; g < G; ++g) {
        if (!gen && !ks[g]->cheb_K) continue;
        kx_sg_problem pb = kx_sg_problem_for(gen, ks[g], *vs[g], items);
        L.p[L.np++] = pb;
        items += pb.MTb * pb.NTi * pb.chunks;
        nmax = std::max(nmax, pb.n);
        nsmax = std::max(nsmax, pb.nsubI);
        wmax = std::max(wmax, std::min(KX_GN, pb.nis));
    }
    if (!L.np) return cudaSuccess;
    L.items = items;
    auto launch = [&](const kx_sg_plan &pl) {
        if (gen)
            k_split_gemm<true><<<kx_sg_grid(items), KX_SG_THREADS, pl.smem, s>>>(L, pl, d_err);
        else
            k_split_gemm<false><<<kx_sg_grid(items), KX_SG_THREADS, pl.smem, s>>>(L, pl, d_err);
        return cudaGetLastError();
    };
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, gen ? 1 : 0, nmax, nsmax, items);
    bool tune = false;
    int operand = 0;
    kx_sg_choice ch;
    {
        std::lock_guard<std::mutex> lock(g_sg_mu);
        operand = g_gain_operand;
        ch = {0, 1, operand != 1};
        auto it = g_sg_tuned.find(key);
        if (it != g_sg_tuned.end()) ch = it->second;
        else tune = g_split_tuning;
    }
    if (tune && !kx_capturing(s)) {
        // the gain's A operand in tensor or shared memory (as allowed), ring
        // depths 2 .. the most that fit, with and without the f' stage
        std::vector<kx_sg_choice> cand;
        for (int atm = (gen && operand != 1) ? 1 : 0; atm >= (operand == 2 ? 1 : 0); --atm)
            for (int fs = (gen && nmax <= 256) ? 1 : 0; fs >= 0; --fs) {
                const int smax = kx_sg_plan_for(gen, nmax, nsmax, wmax, 0, fs, atm).S;
                for (int S = smax; S >= 2; --S) cand.push_back({S, fs, atm});
            }
        if (!cand.empty()) {
            const int best = kx_time_candidates((int)cand.size(), s, [&](int c) {
                return launch(kx_sg_plan_for(gen, nmax, nsmax, wmax, cand[c].S, cand[c].fs, cand[c].atm));
            });
            ch = cand[best];
        }
        std::lock_guard<std::mutex> lock(g_sg_mu);
        g_sg_tuned[key] = ch;
    }
    return launch(kx_sg_plan_for(gen, nmax, nsmax, wmax, ch.S, ch.fs, ch.atm));
}

// The exact loss kernel (all instances, or the Chebyshev path's flagged ones).
static cudaError_t kx_launch_batch_loss(const kx_kernel *k, int B, const kx_batch_views &v,
                                        const kx_inst_state *st, int stage, cudaStream_t s) {
    if (k->stats) {
        // quantum statistics: L, P and Q (the loss list's warps; instances per
        // lane by n alone, so that an instance's sums do not depend on the batch)
        const int warps = kx_loss_shape_for(k->n).warps, ipl = kx_loss_q_ipl(k->n);
        dim3 g2((B + 32 * ipl - 1) / (32 * ipl), k->n);
        const size_t smem = kx_loss_q_smem(k->n, warps, ipl);
#define KX_LQ(I, W)                                                                                             \
    k_batch_loss_q<I, W><<<g2, W * 32, smem, s>>>(k->n, B, v.B, k->d_lel, k->d_lnm, k->d_lseg, k->d_lsw,        \
                                                  k->d_lorder, v.td, v.fT, v.fmax, v.partial, v.qsum, st, stage, \
                                                  (int)k->nlel)
        if (ipl == 2 && warps == 16) KX_LQ(2, 16);
        else if (ipl == 2) KX_LQ(2, 32);
        else if (warps == 16) KX_LQ(1, 16);
        else KX_LQ(1, 32);
#undef KX_LQ
        return cudaGetLastError();
    }
    const int *flags = k->cheb_K ? v.cflag : nullptr;
    auto launch = [&](kx_loss_shape sh) {
        const int per = 32 * sh.ipl;
        dim3 g2((B + per - 1) / per, k->n);
        const size_t smem = kx_loss_smem(k->n, sh);
        if (sh.ipl == 2 && sh.warps == 16)
            k_batch_loss<2, 16><<<g2, 512, smem, s>>>(k->n, B, v.B, k->d_lel, k->d_lseg, k->d_lsw, k->d_lorder,
                                                      v.td, v.fmax, v.partial, st, stage, flags, (int)k->nlel);
        else if (sh.warps == 16)
            k_batch_loss<1, 16><<<g2, 512, smem, s>>>(k->n, B, v.B, k->d_lel, k->d_lseg, k->d_lsw, k->d_lorder,
                                                      v.td, v.fmax, v.partial, st, stage, flags, (int)k->nlel);
        else if (sh.ipl == 2)
            k_batch_loss<2, 32><<<g2, 1024, smem, s>>>(k->n, B, v.B, k->d_lel, k->d_lseg, k->d_lsw, k->d_lorder,
                                                       v.td, v.fmax, v.partial, st, stage, flags, (int)k->nlel);
        else
            k_batch_loss<1, 32><<<g2, 1024, smem, s>>>(k->n, B, v.B, k->d_lel, k->d_lseg, k->d_lsw, k->d_lorder,
                                                       v.td, v.fmax, v.partial, st, stage, flags, (int)k->nlel);
        return cudaGetLastError();
    };
    kx_loss_shape sh = kx_loss_shape_for(k->n);
    // (the Chebyshev path runs the exact loss only for flagged instances: not tuned)
    if (!k->cheb_K) {
        int dev = 0;
        cudaGetDevice(&dev);
        const auto key = std::make_tuple(dev, k->n, B);
        bool tune = false;
        {
            std::lock_guard<std::mutex> lock(g_sg_mu);
            auto it = g_loss_tuned.find(key);
            if (it != g_loss_tuned.end()) sh.ipl = it->second;
            else tune = g_split_tuning;
        }
        if (tune && !kx_capturing(s)) {
            // the rule's shape and the other instances-per-lane count (two
            // instances per lane with 32 warps fit only up to n = 400)
            const kx_loss_shape c2[2] = {sh, {3 - sh.ipl, sh.warps}};
            const int nc = (sh.ipl == 1 && sh.warps == 32) ? 1 : 2;
            const int best = kx_time_candidates(nc, s, [&](int c) { return launch(c2[c]); });
            sh.ipl = c2[best].ipl;
            std::lock_guard<std::mutex> lock(g_sg_mu);
            g_loss_tuned[key] = sh.ipl;
        }
    }
    return launch(sh);
}

cudaError_t kx_launch_batch_contract(const kx_kernel *k, int B, const kx_batch_views &v,
                                     const kx_inst_state *st, int stage, int *d_err,
                                     cudaStream_t s) {
    const kx_batch_views *vp = &v;
    cudaError_t e = kx_launch_split_gemm(true, 1, &k, &vp, d_err, s);
    if (e == cudaSuccess && k->cheb_K) e = kx_launch_split_gemm(false, 1, &k, &vp, d_err, s);
    if (e == cudaSuccess) e = kx_launch_batch_loss(k, B, v, st, stage, s);
    return e;
}

// Grouped contraction of G kernels (the uneven batch): one gain-GEMM launch
// and one loss-GEMM launch over all their work items; the exact loss per kernel.
cudaError_t kx_launch_batch_contract_grouped(int G, const kx_kernel *const *ks, const int *B,
                                             const kx_batch_views *const *vs, const kx_inst_state *const *sts,
                                             int stage, int *d_err, cudaStream_t s, const cudaStream_t *side,
                                             const cudaEvent_t *ev) {
    cudaError_t e = kx_launch_split_gemm(true, G, ks, vs, d_err, s);
    if (e == cudaSuccess) e = kx_launch_split_gemm(false, G, ks, vs, d_err, s);
    if (!side || !ev) {
        for (int g = 0; g < G && e == cudaSuccess; ++g) e = kx_launch_batch_loss(ks[g], B[g], *vs[g], sts[g], stage, s);
        return e;
    }
    // the exact loss kernels of the G grids side by side: forked from s after the
    // GEMMs (ev[0]) onto the side streams and joined back (ev[1 + g])
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        e = cudaStreamWaitEvent(side[g], ev[0], 0);
        if (e == cudaSuccess) e = kx_launch_batch_loss(ks[g], B[g], *vs[g], sts[g], stage, side[g]);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1 + g], side[g]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1 + g], 0);
    }
    return e;
}

// ------------------------------------------------------ host table build
// From the device FP64 tables (symmetrised S over n <= m, j_L, omega):
//  gain operand: S_ip (p = pair n <= m) as TF32 hi/lo (hi rounded to nearest
//           TF32, lo = S - hi) in 64-row tiles of the rows i;
//  Chebyshev loss operand (loss_terms = K): M_k[i][j] likewise, column j K + k;
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

// Shapes of the batched path's GEMMs for an n-point grid (and cheb_K terms):
// fixed by the kernel alone, so that an instance's sums do not depend on the
// batch it is evaluated in.
void kx_split_geometry(kx_kernel *k) {
    const int n = k->n;
    const long long P = (long long)n * (n + 1) / 2;
    k->nsubI = (n + 63) / 64;
    k->nis = (n + 15) / 16 * 16;
    k->KBG = (int)((P + KX_TILE_K - 1) / KX_TILE_K);
    k->gsk = (k->KBG + KX_GAIN_KC - 1) / KX_GAIN_KC;
    if (k->cheb_K) {
        k->KBL = ((n - 1) * k->cheb_K + KX_TILE_K - 1) / KX_TILE_K;
        k->lsk = (k->KBL + KX_LOSS_KC - 1) / KX_LOSS_KC;
    } else {
        k->KBL = k->lsk = 0;
    }
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
    kx_split_geometry(k);
    // gain GEMM operand: S_ip (p = pairs n <= m in packed order) as TF32 hi/lo;
    // per (i tile of up to 256 rows, k block of 16 pairs) the hi part, then the
    // lo part, each nsb 64-row tiles in MMA operand layout (one bulk copy each)
    const int nsb = std::min(4, k->nsubI), NTi = (k->nis + 255) / 256;
    auto bt_index = [&](int i, long long c, int KB, int h) {
        const size_t blk = (((size_t)(i / 256) * KB + (size_t)(c / KX_TILE_K)) * 2 + h) * nsb;
        return (blk + (size_t)((i % 256) / 64)) * KX_BTILE + kx_tile_offset(i % 64, (int)(c % KX_TILE_K));
    };
    std::vector<float> Sg((size_t)NTi * k->KBG * 2 * nsb * KX_BTILE, 0.f);
    for (int i = 0; i < n; ++i)
        for (long long p = 0; p < P; ++p) {
            const float w = (float)W[(size_t)i * P + p];
            const float wh = kx_tf32_round(w), wl = w - wh;
            Sg[bt_index(i, p, k->KBG, 0)] = wh;
            Sg[bt_index(i, p, k->KBG, 1)] = wl;
        }
    std::vector<float2> lel;
    std::vector<uint32_t> lnm;   // quantum statistics: the elements' pairs
    std::vector<int2> lseg;
    const int WARPS = kx_loss_shape_for(n).warps;
    std::vector<int> lsw((size_t)n * WARPS + 1, 0), rlen(n, 0);
    std::vector<long long> base(n);
    for (int a = 0; a < n; ++a) base[a] = (long long)a * n - (long long)a * (a - 1) / 2;
    struct El {
        int j;
        float w, om;
        uint32_t nm;   // the element's pair n | m << 16
    };
    std::vector<El> row;
    std::vector<std::pair<size_t, size_t>> seg;
    std::vector<size_t> ord;
    std::vector<int> owner;
    std::vector<long long> load;
    for (int i = 0; i < n; ++i) {
        row.clear();
        for (int a = 0; a < n; ++a) {
            for (int b = a; b < n; ++b) {
                const size_t e = (size_t)i * P + base[a] + (b - a);
                if (W[e] != 0.0) row.push_back({(int)jl[e], (float)W[e], (float)om[e], (uint32_t)a | ((uint32_t)b << 16)});
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
                // the pairs in element order (c4 words: lnm and lel share the segments' offsets)
                if (k->stats)
                    for (size_t e = 0; e < (size_t)c4; ++e) lnm.push_back(p0 + e < p1 ? row[p0 + e].nm : 0u);
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
        Mt.assign((size_t)NTi * k->KBL * 2 * nsb * KX_BTILE, 0.f);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j + 1 < n; ++j)
                for (int kk = 0; kk < K; ++kk) {
                    const float w = (float)M[((size_t)i * (n - 1) + j) * K + kk];
                    const float wh = kx_tf32_round(w), wl = w - wh;
                    const long long c = (long long)j * K + kk;
                    Mt[bt_index(i, c, k->KBL, 0)] = wh;
                    Mt[bt_index(i, c, k->KBL, 1)] = wl;
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
    if (cudaMalloc(&k->d_Sg, sizeof(float) * Sg.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lel, sizeof(float2) * lel.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lseg, sizeof(int2) * lseg.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lsw, sizeof(int) * lsw.size()) != cudaSuccess ||
        cudaMalloc(&k->d_lorder, sizeof(int) * lorder.size()) != cudaSuccess) {
        cudaGetLastError();
        return kx_set_error(ctx, KX_ENOMEM, "batched build: allocation failed");
    }
    k->nseg = (long long)lsw[(size_t)n * WARPS];
    k->nlel = (long long)lel.size();
    k->bytes += (long long)(sizeof(float) * Sg.size() + sizeof(float2) * lel.size() +
                            sizeof(int2) * lseg.size() + sizeof(int) * (lsw.size() + lorder.size()));
    if (cudaMemcpy(k->d_Sg, Sg.data(), sizeof(float) * Sg.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lel, lel.data(), sizeof(float2) * lel.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lseg, lseg.data(), sizeof(int2) * lseg.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lsw, lsw.data(), sizeof(int) * lsw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(k->d_lorder, lorder.data(), sizeof(int) * lorder.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return kx_set_error(ctx, KX_ECUDA, "batched build: table upload failed");
    if (k->stats) {
        if (lnm.empty()) lnm.push_back(0u);
        if (lnm.size() != lel.size() && !(lel.size() == 1 && lnm.size() == 1))
            return kx_set_error(ctx, KX_ECUDA, "batched build: pair list out of step with the loss list");
        if (cudaMalloc(&k->d_lnm, sizeof(uint32_t) * lnm.size()) != cudaSuccess) {
            cudaGetLastError();
            return kx_set_error(ctx, KX_ENOMEM, "batched build: allocation failed");
        }
        k->bytes += (long long)(sizeof(uint32_t) * lnm.size());
        if (cudaMemcpy(k->d_lnm, lnm.data(), sizeof(uint32_t) * lnm.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return kx_set_error(ctx, KX_ECUDA, "batched build: table upload failed");
    }
    return KX_OK;
}

int kx_chk_read_batch(unsigned int *out, bool reset) { return kx_chk_read(out, reset); }
