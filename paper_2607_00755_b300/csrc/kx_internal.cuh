// kx_internal.cuh -- internal structures of libkx (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/kx.h"

#define KX_MAX_N 512
#define KX_MAX_NMU 64
#define KX_MAX_SRC 4
#define KX_LOG_FLOOR 1e-300   // floor of f inside the logarithm (Appendix A, "small positive floor")
#define KX_EPS_SUPP 1e-12     // epsilon_supp of the projection (Appendix B)
#define KX_DET_GUARD 1e-14    // relative guard of the 2x2 projection system

// Chunking of the contraction work (elements of one row i are split in chunks
// whose partial sums are combined in a fixed order: results are deterministic).
#define KX_T64 256            // threads per FP64 contraction block
#define KX_EPT64 8            // pairs per thread
#define KX_CH64 (KX_T64 * KX_EPT64)
#define KX_T32 256            // threads per FP32 contraction block
#define KX_BINS 2368          // equal-work bins of the FP32 contraction (148 SMs x 16 warps)
#define KX_FIN_THREADS 512    // finalize / stage kernels: one block per instance, thread = grid point
#define KX_FIT_W 17           // per-warp partial slots of the FP32 path's line fit (up to 17 warps)
#define KX_WAIT_CYCLES_MAX (4ll << 30)   // longest bounded device wait (the kernels' own limit, ~2 s)

// ---------------------------------------------------------------- KX_CHECK
// Bounds-checked build (compiled with -DKX_CHECK; libkx_check.so): the hot
// kernels pass their table, bracket, task, bin and slot indices through
// KX_IDX(i, limit, site), which in that build tests 0 <= i < limit and, when
// it fails, records the site and the index (the first failure of the
// translation unit, and a count) and returns 0 instead, so that the access
// stays inside its array and the kernel runs to its end.  In the normal build
// KX_IDX(i, limit, site) is i and the limits are not used.  Sites:
#define KX_SITE_TAB_N 1       // FP32 streaming: the n-row of the (l2, delta) table
#define KX_SITE_TAB_M 2       // FP32 streaming: the m-row of the (l2, delta) table
#define KX_SITE_BRACKET 3     // FP32 streaming: bracket j of (delta - D, D)
#define KX_SITE_TASK 4        // FP32 streaming: task index
#define KX_SITE_VECTOR 5      // FP32 streaming: kept-vector index of a unit
#define KX_SITE_SLOT 6        // FP32 streaming / row combine: partial slot
#define KX_SITE_F64_BRACKET 7 // FP64 contraction: bracket j, j + 1 of the log table
#define KX_SITE_F64_PAIR 8    // FP64 contraction: pair (n, m)
#define KX_SITE_LOSS_ELEM 9   // batched exact loss: a segment's element range
#define KX_SITE_LOSS_BRACKET 10   // batched exact loss: bracket j of a segment
#define KX_SITE_LOSS_ROW 11   // batched exact loss: row i
#define KX_SITE_GAIN_PAIR 12  // batched gain GEMM: decoded pair (n, m)
#define KX_SITE_BIN 13        // FP32 streaming: bin index
#define KX_SITE_LOSS_PAIR 14  // batched exact loss with quantum statistics: an element's (n, m)
#define KX_SITE_PROBE 99      // kx_check_probe
#ifdef KX_CHECK
static __device__ unsigned int kx_chk_state[3];   // failures, first site, first index (this unit)
__device__ __forceinline__ int kx_chk_idx(long long i, long long lim, int site) {
    if (i >= 0 && i < lim) return (int)i;
    if (atomicAdd(&kx_chk_state[0], 1u) == 0u) {
        kx_chk_state[1] = (unsigned)site;
        kx_chk_state[2] = (unsigned)i;
    }
    return 0;
}
#define KX_IDX(i, lim, site) kx_chk_idx((long long)(i), (long long)(lim), (site))
// failures, first site and index of this translation unit; reset = clear them
static inline int kx_chk_read(unsigned int *out, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out, kx_chk_state, sizeof(unsigned int) * 3);
    if (e == cudaSuccess && reset) {
        const unsigned int z[3] = {0u, 0u, 0u};
        e = cudaMemcpyToSymbol(kx_chk_state, z, sizeof(z));
    }
    return e == cudaSuccess ? 0 : -1;
}
#define KX_CHECKED 1
#else
#define KX_IDX(i, lim, site) (i)
static inline int kx_chk_read(unsigned int *out, bool) {
    out[0] = out[1] = out[2] = 0u;
    return 0;
}
#define KX_CHECKED 0
#endif
// each translation unit with checked kernels defines its reader
int kx_chk_read_contract(unsigned int *out, bool reset);
int kx_chk_read_batch(unsigned int *out, bool reset);
cudaError_t kx_launch_chk_probe(int index, int limit, int *out, cudaStream_t s);
// limits of the FP32 streaming kernels' indices (KX_CHECK)
struct kx_lim {
    int ntask;
    long long Vt;
};

struct kx_gl_nodes {
    double x[KX_MAX_NMU];
    double w[KX_MAX_NMU];
};

struct kx_kernel {
    int refcount;
    int device;
    int n, n_mu, measure, precision;
    int stats;           // 0 dilute, +1 Bose-Einstein, -1 Fermi-Dirac (FP64 and FP32 paths)
    double a, mass;
    long long P;         // pairs n <= m: n(n+1)/2
    int V;               // 4-element vectors per row (FP32 layout, segments padded to 4)
    // grid (device, FP64)
    double *d_p, *d_E, *d_dp, *d_dE, *d_h;
    std::vector<double> p, E, dp, dE, h, q;
    // FP64 tables [n][P]
    uint32_t *d_pair;    // [P]: n | m << 16
    double *d_W64;
    double *d_om64;
    uint16_t *d_jl;
    // FP32 tables: per row i only the 4-element vectors with an element inside
    // the kinematic support, rows concatenated (row i at d_roff[i] .. d_roff[i+1])
    uint32_t *d_vt;      // [Vt]: n | m0 << 16 (first m of the vector)
    float *d_W32;        // [Vt][4], slots rotated by (k >> 2) & 3, k = index in the row
    uint32_t *d_pk;      // [Vt][4]: j_L << 23 | round(omega 2^23), same slots
    int *d_roff;         // [n + 1] first kept vector of each row
    int2 *d_rtask;       // [n]: (first partial slot = i, tasks) of each row; slot k at k n + i
    int4 *d_task;        // [ntask]: (row, first unit, end unit, partial slot)
    int *d_bins;         // [KX_BINS + 1]: first task of each equal-work bin
    long long Vt;        // kept vectors, all rows
    int vpl;             // vectors per lane of a unit
    int ntask;           // streaming tasks
    int bin_units;       // the most units in one bin (sizes the staged variant's shared memory)
    int tslots;          // partial slots per instance: n x MT, MT = largest row task count rounded up to even
    // batched (split TF32) tables: the GEMMs take the instances as rows and the
    // grid points i as columns (64-row operand tiles of i, 16-wide k blocks)
    int nsubI;           // 64-row tiles of the rows i: ceil(n / 64)
    int nis;             // columns of the GEMM partials: n rounded up to 16
    int KBG;             // k blocks of the gain GEMM: ceil(P / 16), P pairs n <= m
    int gsk;             // k chunks of the gain GEMM
    float *d_Sg;         // [nsubI][KBG][hi, lo][1024]: S_ip as TF32 hi/lo operand tiles
    float2 *d_lel;       // per row i: nonzero (S_inm, omega) sorted by j_L, element pairs as
                         // (S_0, S_1), (omega_0, omega_1)
    uint32_t *d_lnm;     // quantum statistics: per loss element (same order and padding as the
                         // elements of d_lel) its pair n | m << 16 (padding: 0)
    int2 *d_lseg;        // segments of <= 64 elements of one j_L: (first element, j_L << 8 | count)
    int *d_lsw;          // [n * warps + 1] first segment of each (row, loss-kernel warp)
    int *d_lorder;       // [n] rows by element count, longest first
    // Chebyshev loss GEMM (loss_terms > 0): M_k[i][j] as TF32 hi/lo operand tiles
    int cheb_K;          // terms (0: exact loss only)
    int KBL;             // 16-wide k blocks of the flattened (j, k) dimension: ceil((n - 1) K / 16)
    int lsk;             // k chunks of the loss GEMM (each CTA work item sums one chunk)
    float *d_Mtile;      // [nsubI][KBL][hi, lo][1024]
    long long nseg;      // segments, all rows
    long long nlel;      // loss elements with the segments' zero padding
    long long nnz;
    long long bytes;
    long long stream_bytes;   // table bytes one contraction launch reads
    double build_ms;
    // rescalable kernels (expanding universe): rebuilt in place for each scale
    // factor; FP64 tables kept, FP32 tables keep every vector (layout fixed)
    bool rescalable;
    kx_gl_nodes gl;
    uint32_t *d_vt_all;  // [V] global vector list (n | m0 << 16)
    int *d_pos;          // [n][V] vector positions in the rows (identity)
};

// Per-instance integration state (device resident).
struct kx_inst_state {
    double t, h, h_try, t_end, err;
    double l1, T, lnz;
    double env_t;               // time of the stored source envelopes
    double env[KX_MAX_SRC];     // envelopes rate_k exp(-(env_t - t_on_k) / tau_k), made by the
                                // previous stage kernel for the next stage's time
    long long steps, rejects, evals;
    int status;      // KX_OK or error
    int done;        // 1: finished (converged, t_end, error)
    int converged;
    int skip2;       // stage 1 rejected: skip stage 2 of this attempt
    int last;        // this attempt ends exactly at t_end
    int env_ok;      // env holds the envelopes at env_t (0 in a new state)
};

struct kx_src_dev {
    int n_src;
    int pad;
    double rate[KX_MAX_SRC];
    double tau[KX_MAX_SRC];
    double t_on[KX_MAX_SRC];
    double t_off;            // all envelopes < 1e-12 of their peak for t >= t_off
    long long shape_off;     // offset (doubles) of this instance's normalised shapes
};

struct kx_ctx {
    int device;
    cudaStream_t stream;
    std::string last_error;
    void *d_arena;
    size_t arena_bytes;
    void *h_pinned;
    size_t pinned_bytes;
    long long launches;      // kernels enqueued through this context
};

// error helpers ---------------------------------------------------------------
int kx_set_error(kx_ctx *ctx, int code, const std::string &msg);
// NVTX range over a host call (visible to profilers that record NVTX).
#include <nvtx3/nvToolsExt.h>
struct kx_nvtx {
    explicit kx_nvtx(const char *name) { nvtxRangePushA(name); }
    ~kx_nvtx() { nvtxRangePop(); }
};
// Host-side fault injection (KX_FAULT, a comma-separated list read at each
// check): true if `what` is listed.  Nothing it does touches the GPU's state.
bool kx_fault(const char *what);
#define KX_CUDA_TRY(ctx, expr)                                                         \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess)                                                         \
            return kx_set_error((ctx), KX_ECUDA, std::string(#expr) + ": " +           \
                                                   cudaGetErrorString(_e));            \
    } while (0)

// launch wrappers (defined in the .cu files) ----------------------------------
struct kx_batch_views {
    // per call scratch carved from the context arena
    double *fmax;          // [B]
    double *lf64;          // [B][n]       FP64 path: ln max(f, floor)
    float2 *tl;            // [B][n + 4]   FP32 path: (l2_j, delta_j), l2 = log2(max(f, floor)/f_max)
    float2 *td;            // FP32 path: [B][n] (delta_j - D_j, D_j), D_j = delta_{j+1} - delta_j;
                           // split path: [n][B] (l2_j, D_j), D_j = l2_{j+1} - l2_j (instance-minor)
    float4 *tq;            // FP32 path with quantum statistics: [B][n] (eps_j - De_j, De_j,
                           //   l2_j - Dl_j, Dl_j), eps = l2 - line, De/Dl forward differences
    float *tlam;           // FP32 path with quantum statistics: [B][n] lambda_j = log2(1 + eta f_j)
    int eta;               // quantum statistics of the kernel: 0 dilute, +1 BE, -1 FD
    int grid_div;          // FP32 streaming launches use 1/grid_div of the resident blocks
    int tune_tag;          // FP32 streaming variant choice: 0, or the number of concurrent
                           // solve chains the launch runs beside (a separate tuning key)
                           // (1: the whole GPU; the server shares it among its groups)
    double2 *partial;      // [B][n][chunks]  (FP32 path: float2 (hi, lo) task partials, [B][chunks])
    const int2 *rtask;     // FP32 path: [n] (first partial slot i, tasks) per row; slot k at k n + i
    double *rfmax;         // [B]          1 / scale of the tables (FP32 dilute path: 2^-e, f_max = 2^e m)
    double *fsc;           // [B]          scale of the FP32 path's tables: 2^e (dilute) or f_max (quantum)
    float *fitp;           // [B][5][KX_FIT_W] FP32 dilute path: per-warp partial sums of the line fit
    float4 *fit;           // [B]          FP32 path: reference lines (icpt, slope) of the current
                           //              tables and of the fit of their f
    int *flags;            // [B] non-finite flags
    double *M2;            // [B] |M|^2 per instance
    kx_diag *diag;         // [B]
    int chunks;            // partials per row (FP32 path: partial slots per instance)
    // batched (split TF32) path; Bpad = B rounded up to 128 (one GEMM row tile)
    float *fT;             // [Bpad/128][n][128]: f/f_max, instance-minor within 128-instance tiles
    float *Gs;             // [gsk][Bpad][nis]: FP32 gain partials per k chunk of the gain GEMM
    float *yt;             // Chebyshev loss: [Bpad/64][KBL][hi, lo][1024] coefficient operand tiles
    float *Lp;             // Chebyshev loss: [lsk][Bpad][nis] FP32 loss partials per k chunk
    int *cflag;            // Chebyshev loss: [B] 1 = an instance bracket beyond the truncation bound
    double *qsum;          // split path with quantum statistics: [B][n] Q_i = sum S f~ f_n f_m (the
                           // loss kernel's third row sum; P_i = sum S f~ (f_n + f_m) goes to partial.x)
    int cheb_K, KBL;       // Chebyshev loss: terms (0: exact loss), k blocks of the coefficient tiles
    int gsk, lsk, nis;     // split path: k chunks of the gain and loss GEMMs, partial row length
    int *err;              // tensor-core stage timeout flag (bounded waits)
    int B;                 // instances the views were carved for (td's stride on the split path)
    int Bpad;
};

// The MMA operand tile layout (K-major, no swizzle, 8-row x 16-byte core
// matrices): element (row r, k) of a 128-row (A) or 64-row (B) tile with 16
// TF32 values of k per row sits at float offset
//   (r / 8) * 128 + (k / 4) * 32 + (r % 8) * 4 + (k % 4),
// i.e. leading-dimension (k) stride 128 B between core matrices and
// stride-dimension (row) stride 512 B between 8-row groups.
#define KX_TILE_K 16
__host__ __device__ __forceinline__ int kx_tile_offset(int r, int k) {
    return (r >> 3) * 128 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

int kx_chunks_per_row(const kx_kernel *k);
// Zero the per-call flags of freshly carved views (before the first launch).
cudaError_t kx_views_clear(const kx_kernel *k, int B, const kx_batch_views &v, cudaStream_t s);
cudaError_t kx_contract_prepare();  // one-time launch-shape queries (call outside stream capture)
size_t kx_views_bytes(const kx_kernel *k, int B);
void kx_carve_views(const kx_kernel *k, int B, void *base, kx_batch_views *v);

cudaError_t kx_launch_build_fp64(const kx_kernel *k, const kx_gl_nodes &gl, cudaStream_t s);
cudaError_t kx_launch_keep_scan(const kx_kernel *k, const uint32_t *d_vt_all, int V, int *d_pos,
                                int *d_cnt, cudaStream_t s, bool keep_all = false);
cudaError_t kx_launch_pack_fp32(const kx_kernel *k, const uint32_t *d_vt_all, int V,
                                const int *d_pos, cudaStream_t s);
cudaError_t kx_launch_count_nnz(const kx_kernel *k, unsigned long long *d_count, cudaStream_t s);

// prep: f -> (fmax, lf64 | sf, sld); mode selects path
cudaError_t kx_launch_prep(const kx_kernel *k, int B, const double *f, const kx_batch_views &v,
                           const kx_inst_state *st, cudaStream_t s, bool pdl = false);
// Times the FP32 path's streaming variants once per (device, grid size, batch)
// on the caller's prepared views and keeps the fastest for later launches
// (including graph captures).  Synchronises the stream; call outside capture.
// Adds the launches it made to *launches.  0 on success, -1 on a CUDA error.
int kx_tune_contraction(const kx_kernel *k, int B, const double *f, const kx_batch_views &v,
                        const kx_inst_state *st, cudaStream_t s, long long *launches);
// The solve tunes in place instead (its own attempt graphs, one per candidate,
// timed on real attempts): the candidate variants of a launch (0 or 1: nothing
// to choose), whether its (device, n, batch, grid share) has a choice, and
// pinning one for later launches and captures.
int kx_stream_candidate_list(const kx_kernel *k, int B, int grid_div, int *cand);
bool kx_stream_is_tuned(const kx_kernel *k, int B, int grid_div, int tag);
void kx_stream_pin(const kx_kernel *k, int B, int grid_div, int tag, int variant);
// pdl: launch with programmatic stream serialization where the kernel supports
// it (the FP32 streaming contraction and the stage kernel wait for their
// predecessor inside; other kernels launch in full stream order).
cudaError_t kx_launch_contract(const kx_kernel *k, int B, const double *f, const kx_batch_views &v,
                               const kx_inst_state *st, int stage, cudaStream_t s, bool pdl = false);
// finalize for kx_collision: C_out = (proj) C_raw
cudaError_t kx_launch_finalize(const kx_kernel *k, int B, const double *f, const kx_batch_views &v,
                               double *C_out, int project, int want_diag, cudaStream_t s);

// integration stage kernels
struct kx_step_views {
    double *f;          // [B][n] state
    double *k1;         // [B][n]
    double *fp;         // [B][n] predictor
    kx_inst_state *st;  // [B]
    const kx_src_dev *src;   // [B]
    const double *shapes;    // normalised source shapes
    double rtol, atol, h_min, h_max, l1_tol;
    long long max_attempts;
    int fixed, check_every, project;
    double hscale;      // right-hand side factor: 1 (static box), 1/H (expanding universe, d/du)
};
cudaError_t kx_launch_stage(const kx_kernel *k, int B, const kx_batch_views &v,
                            const kx_step_views &sv, int stage, cudaStream_t s, bool pdl = false);
// MB fit of nb instances: block b fits instance idx[b] (b when idx is null);
// st (nullable) gives each instance's last in-solve temperature as the start.
cudaError_t kx_launch_mbfit(const kx_kernel *k, int nb, const double *f, double *out3,
                            cudaStream_t s, const kx_inst_state *st = nullptr, const int *idx = nullptr);

// expanding universe: one RK4 step on the sources only (one instance, block of n
// threads): f += d/6 (k1 i0 + 2 k2 i1 + 2 k3 i1 + k4 i2), k = S(u), S(u1), S(u1),
// S(u2), i = 1/H at u, u1 = u + d/2, u2 = u + d
cudaError_t kx_launch_rk4_sources(const kx_kernel *k, double *f, const kx_src_dev *src, const double *shapes,
                                  double u, double d, double i0, double i1, double i2, cudaStream_t s);
// expanding universe: loss rate nu_i = sum_{n<=m} S_inm f_t of each row from the FP64 tables
cudaError_t kx_launch_loss_rate64(const kx_kernel *k, const double *f, double *nu, cudaStream_t s);

// bounded-wait self-check: *out = 1 if a wait on an mbarrier nothing arrives
// on gave up after `cycles` SM clock cycles
cudaError_t kx_launch_wait_check(long long cycles, int *out, cudaStream_t s);

// batched split-TF32 path (kx_batch.cu)
int kx_batch_build_tables(kx_ctx *ctx, kx_kernel *k);   // after the FP64 build
void kx_split_geometry(kx_kernel *k);   // GEMM shapes of the batched path from n and cheb_K
cudaError_t kx_launch_batch_contract(const kx_kernel *k, int B, const kx_batch_views &v,
                                     const kx_inst_state *st, int stage, int *d_err, cudaStream_t s);
void kx_batch_prepare();   // one-time kernel attribute setup (outside stream capture)
// grouped (uneven batch) contraction of G split-path kernels: one gain-GEMM and
// one loss-GEMM launch over all their work items, the exact loss per kernel
cudaError_t kx_launch_batch_contract_grouped(int G, const kx_kernel *const *ks, const int *B,
                                             const kx_batch_views *const *vs, const kx_inst_state *const *sts,
                                             int stage, int *d_err, cudaStream_t s, const cudaStream_t *side = nullptr,
                                             const cudaEvent_t *ev = nullptr);
// grouped stage: one launch over the instances of G kernels (block = instance,
// threads = the largest grid of the group rounded up to whole warps)
cudaError_t kx_launch_stage_grouped(int G, const kx_kernel *const *ks, const int *B,
                                    const kx_batch_views *const *vs, const kx_step_views *const *svs, int stage,
                                    cudaStream_t s);
