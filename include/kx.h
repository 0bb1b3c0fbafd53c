/*
 * kx.h -- C ABI of the B300 collision-operator library (libkx.so).
 *
 * The library evaluates the discretised 2->2 elastic self-collision term of a
 * dark-sector momentum distribution (arXiv 2607.00755, "KineticXGPU"):
 *
 *   C_i[f] = sum_{n,m} W_inm [ f_n f_m - f_i f_t(i,n,m) ]            (Sec. 4.1,
 *            eq. discrete_collision_operator; Appendix A, eq. app_dense_collision)
 *
 * with the precomputed kernel tensor W (eq. discrete_weight, eq. app_F_1d), the
 * log-energy interpolation of f at the fourth momentum (eqs. app_interp_weights,
 * app_log_interp), the two-moment conservation projection (Appendix B,
 * eqs. app_self_projection, app_projection_system) and the adaptive Heun time
 * integration of df/dt = C[f] + S(t) (Sec. 4.2) in the static box (a fixed,
 * H = 0) with synthetic freeze-in sources.
 *
 * Conventions for every entry point:
 *  - Return value: KX_OK (0), KX_PENDING (1) or a negative KX_E* code.  No C++
 *    exception crosses the ABI.  kx_strerror() names a code; kx_last_error()
 *    returns the last detailed message of a context.
 *  - Pointers named *_dev are device pointers owned by the caller; they must be
 *    valid for the context's device and are used on the context's stream.
 *    Pointers named *_host (and all struct members) are host memory, read during
 *    the call only.  Device arrays of a batch are row-major [batch][n] FP64.
 *  - The library owns kernels (reference counted), the context's scratch space
 *    and the serving state.
 *  - Units: momenta and mass in the same unit; the cross-section sigma enters
 *    as |M|^2 = 64 pi m^2 sigma (Table 1 caption: sigma_T/m = lambda^2/(64 pi m^3)
 *    with |M|^2 = lambda^2 for the contact interaction of Sec. 3), g_chi = 1.
 *  - Threading: one context per host thread.  Calls on one context are not
 *    re-entrant.  kx_submit/kx_poll may be called from the owning thread while
 *    the serving loop runs on its own worker thread.
 */
#ifndef KX_H_
#define KX_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define KX_OK 0
#define KX_PENDING 1       /* kx_poll: request not finished yet */
#define KX_EINVAL -1       /* bad argument: n < 4 or > 512, q not ascending/positive, m <= 0, ... */
#define KX_ENOMEM -2       /* device or host allocation failed */
#define KX_EADMIT -3       /* serving: footprint above the configured budget; retry later */
#define KX_ENEG -4         /* fixed-step integration produced a negative f */
#define KX_ENONFINITE -5   /* a NaN/Inf appeared in f or C */
#define KX_ESINGULAR -6    /* projection 2x2 system singular; alpha = beta = 0 used */
#define KX_ENOCONV -7      /* integration hit max_attempts before finishing */
#define KX_ETIMEOUT -8     /* a bounded device or host wait expired */
#define KX_ECUDA -9        /* a CUDA runtime/driver call failed (see kx_last_error) */
#define KX_ENOTSUP -10     /* option not supported by the library (e.g. quantum statistics on the split-TF32 path) */

/* -------------------------------------------------------------- options */
#define KX_MEASURE_ENERGY 0   /* W = dE_n dE_m F / (2 E_i g): F of eq. app_F_2d is the kernel of dE_n dE_m (default) */
#define KX_MEASURE_LITERAL 1  /* W = Dp_n Dp_m F / (2 E_i g): eq. discrete_weight read literally */

#define KX_FP64 0        /* plain FP64 path: FP64 tensor (18 B/element), FP64 contraction */
#define KX_FP32 1        /* FP32 streaming path: FP32 W + packed (j_L, omega) (8 B/element), FP32 math, FP64 sums */
#define KX_SPLIT_TF32 2  /* batched path for many f sharing one kernel: gain G = f^T W f with T = W F on the
                            tcgen05 tensor cores in split TF32 (hi*hi + hi*lo + lo*hi, FP32 accumulation in
                            tensor memory), exact FP32 loss with one exp2 per element and instance, FP64 combine */

typedef struct kx_ctx kx_ctx;
typedef struct kx_kernel kx_kernel;
typedef uint64_t kx_ticket;

/* Momentum grid and kernel options (Appendix A).  q is the comoving momentum
 * grid (host, length n, strictly ascending, > 0); p_i = q_i / a, E_i = sqrt(p_i^2 + m^2);
 * widths Dq_i are the trapezoid widths in q (the paper leaves w_i unspecified).
 * n_mu = Gauss-Legendre nodes of the mu integral of eq. app_F_1d (the paper uses 18);
 * n_mu = 0 builds the exact N_mu -> infinity kernel instead: the mu integral in
 * closed form, F = |M|^2 pi L / (4 (2 pi)^4 p_i) with L the overlap of
 * [|p_i - p_n|, p_i + p_n] and [|p_t - p_m|, p_t + p_m] (no quadrature error). */
typedef struct {
    int n;            /* 4 <= n <= 512 */
    const double *q;  /* host [n] */
    double a;         /* scale factor > 0 (1 for the static box) */
    double mass;      /* m_chi > 0 */
    int n_mu;         /* 1 <= n_mu <= 64, or 0 (exact angular kernel) */
    int measure;      /* KX_MEASURE_ENERGY | KX_MEASURE_LITERAL */
    int stats;        /* 0 = dilute f3 f4 - f1 f2 (eq. Lambda dilute); +1 Bose-Einstein, -1
                         Fermi-Dirac: the factor of eq. Lambda_quantum per element, f_t from the
                         log interpolation of f (every path; KX_SPLIT_TF32 with the exact
                         loss only: loss_terms != 0 -> KX_ENOTSUP) */
    int precision;    /* KX_FP64 | KX_FP32 | KX_SPLIT_TF32 */
    int loss_terms;   /* KX_SPLIT_TF32 only (else must be 0): 0 = exact loss (one exp2 per element
                         and instance); 8, 16 or 32 = the loss rate as a second tensor-core GEMM
                         L = M Y with the interpolated f_t of eq. app_log_interp expanded in that
                         many Chebyshev polynomials of t = 2 omega - 1:
                           f_t = f_j e^{d/2} sum_k eps_k I_k(d/2) T_k(t), d = ln f_{j+1} - ln f_j,
                           M_k[i][j] = sum_{(n,m): j_L = j} S_inm T_k(2 omega_inm - 1) (kernel table),
                           Y_k[j][b] = f_jb e^{d/2} eps_k I_k(d/2) (per call, from f).
                         Truncation error of a bracket <= max(f_j, f_{j+1}) 2 sum_{k>=K} e^{-|d|/2}
                         I_k(|d|/2); an instance with a bracket whose bound exceeds 2^-30 f_max
                         has its loss evaluated exactly instead (same result as loss_terms = 0). */
} kx_grid_desc;

/* Synthetic freeze-in sources: S_i(t) = sum_k rate_k env_k(t) shape_k,i / sum_j h_j shape_k,j,
 * env_k(t) = exp(-(t - t_on_k)/tau_k) for t >= t_on_k, else 0.  The library
 * normalises each shape row so that rate_k is the number injection rate. */
typedef struct {
    int n_src;             /* 0..4 */
    const double *shape;   /* host [n_src][n], >= 0 */
    const double *rate;    /* host [n_src] */
    const double *tau;     /* host [n_src], > 0 */
    const double *t_on;    /* host [n_src] */
} kx_source;

/* Integration controls (Sec. 4.2 adaptive Heun; controller details are this
 * library's reading: err = max_i |f_c - f_p| / (atol + rtol |f_c|), accept if
 * err <= 1 and no negative stage, h <- h min(5, max(0.2, 0.9 err^-1/2)),
 * a negative stage halves h). */
typedef struct {
    double t0, t_end, h0;
    double rtol, atol;      /* typical: 1e-6, 1e-12 max f0 */
    double h_min, h_max;
    double l1_tol;          /* stop when sources are off and L1(f, MB fit) <= l1_tol (<= 0: run to t_end) */
    int max_attempts;       /* accepted + rejected attempts before KX_ENOCONV */
    int fixed_step;         /* 1: constant h = h0, always accept, negative stage -> KX_ENEG */
    int check_every;        /* MB test every k accepted steps */
    int project;            /* 1: use the projected operator (Appendix B) */
    int chains;             /* kx_solve / kx_solve_host only (no counterpart in the paper):
                               0 = the library's rule: on the FP32 path a batch of 2..4
                               instances runs as concurrent chains, one per instance (its
                               own state, captured graph of attempts and stream), which
                               overlap one another's kernel dependency gaps; else one
                               batch; 1 = one batch; 2 = one chain per instance (batches of
                               up to 8, any path).  The results are the same bits either
                               way: an instance's arithmetic does not depend on its batch. */
} kx_solve_params;

/* Projection diagnostics (Appendix B: eq. app_epsilon_definition and
 * eq. app_projection_relative_correction). */
typedef struct {
    double eps_N_raw, eps_E_raw, eps_N_proj, eps_E_proj;
    double R_N, R_E, alpha, beta;
    double f_max;
    int singular;   /* det guard fired (alpha = beta = 0) */
    int status;     /* KX_OK or KX_ENONFINITE for this instance */
} kx_diag;

typedef struct {
    double t, h, l1_to_mb, T_mb, ln_z_mb, latency_s;
    long long steps, rejects, evals;
    int status;       /* KX_OK, KX_ENEG, KX_ENONFINITE, KX_ENOCONV, KX_ETIMEOUT */
    int converged;    /* stopping test met */
} kx_result;

typedef struct {
    int n, n_mu, measure, precision;
    long long unique_elements;   /* U = n^2 (n+1)/2 (i, n <= m) elements */
    long long nonzero_elements;  /* elements inside the kinematic support */
    long long tensor_bytes;      /* device bytes of the kernel tables */
    double build_ms;             /* device time of the build */
    long long stream_bytes;      /* table bytes one contraction launch reads: FP32 path = 36 B per
                                    4-element vector inside the kinematic support (W, packed
                                    (j_L, omega), (n, m0)) + the task table; FP64 path = 18 B per
                                    (i, n <= m) element + 4 B per pair; split path = the TF32
                                    operand tiles + the loss list */
} kx_kernel_info;

/* ------------------------------------------------------------- context */
/* Create a context on CUDA device `device` that enqueues work on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  KX_EINVAL/KX_ECUDA on failure. */
int kx_create(kx_ctx **out, int device, void *cuda_stream);
void kx_destroy(kx_ctx *ctx);
int kx_set_stream(kx_ctx *ctx, void *cuda_stream);
const char *kx_strerror(int code);
const char *kx_last_error(const kx_ctx *ctx);

/* --------------------------------------------------------------- kernel */
/* Build the kernel tensor of eq. discrete_weight for one grid (Appendix A):
 * W_inm = mu_n mu_m F_inm / (2 E_i g) with |M|^2 = 1 (sigma scales it at call
 * time), F from Gauss-Legendre over the closed-form nu integral (equal to the
 * printed arcsin form, eq. app_I_mu), zero outside E_0 <= E_n + E_m - E_i <= E_{n-1};
 * symmetrised over (n, m) and stored for n <= m, with the interpolation bracket
 * j_L and weight omega per element.  Runs on the device (FP64), synchronises
 * the stream.  The handle starts with reference count 1. */
int kx_build_kernel(kx_ctx *ctx, const kx_grid_desc *desc, kx_kernel **out);
void kx_kernel_retain(kx_kernel *k);
void kx_kernel_release(kx_kernel *k);
int kx_kernel_get_info(const kx_kernel *k, kx_kernel_info *info);
/* Copy the grid as the library sees it (host arrays [n], any may be NULL). */
int kx_kernel_grid(const kx_kernel *k, double *p, double *E, double *dp, double *dE, double *h);
/* Copy the symmetrised FP64 tables of row i (host arrays [n(n+1)/2] in
 * (n, m >= n) row-major pair order; any may be NULL).  KX_FP64 kernels only. */
int kx_kernel_row(const kx_kernel *k, int i, double *W, int *jL, double *omega);

/* ------------------------------------------------------------ collision */
/* Evaluate C[f] for `batch` distributions sharing one kernel (eq.
 * discrete_collision_operator, dilute), scaled by |M|^2 = 64 pi m^2 sigma_b.
 * f_dev, C_dev: device [batch][n] FP64.  project = 1 applies the two-moment
 * projection (Appendix B).  diag_host: NULL, or host [batch] (requires a
 * stream synchronisation inside the call).  Without diag the call only
 * enqueues work on the stream.  KX_ENONFINITE is reported through diag. */
int kx_collision(kx_ctx *ctx, const kx_kernel *k, int batch, const double *sigma_host,
                 const double *f_dev, double *C_dev, int project, kx_diag *diag_host);

/* Same as kx_collision with host input/output arrays (host [batch][n]); the
 * copies run on the context's stream; returns after C_host is written. */
int kx_collision_host(kx_ctx *ctx, const kx_kernel *k, int batch, const double *sigma_host,
                      const double *f_host, double *C_host, int project, kx_diag *diag_host);

/* Allocation-free variant of kx_collision (no counterpart in the paper; it
 * exists for callers that must not allocate GPU memory during the call, such
 * as code running inside an allocator or memory-pool callback, or a host that
 * reserved all device memory up front).  Same inputs, outputs and arithmetic as
 * kx_collision without diagnostics: f_dev, C_dev are the caller's device
 * arrays [batch][n].  Instead of the context arena it uses one scratch array
 * of 8 MiB compiled into the library (one copy per GPU that loads it, resident
 * until the process exits); it calls no cudaMalloc/cudaFree and no allocating
 * library routine.  Limits: batch <= 64 and the call's scratch (per instance:
 * the partial row sums and prepared tables) <= 8 MiB, e.g. 64 instances at
 * n = 512 on the FP32 path or 15 on the FP64 path; larger requests return KX_EINVAL
 * with a message in kx_last_error.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call outside
 * any stream capture.  That address is kept for the life of the process and
 * is not looked up again: a caller that resets the device (cudaDeviceReset, or
 * anything else that tears down its primary context) must not call this entry
 * point afterwards.  If a bounded device wait of the contraction expires, C
 * holds NaN.  All calls share the one array: calls whose work can
 * overlap on the GPU (other streams, other contexts on the same device) race
 * and must be serialised by the caller.  Only enqueues work on the stream. */
int kx_collision_noalloc(kx_ctx *ctx, const kx_kernel *k, int batch, const double *sigma_host,
                         const double *f_dev, double *C_dev, int project);

/* ---------------------------------------------------------- integration */
/* One Heun attempt per instance (Sec. 4.2): k1 = RHS(f, t), f_p = f + h k1,
 * k2 = RHS(f_p, t + h), f_c = f + h/2 (k1 + k2); accept/reject and the next h
 * as described at kx_solve_params.  t_host, h_host: host [batch], updated.
 * src: NULL, one source set shared by all instances (n_src_sets = 1) or one per
 * instance (n_src_sets = batch).  res_host: host [batch] (may be NULL). */
int kx_step(kx_ctx *ctx, const kx_kernel *k, int batch, const double *sigma_host,
            const kx_source *src, int n_src_sets, const kx_solve_params *par,
            double *t_host, double *h_host, double *f_dev, kx_result *res_host);

/* Integrate every instance until its stopping test, t_end or max_attempts.
 * The step loop is device resident (captured CUDA graph of Heun attempts with
 * on-device accept/reject, step-size control and MB stopping test); the host
 * only polls a status word.  f_dev: device [batch][n], in/out. */
int kx_solve(kx_ctx *ctx, const kx_kernel *k, int batch, const double *sigma_host,
             const kx_source *src, int n_src_sets, const kx_solve_params *par,
             double *f_dev, kx_result *res_host);

/* Same as kx_solve with host f (host [batch][n], in/out). */
int kx_solve_host(kx_ctx *ctx, const kx_kernel *k, int batch, const double *sigma_host,
                  const kx_source *src, int n_src_sets, const kx_solve_params *par,
                  double *f_host, kx_result *res_host);

/* ----------------------------------------------------------- uneven batch */
/* Integrates G batches on G different grids (an uneven batch: G <= 8
 * KX_SPLIT_TF32 kernels, kernel g with B[g] instances of sigma[g] (host
 * [B[g]]) and distributions f_dev[g] (device [B[g]][n_g], updated in place))
 * as one sequence of grouped launches: per Heun stage one gain-GEMM launch and
 * one Chebyshev-loss-GEMM launch over the work items of all G kernels, the
 * exact loss per kernel (all instances, or the Chebyshev path's flagged ones),
 * and one stage launch over all instances; eight attempts per captured CUDA
 * graph.  Each instance's arithmetic is that of kx_solve on its own kernel
 * (results are bit-identical).  par as for kx_solve (no sources, adaptive
 * steps); res[g] host [B[g]] (may be NULL).  KX_ENOTSUP for other precisions
 * or fixed steps. */
int kx_solve_grouped(kx_ctx *ctx, int G, const kx_kernel *const *kernels, const int *batch,
                     const double *const *sigma_host, const kx_solve_params *par, double *const *f_dev,
                     kx_result *const *res_host);

/* ------------------------------------------------------ expanding universe */
/* Hubble rate and the two regimes of the integration in u = ln a (Sec. 4,
 * eq. numerical_evolution_loga; Sec. 4.2).  The paper's H(a) comes from
 * Standard-Model thermodynamics that it does not list, so it is an input:
 * H(u) = exp of the piecewise-linear interpolation of ln H through the table
 * (linear extrapolation beyond it; n_h = 1: constant H; radiation domination
 * is a two-point table of slope -2). */
typedef struct {
    int n_h;               /* points of the table, >= 1 */
    const double *u;       /* host [n_h], strictly ascending (may be NULL when n_h = 1) */
    const double *ln_H;    /* host [n_h] */
    double u0, u_end;      /* integration range in u = ln a */
    double du_rk4;         /* fixed interval of the source-only RK4 regime, > 0 */
    int check_every;       /* RK4 steps between checks of Gamma_2->2 / H, >= 1 */
    double eps_switch;     /* the collisions start once Gamma_2->2 / H > eps_switch (the paper: 1e-2) */
} kx_expansion;

typedef struct {
    kx_result r;           /* u reached (r.t), Heun steps, rejects, evaluations, status */
    double u_switch;       /* u where the collisions started (NaN: never) */
    double gamma_over_H;   /* Gamma_2->2 / H at the switch, or at the last check */
    long long rk4_steps;   /* RK4 steps of the source-only regime */
    long long checks;      /* Gamma_2->2 / H evaluations */
} kx_expansion_result;

/* One distribution in an expanding universe (Sec. 4): the comoving grid q of
 * grid (grid->a is ignored; a = e^u), physical momenta p = q/a, and
 *   df/du = [C_el[f; a] + S(u)] / H(u)             (eq. numerical_evolution_loga)
 * with the kernel tensor rebuilt at the scale factor of every evaluation (it
 * depends on a through p = q/a).  Regime 1: the collisions are off and f
 * advances by classical RK4 on fixed intervals du_rk4 (the right-hand side
 * S/H does not depend on f); Gamma_2->2 = n <sigma v> -- read as the
 * number-weighted loss rate of the operator, |M|^2 sum h f nu / sum h f,
 * nu_i = sum W_inm f_t -- is compared with H at u0 and every check_every RK4
 * steps.  Regime 2, from the first check with Gamma_2->2 / H > eps_switch:
 * adaptive Heun in u (the controller of kx_solve_params: h0, rtol, atol,
 * h_min, h_max, max_attempts; t0, t_end, fixed_step, l1_tol, check_every are
 * not used) on the projected operator until u_end.  Sources: u is their clock
 * (t_on in u), shapes normalised with the comoving weights q_i^2 Dq_i, so rate_k
 * is the comoving number injected per unit time.  One instance per call (every
 * evaluation needs the kernel at its own a); f_dev is the caller's device
 * array [n], updated in place.  Precision KX_FP64 or KX_FP32 (dilute
 * statistics, exact loss); else KX_ENOTSUP.  Synchronises the stream once per
 * Heun attempt and per check. */
int kx_solve_expanding(kx_ctx *ctx, const kx_grid_desc *grid, double sigma, const kx_source *src,
                       const kx_expansion *ex, const kx_solve_params *par, double *f_dev,
                       kx_expansion_result *res);

/* -------------------------------------------------------------- serving */
/* A solve server for parameter scans (continuous batching; no counterpart in
 * the paper, which integrates one distribution at a time): requests (grid,
 * mass, sigma, sources, initial f) are queued by kx_submit; a worker thread
 * owning the context's device admits them into free slots of a per-kernel
 * group (kernel tensors are built once per grid and shared between requests,
 * kept in an LRU cache), subject to an HBM budget for kernel tables plus
 * per-slot state; every group integrates all its slots together with captured
 * CUDA graphs of Heun attempts (the Sec. 4.2 step, device-resident
 * accept/reject and stopping test), and finished requests leave their slot at
 * the next graph boundary while new ones join.  A request's result does not
 * depend on the other requests in flight (per-instance arithmetic is
 * independent of co-scheduling). */
typedef struct kx_server kx_server;
typedef struct {
    long long hbm_budget_bytes;  /* kernel tables + slot state admitted at once (> 0) */
    int slots_per_group;         /* instances integrated together per kernel tensor, 1..256 */
    int attempts_per_tick;       /* Heun attempts per captured graph launch, 1..64 */
    int precision;               /* KX_FP32 | KX_FP64 | KX_SPLIT_TF32 for every kernel */
    int n_mu, measure;           /* kernel options of every request */
    kx_solve_params par;         /* integration controls of every request (t0, t_end, h0
                                    are per request; see kx_submit) */
    int grid_div;                /* while more than 8 groups have work, the FP32 streaming
                                    contraction of each group launches with 1/grid_div of
                                    the GPU's resident blocks, so that several groups'
                                    contractions run side by side; with fewer, with all of
                                    them (results do not depend on it); 1..16, 0 = 2 */
    int loss_terms;              /* kx_grid_desc.loss_terms of every kernel (KX_SPLIT_TF32) */
} kx_server_config;

typedef struct {
    long long submitted, completed, failed, queued, active;
    long long kernels_built, kernel_cache_hits, evictions;
    double p50_latency_s, p99_latency_s, mean_latency_s;   /* submit -> result available */
    double p50_wait_s;                                     /* submit -> admitted */
    long long evals;                                       /* collision evaluations done */
    long long converged;          /* completed solves that met the L1 stopping test */
    long long ticks_shared;       /* group graph launches on a share (1/grid_div) of the GPU */
    long long ticks_whole;        /* group graph launches on the whole GPU */
    double p99_wait_s;            /* submit -> admitted */
    double p50_service_s, p99_service_s;   /* admitted -> result available */
    long long stream_bytes;       /* sum over the completed solves of evaluations x the
                                     kernel's stream_bytes: the table bytes the solves'
                                     contractions stream when each runs alone (the two
                                     slots of a group share one pass; small tables can
                                     stay in L2), an upper bound of the algorithmic reads */
} kx_server_stats;

/* Start a server on the context's device (the context's stream is not used).
 * KX_EINVAL on a bad configuration. */
int kx_server_start(kx_ctx *ctx, const kx_server_config *cfg, kx_server **out);
/* Queue one solve.  grid: n, q (host, copied), a, mass (n_mu, measure and
 * precision come from the server).  src: NULL or one source set (copied).
 * f0_host: [n] (copied).  t0, t_end, h0: this request's interval and first
 * step.  Returns KX_EADMIT when the request can never fit the budget. */
int kx_submit(kx_server *srv, const kx_grid_desc *grid, double sigma, const kx_source *src,
              double t0, double t_end, double h0, const double *f0_host, kx_ticket *ticket);
/* Wait up to timeout_s (>= 0) for a request.  KX_OK: done, f_out_host [n]
 * (nullable) and *res filled, ticket released; KX_PENDING: not finished;
 * other codes: the request failed (ticket released) or the ticket is unknown. */
int kx_poll(kx_server *srv, kx_ticket ticket, double timeout_s, double *f_out_host,
            kx_result *res);
int kx_server_get_stats(kx_server *srv, kx_server_stats *out);
/* Starts a new sample for the latency quantiles of kx_server_get_stats (the
 * requests completed from now on); the counters stay cumulative.  KX_EINVAL
 * for a null server. */
int kx_server_reset_latency(kx_server *srv);
/* Finish the requests in flight, stop the worker and free the server. */
void kx_server_stop(kx_server *srv);

/* ------------------------------------------------------ fault injection */
/* For tests of the failure paths, the environment variable KX_FAULT (read at
 * each check; a comma-separated list) makes the host side of the library fail
 * on purpose.  No injected failure touches the GPU: kernels never fault, trap
 * or wait on anything that is not set.
 *   alloc    every device allocation the library makes (context arena, kernel
 *            tables) fails: KX_ENOMEM, with the message in kx_last_error;
 *   admit    kx_submit refuses every request: KX_EADMIT;
 *   nan      kx_collision_host and kx_solve_host stage f[0][0] = NaN after the
 *            host->device copy: KX_ENONFINITE (in the diagnostics / the first
 *            instance's result);
 *   timeout  kx_solve and kx_solve_host stop polling at once: the graphs
 *            already launched run to their end, then KX_ETIMEOUT. */

/* ------------------------------------------------------------ profiling */
/* Number of this library's kernels enqueued through `ctx` so far (a captured
 * graph counts each of its kernel nodes at every launch). */
long long kx_launch_count(const kx_ctx *ctx);

/* Time the contraction kernel alone (eq. discrete_collision_operator, the
 * O(N^3) step) for `batch` instances of f_dev: prepares the inputs once, then
 * launches the contraction `iters` times on the context's stream bracketed by
 * CUDA events and returns the mean device time per launch in *avg_ms.  If
 * flush_bytes > 0, a device buffer of that size (allocated here) is rewritten
 * between launches, outside the timed events, so each launch starts with a
 * cold L2.  Synchronises the stream. */
int kx_time_contraction(kx_ctx *ctx, const kx_kernel *k, int batch, const double *f_dev,
                        int iters, long long flush_bytes, double *avg_ms);

/* Time one full evaluation of C[f] for `batch` instances: the work of
 * kx_collision without diagnostics (prepare f, contraction, row combine and
 * the projection if `project`), captured once as a CUDA graph and launched
 * `iters` times back to back between two CUDA events on the context's stream;
 * *avg_ms = device time per evaluation.  Arguments as in kx_collision; C_dev
 * [batch][n] (device) receives C[f].  Errors as kx_collision, KX_EINVAL for
 * iters < 1 or a null avg_ms.  Synchronises the stream. */
int kx_time_collision(kx_ctx *ctx, const kx_kernel *k, int batch, const double *sigma_host,
                      const double *f_dev, double *C_dev, int project, int iters, double *avg_ms);

/* Time contractions of several kernels of one grid size issued back to back:
 * prepares f_dev [batch][n] (device) for each of the nk kernels ks[0..nk-1]
 * (library-owned, all with the same n), then launches the contraction of
 * ks[0], ks[1], ..., ks[nk-1], `iters` times over, on the context's stream
 * between two CUDA events; *avg_ms = device time / (iters * nk).  With
 * kernels whose tables together exceed the L2 cache, every launch streams its
 * tables from HBM (rotating buffers) while the launches still follow each
 * other as in a solve.  pdl != 0: the FP32 streaming contractions launch with
 * programmatic stream serialization, as inside the solve's graphs (a launch
 * issues its first table loads while its predecessor finishes; the other
 * paths ignore the flag).  KX_EINVAL for nk < 1, a null kernel, mixed sizes or
 * bad arguments; KX_ECUDA on a CUDA error.  Synchronises the stream. */
int kx_time_contractions(kx_ctx *ctx, int nk, const kx_kernel *const *ks, int batch,
                         const double *f_dev, int iters, int pdl, double *avg_ms);

/* Moment-matched discrete Maxwell-Boltzmann fit used by the stopping test:
 * out_host[batch][3] = (T, ln z, L1) with L1 = sum h |f - f_MB| / sum h f. */
int kx_mb_fit(kx_ctx *ctx, const kx_kernel *k, int batch, const double *f_dev, double *out_host);

/* ------------------------------------------------ the paper's sources */
/* The two freeze-in source terms of Sec. 2 as rows for kx_source (host
 * functions, no device work).  q: host [n] comoving grid (ascending, > 0) and
 * a the scale factor, as in kx_grid_desc (p_i = q_i / a); mass = m_chi.
 * shape: host [n] out; rate: out, the row's number injection rate
 * (sum_i h_i S_i with h_i = p_i^2 dp_i, the grid's weights), so that
 * {shape, rate, tau, t_on} in kx_source reproduce the formula times the
 * envelope.  KX_EINVAL for a bad grid or parameters.
 *
 * Higgs decay into dark matter (eq. C_higgs_decay):
 *   S(p) = coupling^2 / (8 pi g_chi) * T / (E p) * (exp(-E_h^-(p)/T) - exp(-E_h^+(p)/T)),
 *   E_h^(+/-) = (m_h^2 E +/- m_h p sqrt(m_h^2 - 4 m_chi^2)) / (2 m_chi^2),
 * coupling = lambda_Hchi v, T the bath temperature (m_h > 2 m_chi, T > 0);
 * shape = S(p_i), rate = sum_i h_i S(p_i). */
int kx_source_higgs_decay(int n, const double *q, double a, double mass, double m_h, double T,
                          double coupling, double g_chi, double *shape, double *rate);

/* Decay of a cold condensate (eq. C_condensate_decay):
 *   S(p) = (2 pi^2 / g_chi) gamma_n delta(p - p0) / p0^2,  p0 = sqrt(m_phi^2 - 4 m_chi^2) / 2,
 * gamma_n = 2 Gamma_Phi n_Phi.  The delta function is binned into the one grid
 * cell (trapezoid widths in q) containing a p0: shape = 1 there, 0 elsewhere,
 * rate = (2 pi^2 / g_chi) gamma_n, the formula's number injection exactly.
 * KX_EINVAL also when p0 lies outside the grid. */
int kx_source_condensate(int n, const double *q, double a, double mass, double m_phi, double g_chi,
                         double gamma_n, double *shape, double *rate);

/* ----------------------------------------------------------- diagnostics */
/* The split-TF32 path's launch choices (no counterpart in the paper): the
 * gain and Chebyshev-loss GEMMs' ring depth and f' staging, the gain's A
 * operand (the generated f'_n f'_m tile) in tensor or shared memory, per
 * launch shape, and the exact loss kernel's instances per lane, per
 * (n, batch).  None of
 * them changes a result; each is timed on the launch's own operands the first
 * time the shape is launched outside a stream capture and kept for the
 * process.  kx_set_split_tuning(0) switches the timing off and forgets the
 * choices (the default rule applies), 1 switches it on.  kx_get_split_tuning
 * reports the choices a whole-batch launch of kernel k with B instances uses:
 * *gain_S, *gain_fs (1: f' staged), *loss_S (0 without the Chebyshev loss),
 * *loss_ipl, *tuned (bit 0 gain, bit 1 Chebyshev loss, bit 2 exact loss:
 * timed rather than the rule) and *gain_atm (1: A in tensor memory).
 * kx_set_gain_operand(where) restricts the gain's A operand for later
 * launches (and forgets the timed GEMM choices): 0 either (the default; the
 * rule takes tensor memory), 1 shared memory only, 2 tensor memory only.
 * KX_EINVAL for bad arguments, KX_ENOTSUP for a kernel of another path. */
int kx_set_split_tuning(int enabled);
int kx_set_gain_operand(int where);
int kx_get_split_tuning(const kx_kernel *k, int B, int *gain_S, int *gain_fs, int *loss_S, int *loss_ipl,
                        int *tuned, int *gain_atm);

/* Bounds-checked build (no counterpart in the paper): libkx_check.so is this
 * library compiled with -DKX_CHECK.  Its contraction and loss kernels test
 * their table, bracket, task and slot indices against the arrays' lengths;
 * a failed test records the first failing site and index (and a count) and
 * uses index 0 instead, so that no access leaves its array.  kx_check_status
 * reports *checked = 1 in that build (0 in libkx.so, whose records stay 0),
 * the failures since the last reset, and the first failure's site and index
 * (reset != 0 clears the records after reading them).  Synchronises the
 * context's stream.  KX_EINVAL for null arguments, KX_ECUDA on a CUDA error. */
int kx_check_status(kx_ctx *ctx, int reset, int *checked, long long *failures, int *first_site,
                    long long *first_index);
/* Passes `index` through the same check with the bound `limit` (>= 0) in a
 * one-thread kernel and writes its result to *result (host): index when
 * 0 <= index < limit, else 0 and a recorded failure in the checked build;
 * index in the normal build.  No memory is addressed with the index.
 * KX_EINVAL for bad arguments, KX_ECUDA on a CUDA error. */
int kx_check_probe(kx_ctx *ctx, int index, int limit, int *result);

/* ALU throughput of the device (a diagnostic for rooflines, no counterpart in
 * the paper): times a grid of 8 blocks per SM running independent chains of
 * FP64 fused multiply-adds and of ex2.approx (the special-function unit) and
 * writes the best of three runs: *fp64_flops (FMA = 2 flops, per second) and
 * *ex2_per_s (host pointers).  Synchronises the context's stream.  KX_EINVAL
 * for null arguments, KX_ECUDA on a CUDA error. */
int kx_measure_peaks(kx_ctx *ctx, double *fp64_flops, double *ex2_per_s);

/* Tensor-core issue rate (a diagnostic for the batched path's roofline, no
 * counterpart in the paper): one thread per SM issues 4096 tcgen05.mma of
 * M = 128, N = n (16 .. 256, a multiple of 16), K = 8 with TF32 operands (kind
 * 0) or K = 16 with BF16 operands (kind 1) from shared-memory tiles into tensor
 * memory and waits for them; writes the FLOP per clock per SM and the cycles
 * per MMA (host pointers).  Synchronises the context's stream.  KX_EINVAL for
 * bad arguments, KX_ECUDA on a CUDA error or an expired wait. */
int kx_measure_mma_rate(kx_ctx *ctx, int kind, int n, double *flop_per_clk_sm, double *cycles_per_mma);

/* Per-kernel timing of the solve's attempts (a diagnostic, no counterpart in
 * the paper): sets up a solve of the B instances of f_dev exactly as kx_solve
 * does (same arguments), prepares f and runs `attempts` (1 .. 100000) real
 * Heun attempts whose four kernels (contraction, stage 1, contraction, stage
 * 2) are launched in plain stream order with CUDA events between them, then
 * writes to us[0..3] (host) the average microseconds of each of the four.
 * Without the programmatic overlap of the solve's graphs each time includes
 * the kernel's launch and its wait on its predecessor's tail.  f_dev is
 * advanced by the attempts (pass a copy).  Synchronises the context's stream.
 * KX_EINVAL for bad arguments, KX_ECUDA on a CUDA error. */
int kx_profile_attempts(kx_ctx *ctx, const kx_kernel *k, int B, const double *sigma, const kx_source *src,
                        int nsets, const kx_solve_params *par, double *f_dev, int attempts, double *us);

/* Self-check of the library's own arithmetic helpers (the stage kernels use
 * them for the per-point log of f, the source envelopes, the Maxwell-Boltzmann
 * fit and the FP32 path's integer-pipe conversions; they have no counterpart
 * in the paper).  For n arguments x_dev (device, n doubles), writes
 * out_dev[2i] = the library's value and out_dev[2i+1] = CUDA's value, for
 *   which = 0: the table-driven FP64 log2 (x >= 1e-300);
 *   which = 1: the FP64 exp;
 *   which = 2: the double-float log2 of the FP32 path's tables, e + hi + lo
 *              (positive normal x);
 *   which = 3: double -> float rounding on the integer pipe (as a double;
 *              the library flushes results below 2^-126 to zero);
 *   which = 4: float -> double on the integer pipe, of the float nearest x.
 * Enqueues on the context's stream.  KX_EINVAL for bad arguments, KX_ECUDA
 * if the launch fails. */
int kx_math_check(kx_ctx *ctx, int which, int n, const double *x_dev, double *out_dev);

/* Self-check of the bounded device waits (no counterpart in the paper): every
 * mbarrier wait of the library's kernels gives up after a cycle limit, sets an
 * error flag and lets the kernel return, so that a lost copy cannot hang the
 * GPU (the contraction then reports KX_ETIMEOUT: NaN in C, the diag status and
 * the return value of kx_collision with diag, the instance status of a solve).
 * This call launches one thread that waits, with a limit of `cycles` SM clock
 * cycles (1 .. 2^32), on an mbarrier that nothing arrives on; *expired_host = 1
 * when the wait gave up, as it must.  Synchronises the context's stream. */
int kx_wait_check(kx_ctx *ctx, long long cycles, int *expired_host);

/* Pins the FP32 path's streaming variant for grids of n points and batches of
 * `batch` instances on the context's device, in place of the autotuner's
 * choice (which is otherwise timed once per (device, n, batch) before the
 * first launch): 0 = one instance per pass, 1 = two per pass (batch >= 2),
 * 2 = four per pass, bulk-copy staged (n > 160, batch >= 4), 3 = four per
 * pass, register pipeline (batch >= 4), 4 = the whole batch per pass with
 * every warp's share of the tables staged in shared memory before the
 * contraction waits for its predecessor (batch <= 4; used where the kernel's
 * bins fit in shared memory and the launch has the whole GPU, else the
 * default rule applies); -1 forgets the pinned or tuned choice.  The pin applies to whole-GPU launches and to the
 * serving groups' launches on a share of the GPU alike (the autotuner keys its
 * choice by that share as well).  All variants give bit-identical results; this is
 * for reproducible timing and for tests.  KX_EINVAL for a variant that does
 * not apply. */
int kx_set_stream_variant(kx_ctx *ctx, int n, int batch, int variant);

/* The FP32 streaming variant (numbering as for kx_set_stream_variant) that
 * whole-GPU contractions of n-point grids with `batch` instances use on the
 * context's device: the pinned or tuned one (*tuned = 1; tuned = NULL allowed), else the
 * rule used before tuning (*tuned = 0).  KX_EINVAL for bad arguments. */
int kx_get_stream_variant(kx_ctx *ctx, int n, int batch, int *variant, int *tuned);

#ifdef __cplusplus
}
#endif
#endif /* KX_H_ */
