// kx_build.cu -- device build of the collision-kernel tensor (Appendix A).
//
// Compiled with -fmad=false: every expression below is evaluated as written,
// operation by operation, in IEEE FP64, so that the kinematic-support and
// Theta(K^2 + A1^2 - A0^2) decisions are reproducible bit for bit from the
// same grid values.
#include "kx_internal.cuh"

#define KX_PI 3.14159265358979323846

// Index of pair (n, n) in the row-major n <= m pair order.
__device__ __forceinline__ long long kx_pair_base(int n, int N) {
    return (long long)n * N - (long long)n * (n - 1) / 2;
}

// Largest j <= N-2 with E[j] <= Et, for E[0] <= Et (bisection on ascending E).
__device__ __forceinline__ int kx_bracket(const double *E, int N, double Et) {
    int lo = 0, hi = N - 2;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (E[mid] <= Et) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Angular kernel of eq. (app_F_1d) with |M|^2 = 1:
//   F = p_n p_m / (4 (2 pi)^4) sum_k w_k I(mu_k),
// I(mu) = pi / sqrt(K^2 + A1^2) when K^2 + A1^2 - A0^2 >= 0 (the nu integral of
// eq. app_I_mu over its root interval, which lies inside [-1, 1]), else 0;
// A0, A1, K^2 as defined below eq. (app_cosphi).
__device__ double kx_F_unit(double m, double pi, double pn, double pm, double Ei, double En,
                            double Em, const kx_gl_nodes &gl, int n_mu) {
    double acc = 0.0;
    for (int k = 0; k < n_mu; ++k) {
        double mu = gl.x[k];
        double A0 = m * m + En * Em - En * Ei - Em * Ei + pi * pn * mu;
        double A1 = pi * pm - pn * pm * mu;
        double K2 = pn * pn * pm * pm * (1.0 - mu * mu);
        double s = K2 + A1 * A1;
        double D = s - A0 * A0;
        if (s > 0.0 && D >= 0.0) acc += gl.w[k] * (KX_PI / sqrt(s));
    }
    double two_pi = 2.0 * KX_PI;
    return 1.0 * pn * pm / (4.0 * two_pi * two_pi * two_pi * two_pi) * acc;
}

// The N_mu -> infinity limit of kx_F_unit in closed form (|M|^2 = 1): with
// k^2 = p_i^2 + p_n^2 - 2 p_i p_n mu, K^2 + A1^2 = p_m^2 k^2 and the Theta
// condition is the triangle condition k in [|p_t - p_m|, p_t + p_m]; the mu
// integral of pi / (p_m k) dmu = pi / (p_i p_n p_m) dk gives
//   F = pi L / (4 (2 pi)^4 p_i),
// L = max(0, min(p_i + p_n, p_t + p_m) - max(|p_i - p_n|, |p_t - p_m|)).
__device__ double kx_F_exact_unit(double pi, double pn, double pm, double pt) {
    double lo1 = fabs(pi - pn), hi1 = pi + pn;
    double lo2 = fabs(pt - pm), hi2 = pt + pm;
    double lo = lo1 > lo2 ? lo1 : lo2;
    double hi = hi1 < hi2 ? hi1 : hi2;
    double L = hi - lo;
    if (L < 0.0) L = 0.0;
    double two_pi = 2.0 * KX_PI;
    return 1.0 * KX_PI * L / (4.0 * two_pi * two_pi * two_pi * two_pi * pi);
}

// One thread per (i, pair n <= m).  Writes the symmetrised weight
// S_inm = W_inm + W_imn (n < m) or W_inn, the bracket j_L and omega_R of
// eq. (app_interp_weights).  W_inm = mu_n mu_m F_inm / (2 E_i g), g = 1, with
// mu = dE (energy measure) or Dp (literal measure).  Outside the support
// E_0 <= E_t <= E_{N-1}, E_t = (E_n + E_m) - E_i (eq. app_fourth_momentum),
// everything is zero.
__global__ void k_build_fp64(int N, long long P, int n_mu, int measure, double m,
                             const double *__restrict__ p, const double *__restrict__ E,
                             const double *__restrict__ dp, const double *__restrict__ dE,
                             const uint32_t *__restrict__ pair, kx_gl_nodes gl,
                             double *__restrict__ W, double *__restrict__ om,
                             uint16_t *__restrict__ jl) {
    long long pidx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (pidx >= P) return;
    uint32_t pr = pair[pidx];
    int n = pr & 0xffff, mm = pr >> 16;
    long long e = (long long)i * P + pidx;
    double Et = (E[n] + E[mm]) - E[i];
    if (!(Et >= E[0] && Et <= E[N - 1])) {
        W[e] = 0.0;
        om[e] = 0.0;
        jl[e] = 0;
        return;
    }
    int j = kx_bracket(E, N, Et);
    double omega = (Et - E[j]) / (E[j + 1] - E[j]);
    double mun = measure == KX_MEASURE_LITERAL ? dp[n] : dE[n];
    double mum = measure == KX_MEASURE_LITERAL ? dp[mm] : dE[mm];
    // n_mu = 0: the exact angular kernel (no quadrature)
    const double pt = n_mu == 0 ? sqrt(Et * Et - m * m) : 0.0;
    double F1 = n_mu == 0 ? kx_F_exact_unit(p[i], p[n], p[mm], pt)
                          : kx_F_unit(m, p[i], p[n], p[mm], E[i], E[n], E[mm], gl, n_mu);
    double W1 = mun * mum * F1 / (2.0 * E[i] * 1.0);
    double S = W1;
    if (n != mm) {
        double F2 = n_mu == 0 ? kx_F_exact_unit(p[i], p[mm], p[n], pt)
                              : kx_F_unit(m, p[i], p[mm], p[n], E[i], E[mm], E[n], gl, n_mu);
        double W2 = mum * mun * F2 / (2.0 * E[i] * 1.0);
        S = W1 + W2;
    }
    W[e] = S;
    om[e] = omega;
    jl[e] = (uint16_t)j;
}

cudaError_t kx_launch_build_fp64(const kx_kernel *k, const kx_gl_nodes &gl, cudaStream_t s) {
    dim3 block(128);
    dim3 grid((unsigned)((k->P + block.x - 1) / block.x), k->n);
    k_build_fp64<<<grid, block, 0, s>>>(k->n, k->P, k->n_mu, k->measure, k->mass, k->d_p, k->d_E,
                                        k->d_dp, k->d_dE, k->d_pair, gl, k->d_W64, k->d_om64,
                                        k->d_jl);
    return cudaGetLastError();
}

// Kinematic support per 4-element vector (n, m0..m0+3) of the global vector
// list, one block per row i: pos[i][v] = index of vector v among row i's
// vectors with an element inside the support (W != 0), or -1; cnt[i] = their
// number.  Block-wide exclusive scan in tiles of blockDim vectors.
// keep_all: every vector kept (pos[i][v] = v), for kernels rebuilt at other
// scale factors, whose layout must not depend on the support.
__global__ void k_keep_scan(int N, long long P, int V, const uint32_t *__restrict__ vt,
                            const double *__restrict__ W64, int *__restrict__ pos,
                            int *__restrict__ cnt, int keep_all) {
    __shared__ int s_warp[32];
    __shared__ int s_base;
    const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int v0 = 0; v0 < V; v0 += blockDim.x) {
        const int v = v0 + tid;
        int keep = 0;
        if (v < V && keep_all) keep = 1;
        else if (v < V) {
            const uint32_t t = vt[v];
            const int n = t & 0xffff, m0 = t >> 16;
            const long long base = (long long)i * P + kx_pair_base(n, N);
            for (int c = 0; c < 4; ++c) {
                const int m = m0 + c;
                if (m < N && W64[base + (m - n)] != 0.0) keep = 1;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int wpre = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) s_warp[w] = __popc(bal);
        __syncthreads();
        if (w == 0) {
            int x = lane < nw ? s_warp[lane] : 0;
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += y;
            }
            if (lane < nw) s_warp[lane] = x;   // inclusive
        }
        __syncthreads();
        const int wbase = w ? s_warp[w - 1] : 0;
        if (v < V) pos[(long long)i * V + v] = keep ? s_base + wbase + wpre : -1;
        __syncthreads();
        if (tid == 0) s_base += s_warp[nw - 1];
        __syncthreads();
    }
    if (tid == 0) cnt[i] = s_base;
}

cudaError_t kx_launch_keep_scan(const kx_kernel *k, const uint32_t *d_vt_all, int V, int *d_pos,
                                int *d_cnt, cudaStream_t s, bool keep_all) {
    k_keep_scan<<<k->n, 1024, 0, s>>>(k->n, k->P, V, d_vt_all, k->d_W64, d_pos, d_cnt, keep_all ? 1 : 0);
    return cudaGetLastError();
}

// FP32 streaming tables, rows compacted to their kept vectors.  Kept vector v
// of row i (index k = pos[i][v] in the row) goes to d_roff[i] + k with its
// (n, m0) in d_vt and its four elements (W as float, pk = j_L << 23 |
// round(omega 2^23)) in slots rotated by r = (k >> 2) & 3: slot s holds
// element m0 + ((s + r) & 3).  The streaming kernel reads row vector k in lane
// k mod 32, so at each slot the lanes of a warp touch grid points spread over
// all shared-memory banks.  omega quantised to 2^-23; omega that rounds to 1 is
// stored as (j_L + 1, 0).  Elements outside the support (and past the row end)
// have W = 0 and pk = 0.
__global__ void k_pack_fp32(int N, long long P, int V, const uint32_t *__restrict__ vt_all,
                            const int *__restrict__ pos, const int *__restrict__ roff,
                            const double *__restrict__ W64, const double *__restrict__ om64,
                            const uint16_t *__restrict__ jl, uint32_t *__restrict__ vt,
                            float *__restrict__ W32, uint32_t *__restrict__ pk) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (v >= V) return;
    const int kk = pos[(long long)i * V + v];
    if (kk < 0) return;
    const uint32_t t = vt_all[v];
    const int n = t & 0xffff, m0 = t >> 16;
    const long long dst = (long long)roff[i] + kk;
    vt[dst] = t;
    const long long out = dst * 4;
    const long long base = (long long)i * P + kx_pair_base(n, N);
    const int r = (kk >> 2) & 3;
    for (int sl = 0; sl < 4; ++sl) {
        const int c = (sl + r) & 3;
        const int m = m0 + c;
        float w = 0.f;
        uint32_t word = 0u;
        if (m < N) {
            const long long e = base + (m - n);
            const double wd = W64[e];
            if (wd != 0.0) {
                w = (float)wd;
                uint32_t j = jl[e];
                double q = rint(om64[e] * 8388608.0);
                // omega rounding to 1 is stored as the next grid point with omega = 0,
                // so that E_t on a grid point interpolates exactly (j + 1 <= N - 1)
                if (q >= 8388608.0) {
                    j += 1;
                    q = 0.0;
                }
                word = (j << 23) | (uint32_t)q;
            }
        }
        W32[out + sl] = w;
        pk[out + sl] = word;
    }
}

cudaError_t kx_launch_pack_fp32(const kx_kernel *k, const uint32_t *d_vt_all, int V,
                                const int *d_pos, cudaStream_t s) {
    dim3 block(128);
    dim3 grid((unsigned)((V + block.x - 1) / block.x), k->n);
    k_pack_fp32<<<grid, block, 0, s>>>(k->n, k->P, V, d_vt_all, d_pos, k->d_roff, k->d_W64,
                                       k->d_om64, k->d_jl, k->d_vt, k->d_W32, k->d_pk);
    return cudaGetLastError();
}

__global__ void k_count_nnz(long long total, const double *__restrict__ W,
                            unsigned long long *count) {
    unsigned long long local = 0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        local += W[e] != 0.0;
    for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(count, local);
}

cudaError_t kx_launch_count_nnz(const kx_kernel *k, unsigned long long *d_count, cudaStream_t s) {
    k_count_nnz<<<592, 256, 0, s>>>((long long)k->n * k->P, k->d_W64, d_count);
    return cudaGetLastError();
}
