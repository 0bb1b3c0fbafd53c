/*
 * kx_oracle.c -- plain, slow, FP64 CPU oracle for the discretised 2->2 elastic
 * self-collision operator of "KineticXGPU: A Tensorized Collision Operator for
 * Dark-Sector Self-Scattering" (arXiv 2607.00755).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; it is used by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline / reference leg of bench.py.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * Every function follows the paper's definitions in the paper's order, with no
 * blocking, fusion or reordering:
 *   grid                Appendix A (p_i = q_i/a, E_i, Delta p_i, h_i = p_i^2 Delta p_i)
 *   Gauss-Legendre      Appendix A, eq. (app_F_1d): "remaining mu integral ... Gauss-Legendre"
 *   nu integral         Appendix A, eqs. (app_cosphi)-(app_I_mu)
 *   kernel F, W         eqs. (app_F_1d), (discrete_weight)
 *   interpolation       eqs. (app_interp_weights), (app_log_interp)
 *   C_raw               eqs. (discrete_collision_operator) / (app_dense_collision)
 *   projection          Appendix B, eqs. (app_self_projection), (app_projection_system)
 *   diagnostics         eqs. (app_epsilon_definition), (app_projection_relative_correction)
 *   Heun integrator     Sec. 4.2 ("Euler predictor ... corrected using the average of the slopes")
 *
 * Readings where the paper is silent or ambiguous (energy measure, trapezoid
 * weights, log floor, bracket tie-break, det guard, Heun controller, synthetic
 * sources) are listed in the design notes and repeated at each use below.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 * (no FMA contraction, so that the support and Theta decisions are exactly the
 * IEEE results of the written expressions).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_LOG_FLOOR 1e-300   /* "small positive floor" in the log, Appendix A (reading A5) */
#define OR_EPS_SUPP 1e-12     /* support cutoff epsilon_supp, Appendix B */
#define OR_DET_GUARD 1e-14    /* relative det guard of the 2x2 system (reading A10) */

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2, OR_ENEG = -4, OR_ENONFINITE = -5,
       OR_ESINGULAR = -6, OR_ENOCONV = -7 };

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ grid --- */
/* Appendix A: p_i = q_i / a, E_i = sqrt(p_i^2 + m^2), Delta p_i = Delta q_i / a,
 * h_i = p_i^2 Delta p_i.  The paper leaves the quadrature weights w_i / Delta q_i
 * unspecified; reading A2: trapezoid in q,
 *   Dq_0 = (q_1-q_0)/2,  Dq_i = (q_{i+1}-q_{i-1})/2,  Dq_{N-1} = (q_{N-1}-q_{N-2})/2.
 * dE_i = p_i Dp_i / E_i is the energy width used by the energy measure (reading A1). */
int oracle_grid(int n, const double *q, double a, double mass,
                double *p, double *E, double *dp, double *dE, double *h) {
    if (n < 4 || !(a > 0) || !(mass > 0)) return OR_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!(q[i] > 0)) return OR_EINVAL;
        if (i > 0 && !(q[i] > q[i - 1])) return OR_EINVAL;
    }
    for (int i = 0; i < n; ++i) {
        double dq;
        if (i == 0) dq = (q[1] - q[0]) / 2.0;
        else if (i == n - 1) dq = (q[n - 1] - q[n - 2]) / 2.0;
        else dq = (q[i + 1] - q[i - 1]) / 2.0;
        p[i] = q[i] / a;
        E[i] = sqrt(p[i] * p[i] + mass * mass);
        dp[i] = dq / a;
        dE[i] = p[i] * dp[i] / E[i];
        h[i] = p[i] * p[i] * dp[i];
    }
    return OR_OK;
}

/* ------------------------------------------------------- Gauss-Legendre --- */
/* Nodes/weights on [-1,1]: Newton iteration on P_n from the classical cosine
 * initial guesses; P_n and P_n' from the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};  w = 2 / ((1-x^2) P_n'(x)^2).
 * Nodes are returned in ascending order. */
int oracle_gauss_legendre(int n, double *x, double *w) {
    if (n < 1) return OR_EINVAL;
    for (int k = 0; k < n; ++k) {
        double z = cos(OR_PI * (k + 0.75) / (n + 0.5));
        double dpn = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 1; j < n; ++j) {
                double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? z : p1;
            double pnm1 = (n == 1) ? 1.0 : p0;
            dpn = n * (z * pn - pnm1) / (z * z - 1.0);
            double dz = pn / dpn;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged node */
        {
            double p0 = 1.0, p1 = z;
            for (int j = 1; j < n; ++j) {
                double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? z : p1;
            double pnm1 = (n == 1) ? 1.0 : p0;
            dpn = n * (z * pn - pnm1) / (z * z - 1.0);
        }
        x[n - 1 - k] = z;  /* cos guesses descend in k: store ascending */
        w[n - 1 - k] = 2.0 / ((1.0 - z * z) * dpn * dpn);
    }
    return OR_OK;
}

/* ------------------------------------------------ angular coefficients --- */
/* Appendix A, definitions below eq. (app_cosphi):
 *   A0 = m^2 + E_n E_m - E_n E_i - E_m E_i + p_i p_n mu
 *   A1 = p_i p_m - p_n p_m mu
 *   K^2 = p_n^2 p_m^2 (1 - mu^2)                                        */
void oracle_angular_coeffs(double m, double pi, double pn, double pm,
                           double Ei, double En, double Em, double mu,
                           double *A0, double *A1, double *K2) {
    *A0 = m * m + En * Em - En * Ei - Em * Ei + pi * pn * mu;
    *A1 = pi * pm - pn * pm * mu;
    *K2 = pn * pn * pm * pm * (1.0 - mu * mu);
}

/* nu integral, "direct" form exactly as printed in eq. (app_I_mu):
 * a = -(K^2 + A1^2), b = -2 A0 A1, c = K^2 - A0^2, Delta = b^2 - 4ac;
 * zero if Delta < 0 or the root interval misses [-1,1]; otherwise the roots are
 * clipped to [-1,1] and I = [asin((2a nu_- + b)/sqrt(Delta)) - asin((2a nu_+ + b)/sqrt(Delta))]/sqrt(-a).
 * A tie Delta == 0 is the limit of a vanishing interval whose integral tends to
 * pi/sqrt(-a) (reading A8); asin arguments are clamped to [-1,1]. */
double oracle_nu_integral_arcsin(double A0, double A1, double K2) {
    double a = -(K2 + A1 * A1);
    double b = -2.0 * A0 * A1;
    double c = K2 - A0 * A0;
    if (!(a < 0.0)) return 0.0;
    double disc = b * b - 4.0 * a * c;
    if (disc < 0.0) return 0.0;
    if (disc == 0.0) return OR_PI / sqrt(-a);
    double sq = sqrt(disc);
    double r1 = (-b + sq) / (2.0 * a);
    double r2 = (-b - sq) / (2.0 * a);
    double lo = r1 < r2 ? r1 : r2;
    double hi = r1 < r2 ? r2 : r1;
    int clip_lo = 0, clip_hi = 0;
    if (lo < -1.0) { lo = -1.0; clip_lo = 1; }
    if (hi > 1.0) { hi = 1.0; clip_hi = 1; }
    if (!(lo < hi)) return 0.0;
    /* At an unclipped root the asin argument is exactly +1 (lower root) or -1
     * (upper root, a < 0) by the quadratic formula: 2 a r + b = +-sqrt(Delta).
     * Substituting the rounded root instead would lose ~8 digits (asin is
     * ill-conditioned at +-1), so the exact value is used there. */
    double s_lo = clip_lo ? (2.0 * a * lo + b) / sq : 1.0;
    double s_hi = clip_hi ? (2.0 * a * hi + b) / sq : -1.0;
    if (s_lo > 1.0) s_lo = 1.0;
    if (s_lo < -1.0) s_lo = -1.0;
    if (s_hi > 1.0) s_hi = 1.0;
    if (s_hi < -1.0) s_hi = -1.0;
    return (asin(s_lo) - asin(s_hi)) / sqrt(-a);
}

/* nu integral, closed form: with Delta = 4 K^2 (K^2 + A1^2 - A0^2) >= 0 the
 * quadratic is <= 0 at nu = +-1 (it equals -(A0 +- A1)^2 there) and its vertex
 * lies in [-1,1], so the whole root interval is inside [-1,1] and the integral
 * of 1/sqrt(a nu^2 + b nu + c) over it is pi/sqrt(-a) = pi/sqrt(K^2 + A1^2).
 * Theta(K^2 + A1^2 - A0^2), tie included (reading A8). */
double oracle_nu_integral_closed(double A0, double A1, double K2) {
    double s = K2 + A1 * A1;
    double D = s - A0 * A0;
    if (!(s > 0.0)) return 0.0;
    if (D < 0.0) return 0.0;
    return OR_PI / sqrt(s);
}

/* ---------------------------------------------------------- kernel F ----- */
/* eq. (app_F_1d): F_inm = |M|^2 p_n p_m / (4 (2 pi)^4) * sum_k w_k I(mu_k).
 * form 0: closed-form nu integral, form 1: arcsin form. */
double oracle_F(double m, double M2, double pi, double pn, double pm,
                double Ei, double En, double Em, int n_mu,
                const double *x, const double *w, int form) {
    double acc = 0.0;
    for (int k = 0; k < n_mu; ++k) {
        double A0, A1, K2;
        oracle_angular_coeffs(m, pi, pn, pm, Ei, En, Em, x[k], &A0, &A1, &K2);
        double I = (form == 1) ? oracle_nu_integral_arcsin(A0, A1, K2)
                               : oracle_nu_integral_closed(A0, A1, K2);
        acc += w[k] * I;
    }
    double two_pi = 2.0 * OR_PI;
    return M2 * pn * pm / (4.0 * two_pi * two_pi * two_pi * two_pi) * acc;
}

/* N_mu -> infinity limit of F (derived, not printed in the paper): with
 * k^2 = p_i^2 + p_n^2 - 2 p_i p_n mu one has K^2 + A1^2 = p_m^2 k^2 and the
 * Theta condition becomes the triangle condition |p_t - p_m| <= k <= p_t + p_m,
 * so  int dmu I = pi L / (p_i p_n),  L = overlap of [|p_i-p_n|, p_i+p_n] and
 * [|p_t-p_m|, p_t+p_m], and F_exact = |M|^2 pi L / (4 (2pi)^4 p_i). */
double oracle_F_exact(double M2, double pi, double pn, double pm, double pt) {
    double lo1 = fabs(pi - pn), hi1 = pi + pn;
    double lo2 = fabs(pt - pm), hi2 = pt + pm;
    double lo = lo1 > lo2 ? lo1 : lo2;
    double hi = hi1 < hi2 ? hi1 : hi2;
    double L = hi - lo;
    if (L < 0.0) L = 0.0;
    double two_pi = 2.0 * OR_PI;
    return M2 * OR_PI * L / (4.0 * two_pi * two_pi * two_pi * two_pi * pi);
}

/* ---------------------------------------------------- support, bracket --- */
/* Kept configurations (Appendix A): E_t >= m and q_min <= q_t <= q_max, i.e.
 * E_0 <= E_t <= E_{N-1} (reading A6, tested in E, closed interval), with
 * E_t = (E_n + E_m) - E_i evaluated in this order (eq. app_fourth_momentum). */
static int in_support(int n, const double *E, double Et) {
    return (Et >= E[0]) && (Et <= E[n - 1]);
}

/* Bracket q_jL <= q_t <= q_jR (Appendix A) with jR = jL + 1; reading A6: jL is
 * the largest j <= N-2 with E_j <= E_t (bisection on the ascending E array;
 * E_0 <= E_t holds inside the support, so j = 0 always qualifies).
 * omega_R = (E_t - E_jL) / (E_jR - E_jL), eq. (app_interp_weights). */
int oracle_bracket(int n, const double *E, double Et, int *jL, double *omega) {
    if (!in_support(n, E, Et)) return 0;
    int lo = 0, hi = n - 2;          /* invariant: E[lo] <= Et; answer in [lo, hi] */
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (E[mid] <= Et) lo = mid; else hi = mid - 1;
    }
    int j = lo;
    *jL = j;
    *omega = (Et - E[j]) / (E[j + 1] - E[j]);
    return 1;
}

/* eq. (app_log_interp): f_t = exp(omega_L log f_jL + omega_R log f_jR), with
 * the log taken of max(f, 1e-300) (reading A5). */
static double log_floor(double f) {
    return log(f > OR_LOG_FLOOR ? f : OR_LOG_FLOOR);
}

/* ------------------------------------------------------- W tensor -------- */
/* eq. (discrete_weight): W_inm = mu_n mu_m F_inm / (2 E_i g_chi), g_chi = 1
 * (reading A4).  measure 0 (reading A1, default): mu_n = dE_n (the kernel F of
 * eq. app_F_2d is the kernel of dE_n dE_m); measure 1: the literal mu_n = Dp_n.
 * angular 0: GL closed form; 1: GL arcsin form; 2: exact N_mu -> inf kernel.
 * W has layout [i][n][m] (N^3 doubles); W = 0 outside the support. */
int oracle_kernel_tensor(int n, const double *q, double a, double mass, double M2,
                         int n_mu, int measure, int angular, double *W) {
    double *p = malloc(sizeof(double) * n), *E = malloc(sizeof(double) * n);
    double *dp = malloc(sizeof(double) * n), *dE = malloc(sizeof(double) * n);
    double *h = malloc(sizeof(double) * n);
    double *x = malloc(sizeof(double) * (n_mu > 0 ? n_mu : 1));
    double *w = malloc(sizeof(double) * (n_mu > 0 ? n_mu : 1));
    int rc = OR_OK;
    if (!p || !E || !dp || !dE || !h || !x || !w) { rc = OR_ENOMEM; goto out; }
    rc = oracle_grid(n, q, a, mass, p, E, dp, dE, h);
    if (rc) goto out;
    if (angular != 2) {
        if (n_mu < 1) { rc = OR_EINVAL; goto out; }
        oracle_gauss_legendre(n_mu, x, w);
    }
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n; ++i) {
        for (int nn = 0; nn < n; ++nn) {
            for (int mm = 0; mm < n; ++mm) {
                double Et = (E[nn] + E[mm]) - E[i];
                double val = 0.0;
                if (in_support(n, E, Et)) {
                    double F;
                    if (angular == 2) {
                        double pt = sqrt(Et * Et - mass * mass);
                        F = oracle_F_exact(M2, p[i], p[nn], p[mm], pt);
                    } else {
                        F = oracle_F(mass, M2, p[i], p[nn], p[mm], E[i], E[nn], E[mm],
                                     n_mu, x, w, angular);
                    }
                    double mun = measure == 1 ? dp[nn] : dE[nn];
                    double mum = measure == 1 ? dp[mm] : dE[mm];
                    val = mun * mum * F / (2.0 * E[i] * 1.0);
                }
                W[((size_t)i * n + nn) * n + mm] = val;
            }
        }
    }
out:
    free(p); free(E); free(dp); free(dE); free(h); free(x); free(w);
    return rc;
}

/* Interpolation table of the tensor: jL and omega for every (i,n,m) in the
 * support (jL = -1 outside). */
int oracle_bracket_tensor(int n, const double *q, double a, double mass,
                          int *jL, double *omega) {
    double *p = malloc(sizeof(double) * n), *E = malloc(sizeof(double) * n);
    double *dp = malloc(sizeof(double) * n), *dE = malloc(sizeof(double) * n);
    double *h = malloc(sizeof(double) * n);
    int rc = OR_OK;
    if (!p || !E || !dp || !dE || !h) { rc = OR_ENOMEM; goto out; }
    rc = oracle_grid(n, q, a, mass, p, E, dp, dE, h);
    if (rc) goto out;
    for (int i = 0; i < n; ++i)
        for (int nn = 0; nn < n; ++nn)
            for (int mm = 0; mm < n; ++mm) {
                size_t e = ((size_t)i * n + nn) * n + mm;
                double Et = (E[nn] + E[mm]) - E[i];
                int j;
                double om;
                if (oracle_bracket(n, E, Et, &j, &om)) { jL[e] = j; omega[e] = om; }
                else { jL[e] = -1; omega[e] = 0.0; }
            }
out:
    free(p); free(E); free(dp); free(dE); free(h);
    return rc;
}

/* ------------------------------------------------------- C_raw ----------- */
/* eq. (discrete_collision_operator), dilute limit:
 *   C_i = sum_{n,m} W_inm [ f_n f_m - f_i f_t(i,n,m) ]
 * Also returns the gain G_i = sum W f_n f_m and the loss rate
 * nu_i = sum W f_t (so that C_i = G_i - f_i nu_i); either may be NULL. */
int oracle_collision_tensor(int n, const double *q, double a, double mass,
                            const double *W, const double *f,
                            double *C, double *gain, double *loss_rate) {
    double *p = malloc(sizeof(double) * n), *E = malloc(sizeof(double) * n);
    double *dp = malloc(sizeof(double) * n), *dE = malloc(sizeof(double) * n);
    double *h = malloc(sizeof(double) * n), *lf = malloc(sizeof(double) * n);
    int rc = OR_OK;
    if (!p || !E || !dp || !dE || !h || !lf) { rc = OR_ENOMEM; goto out; }
    rc = oracle_grid(n, q, a, mass, p, E, dp, dE, h);
    if (rc) goto out;
    for (int j = 0; j < n; ++j) lf[j] = log_floor(f[j]);
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n; ++i) {
        double Ci = 0.0, Gi = 0.0, Li = 0.0;
        for (int nn = 0; nn < n; ++nn) {
            for (int mm = 0; mm < n; ++mm) {
                double Wv = W[((size_t)i * n + nn) * n + mm];
                if (Wv == 0.0) continue;
                double Et = (E[nn] + E[mm]) - E[i];
                int j;
                double om;
                if (!oracle_bracket(n, E, Et, &j, &om)) continue;
                double ft = exp((1.0 - om) * lf[j] + om * lf[j + 1]);
                Ci += Wv * (f[nn] * f[mm] - f[i] * ft);
                Gi += Wv * (f[nn] * f[mm]);
                Li += Wv * ft;
            }
        }
        C[i] = Ci;
        if (gain) gain[i] = Gi;
        if (loss_rate) loss_rate[i] = Li;
    }
out:
    free(p); free(E); free(dp); free(dE); free(h); free(lf);
    return rc;
}

/* Quantum statistics (eq. Lambda_quantum): the statistical factor of the
 * collision integral with eta = +1 (Bose-Einstein) or -1 (Fermi-Dirac),
 *   f_n f_m (1 + eta f_i)(1 + eta f_t) - f_i f_t (1 + eta f_n)(1 + eta f_m),
 * in the discrete sum of eq. (discrete_collision_operator) with f_t from the
 * log-energy interpolation of f itself (reading A14); eta = 0 is the dilute
 * factor.  C[i] = sum_nm W_inm * factor (raw, no projection). */
int oracle_collision_tensor_stats(int n, const double *q, double a, double mass,
                                  const double *W, const double *f, int eta, double *C) {
    double *p = malloc(sizeof(double) * n), *E = malloc(sizeof(double) * n);
    double *dp = malloc(sizeof(double) * n), *dE = malloc(sizeof(double) * n);
    double *h = malloc(sizeof(double) * n), *lf = malloc(sizeof(double) * n);
    int rc = OR_OK;
    if (eta < -1 || eta > 1) return OR_EINVAL;
    if (!p || !E || !dp || !dE || !h || !lf) { rc = OR_ENOMEM; goto out; }
    rc = oracle_grid(n, q, a, mass, p, E, dp, dE, h);
    if (rc) goto out;
    for (int j = 0; j < n; ++j) lf[j] = log_floor(f[j]);
    const double et = (double)eta;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n; ++i) {
        double Ci = 0.0;
        for (int nn = 0; nn < n; ++nn) {
            for (int mm = 0; mm < n; ++mm) {
                double Wv = W[((size_t)i * n + nn) * n + mm];
                if (Wv == 0.0) continue;
                double Et = (E[nn] + E[mm]) - E[i];
                int j;
                double om;
                if (!oracle_bracket(n, E, Et, &j, &om)) continue;
                double ft = exp((1.0 - om) * lf[j] + om * lf[j + 1]);
                double gain = f[nn] * f[mm] * (1.0 + et * f[i]) * (1.0 + et * ft);
                double loss = f[i] * ft * (1.0 + et * f[nn]) * (1.0 + et * f[mm]);
                Ci += Wv * (gain - loss);
            }
        }
        C[i] = Ci;
    }
out:
    free(p); free(E); free(dp); free(dE); free(h); free(lf);
    return rc;
}

/* Direct form: the same sum with F evaluated on the fly from the printed
 * arcsin form of eq. (app_I_mu) (no stored tensor). */
int oracle_collision_direct(int n, const double *q, double a, double mass, double M2,
                            int n_mu, int measure, const double *f, double *C) {
    double *p = malloc(sizeof(double) * n), *E = malloc(sizeof(double) * n);
    double *dp = malloc(sizeof(double) * n), *dE = malloc(sizeof(double) * n);
    double *h = malloc(sizeof(double) * n), *lf = malloc(sizeof(double) * n);
    double *x = malloc(sizeof(double) * (n_mu > 0 ? n_mu : 1));
    double *w = malloc(sizeof(double) * (n_mu > 0 ? n_mu : 1));
    int rc = OR_OK;
    if (!p || !E || !dp || !dE || !h || !lf || !x || !w) { rc = OR_ENOMEM; goto out; }
    rc = oracle_grid(n, q, a, mass, p, E, dp, dE, h);
    if (rc) goto out;
    if (n_mu < 1) { rc = OR_EINVAL; goto out; }
    oracle_gauss_legendre(n_mu, x, w);
    for (int j = 0; j < n; ++j) lf[j] = log_floor(f[j]);
    for (int i = 0; i < n; ++i) {
        double Ci = 0.0;
        for (int nn = 0; nn < n; ++nn) {
            for (int mm = 0; mm < n; ++mm) {
                double Et = (E[nn] + E[mm]) - E[i];
                int j;
                double om;
                if (!oracle_bracket(n, E, Et, &j, &om)) continue;
                double F = oracle_F(mass, M2, p[i], p[nn], p[mm], E[i], E[nn], E[mm],
                                    n_mu, x, w, 1);
                double mun = measure == 1 ? dp[nn] : dE[nn];
                double mum = measure == 1 ? dp[mm] : dE[mm];
                double Wv = mun * mum * F / (2.0 * E[i] * 1.0);
                double ft = exp((1.0 - om) * lf[j] + om * lf[j + 1]);
                Ci += Wv * (f[nn] * f[mm] - f[i] * ft);
            }
        }
        C[i] = Ci;
    }
out:
    free(p); free(E); free(dp); free(dE); free(h); free(lf); free(x); free(w);
    return rc;
}

/* ------------------------------------------------------- projection ------ */
/* Appendix B.  xi_i = |f_i|/f_max if > eps_supp else 0;
 * A00 = sum h xi, A01 = sum h E xi, A11 = sum h E^2 xi; R0 = sum h C, R1 = sum h E C;
 * (alpha, beta) from the 2x2 system, C_proj = C - xi (alpha + beta E).
 * diag (may be NULL), 10 entries:
 *   [0] eps_N raw  [1] eps_E raw  [2] eps_N proj  [3] eps_E proj
 *   [4] R_N        [5] R_E        [6] alpha       [7] beta
 *   [8] singular flag (reading A10: det <= 1e-14 A00 A11 -> alpha = beta = 0)
 *   [9] f_max
 * Returns OR_ESINGULAR when the guard fired (C_proj = C then). */
int oracle_project(int n, const double *E, const double *h, const double *f,
                   const double *C, double *Cproj, double *diag) {
    double fmax = 0.0;
    for (int i = 0; i < n; ++i) if (fabs(f[i]) > fmax) fmax = fabs(f[i]);
    double A00 = 0, A01 = 0, A11 = 0, R0 = 0, R1 = 0;
    for (int i = 0; i < n; ++i) {
        double xi = 0.0;
        if (fmax > 0.0) {
            double r = fabs(f[i]) / fmax;
            xi = r > OR_EPS_SUPP ? r : 0.0;
        }
        A00 += h[i] * xi;
        A01 += h[i] * E[i] * xi;
        A11 += h[i] * E[i] * E[i] * xi;
        R0 += h[i] * C[i];
        R1 += h[i] * E[i] * C[i];
    }
    double det = A00 * A11 - A01 * A01;
    double alpha = 0.0, beta = 0.0;
    int singular = 0;
    if (!(det > OR_DET_GUARD * A00 * A11)) singular = 1;
    else {
        alpha = (R0 * A11 - R1 * A01) / det;
        beta = (R1 * A00 - R0 * A01) / det;
    }
    for (int i = 0; i < n; ++i) {
        double xi = 0.0;
        if (fmax > 0.0) {
            double r = fabs(f[i]) / fmax;
            xi = r > OR_EPS_SUPP ? r : 0.0;
        }
        Cproj[i] = C[i] - xi * (alpha + beta * E[i]);
    }
    if (diag) {
        double sN = 0, sE = 0, aN = 0, aE = 0, pN = 0, pE = 0, paN = 0, paE = 0, dN = 0, dEs = 0;
        for (int i = 0; i < n; ++i) {
            sN += h[i] * C[i];
            sE += h[i] * E[i] * C[i];
            aN += h[i] * fabs(C[i]);
            aE += h[i] * E[i] * fabs(C[i]);
            pN += h[i] * Cproj[i];
            pE += h[i] * E[i] * Cproj[i];
            paN += h[i] * fabs(Cproj[i]);
            paE += h[i] * E[i] * fabs(Cproj[i]);
            dN += h[i] * fabs(Cproj[i] - C[i]);
            dEs += h[i] * E[i] * fabs(Cproj[i] - C[i]);
        }
        diag[0] = aN > 0 ? sN / aN : 0.0;
        diag[1] = aE > 0 ? sE / aE : 0.0;
        diag[2] = paN > 0 ? pN / paN : 0.0;
        diag[3] = paE > 0 ? pE / paE : 0.0;
        diag[4] = aN > 0 ? dN / aN : 0.0;
        diag[5] = aE > 0 ? dEs / aE : 0.0;
        diag[6] = alpha;
        diag[7] = beta;
        diag[8] = singular;
        diag[9] = fmax;
    }
    return singular ? OR_ESINGULAR : OR_OK;
}

/* ------------------------------------------------------- sources --------- */
/* Synthetic freeze-in sources (reading A12; the paper's own sources,
 * eqs. (C_higgs_decay) and (C_condensate_decay), need a cosmology):
 *   S_i(t) = sum_k R_k env_k(t) s_k,i / (sum_j h_j s_k,j),
 *   env_k(t) = exp(-(t - t_k)/tau_k) for t >= t_k, else 0.
 * The shape rows are normalised here so that R_k is the number injection
 * rate (sum_i h_i S_i = sum_k R_k env_k). shape layout [n_src][n]. */
void oracle_source(int n, const double *h, double t, int n_src, const double *shape,
                   const double *rate, const double *tau, const double *t_on, double *S) {
    for (int i = 0; i < n; ++i) S[i] = 0.0;
    for (int k = 0; k < n_src; ++k) {
        if (t < t_on[k]) continue;
        double norm = 0.0;
        for (int j = 0; j < n; ++j) norm += h[j] * shape[(size_t)k * n + j];
        if (!(norm > 0.0)) continue;
        double env = exp(-(t - t_on[k]) / tau[k]);
        for (int i = 0; i < n; ++i) S[i] += rate[k] * env * shape[(size_t)k * n + i] / norm;
    }
}

/* All sources are below 1e-12 of their peak: t >= t_k + tau_k ln(1e12). */
static int sources_off(double t, int n_src, const double *tau, const double *t_on) {
    for (int k = 0; k < n_src; ++k)
        if (t < t_on[k] + tau[k] * log(1e12)) return 0;
    return 1;
}

/* ------------------------------------------------------- MB fit ---------- */
/* Stopping test: the discrete Maxwell-Boltzmann f_MB = z exp(-E/T) with the
 * same number and energy moments as f (sum h f, sum h E f).  T by bisection in
 * ln T on the monotone mean energy <E>(T) = sum h E e^{-E/T} / sum h e^{-E/T};
 * z from the number moment.  L1 = sum h |f - f_MB| / sum h f.
 * out[0] = T, out[1] = ln z, out[2] = L1. */
int oracle_mb_fit(int n, const double *E, const double *h, const double *f, double *out) {
    double N0 = 0.0, E1 = 0.0;
    for (int i = 0; i < n; ++i) { N0 += h[i] * f[i]; E1 += h[i] * E[i] * f[i]; }
    if (!(N0 > 0.0)) { out[0] = 0; out[1] = 0; out[2] = INFINITY; return OR_EINVAL; }
    double ebar = E1 / N0;
    double lo = log(1e-12), hi = log(1e12);
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double T = exp(mid);
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i < n; ++i) {
            double wgt = h[i] * exp(-(E[i] - E[0]) / T);
            s0 += wgt;
            s1 += wgt * E[i];
        }
        if (s1 / s0 < ebar) lo = mid; else hi = mid;
    }
    double T = exp(0.5 * (lo + hi));
    double s0 = 0.0;
    for (int i = 0; i < n; ++i) s0 += h[i] * exp(-(E[i] - E[0]) / T);
    double l1 = 0.0;
    for (int i = 0; i < n; ++i) {
        double fmb = N0 * exp(-(E[i] - E[0]) / T) / s0;
        l1 += h[i] * fabs(f[i] - fmb);
    }
    out[0] = T;
    out[1] = log(N0 / s0) + E[0] / T;
    out[2] = l1 / N0;
    return OR_OK;
}

/* ------------------------------------------------------- RHS, Heun ------- */
typedef struct {
    int n;
    const double *q; double a, mass;
    const double *W;      /* [N^3], built with |M|^2 = 1 */
    double M2;            /* |M|^2 = 64 pi m^2 sigma (reading A3) */
    int project;
    int n_src; const double *shape, *rate, *tau, *t_on;
    const double *E, *h;
} rhs_ctx;

/* RHS(f, t) = C_proj[f] + S(t) (Sec. 4: df_i/dt = C_el,i[f] + C_FI,i with a = 1,
 * H = 0, reading A13).  C = |M|^2 C_unit since W is linear in |M|^2. */
static int rhs_eval(const rhs_ctx *c, const double *f, double t, double *out, double *work) {
    int n = c->n;
    int rc = oracle_collision_tensor(n, c->q, c->a, c->mass, c->W, f, work, NULL, NULL);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) work[i] *= c->M2;
    if (c->project) {
        rc = oracle_project(n, c->E, c->h, f, work, out, NULL);
        if (rc == OR_ESINGULAR) rc = OR_OK;  /* C_proj = C_raw, flagged only in diag */
        if (rc) return rc;
    } else {
        for (int i = 0; i < n; ++i) out[i] = work[i];
    }
    double *S = work + n;
    oracle_source(n, c->h, t, c->n_src, c->shape, c->rate, c->tau, c->t_on, S);
    for (int i = 0; i < n; ++i) out[i] += S[i];
    return OR_OK;
}

/* One Heun attempt (Sec. 4.2): k1 = RHS(f,t); f_p = f + h k1 (Euler predictor);
 * k2 = RHS(f_p, t+h); f_c = f + h/2 (k1 + k2) (trapezoid corrector);
 * err = max_i |f_c - f_p| / (atol + rtol |f_c|) (reading A11).
 * Adaptive: accept iff err <= 1 and f_p, f_c >= 0; h <- h min(5, max(0.2, 0.9 err^-1/2)),
 * a negative stage halves h.  Fixed: always accept; a negative stage is OR_ENEG.
 * Returns 1 accepted, 0 rejected, <0 error.  *err_out receives err. */
static int heun_attempt(const rhs_ctx *c, double *f, double t, double h, int fixed,
                        double rtol, double atol, double *h_next, double *err_out,
                        double *k1, double *k2, double *fp, double *fc, double *work) {
    int n = c->n;
    int rc = rhs_eval(c, f, t, k1, work);
    if (rc) return rc;
    int neg = 0;
    for (int i = 0; i < n; ++i) {
        fp[i] = f[i] + h * k1[i];
        if (!isfinite(fp[i])) return OR_ENONFINITE;
        if (fp[i] < 0.0) neg = 1;
    }
    if (neg) {
        if (fixed) return OR_ENEG;
        *h_next = 0.5 * h;
        *err_out = INFINITY;
        return 0;
    }
    rc = rhs_eval(c, fp, t + h, k2, work);
    if (rc) return rc;
    double err = 0.0;
    for (int i = 0; i < n; ++i) {
        fc[i] = f[i] + 0.5 * h * (k1[i] + k2[i]);
        if (!isfinite(fc[i])) return OR_ENONFINITE;
        if (fc[i] < 0.0) neg = 1;
        double e = fabs(fc[i] - fp[i]) / (atol + rtol * fabs(fc[i]));
        if (e > err) err = e;
    }
    *err_out = err;
    if (fixed) {
        if (neg) return OR_ENEG;
        for (int i = 0; i < n; ++i) f[i] = fc[i];
        *h_next = h;
        return 1;
    }
    if (neg) { *h_next = 0.5 * h; return 0; }
    double fac = err > 0.0 ? 0.9 / sqrt(err) : 5.0;
    if (fac > 5.0) fac = 5.0;
    if (fac < 0.2) fac = 0.2;
    *h_next = h * fac;
    if (err <= 1.0) {
        for (int i = 0; i < n; ++i) f[i] = fc[i];
        return 1;
    }
    return 0;
}

/* Time integration.  params (12 doubles):
 *  [0] t0 [1] t_end [2] h0 [3] rtol [4] atol [5] h_min [6] h_max [7] l1_tol
 *  [8] max_attempts [9] fixed_step [10] check_every [11] project
 * Stops when (sources off and L1 <= l1_tol, checked every check_every accepted
 * steps), or t reaches t_end, or max_attempts attempts were made (OR_ENOCONV).
 * res (10 doubles): [0] t [1] steps [2] rejects [3] L1 [4] T_mb [5] ln z_mb
 *  [6] status [7] h [8] evaluations [9] converged flag */
int oracle_solve(int n, const double *q, double a, double mass, const double *W, double M2,
                 int n_src, const double *shape, const double *rate, const double *tau,
                 const double *t_on, const double *params, double *f, double *res) {
    double *p = malloc(sizeof(double) * n), *E = malloc(sizeof(double) * n);
    double *dp = malloc(sizeof(double) * n), *dE = malloc(sizeof(double) * n);
    double *h = malloc(sizeof(double) * n);
    double *k1 = malloc(sizeof(double) * n), *k2 = malloc(sizeof(double) * n);
    double *fp = malloc(sizeof(double) * n), *fc = malloc(sizeof(double) * n);
    double *work = malloc(sizeof(double) * 2 * n);
    int rc = OR_OK;
    if (!p || !E || !dp || !dE || !h || !k1 || !k2 || !fp || !fc || !work) { rc = OR_ENOMEM; goto out; }
    rc = oracle_grid(n, q, a, mass, p, E, dp, dE, h);
    if (rc) goto out;
    rhs_ctx c = { n, q, a, mass, W, M2, (int)params[11], n_src, shape, rate, tau, t_on, E, h };
    double t = params[0], t_end = params[1], hs = params[2];
    double rtol = params[3], atol = params[4], h_min = params[5], h_max = params[6];
    double l1_tol = params[7];
    long max_att = (long)params[8];
    int fixed = (int)params[9];
    int check_every = (int)params[10];
    long steps = 0, rejects = 0, evals = 0;
    int converged = 0;
    double fit[3] = {0, 0, INFINITY};
    int status = OR_OK;
    while (1) {
        if (t >= t_end) break;
        if (steps + rejects >= max_att) { status = OR_ENOCONV; break; }
        double htry = hs;
        if (!fixed) {
            if (htry > h_max) htry = h_max;
            if (htry < h_min) htry = h_min;
        }
        int last = 0;
        if (t + htry >= t_end) { htry = t_end - t; last = 1; }
        double hn, err;
        int r = heun_attempt(&c, f, t, htry, fixed, rtol, atol, &hn, &err, k1, k2, fp, fc, work);
        evals += (err == INFINITY && r == 0) ? 1 : 2;
        if (r < 0) { status = r; break; }
        if (r == 1) {
            steps++;
            t = last ? t_end : t + htry;
            if (check_every > 0 && l1_tol > 0 && steps % check_every == 0 &&
                sources_off(t, n_src, tau, t_on)) {
                oracle_mb_fit(n, E, h, f, fit);
                if (fit[2] <= l1_tol) { converged = 1; hs = hn; break; }
            }
        } else {
            rejects++;
        }
        /* the step actually tried bounds the next proposal when it was clipped at t_end */
        hs = hn;
    }
    oracle_mb_fit(n, E, h, f, fit);
    res[0] = t; res[1] = (double)steps; res[2] = (double)rejects; res[3] = fit[2];
    res[4] = fit[0]; res[5] = fit[1]; res[6] = status; res[7] = hs; res[8] = (double)evals;
    res[9] = converged;
    rc = status;
out:
    free(p); free(E); free(dp); free(dE); free(h); free(k1); free(k2); free(fp); free(fc); free(work);
    return rc;
}

/* ------------------------------------------------------- sigma -> |M|^2 -- */
/* Contact interaction lambda chi^4/4!: |M|^2 = lambda^2 (Sec. 3), and the
 * Table 1 caption gives sigma_T/m = lambda^2/(64 pi m^3); hence
 * |M|^2 = 64 pi m^2 sigma (reading A3, no extra identical-particle 1/2). */
double oracle_M2_from_sigma(double mass, double sigma) {
    return 64.0 * OR_PI * mass * mass * sigma;
}

/* Selected rows of C_raw (direct form, F on the fly from eq. app_F_1d with the
 * closed-form nu integral) for sampled checks at sizes where the full N^3 tensor
 * is too large for the oracle.  rows[nrows] are row indices; C[nrows]; the gain
 * G and loss rate nu of those rows are returned too (may be NULL). */
int oracle_collision_rows(int n, const double *q, double a, double mass, double M2,
                          int n_mu, int measure, const double *f, int nrows, const int *rows,
                          double *C, double *gain, double *loss_rate) {
    double *p = malloc(sizeof(double) * n), *E = malloc(sizeof(double) * n);
    double *dp = malloc(sizeof(double) * n), *dE = malloc(sizeof(double) * n);
    double *h = malloc(sizeof(double) * n), *lf = malloc(sizeof(double) * n);
    double *x = malloc(sizeof(double) * (n_mu > 0 ? n_mu : 1));
    double *w = malloc(sizeof(double) * (n_mu > 0 ? n_mu : 1));
    int rc = OR_OK;
    if (!p || !E || !dp || !dE || !h || !lf || !x || !w) { rc = OR_ENOMEM; goto out; }
    rc = oracle_grid(n, q, a, mass, p, E, dp, dE, h);
    if (rc) goto out;
    if (n_mu < 1) { rc = OR_EINVAL; goto out; }
    oracle_gauss_legendre(n_mu, x, w);
    for (int j = 0; j < n; ++j) lf[j] = log_floor(f[j]);
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < nrows; ++r) {
        int i = rows[r];
        double Ci = 0.0, Gi = 0.0, Li = 0.0;
        for (int nn = 0; nn < n; ++nn) {
            for (int mm = 0; mm < n; ++mm) {
                double Et = (E[nn] + E[mm]) - E[i];
                int j;
                double om;
                if (!oracle_bracket(n, E, Et, &j, &om)) continue;
                double F = oracle_F(mass, M2, p[i], p[nn], p[mm], E[i], E[nn], E[mm], n_mu, x, w, 0);
                double mun = measure == 1 ? dp[nn] : dE[nn];
                double mum = measure == 1 ? dp[mm] : dE[mm];
                double Wv = mun * mum * F / (2.0 * E[i] * 1.0);
                double ft = exp((1.0 - om) * lf[j] + om * lf[j + 1]);
                Ci += Wv * (f[nn] * f[mm] - f[i] * ft);
                Gi += Wv * (f[nn] * f[mm]);
                Li += Wv * ft;
            }
        }
        C[r] = Ci;
        if (gain) gain[r] = Gi;
        if (loss_rate) loss_rate[r] = Li;
    }
out:
    free(p); free(E); free(dp); free(dE); free(h); free(lf); free(x); free(w);
    return rc;
}

/* ------------------------------------------- Chebyshev loss expansion --- */
/* Exponentially scaled modified Bessel functions of the first kind,
 *   ive[k] = e^{-x} I_k(x),  k = 0 .. K-1,  x >= 0,
 * from the power series I_k(x) = sum_{m>=0} (x/2)^{2m+k} / (m! (m+k)!)
 * (Abramowitz & Stegun 9.6.10), each term formed as exp of its logarithm
 * (lgamma) so that large x does not overflow; summed until past the largest
 * term and below 1e-20 of the sum. */
int oracle_bessel_ive(int K, double x, double *ive) {
    if (K < 1 || !(x >= 0.0)) return OR_EINVAL;
    for (int k = 0; k < K; ++k) {
        if (x == 0.0) { ive[k] = k == 0 ? 1.0 : 0.0; continue; }
        double lx = log(0.5 * x), s = 0.0;
        for (int m = 0; m < 100000; ++m) {
            double lt = (2.0 * m + k) * lx - lgamma(m + 1.0) - lgamma(m + k + 1.0) - x;
            double t = exp(lt);
            s += t;
            if (m > 0.5 * x + 2 && t < 1e-20 * s) break;
        }
        ive[k] = s;
    }
    return OR_OK;
}

/* Loss rate of eq. (discrete_collision_operator) with the interpolated f_t of
 * eq. (app_log_interp) expanded in Chebyshev polynomials of t = 2 omega - 1.
 * With d = ln f_{jL+1} - ln f_jL (logs of max(f, 1e-300), reading A5),
 *   f_t = f_jL e^{omega d} = f_jL e^{d/2} e^{t d/2}
 *       = f_jL e^{d/2} sum_k eps_k I_k(d/2) T_k(t),   eps_0 = 1, eps_k = 2
 * (the generating function of I_k: e^{x cos theta} = sum eps_k I_k(x) cos k theta),
 * truncated after K terms:
 *   M_k[i][j] = sum_{n,m: jL(i,n,m) = j} W_inm T_k(2 omega_inm - 1),
 *   Y_k[j]    = f_j e^{d_j/2} eps_k I_k(d_j/2),      I_k(-x) = (-1)^k I_k(x),
 *   L_i       = sum_j sum_{k<K} M_k[i][j] Y_k[j].
 * Since f_j e^{d/2} I_k(d/2) = max(f_j, f_{j+1}) (+-1)^k e^{-|d|/2} I_k(|d|/2) and
 * |T_k| <= 1, the truncation error of row i is at most
 *   bound[i] = sum_{n,m} W_inm max(f_j, f_{j+1}) 2 sum_{k>=K} e^{-|d_j|/2} I_k(|d_j|/2).
 * C[i] = sum W f_n f_m - f_i L_i (dilute), G[i] the gain.  W as from
 * oracle_kernel_tensor ([i][n][m]).  T_k from the three-term recurrence. */
int oracle_loss_chebyshev(int n, const double *q, double a, double mass, const double *W,
                          const double *f, int K, double *C, double *G, double *L, double *bound) {
    if (n < 2 || K < 1) return OR_EINVAL;
    const int KT = K + 80;   /* terms of the tail sum (enough for |d|/2 up to ~40) */
    double *p = malloc(sizeof(double) * n), *E = malloc(sizeof(double) * n);
    double *dp = malloc(sizeof(double) * n), *dE = malloc(sizeof(double) * n);
    double *h = malloc(sizeof(double) * n), *lf = malloc(sizeof(double) * n);
    double *M = calloc((size_t)n * n * K, sizeof(double));     /* M[i][j][k] */
    double *Y = malloc(sizeof(double) * (size_t)n * K);        /* Y[j][k] */
    double *tail = malloc(sizeof(double) * n);                 /* per bracket j */
    double *iv = malloc(sizeof(double) * KT);
    int rc = OR_OK;
    if (!p || !E || !dp || !dE || !h || !lf || !M || !Y || !tail || !iv) { rc = OR_ENOMEM; goto out; }
    rc = oracle_grid(n, q, a, mass, p, E, dp, dE, h);
    if (rc) goto out;
    for (int j = 0; j < n; ++j) lf[j] = log_floor(f[j]);
    /* Y_k[j] and the truncation tail of bracket j */
    for (int j = 0; j + 1 < n; ++j) {
        double d = lf[j + 1] - lf[j], x = 0.5 * fabs(d);
        double fmx = exp(lf[j] > lf[j + 1] ? lf[j] : lf[j + 1]);
        rc = oracle_bessel_ive(KT, x, iv);
        if (rc) goto out;
        for (int k = 0; k < K; ++k) {
            double sg = (d < 0.0 && (k & 1)) ? -1.0 : 1.0;
            Y[(size_t)j * K + k] = fmx * (k == 0 ? 1.0 : 2.0) * sg * iv[k];
        }
        double tl = 0.0;
        for (int k = KT - 1; k >= K; --k) tl += iv[k];
        tail[j] = fmx * 2.0 * tl;
    }
    /* M_k[i][j] */
    for (int i = 0; i < n; ++i) {
        double bi = 0.0;
        for (int nn = 0; nn < n; ++nn) {
            for (int mm = 0; mm < n; ++mm) {
                double Wv = W[((size_t)i * n + nn) * n + mm];
                if (Wv == 0.0) continue;
                double Et = (E[nn] + E[mm]) - E[i];
                int j;
                double om;
                if (!oracle_bracket(n, E, Et, &j, &om)) continue;
                double t = 2.0 * om - 1.0, T0 = 1.0, T1 = t;
                double *Mij = M + ((size_t)i * n + j) * K;
                for (int k = 0; k < K; ++k) {
                    double Tk = k == 0 ? 1.0 : (k == 1 ? t : 2.0 * t * T1 - T0);
                    if (k >= 2) { T0 = T1; T1 = Tk; }
                    Mij[k] += Wv * Tk;
                }
                bi += Wv * tail[j];
            }
        }
        bound[i] = bi;
    }
    /* L_i = sum_j sum_k M_k[i][j] Y_k[j];  C_i = G_i - f_i L_i */
    for (int i = 0; i < n; ++i) {
        double Li = 0.0, Gi = 0.0;
        for (int j = 0; j + 1 < n; ++j)
            for (int k = 0; k < K; ++k) Li += M[((size_t)i * n + j) * K + k] * Y[(size_t)j * K + k];
        for (int nn = 0; nn < n; ++nn)
            for (int mm = 0; mm < n; ++mm) Gi += W[((size_t)i * n + nn) * n + mm] * (f[nn] * f[mm]);
        L[i] = Li;
        G[i] = Gi;
        C[i] = Gi - f[i] * Li;
    }
out:
    free(p); free(E); free(dp); free(dE); free(h); free(lf); free(M); free(Y); free(tail); free(iv);
    return rc;
}

/* --------------------------------------------- expanding universe, u = log a */
/* Sec. 4 with the scale factor as clock: q is the comoving grid (fixed), the
 * physical momenta are p_i = q_i / a, a = e^u, and eq. (numerical_evolution_loga)
 *   df_i/du = [C_el,i[f; a] + C_FI,i(u)] / H(u).
 * The kernel W depends on a through p = q/a and is rebuilt (eq. discrete_weight
 * at that a) for every evaluation.  H(u): exp of the piecewise-linear
 * interpolation of ln H through (hu_k, hlnH_k) (n_h >= 1 points, linear
 * extrapolation beyond them; n_h = 1: constant H) -- the paper's H(a) comes
 * from Standard-Model thermodynamics it does not list, so it is an input
 * (reading).  C_FI (reading): the synthetic sources of the static box with u as
 * their clock, shapes normalised with the comoving weights q_i^2 Dq_i, so that
 * rate_k is the comoving number injected per unit time.
 * Two regimes (Sec. 4.2): while Gamma_2->2 / H <= eps_switch the collisions are
 * off and f advances by classical RK4 on fixed intervals du (the right-hand
 * side S(u)/H(u) does not depend on f); Gamma_2->2 = n <sigma v> is read here
 * as the number-weighted loss rate of the discrete operator,
 *   Gamma = |M|^2 sum_i h_i f_i nu_i / sum_i h_i f_i,  nu_i = sum_nm W_inm f_t,
 * checked at u0 and after every check_every RK4 steps.  Once it exceeds
 * eps_switch H, adaptive Heun in u (the controller of oracle_solve, projected
 * operator) runs to u_end.
 * p[12]: u0 u_end du_rk4 check_every eps_switch h0 rtol atol h_min h_max
 *        max_attempts M2
 * res[10]: [0] u [1] u_switch (NaN: never) [2] rk4 steps [3] heun steps
 *          [4] rejects [5] evaluations [6] status [7] h [8] Gamma/H at the switch
 *          (or at the last check) [9] checks */
static double oracle_H(int n_h, const double *hu, const double *hl, double u) {
    if (n_h == 1) return exp(hl[0]);
    int k = 0;
    while (k + 2 < n_h && u > hu[k + 1]) ++k;
    double s = (hl[k + 1] - hl[k]) / (hu[k + 1] - hu[k]);
    return exp(hl[k] + s * (u - hu[k]));
}

typedef struct {
    int n; const double *q; double mass, M2; int n_mu, measure;
    int n_src; const double *shape, *rate, *tau, *u_on, *hc;
    int n_h; const double *hu, *hl;
    double *W, *p, *E, *dp, *dE, *h;
} exp_ctx;

/* grid and kernel at a = e^u */
static int exp_at(const exp_ctx *c, double u) {
    double a = exp(u);
    int rc = oracle_grid(c->n, c->q, a, c->mass, c->p, c->E, c->dp, c->dE, c->h);
    if (rc) return rc;
    return oracle_kernel_tensor(c->n, c->q, a, c->mass, 1.0, c->n_mu, c->measure, 0, c->W);
}

/* S(u) with comoving-weight normalisation */
static void exp_source(const exp_ctx *c, double u, double *S) {
    oracle_source(c->n, c->hc, u, c->n_src, c->shape, c->rate, c->tau, c->u_on, S);
}

/* RHS(f, u) = (C_proj[f; a(u)] + S(u)) / H(u) */
static int exp_rhs(const exp_ctx *c, const double *f, double u, double *out, double *work) {
    int n = c->n;
    int rc = exp_at(c, u);
    if (rc) return rc;
    rc = oracle_collision_tensor(n, c->q, exp(u), c->mass, c->W, f, work, NULL, NULL);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) work[i] *= c->M2;
    rc = oracle_project(n, c->E, c->h, f, work, out, NULL);
    if (rc == OR_ESINGULAR) rc = OR_OK;
    if (rc) return rc;
    double *S = work + n;
    exp_source(c, u, S);
    double inv = 1.0 / oracle_H(c->n_h, c->hu, c->hl, u);
    for (int i = 0; i < n; ++i) out[i] = (out[i] + S[i]) * inv;
    return OR_OK;
}

/* Gamma_2->2 / H at u */
static int exp_gamma_over_H(const exp_ctx *c, const double *f, double u, double *g, double *work) {
    int n = c->n;
    int rc = exp_at(c, u);
    if (rc) return rc;
    double *L = work;
    rc = oracle_collision_tensor(n, c->q, exp(u), c->mass, c->W, f, work + n, work + 2 * n, L);
    if (rc) return rc;
    double num = 0.0, den = 0.0;
    for (int i = 0; i < n; ++i) {
        num += c->h[i] * f[i] * L[i];
        den += c->h[i] * f[i];
    }
    *g = den > 0.0 ? c->M2 * num / den / oracle_H(c->n_h, c->hu, c->hl, u) : 0.0;
    return OR_OK;
}

int oracle_solve_expanding(int n, const double *q, double mass, int n_mu, int measure,
                           int n_src, const double *shape, const double *rate, const double *tau,
                           const double *u_on, int n_h, const double *hu, const double *hlnH,
                           const double *p, double *f, double *res) {
    if (n < 4 || n_h < 1) return OR_EINVAL;
    double *buf = malloc(sizeof(double) * ((size_t)n * n * n + 16 * (size_t)n));
    if (!buf) return OR_ENOMEM;
    double *W = buf, *v = buf + (size_t)n * n * n;
    double *pp = v, *E = v + n, *dp = v + 2 * n, *dE = v + 3 * n, *h = v + 4 * n, *hc = v + 5 * n;
    double *k1 = v + 6 * n, *k2 = v + 7 * n, *fp = v + 8 * n, *fc = v + 9 * n, *work = v + 10 * n;
    double *k3 = v + 13 * n, *k4 = v + 14 * n;
    int rc = oracle_grid(n, q, 1.0, mass, pp, E, dp, dE, hc);   /* comoving weights q^2 Dq */
    if (rc) { free(buf); return rc; }
    exp_ctx c = { n, q, mass, p[11], n_mu, measure, n_src, shape, rate, tau, u_on, hc, n_h, hu, hlnH,
                  W, pp, E, dp, dE, h };
    double u = p[0], u_end = p[1], du = p[2], eps = p[4];
    int check_every = (int)p[3];
    double hs = p[5], rtol = p[6], atol = p[7], h_min = p[8], h_max = p[9];
    long max_att = (long)p[10];
    long rk4 = 0, steps = 0, rejects = 0, evals = 0, checks = 0;
    double u_switch = NAN, gh = 0.0;
    int status = OR_OK, switched = 0;
    /* regime 1: sources only, RK4 on fixed intervals, Gamma/H checks */
    rc = exp_gamma_over_H(&c, f, u, &gh, work);
    if (rc) { free(buf); return rc; }
    checks++;
    if (gh > eps) { switched = 1; u_switch = u; }
    while (!switched && u < u_end) {
        /* step k spans [u0 + k du, u0 + (k+1) du], the last one clipped at u_end */
        double d = du;
        u = p[0] + (double)rk4 * du;
        if (u + d >= u_end) d = u_end - u;
        double u1 = u + 0.5 * d, u2 = u + d;
        double i0 = 1.0 / oracle_H(n_h, hu, hlnH, u), i1 = 1.0 / oracle_H(n_h, hu, hlnH, u1);
        double i2 = 1.0 / oracle_H(n_h, hu, hlnH, u2);
        exp_source(&c, u, k1);
        exp_source(&c, u1, k2);
        exp_source(&c, u1, k3);
        exp_source(&c, u2, k4);
        for (int i = 0; i < n; ++i)
            f[i] = f[i] + d / 6.0 * (((k1[i] * i0 + 2.0 * (k2[i] * i1)) + 2.0 * (k3[i] * i1)) + k4[i] * i2);
        u = (u + d >= u_end) ? u_end : u + d;
        rk4++;
        if (check_every > 0 && rk4 % check_every == 0) {
            rc = exp_gamma_over_H(&c, f, u, &gh, work);
            if (rc) { free(buf); return rc; }
            checks++;
            if (gh > eps) { switched = 1; u_switch = u; }
        }
    }
    /* regime 2: adaptive Heun in u with collisions (controller of oracle_solve) */
    while (switched && u < u_end) {
        if (steps + rejects >= max_att) { status = OR_ENOCONV; break; }
        double htry = hs;
        if (htry > h_max) htry = h_max;
        if (htry < h_min) htry = h_min;
        int last = 0;
        if (u + htry >= u_end) { htry = u_end - u; last = 1; }
        rc = exp_rhs(&c, f, u, k1, work);
        if (rc) { status = rc; break; }
        evals++;
        int neg = 0;
        for (int i = 0; i < n; ++i) {
            fp[i] = f[i] + htry * k1[i];
            if (!isfinite(fp[i])) { status = OR_ENONFINITE; break; }
            if (fp[i] < 0.0) neg = 1;
        }
        if (status) break;
        if (neg) { hs = 0.5 * htry; rejects++; continue; }
        rc = exp_rhs(&c, fp, u + htry, k2, work);
        if (rc) { status = rc; break; }
        evals++;
        double err = 0.0;
        for (int i = 0; i < n; ++i) {
            fc[i] = f[i] + 0.5 * htry * (k1[i] + k2[i]);
            if (!isfinite(fc[i])) { status = OR_ENONFINITE; break; }
            if (fc[i] < 0.0) neg = 1;
            double e = fabs(fc[i] - fp[i]) / (atol + rtol * fabs(fc[i]));
            if (e > err) err = e;
        }
        if (status) break;
        if (neg) { hs = 0.5 * htry; rejects++; continue; }
        double fac = err > 0.0 ? 0.9 / sqrt(err) : 5.0;
        if (fac > 5.0) fac = 5.0;
        if (fac < 0.2) fac = 0.2;
        if (err <= 1.0) {
            for (int i = 0; i < n; ++i) f[i] = fc[i];
            u = last ? u_end : u + htry;
            steps++;
        } else {
            rejects++;
        }
        hs = htry * fac;
    }
    res[0] = u; res[1] = u_switch; res[2] = (double)rk4; res[3] = (double)steps;
    res[4] = (double)rejects; res[5] = (double)evals; res[6] = status; res[7] = hs; res[8] = gh;
    res[9] = (double)checks;
    free(buf);
    return status;
}
