// kx_sources.cu -- the paper's two freeze-in source terms as source shapes for
// the solve API (host code).
//
//   Higgs decay (eq. C_higgs_decay, Sec. 2):
//     C(p) = c^2 / (8 pi g) * T / (E p) * (exp(-E_h^-(p)/T) - exp(-E_h^+(p)/T)),
//     E_h^(+/-)(p) = (m_h^2 E +/- m_h p sqrt(m_h^2 - 4 m^2)) / (2 m^2),  c = lambda v;
//   condensate decay (eq. C_condensate_decay):
//     C(p) = (2 pi^2 / g) (2 Gamma n_Phi) delta(p - p0) / p0^2,
//     p0 = sqrt(m_Phi^2 - 4 m^2) / 2.
// The solve API normalises a shape row by its number weight (sum_i h_i shape_i)
// and multiplies by the row's rate, so each helper returns the profile and the
// rate that reproduce the formula: rate = sum_i h_i C(p_i) for the Higgs term
// (pointwise on the grid), and (2 pi^2 / g) (2 Gamma n_Phi) for the condensate,
// whose delta function is binned into the one cell (of the trapezoid widths in
// q) that contains p0: the number it injects is the formula's exactly.
#include <cmath>
#include <vector>

#include "kx_internal.cuh"

namespace {
// grid p_i = q_i / a and weights h_i = p_i^2 dp_i (trapezoid widths in q), as
// the kernel build uses them; false for a bad grid
bool kx_src_grid(int n, const double *q, double a, std::vector<double> &p, std::vector<double> &h) {
    if (n < 2 || !q || !(a > 0)) return false;
    for (int i = 0; i < n; ++i)
        if (!(q[i] > 0) || (i > 0 && !(q[i] > q[i - 1]))) return false;
    p.resize(n);
    h.resize(n);
    for (int i = 0; i < n; ++i) {
        double dq;
        if (i == 0) dq = (q[1] - q[0]) / 2.0;
        else if (i == n - 1) dq = (q[n - 1] - q[n - 2]) / 2.0;
        else dq = (q[i + 1] - q[i - 1]) / 2.0;
        p[i] = q[i] / a;
        h[i] = p[i] * p[i] * (dq / a);
    }
    return true;
}
}  // namespace

extern "C" int kx_source_higgs_decay(int n, const double *q, double a, double mass, double m_h,
                                     double T, double coupling, double g_chi, double *shape,
                                     double *rate) {
    std::vector<double> p, h;
    if (!shape || !rate || !kx_src_grid(n, q, a, p, h)) return KX_EINVAL;
    if (!(mass > 0) || !(m_h > 2 * mass) || !(T > 0) || !(g_chi > 0) || !std::isfinite(coupling))
        return KX_EINVAL;
    const double k = std::sqrt(m_h * m_h - 4 * mass * mass);
    const double pre = coupling * coupling / (8 * M_PI * g_chi);
    double r = 0.0;
    for (int i = 0; i < n; ++i) {
        const double E = std::sqrt(p[i] * p[i] + mass * mass);
        const double em = (m_h * m_h * E - m_h * p[i] * k) / (2 * mass * mass);
        const double ep = (m_h * m_h * E + m_h * p[i] * k) / (2 * mass * mass);
        // exp(-em/T) - exp(-ep/T) = exp(-em/T) (1 - exp(-(ep - em)/T)), without cancellation
        const double v = pre * T / (E * p[i]) * std::exp(-em / T) * -std::expm1(-(ep - em) / T);
        shape[i] = v;
        r += h[i] * v;
    }
    *rate = r;
    return KX_OK;
}

extern "C" int kx_source_condensate(int n, const double *q, double a, double mass, double m_phi,
                                    double g_chi, double gamma_n, double *shape, double *rate) {
    std::vector<double> p, h;
    if (!shape || !rate || !kx_src_grid(n, q, a, p, h)) return KX_EINVAL;
    if (!(mass > 0) || !(m_phi > 2 * mass) || !(g_chi > 0) || !(gamma_n >= 0)) return KX_EINVAL;
    const double p0 = 0.5 * std::sqrt(m_phi * m_phi - 4 * mass * mass);
    // cell i spans [(q_{i-1} + q_i)/2, (q_i + q_{i+1})/2) in q (the ends at q_0, q_{n-1}]
    const double x = p0 * a;
    int cell = -1;
    for (int i = 0; i < n; ++i) {
        const double lo = i == 0 ? q[0] : 0.5 * (q[i - 1] + q[i]);
        const double hi = i == n - 1 ? q[n - 1] : 0.5 * (q[i] + q[i + 1]);
        if (x >= lo && (x < hi || (i == n - 1 && x <= hi))) {
            cell = i;
            break;
        }
    }
    if (cell < 0) return KX_EINVAL;   // p0 outside the grid
    for (int i = 0; i < n; ++i) shape[i] = i == cell ? 1.0 : 0.0;
    *rate = 2 * M_PI * M_PI / g_chi * gamma_n;
    return KX_OK;
}
