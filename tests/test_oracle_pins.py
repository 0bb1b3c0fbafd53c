"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against something the paper or mathematics fixes:
library routines for special cases, closed forms derived independently,
textbook two-body phase space, exact invariants, dimensional analysis, and the
paper's printed Table 1.  A plausible slip (dropped term, wrong sign or index,
transposed operand, wrong measure or normalisation) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
import kx_inputs as ki

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- grid -----
def test_grid_trapezoid_closed_form():
    """Appendix A grid with trapezoid widths (reading A2): on a uniform grid the
    widths are the spacing (half at the ends) and sum to q_max - q_min; E, h,
    dE follow their definitions; p = q/a."""
    q = np.linspace(0.5, 4.0, 8)
    g = oracle.grid(q, a=2.0, mass=1.5)
    d = q[1] - q[0]
    dq = np.full(8, d)
    dq[0] = dq[-1] = d / 2
    np.testing.assert_allclose(g["dp"], dq / 2.0, rtol=1e-15)
    np.testing.assert_allclose(g["p"], q / 2.0, rtol=1e-15)
    assert abs(g["dp"].sum() * 2.0 - (q[-1] - q[0])) < 1e-14
    np.testing.assert_allclose(g["E"], np.hypot(q / 2.0, 1.5), rtol=1e-15)
    np.testing.assert_allclose(g["h"], (q / 2) ** 2 * dq / 2, rtol=1e-15)
    np.testing.assert_allclose(g["dE"], (q / 2) * (dq / 2) / g["E"], rtol=1e-15)


def test_grid_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.grid(np.array([1.0, 2.0, 2.0, 3.0]))
    with pytest.raises(ValueError):
        oracle.grid(np.array([1.0, 2.0, 3.0]))
    with pytest.raises(ValueError):
        oracle.grid(np.array([-1.0, 2.0, 3.0, 4.0]))


# ------------------------------------------------------- Gauss-Legendre ----
@pytest.mark.parametrize("n", [1, 2, 5, 18, 36, 144])
def test_gauss_legendre_matches_library(n):
    """P10: nodes/weights equal numpy's Golub-Welsch leggauss (different
    algorithm) and integrate polynomials of degree 2n-1 exactly."""
    x, w = oracle.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=2e-15)
    np.testing.assert_allclose(w, wr, atol=5e-15, rtol=1e-13)
    for k in range(0, 2 * n, 3):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


# --------------------------------------------------------- nu integral -----
def _random_coeffs(rng, count):
    out = []
    while len(out) < count:
        m = 1.0
        pi, pn, pm = np.exp(rng.uniform(np.log(1e-2), np.log(20.0), size=3))
        Ei, En, Em = (math.hypot(v, m) for v in (pi, pn, pm))
        mu = rng.uniform(-0.999, 0.999)
        A0 = m * m + En * Em - En * Ei - Em * Ei + pi * pn * mu
        A1 = pi * pm - pn * pm * mu
        K2 = pn * pn * pm * pm * (1 - mu * mu)
        out.append((A0, A1, K2))
    return out


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_nu_integral_root_interval_inside_unit_interval():
    """P2: whenever Delta >= 0 both roots of a nu^2 + b nu + c lie in [-1, 1]
    (clipping never acts) and a direct numerical quadrature of
    int dnu / sqrt(a nu^2 + b nu + c) over [-1, 1] equals the oracle's value for
    both the printed arcsin form and the closed form."""
    rng = np.random.default_rng(11)
    hits = 0
    for A0, A1, K2 in _random_coeffs(rng, 400):
        a = -(K2 + A1 * A1)
        b = -2 * A0 * A1
        c = K2 - A0 * A0
        disc = b * b - 4 * a * c
        Ic = oracle.nu_integral(A0, A1, K2, "closed")
        Ia = oracle.nu_integral(A0, A1, K2, "arcsin")
        assert abs(Ic - Ia) <= 1e-14 * max(abs(Ic), 1e-300)
        if disc < 0:
            assert Ic == 0.0
            continue
        r = sorted([(-b + math.sqrt(disc)) / (2 * a), (-b - math.sqrt(disc)) / (2 * a)])
        assert -1 - 1e-12 <= r[0] <= r[1] <= 1 + 1e-12
        if hits < 40 and r[1] - r[0] > 1e-3:
            hits += 1
            val, _ = integrate.quad(lambda v: 1.0 / math.sqrt(max(a * v * v + b * v + c, 1e-300)),
                                    r[0], r[1], limit=200, epsabs=0, epsrel=1e-10)
            assert abs(val - Ic) < 1e-6 * Ic
    assert hits >= 10


# ------------------------------------------------------------- kernel F ----
def _support_cases():
    return [(0.7, 1.3, 0.4), (2.0, 1.5, 1.7), (0.05, 0.3, 0.2), (3.0, 3.5, 0.9), (1.0, 0.2, 2.5)]


@pytest.mark.parametrize("pi,pn,pm", _support_cases())
def test_F_converges_to_exact_kernel(pi, pn, pm):
    """P1: the Gauss-Legendre F (eq. app_F_1d) tends to the closed-form
    N_mu -> infinity kernel |M|^2 pi L / (4 (2pi)^4 p_i) (triangle overlap L)
    as N_mu grows, and GL applied piecewise between the Theta breakpoints is
    exact to 1e-10 (the integrand is smooth there)."""
    m, M2 = 1.0, 1.0
    Ei, En, Em = (math.hypot(v, m) for v in (pi, pn, pm))
    Et = En + Em - Ei
    assert Et > m
    pt = math.sqrt(Et * Et - m * m)
    Fx = oracle.F_exact(M2, pi, pn, pm, pt)
    assert Fx > 0
    errs = [abs(oracle.F(m, M2, pi, pn, pm, n_mu=nm) - Fx) / Fx for nm in (18, 72, 288, 1152)]
    assert errs[-1] < 2e-3
    assert errs[-1] < errs[0] or errs[0] < 1e-12
    # piecewise: breakpoints where k(mu) = |pt - pm| or pt + pm
    bps = [-1.0, 1.0]
    for kk in (abs(pt - pm), pt + pm):
        mu_b = (pi * pi + pn * pn - kk * kk) / (2 * pi * pn)
        if -1 < mu_b < 1:
            bps.append(mu_b)
    bps = sorted(bps)
    xg, wg = np.polynomial.legendre.leggauss(60)
    tot = 0.0
    for lo, hi in zip(bps[:-1], bps[1:]):
        nodes = (0.5 * (hi - lo) * xg + 0.5 * (hi + lo), 0.5 * (hi - lo) * wg)
        # only pieces inside the Theta support contribute; the oracle's own Theta decides
        tot += oracle.F(m, M2, pi, pn, pm, nodes=nodes)
    assert abs(tot - Fx) < 1e-10 * Fx


def test_F_is_symmetric_in_outgoing_pair_in_the_limit():
    """The exact kernel is symmetric under n <-> m (identical particles); the
    GL kernel only approximately (this is why the library symmetrises)."""
    m = 1.0
    for pi, pn, pm in _support_cases():
        Ei, En, Em = (math.hypot(v, m) for v in (pi, pn, pm))
        pt = math.sqrt((En + Em - Ei) ** 2 - 1)
        a = oracle.F_exact(1.0, pi, pn, pm, pt)
        b = oracle.F_exact(1.0, pi, pm, pn, pt)
        assert abs(a - b) < 1e-13 * max(a, b)


# --------------------------------------------- measure and normalisation ---
def _nu_two_body(p1, T, m=1.0):
    """Textbook loss rate for constant |M|^2 = 1 and f = exp(-E/T):
    nu(p1) = 1/(2E1) int d^3p2/((2pi)^3 2E2) f(p2) beta(s)/(8 pi),
    beta = sqrt(1 - 4 m^2/s), s = 2m^2 + 2(E1 E2 - p1 p2 cos)."""
    E1 = math.hypot(p1, m)

    def inner(c, p2):
        E2 = math.hypot(p2, m)
        s = 2 * m * m + 2 * (E1 * E2 - p1 * p2 * c)
        beta = math.sqrt(max(0.0, 1 - 4 * m * m / s))
        return p2 * p2 / (4 * math.pi ** 2 * 2 * E2) * math.exp(-E2 / T) * beta / (8 * math.pi)

    v, _ = integrate.dblquad(inner, 1e-6, 40 * T + 10, -1, 1, epsabs=1e-14, epsrel=1e-10)
    return v / (2 * E1)


def test_loss_rate_matches_two_body_phase_space():
    """P3: for f = e^{-E/T} the discrete loss rate nu_i = sum_nm W_inm f_t
    (f_t exact for MB under log interpolation) converges to the textbook
    two-body rate at second order in the grid spacing with the energy measure
    (reading A1); the literal Delta p_n Delta p_m measure misses it by > 50 %.
    This pins |M|^2, 1/(2E_i g), 4(2pi)^4, the p_n p_m factor and A0/A1/K^2."""
    T = 0.5
    probes = (0.1, 0.5, 1.0)
    errs = {}
    for N in (48, 96):
        q = ki.log_grid(N, 1e-3, 1e2)
        g = oracle.grid(q)
        f = np.exp(-g["E"] / T)
        idx = [int(np.argmin(abs(q - x))) for x in probes]
        ref = [_nu_two_body(q[i], T) for i in idx]
        for ang in (oracle.ANG_EXACT, oracle.ANG_GL_CLOSED):
            W = oracle.kernel_tensor(q, angular=ang)
            _, _, L = oracle.collision_tensor(q, W, f, parts=True)
            errs[(N, ang)] = [abs(L[i] / r - 1) for i, r in zip(idx, ref)]
    e48, e96 = np.array(errs[(48, 2)]), np.array(errs[(96, 2)])
    assert e96.max() < 1.2e-2
    assert np.all(e48 / e96 > 3.0)  # second order: ratio ~ 4
    assert np.max(errs[(96, 0)]) < 1.5e-2  # GL-18 adds little
    # the literal measure is far off
    q = ki.log_grid(96, 1e-3, 1e2)
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q, angular=oracle.ANG_EXACT, measure=oracle.MEASURE_LITERAL)
    _, _, L = oracle.collision_tensor(q, W, np.exp(-g["E"] / T), parts=True)
    i = np.argmin(abs(q - 0.5))
    assert abs(L[i] / _nu_two_body(q[i], T) - 1) > 0.5


def test_raw_residuals_vanish_with_grid_refinement():
    """Continuum conservation (eq. C22_conservation): with the energy measure
    the raw moment residuals eps_N, eps_E of eq. (app_epsilon_definition)
    decrease ~N^-2 for a smooth two-bump f; with the literal measure they do not
    (the paper reports non-vanishing residuals, Appendix B)."""
    eps = {}
    for N in (48, 96, 192):
        q = ki.log_grid(N, 1e-3, 1e2)
        g = oracle.grid(q)
        f = ki.lognormal_bumps(q, (0.3, 2.0), (0.3, 0.3), (1.0, 0.5))
        for meas in (0, 1):
            W = oracle.kernel_tensor(q, angular=oracle.ANG_EXACT, measure=meas)
            C = oracle.collision_tensor(q, W, f)
            _, d = oracle.project(g["E"], g["h"], f, C)
            eps[(N, meas)] = max(abs(d["eps_N_raw"]), abs(d["eps_E_raw"]))
    assert eps[(96, 0)] < 0.5 * eps[(48, 0)]
    assert eps[(192, 0)] < 0.5 * eps[(96, 0)]
    assert eps[(192, 0)] < 1e-2
    assert eps[(192, 1)] > 0.1


def test_dimensional_scaling_of_W():
    """P7: W has the dimension of |M|^2 m: scaling q -> lam q and m -> lam m
    multiplies W by lam (for fixed |M|^2), and W is linear in |M|^2."""
    q = ki.log_grid(10, 1e-2, 10.0)
    W1 = oracle.kernel_tensor(q, mass=1.0, M2=1.0)
    W2 = oracle.kernel_tensor(3.0 * q, mass=3.0, M2=1.0)
    W3 = oracle.kernel_tensor(q, mass=1.0, M2=7.0)
    np.testing.assert_allclose(W3, 7.0 * W1, rtol=1e-13, atol=1e-300)
    both = (W1 > 0) & (W2 > 0)
    np.testing.assert_allclose(W2[both], 3.0 * W1[both], rtol=1e-12)
    # elements kept on one side only are exact support ties E_t = E_0 or E_{N-1}
    # (e.g. n = 0, m = i) that rounding of (E_n + E_m) - E_i decides
    E = oracle.grid(q)["E"]
    for i, n, m in zip(*np.nonzero((W1 > 0) != (W2 > 0))):
        Et = E[n] + E[m] - E[i]
        assert min(abs(Et - E[0]), abs(Et - E[-1])) < 1e-14 * Et


def test_sigma_convention_matches_table1():
    """Reading A3 pinned on the paper's printed Table 1: |M|^2 = lambda^2 and
    sigma_T/m = lambda^2/(64 pi m^3) with m = 500 MeV in cm^2/g."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_sigma.txt"))
    m_gev = 0.5
    gev2_to_cm2 = 0.3893794e-27      # (hbar c)^2 in GeV^2 cm^2
    gev_to_g = 1.78266192e-24
    for lam, s_over_m in rows:
        sigma = lam ** 2 / oracle.M2_from_sigma(m_gev, 1.0)   # GeV^-2
        val = sigma / m_gev * gev2_to_cm2 / gev_to_g
        assert abs(val / s_over_m - 1) < 0.03, (lam, val, s_over_m)


# ------------------------------------------------- interpolation / support -
def test_mb_fixed_point():
    """P4: log interpolation is exact for f = z e^{-E/T} (eq. app_log_interp),
    so every element's gain and loss cancel: C_raw(MB) = 0 to rounding, with the
    range cut (whole elements dropped)."""
    for (N, qmax, T, z) in ((24, 10.0, 0.3, 0.5), (40, 1e2, 2.0, 1e-3)):
        q = ki.log_grid(N, 1e-3, qmax)
        g = oracle.grid(q)
        f = z * np.exp(-g["E"] / T)
        W = oracle.kernel_tensor(q)
        C, G, L = oracle.collision_tensor(q, W, f, parts=True)
        assert np.max(abs(C)) <= 2e-14 * np.max(G)


def test_bracket_and_support_brute_force():
    """Support (E_0 <= E_t <= E_{N-1}) and bracket (largest j <= N-2 with
    E_j <= E_t) against numpy searchsorted, for every (i, n, m) at N = 7 on a
    random grid; omega in [0, 1] and reproduces E_t."""
    rng = np.random.default_rng(5)
    q = ki.random_grid(rng, 7, 1e-2, 5.0)
    g = oracle.grid(q)
    E = g["E"]
    jL, om = oracle.bracket_tensor(q)
    for i in range(7):
        for n in range(7):
            for m in range(7):
                Et = (E[n] + E[m]) - E[i]
                inside = E[0] <= Et <= E[-1]
                if not inside:
                    assert jL[i, n, m] == -1
                    continue
                j = min(int(np.searchsorted(E, Et, side="right")) - 1, 5)
                assert jL[i, n, m] == j
                assert 0.0 <= om[i, n, m] <= 1.0
                assert abs(E[j] + om[i, n, m] * (E[j + 1] - E[j]) - Et) < 1e-14 * Et


def test_direct_equals_tensor():
    """P6: the direct form (F on the fly, printed arcsin nu integral) equals the
    tensor form (stored W, closed-form nu integral)."""
    rng = np.random.default_rng(6)
    for N in (6, 12):
        q = ki.random_grid(rng, N, 1e-3, 10.0)
        f = ki.bimodal(rng, q)
        W = oracle.kernel_tensor(q, M2=3.0)
        Ct = oracle.collision_tensor(q, W, f)
        Cd = oracle.collision_direct(q, f, M2=3.0)
        assert np.max(abs(Ct - Cd)) <= 1e-13 * np.max(abs(Ct))


def test_bilinearity_and_loss_structure():
    """P7: C(lam f) = lam^2 C(f) (dilute operator; a loss written with f_t
    alone would be linear) and C = G - f nu elementwise."""
    q = ki.log_grid(16, 1e-3, 10.0)
    f = ki.bimodal(np.random.default_rng(7), q)
    W = oracle.kernel_tensor(q)
    C, G, L = oracle.collision_tensor(q, W, f, parts=True)
    C3 = oracle.collision_tensor(q, W, 3.0 * f)
    np.testing.assert_allclose(C3, 9.0 * C, rtol=1e-12, atol=1e-14 * np.max(abs(C)))
    np.testing.assert_allclose(C, G - f * L, rtol=1e-12, atol=1e-14 * np.max(G))


# ------------------------------------------------------------ projection ---
def test_projection_invariants():
    """P5: the projected operator has zero number and energy moments, C_proj of
    an MB state stays zero, alpha = beta = 0 when the raw moments vanish, the
    correction is restricted to the support (xi = 0 below eps_supp), and a
    one-bin support is flagged singular (reading A10)."""
    q = ki.log_grid(32, 1e-3, 10.0)
    g = oracle.grid(q)
    E, h = g["E"], g["h"]
    f = ki.bimodal(np.random.default_rng(8), q)
    W = oracle.kernel_tensor(q)
    C = oracle.collision_tensor(q, W, f)
    Cp, d = oracle.project(E, h, f, C)
    scale = np.sum(h * abs(C))
    assert abs(np.sum(h * Cp)) < 1e-14 * scale
    assert abs(np.sum(h * E * Cp)) < 1e-14 * np.sum(h * E * abs(C))
    assert abs(d["eps_N_proj"]) < 1e-13 and abs(d["eps_E_proj"]) < 1e-13
    assert d["R_N"] > 0 and d["singular"] == 0
    # restricted to support
    f2 = f.copy()
    f2[:5] = 1e-20 * f.max()
    Cp2, _ = oracle.project(E, h, f2, C)
    np.testing.assert_array_equal(Cp2[:5], C[:5])
    # zero raw moments -> unchanged
    Cz = Cp.copy()
    Cz2, d2 = oracle.project(E, h, f, Cz)
    assert abs(d2["alpha"]) < 1e-12 * np.max(abs(C)) and np.allclose(Cz2, Cz, rtol=1e-12, atol=1e-15 * np.max(abs(C)))
    # singular
    f1 = np.zeros_like(f)
    f1[10] = 1.0
    _, d3 = oracle.project(E, h, f1, C)
    assert d3["singular"] == 1 and d3["rc"] == oracle.ESINGULAR


def test_projection_is_the_two_moment_least_change():
    """The correction xi (alpha + beta E) solves the 2x2 system of eq.
    (app_projection_system): checked against numpy.linalg.solve."""
    q = ki.log_grid(20, 1e-3, 10.0)
    g = oracle.grid(q)
    E, h = g["E"], g["h"]
    rng = np.random.default_rng(9)
    f = ki.bimodal(rng, q)
    C = rng.normal(size=20)
    Cp, d = oracle.project(E, h, f, C)
    xi = np.abs(f) / np.max(np.abs(f))
    A = np.array([[np.sum(h * xi), np.sum(h * E * xi)], [np.sum(h * E * xi), np.sum(h * E * E * xi)]])
    ab = np.linalg.solve(A, [np.sum(h * C), np.sum(h * E * C)])
    assert abs(d["alpha"] - ab[0]) < 1e-10 * abs(ab[0])
    assert abs(d["beta"] - ab[1]) < 1e-10 * abs(ab[1])


# ---------------------------------------------------------------- sources --
def test_source_normalisation_and_envelope():
    q = ki.log_grid(40, 1e-3, 10.0)
    g = oracle.grid(q)
    src = ki.two_sources(q, t_scale=2.0, rate=0.3)
    for t in (-1.0, 0.0, 1.0, 6.0, 9.0):
        S = oracle.source(g["h"], t, **src)
        env = [math.exp(-(t - t0) / tau) if t >= t0 else 0.0 for t0, tau in zip(src["t_on"], src["tau"])]
        assert abs(np.sum(g["h"] * S) - 0.3 * sum(env)) < 1e-14 * max(1e-300, 0.3 * sum(env)) + 1e-300


# ----------------------------------------------------------------- MB fit --
def test_mb_fit_recovers_and_matches_moments():
    q = ki.log_grid(64, 1e-3, 10.0)
    g = oracle.grid(q)
    E, h = g["E"], g["h"]
    f = 0.2 * np.exp(-E / 0.4)
    r = oracle.mb_fit(E, h, f)
    assert abs(r["T"] / 0.4 - 1) < 1e-10 and r["l1"] < 1e-10
    assert abs(r["ln_z"] - math.log(0.2)) < 1e-8
    fb = ki.bimodal(np.random.default_rng(10), q)
    r = oracle.mb_fit(E, h, fb)
    fmb = np.exp(r["ln_z"] - E / r["T"])
    assert abs(np.sum(h * fmb) / np.sum(h * fb) - 1) < 1e-10
    assert abs(np.sum(h * E * fmb) / np.sum(h * E * fb) - 1) < 1e-10
    assert abs(np.sum(h * abs(fb - fmb)) / np.sum(h * fb) - r["l1"]) < 1e-10


# ----------------------------------------------------------------- Heun ----
def _small_problem(N=24, seed=12):
    q = ki.log_grid(N, 1e-3, 10.0)
    f0 = ki.bimodal(np.random.default_rng(seed), q)
    W = oracle.kernel_tensor(q)
    return q, f0, W


def test_heun_conservation_with_constant_source():
    """P9: projection + a constant-rate source: the trapezoid corrector is exact
    for a constant source, so N(t) = N(0) + R t and E(t) = E(0) + R <E>_s t."""
    q, f0, W = _small_problem()
    g = oracle.grid(q)
    shape = ki.lognormal_bumps(q, (1.0,), (0.3,), (1.0,))
    src = dict(shape=shape[None], rate=np.array([0.01]), tau=np.array([1e300]), t_on=np.array([0.0]))
    M2 = oracle.M2_from_sigma(1.0, 1.0)
    f, res = oracle.solve(q, W, f0, M2, sources=src, t_end=2.0, h0=0.01, fixed_step=1)
    assert res["status"] == 0 and res["steps"] == 200
    n0, n1 = np.sum(g["h"] * f0), np.sum(g["h"] * f)
    e_s = np.sum(g["h"] * g["E"] * shape) / np.sum(g["h"] * shape)
    assert abs(n1 - (n0 + 0.01 * 2.0)) < 1e-13 * n1
    assert abs(np.sum(g["h"] * g["E"] * f) - (np.sum(g["h"] * g["E"] * f0) + 0.01 * e_s * 2.0)) < 1e-13 * n1


def test_heun_is_second_order():
    """The Euler-predictor / trapezoid-corrector pair of Sec. 4.2 is second
    order: halving h cuts the global error ~4x (a first-order slip gives 2x)."""
    q, f0, W = _small_problem()
    M2 = oracle.M2_from_sigma(1.0, 1.0)
    ref, _ = oracle.solve(q, W, f0, M2, t_end=0.4, h0=0.4 / 640, fixed_step=1)
    errs = []
    for k in (20, 40, 80):
        f, _ = oracle.solve(q, W, f0, M2, t_end=0.4, h0=0.4 / k, fixed_step=1)
        errs.append(np.max(abs(f - ref)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def test_sigma_collapse_of_trajectories():
    """P7/P8: without sources f(t; sigma) = f(sigma t; 1): fixed-step runs with
    h/sigma coincide with the sigma = 1 run."""
    q, f0, W = _small_problem()
    M2 = oracle.M2_from_sigma(1.0, 1.0)
    f1, _ = oracle.solve(q, W, f0, M2, t_end=0.5, h0=0.01, fixed_step=1)
    f8, _ = oracle.solve(q, W, f0, 8 * M2, t_end=0.5 / 8, h0=0.01 / 8, fixed_step=1)
    assert np.max(abs(f8 - f1)) < 1e-12 * np.max(f1)


def test_relaxation_to_mb_rate_scales_with_sigma():
    """P8: a bimodal f relaxes to the moment-matched MB (L1 <= 1e-3) and the
    time needed scales as 1/sigma; number and energy are conserved."""
    q, f0, W = _small_problem(N=32, seed=13)
    g = oracle.grid(q)
    times = {}
    for s in (1.0, 4.0):
        M2 = oracle.M2_from_sigma(1.0, s)
        f, res = oracle.solve(q, W, f0, M2, t_end=1e6, h0=1e-3 / s, l1_tol=1e-3,
                              check_every=1, rtol=1e-6, atol=1e-12 * f0.max())
        assert res["converged"] == 1 and res["l1"] <= 1e-3
        assert abs(np.sum(g["h"] * f) / np.sum(g["h"] * f0) - 1) < 1e-12
        assert abs(np.sum(g["h"] * g["E"] * f) / np.sum(g["h"] * g["E"] * f0) - 1) < 1e-12
        times[s] = res["t"]
    assert abs(times[1.0] / times[4.0] / 4.0 - 1) < 0.1


def test_fixed_step_negative_stage_is_an_error():
    q, f0, W = _small_problem()
    M2 = oracle.M2_from_sigma(1.0, 1.0)
    f, res = oracle.solve(q, W, f0, M2, t_end=100.0, h0=50.0, fixed_step=1)
    assert res["status"] in (oracle.ENEG, oracle.ENONFINITE)


# ------------------------------------------------ quantum statistics (f2) ---
def test_quantum_statistics_dilute_limit_is_bitwise_the_dilute_operator():
    """eta = 0 in the statistical factor of eq. (Lambda_quantum) is the dilute
    factor f_n f_m - f_i f_t of the same sum."""
    q = ki.log_grid(20, 1e-3, 10.0)
    f = ki.bimodal(np.random.default_rng(41), q)
    W = oracle.kernel_tensor(q)
    np.testing.assert_array_equal(oracle.collision_tensor_stats(q, W, f, 0),
                                  oracle.collision_tensor(q, W, f))


@pytest.mark.parametrize("eta", [1, -1])
def test_quantum_equilibrium_is_a_fixed_point_in_the_continuum_limit(eta):
    """Bose-Einstein (eta = +1) and Fermi-Dirac (eta = -1) equilibria
    f = 1/(exp((E - mu)/T) - eta) make the continuum factor vanish pointwise,
    so the discrete C -> 0 as the grid is refined (second order: the log-energy
    interpolation of a non-log-linear f is the only error); the dilute factor
    on the same f, and the factor with the opposite eta, do not vanish."""
    res, dil, wrong = [], [], []
    for N in (24, 48, 96):
        q = ki.log_grid(N, 1e-2, 20.0)
        E = oracle.grid(q)["E"]
        f = 1.0 / (np.exp((E - 0.6) / 0.7) - eta)
        W = oracle.kernel_tensor(q)
        _, G, _ = oracle.collision_tensor(q, W, f, parts=True)
        sc = np.max(np.abs(G))
        res.append(np.max(np.abs(oracle.collision_tensor_stats(q, W, f, eta))) / sc)
        dil.append(np.max(np.abs(oracle.collision_tensor_stats(q, W, f, 0))) / sc)
        wrong.append(np.max(np.abs(oracle.collision_tensor_stats(q, W, f, -eta))) / sc)
    for a, b in zip(res[:-1], res[1:]):
        assert 3.0 < a / b < 5.5, res
    assert res[-1] < 2e-3
    assert min(dil) > 0.05 and min(wrong) > 0.05


# ------------------------------------------------ Chebyshev loss expansion ---
def test_bessel_ive_against_scipy():
    """The oracle's own power-series e^{-x} I_k(x) against scipy's (Amos)."""
    import scipy.special as sp
    for x in (0.0, 1e-4, 0.3, 2.0, 9.0, 35.0, 150.0):
        a = oracle.bessel_ive(48, x)
        b = sp.ive(np.arange(48), x)
        m = b > 1e-290
        assert np.all(np.abs(a[m] - b[m]) <= 1e-12 * b[m]), x


def test_chebyshev_generating_function():
    """sum_k eps_k e^{-x} I_k(x) T_k(t) = e^{x (t - 1)} (the generating function
    behind the expansion of f_t), with T_k from cos(k arccos t)."""
    rng = np.random.default_rng(5)
    for x in (0.0, 0.7, 4.0, 15.0):
        iv = oracle.bessel_ive(90, x)
        for t in rng.uniform(-1, 1, 7):
            T = np.cos(np.arange(90) * np.arccos(t))
            s = iv[0] * T[0] + 2 * np.sum(iv[1:] * T[1:])
            assert abs(s - np.exp(x * (t - 1))) <= 1e-13 * max(1.0, np.exp(x * (t - 1)))


@pytest.mark.parametrize("N", [12, 28])
def test_chebyshev_loss_within_its_bound_and_converges(N):
    """Truncated loss vs the exact tensor-form loss: |L_K - L| <= bound row by
    row for K = 2 .. 32 (the bound is the printed sum over brackets of
    max(f_j, f_j+1) 2 sum_{k>=K} e^{-|d|/2} I_k(|d|/2)), the bound is not
    vacuous (the K = 2 error is at least a tenth of it somewhere), the gain is
    untouched, and K = 32 reproduces the exact loss to rounding; also on an f
    with a steep cold tail (large |d|)."""
    q = ki.log_grid(N, 1e-3, 10.0)
    W = oracle.kernel_tensor(q)
    g = oracle.grid(q)
    fs = [ki.bimodal(np.random.default_rng(N), q),
          0.5 * np.exp(-(g["E"] - 1.0) / 0.02) + 1e-4 * np.exp(-(g["E"] - 1.0) / 3.0)]
    for f in fs:
        C0, G0, L0 = oracle.collision_tensor(q, W, f, parts=True)
        for K in (2, 4, 8, 16, 32):
            C, G, L, B = oracle.collision_chebyshev(q, W, f, K)
            assert np.all(np.abs(L - L0) <= B + 1e-14 * np.abs(L0)), K
            np.testing.assert_array_equal(G, G0)
            np.testing.assert_allclose(C, G - f * L, rtol=0, atol=1e-15 * np.max(np.abs(G)))
            if K == 2:
                assert np.max(np.abs(L - L0) / np.maximum(B, 1e-300)) > 0.1
        C, G, L, B = oracle.collision_chebyshev(q, W, f, 32)
        if np.max(B / L0) < 1e-15:
            assert np.max(np.abs(L - L0) / L0) < 1e-13


# ------------------------------------------------------ expanding universe ---
def _rd_source(q, u_on=0.0, tau=0.3, rate=2e-2):
    return dict(shape=ki.lognormal_bumps(q, (0.5,), (0.3,), (1.0,))[None], rate=np.array([rate]),
                tau=np.array([tau]), t_on=np.array([u_on]))


def test_expanding_rk4_regime_is_fourth_order():
    """Sources only (the switch never fires): f(u_end) against the closed-form
    integral of S(u)/H(u) for H = exp(-2u) (radiation domination) and an
    exponential envelope; the error falls ~16x per halving of du."""
    q = ki.log_grid(16, 1e-3, 10.0)
    f0 = 1e-3 * ki.bimodal(np.random.default_rng(2), q)
    src = _rd_source(q)
    g1 = oracle.grid(q)   # a = 1: the comoving weights q^2 Dq
    s = src["shape"][0] / np.sum(g1["h"] * src["shape"][0])
    alpha, beta = -1.0 / 0.3 + 2.0, 0.0
    integral = (np.exp(alpha * 1.0) - 1.0) * np.exp(beta) / alpha
    exact = f0 + 2e-2 * s * integral
    errs = []
    for du in (0.1, 0.05, 0.025):
        f, r = oracle.solve_expanding(q, f0, 1.0, hu=[0.0, 1.0], hlnH=[0.0, -2.0], u0=0.0, u_end=1.0,
                                      du_rk4=du, eps_switch=np.inf, sources=src)
        assert np.isnan(r["u_switch"]) and r["steps"] == 0 and r["rk4_steps"] == round(1.0 / du)
        errs.append(np.max(np.abs(f - exact)) / np.max(exact))
    assert errs[0] / errs[1] > 12 and errs[1] / errs[2] > 12, errs
    assert errs[2] < 1e-8


def test_expanding_collisions_conserve_comoving_number():
    """Collisions only (switch at u0): the comoving number sum q^2 Dq f stays
    at its initial value to rounding while a grows (the projection zeroes the
    number moment at every a)."""
    q = ki.log_grid(14, 1e-3, 10.0)
    f0 = 1e-3 * ki.bimodal(np.random.default_rng(3), q)
    hc = oracle.grid(q)["h"]
    f, r = oracle.solve_expanding(q, f0, oracle.M2_from_sigma(1.0, 40.0), hu=[0.0, 1.0],
                                  hlnH=[0.0, -2.0], u0=0.0, u_end=0.3, eps_switch=0.0, h0=1e-3)
    assert r["u_switch"] == 0.0 and r["rk4_steps"] == 0 and r["steps"] > 10 and r["status"] == 0
    assert abs(np.sum(hc * f) / np.sum(hc * f0) - 1) < 1e-13


def test_expanding_heun_regime_against_an_independent_integrator():
    """The Heun regime against scipy's DOP853 (tight tolerances) on the same
    right-hand side (C_proj of the kernel at a = e^u plus the source, over
    H(u)), assembled here from the pinned primitives."""
    from scipy.integrate import solve_ivp
    q = ki.log_grid(12, 1e-3, 10.0)
    f0 = 1e-3 * ki.bimodal(np.random.default_rng(4), q)
    src = _rd_source(q, tau=0.5)
    M2 = oracle.M2_from_sigma(1.0, 60.0)
    hc = oracle.grid(q)["h"]
    s = src["shape"][0] / np.sum(hc * src["shape"][0])

    def rhs(u, f):
        a = np.exp(u)
        g = oracle.grid(q, a=a)
        W = oracle.kernel_tensor(q, a=a)
        C = oracle.collision_tensor(q, W, f, a=a) * M2
        Cp, _ = oracle.project(g["E"], g["h"], f, C)
        return (Cp + 2e-2 * np.exp(-u / 0.5) * s) / np.exp(-2.0 * u)

    ref = solve_ivp(rhs, (0.0, 0.25), f0, method="DOP853", rtol=1e-11, atol=1e-16).y[:, -1]
    f, r = oracle.solve_expanding(q, f0, M2, hu=[0.0, 1.0], hlnH=[0.0, -2.0], u0=0.0, u_end=0.25,
                                  eps_switch=0.0, sources=src, h0=1e-4, rtol=1e-9, atol=1e-18)
    assert r["status"] == 0 and r["u"] == 0.25
    assert np.max(np.abs(f - ref)) / np.max(ref) < 1e-6


def test_expanding_switch_rule():
    """eps_switch = 0 switches at u0 without RK4 steps; a finite threshold
    switches at the first check with Gamma/H above it."""
    q = ki.log_grid(16, 1e-3, 10.0)
    f0 = 1e-3 * ki.bimodal(np.random.default_rng(5), q)
    src = _rd_source(q)
    M2 = oracle.M2_from_sigma(1.0, 40.0)
    _, r0 = oracle.solve_expanding(q, f0, M2, hu=[0.0, 1.0], hlnH=[0.0, -2.0], u0=0.0, u_end=0.05,
                                   eps_switch=0.0, sources=src)
    assert r0["u_switch"] == 0.0 and r0["rk4_steps"] == 0
    _, r1 = oracle.solve_expanding(q, f0, oracle.M2_from_sigma(1.0, 80.0), hu=[0.0, 1.0],
                                   hlnH=[0.0, -2.0], u0=0.0, u_end=0.3, du_rk4=0.02, check_every=2,
                                   eps_switch=1e-2, sources=src)
    assert 0.0 < r1["u_switch"] < 0.3 and r1["gamma_over_H"] > 1e-2
    assert r1["rk4_steps"] == round(r1["u_switch"] / 0.02) and r1["checks"] == r1["rk4_steps"] // 2 + 1


@pytest.mark.parametrize("N", [96, 256])
def test_projection_correction_small_on_the_paper_workload(N):
    """The paper reports (Sec. 5, its runtime workload: the two-bump f of eq.
    benchmark_two_bump, m = 1, a = 1, q in [1e-3, 1e2], N_mu = 18, BE factors)
    that the pointwise moment-fixing correction stays below one percent of
    max |C_raw|.  The oracle's correction on that input, under the energy
    measure (reading A1): below 1 %, with and without the quantum factor."""
    q = ki.log_grid(N, 1e-3, 1e2)
    f = ki.paper_two_bump(q)
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q)
    for C in (oracle.collision_tensor_stats(q, W, f, 1), oracle.collision_tensor(q, W, f)):
        Cp, _ = oracle.project(g["E"], g["h"], f, C)
        assert np.max(np.abs(Cp - C)) < 1e-2 * np.max(np.abs(C))
