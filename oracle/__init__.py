"""FP64 CPU oracle for the discretised 2->2 elastic self-collision operator.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product package never imports it, and it imports nothing from the product
package.  The arithmetic lives in ``kx_oracle.c`` (plain C, FP64, no FMA
contraction); this module only compiles it (``gcc``) and marshals numpy arrays.

Parity status per function (pins live in ``tests/test_oracle_pins.py``):
  grid, gauss_legendre, nu integrals, F, F_exact, kernel_tensor, bracket,
  collision_tensor, collision_tensor_stats, collision_direct, project, source,
  mb_fit, solve, bessel_ive, collision_chebyshev, solve_expanding: pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# status codes (same meaning as the product library's, defined independently)
OK, EINVAL, ENOMEM, ENEG, ENONFINITE, ESINGULAR, ENOCONV = 0, -1, -2, -4, -5, -6, -7

MEASURE_ENERGY, MEASURE_LITERAL = 0, 1
ANG_GL_CLOSED, ANG_GL_ARCSIN, ANG_EXACT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, FP64, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    sig = {
        "oracle_grid": (i, [i, vp, d, d, vp, vp, vp, vp, vp]),
        "oracle_gauss_legendre": (i, [i, vp, vp]),
        "oracle_nu_integral_arcsin": (d, [d, d, d]),
        "oracle_nu_integral_closed": (d, [d, d, d]),
        "oracle_F": (d, [d, d, d, d, d, d, d, d, i, vp, vp, i]),
        "oracle_F_exact": (d, [d, d, d, d, d]),
        "oracle_bracket": (i, [i, vp, d, vp, vp]),
        "oracle_kernel_tensor": (i, [i, vp, d, d, d, i, i, i, vp]),
        "oracle_bracket_tensor": (i, [i, vp, d, d, vp, vp]),
        "oracle_collision_tensor": (i, [i, vp, d, d, vp, vp, vp, vp, vp]),
        "oracle_collision_tensor_stats": (i, [i, vp, d, d, vp, vp, i, vp]),
        "oracle_collision_direct": (i, [i, vp, d, d, d, i, i, vp, vp]),
        "oracle_project": (i, [i, vp, vp, vp, vp, vp, vp]),
        "oracle_source": (None, [i, vp, d, i, vp, vp, vp, vp, vp]),
        "oracle_mb_fit": (i, [i, vp, vp, vp, vp]),
        "oracle_solve": (i, [i, vp, d, d, vp, d, i, vp, vp, vp, vp, vp, vp, vp]),
        "oracle_M2_from_sigma": (d, [d, d]),
        "oracle_collision_rows": (i, [i, vp, d, d, d, i, i, vp, i, vp, vp, vp, vp]),
        "oracle_bessel_ive": (i, [i, d, vp]),
        "oracle_loss_chebyshev": (i, [i, vp, d, d, vp, vp, i, vp, vp, vp, vp]),
        "oracle_solve_expanding": (i, [i, vp, d, i, i, i, vp, vp, vp, vp, i, vp, vp, vp, vp, vp]),
        "oracle_num_threads": (i, []),
        "oracle_set_threads": (None, [i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def M2_from_sigma(mass: float, sigma: float) -> float:
    """|M|^2 = 64 pi m^2 sigma (Table 1 caption, contact interaction)."""
    return _load().oracle_M2_from_sigma(float(mass), float(sigma))


def grid(q, a=1.0, mass=1.0):
    """Appendix A grid: returns dict p, E, dp, dE, h."""
    q = _f64(q)
    n = q.size
    out = {k: np.empty(n) for k in ("p", "E", "dp", "dE", "h")}
    rc = _load().oracle_grid(n, _p(q), a, mass, _p(out["p"]), _p(out["E"]),
                             _p(out["dp"]), _p(out["dE"]), _p(out["h"]))
    if rc:
        raise ValueError(f"oracle_grid rc={rc}")
    return out


def gauss_legendre(n: int):
    x = np.empty(n)
    w = np.empty(n)
    rc = _load().oracle_gauss_legendre(n, _p(x), _p(w))
    if rc:
        raise ValueError(rc)
    return x, w


def nu_integral(A0, A1, K2, form="closed"):
    lib = _load()
    fn = lib.oracle_nu_integral_closed if form == "closed" else lib.oracle_nu_integral_arcsin
    return fn(float(A0), float(A1), float(K2))


def F(mass, M2, pi, pn, pm, n_mu=18, form="closed", nodes=None):
    """eq. (app_F_1d) for one (i, n, m); nodes=(x, w) overrides Gauss-Legendre."""
    x, w = nodes if nodes is not None else gauss_legendre(n_mu)
    x, w = _f64(x), _f64(w)
    Ei, En, Em = (np.sqrt(v * v + mass * mass) for v in (pi, pn, pm))
    return _load().oracle_F(mass, M2, pi, pn, pm, Ei, En, Em, x.size, _p(x), _p(w),
                            1 if form == "arcsin" else 0)


def F_exact(M2, pi, pn, pm, pt):
    return _load().oracle_F_exact(M2, pi, pn, pm, pt)


def bracket(E, Et):
    E = _f64(E)
    j = ctypes.c_int(0)
    om = ctypes.c_double(0.0)
    ok = _load().oracle_bracket(E.size, _p(E), float(Et), ctypes.byref(j), ctypes.byref(om))
    return (j.value, om.value) if ok else None


def kernel_tensor(q, a=1.0, mass=1.0, M2=1.0, n_mu=18, measure=MEASURE_ENERGY,
                  angular=ANG_GL_CLOSED):
    """W[i, n, m] of eq. (discrete_weight) (unsymmetrised, N^3 doubles)."""
    q = _f64(q)
    n = q.size
    W = np.empty((n, n, n))
    rc = _load().oracle_kernel_tensor(n, _p(q), a, mass, M2, n_mu, measure, angular, _p(W))
    if rc:
        raise ValueError(f"oracle_kernel_tensor rc={rc}")
    return W


def bracket_tensor(q, a=1.0, mass=1.0):
    q = _f64(q)
    n = q.size
    jL = np.empty((n, n, n), dtype=np.int32)
    om = np.empty((n, n, n))
    rc = _load().oracle_bracket_tensor(n, _p(q), a, mass, _p(jL), _p(om))
    if rc:
        raise ValueError(rc)
    return jL, om


def collision_tensor(q, W, f, a=1.0, mass=1.0, parts=False):
    """C_raw of eq. (discrete_collision_operator); parts=True also returns
    the gain G and the loss rate nu (C = G - f nu)."""
    q, W, f = _f64(q), _f64(W), _f64(f)
    n = q.size
    C, G, L = np.empty(n), np.empty(n), np.empty(n)
    rc = _load().oracle_collision_tensor(n, _p(q), a, mass, _p(W), _p(f), _p(C), _p(G), _p(L))
    if rc:
        raise ValueError(rc)
    return (C, G, L) if parts else C


def collision_tensor_stats(q, W, f, eta, a=1.0, mass=1.0):
    """C_raw with the quantum statistical factor of eq. (Lambda_quantum):
    eta = +1 Bose-Einstein, -1 Fermi-Dirac, 0 dilute."""
    q, W, f = _f64(q), _f64(W), _f64(f)
    n = q.size
    C = np.empty(n)
    rc = _load().oracle_collision_tensor_stats(n, _p(q), a, mass, _p(W), _p(f), int(eta), _p(C))
    if rc:
        raise ValueError(rc)
    return C


def bessel_ive(K, x):
    """e^{-x} I_k(x) for k = 0 .. K-1 (power series; x >= 0)."""
    out = np.empty(int(K))
    rc = _load().oracle_bessel_ive(int(K), float(x), _p(out))
    if rc:
        raise ValueError(rc)
    return out


def collision_chebyshev(q, W, f, K, a=1.0, mass=1.0):
    """C_raw with the loss rate's interpolated f_t expanded in K Chebyshev terms
    of t = 2 omega - 1 (coefficients e^{d/2} eps_k I_k(d/2)); returns
    (C, G, L, bound) with |L - exact L| <= bound row by row."""
    q, W, f = _f64(q), _f64(W), _f64(f)
    n = q.size
    C, G, L, B = (np.empty(n) for _ in range(4))
    rc = _load().oracle_loss_chebyshev(n, _p(q), a, mass, _p(W), _p(f), int(K), _p(C), _p(G),
                                       _p(L), _p(B))
    if rc:
        raise ValueError(rc)
    return C, G, L, B


def solve_expanding(q, f0, M2, hu, hlnH, u0, u_end, du_rk4=0.05, check_every=1, eps_switch=1e-2,
                    h0=1e-3, rtol=1e-6, atol=1e-12, h_min=0.0, h_max=np.inf, max_attempts=1_000_000,
                    sources=None, mass=1.0, n_mu=18, measure=MEASURE_ENERGY):
    """Expanding universe in u = log a (Sec. 4, eq. numerical_evolution_loga):
    RK4 on the sources while Gamma/H <= eps_switch, then adaptive Heun with the
    collisions.  H(u) = exp(piecewise-linear ln H through (hu, hlnH)).  Returns
    (f, result dict)."""
    q, f = _f64(q), _f64(f0).copy()
    n = q.size
    hu, hl = _f64(np.atleast_1d(hu)), _f64(np.atleast_1d(hlnH))
    if sources is None:
        shape = np.zeros((1, n)); rate = tau = u_on = np.zeros(1); ns = 0
    else:
        shape = _f64(np.atleast_2d(sources["shape"]))
        rate, tau, u_on = _f64(sources["rate"]), _f64(sources["tau"]), _f64(sources["t_on"])
        ns = shape.shape[0]
    p = _f64([u0, u_end, du_rk4, check_every, eps_switch, h0, rtol, atol, h_min,
              h_max if np.isfinite(h_max) else 1e300, max_attempts, M2])
    res = np.empty(10)
    rc = _load().oracle_solve_expanding(n, _p(q), mass, n_mu, measure, ns, _p(shape), _p(rate),
                                        _p(tau), _p(u_on), hu.size, _p(hu), _p(hl), _p(p), _p(f),
                                        _p(res))
    keys = ("u", "u_switch", "rk4_steps", "steps", "rejects", "evals", "status", "h",
            "gamma_over_H", "checks")
    out = dict(zip(keys, res))
    out["rc"] = rc
    return f, out


def collision_direct(q, f, a=1.0, mass=1.0, M2=1.0, n_mu=18, measure=MEASURE_ENERGY):
    q, f = _f64(q), _f64(f)
    n = q.size
    C = np.empty(n)
    rc = _load().oracle_collision_direct(n, _p(q), a, mass, M2, n_mu, measure, _p(f), _p(C))
    if rc:
        raise ValueError(rc)
    return C


def collision_rows(q, f, rows, a=1.0, mass=1.0, M2=1.0, n_mu=18, measure=MEASURE_ENERGY):
    """C_raw, G and nu of selected rows (direct form, no stored tensor)."""
    q, f = _f64(q), _f64(f)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    C, G, L = (np.empty(rows.size) for _ in range(3))
    rc = _load().oracle_collision_rows(q.size, _p(q), a, mass, M2, n_mu, measure, _p(f),
                                       rows.size, _p(rows), _p(C), _p(G), _p(L))
    if rc:
        raise ValueError(rc)
    return C, G, L


DIAG_KEYS = ("eps_N_raw", "eps_E_raw", "eps_N_proj", "eps_E_proj", "R_N", "R_E",
             "alpha", "beta", "singular", "f_max")


def project(E, h, f, C):
    E, h, f, C = _f64(E), _f64(h), _f64(f), _f64(C)
    out = np.empty(E.size)
    diag = np.empty(10)
    rc = _load().oracle_project(E.size, _p(E), _p(h), _p(f), _p(C), _p(out), _p(diag))
    d = dict(zip(DIAG_KEYS, diag))
    d["rc"] = rc
    return out, d


def source(h, t, shape, rate, tau, t_on):
    h = _f64(h)
    shape = _f64(np.atleast_2d(shape))
    rate, tau, t_on = _f64(rate), _f64(tau), _f64(t_on)
    S = np.empty(h.size)
    _load().oracle_source(h.size, _p(h), float(t), shape.shape[0], _p(shape), _p(rate),
                          _p(tau), _p(t_on), _p(S))
    return S


def higgs_decay_source(q, mass, m_h, T, coupling, g_chi=1.0, a=1.0):
    """Higgs decay into dark matter, eq. C_higgs_decay (Sec. 2), at p = q / a:
    coupling^2/(8 pi g) T/(E p) (exp(-E_h^-/T) - exp(-E_h^+/T)) with
    E_h^(+/-) = (m_h^2 E +/- m_h p sqrt(m_h^2 - 4 m^2)) / (2 m^2)."""
    p = _f64(q) / a
    E = np.sqrt(p * p + mass * mass)
    k = np.sqrt(m_h * m_h - 4.0 * mass * mass)
    e_minus = (m_h * m_h * E - m_h * p * k) / (2.0 * mass * mass)
    e_plus = (m_h * m_h * E + m_h * p * k) / (2.0 * mass * mass)
    return coupling ** 2 / (8.0 * np.pi * g_chi) * T / (E * p) * (np.exp(-e_minus / T) - np.exp(-e_plus / T))


def condensate_source_cell(q, mass, m_phi, a=1.0):
    """Grid cell of the condensate's delta function, eq. C_condensate_decay:
    p0 = sqrt(m_phi^2 - 4 m^2) / 2, cells = the trapezoid widths in q (edges at
    the midpoints, the ends at q_0 and q_{n-1}); None outside the grid."""
    q = _f64(q)
    x = 0.5 * np.sqrt(m_phi * m_phi - 4.0 * mass * mass) * a
    edges = np.concatenate(([q[0]], 0.5 * (q[1:] + q[:-1]), [q[-1]]))
    if x < edges[0] or x > edges[-1]:
        return None
    return int(min(np.searchsorted(edges, x, side="right") - 1, q.size - 1))


def mb_fit(E, h, f):
    E, h, f = _f64(E), _f64(h), _f64(f)
    out = np.empty(3)
    _load().oracle_mb_fit(E.size, _p(E), _p(h), _p(f), _p(out))
    return {"T": out[0], "ln_z": out[1], "l1": out[2]}


SOLVE_DEFAULTS = dict(t0=0.0, t_end=1.0, h0=1e-3, rtol=1e-6, atol=1e-12, h_min=0.0,
                      h_max=np.inf, l1_tol=0.0, max_attempts=10**6, fixed_step=0,
                      check_every=10, project=1)
RES_KEYS = ("t", "steps", "rejects", "l1", "T_mb", "ln_z_mb", "status", "h", "evals",
            "converged")


def solve(q, W, f0, M2, sources=None, a=1.0, mass=1.0, **params):
    """Heun time integration of df/dt = C_proj[f] + S(t) (static box).

    W must be built with |M|^2 = 1; M2 scales it.  sources: dict with
    shape [K][N], rate, tau, t_on (or None).  Returns (f, result dict)."""
    p = dict(SOLVE_DEFAULTS)
    p.update(params)
    par = _f64([p[k] for k in ("t0", "t_end", "h0", "rtol", "atol", "h_min", "h_max",
                                "l1_tol", "max_attempts", "fixed_step", "check_every",
                                "project")])
    q, W = _f64(q), _f64(W)
    f = _f64(f0).copy()
    n = q.size
    if sources:
        shape = _f64(np.atleast_2d(sources["shape"]))
        rate, tau, t_on = (_f64(sources[k]) for k in ("rate", "tau", "t_on"))
        ns = shape.shape[0]
    else:
        shape = rate = tau = t_on = None
        ns = 0
    res = np.empty(10)
    _load().oracle_solve(n, _p(q), a, mass, _p(W), float(M2), ns, _p(shape), _p(rate),
                         _p(tau), _p(t_on), _p(par), _p(f), _p(res))
    return f, dict(zip(RES_KEYS, res))

