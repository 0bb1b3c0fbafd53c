"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle legs.

This module holds no arithmetic of the collision method: it only draws grids,
distributions, source shapes, cross-sections and arrival streams from
``numpy.random.default_rng(seed)`` following the workload recipes.  Both the
CUDA library and the FP64 oracle receive exactly these arrays.

Shapes follow the paper's workloads: log-spaced comoving-momentum grids
(Sec. 4, Appendix A), bimodal freeze-in distributions made of two log-normal
bumps in ln p (the two-bump input of eq. (benchmark_two_bump), Sec. 5, and the
two-source scenario of Sec. 3), and source terms injecting at two momenta.
"""
from __future__ import annotations

import numpy as np

SIGMAS_CONFIG2 = (0.1, 1.0, 10.0, 100.0)


def log_grid(n: int, q_min: float, q_max: float) -> np.ndarray:
    """q_i = q_min (q_max/q_min)^(i/(n-1)), i = 0..n-1 (ascending)."""
    i = np.arange(n, dtype=np.float64)
    return q_min * (q_max / q_min) ** (i / (n - 1))


def lognormal_bumps(q, centres, widths, amps) -> np.ndarray:
    """sum_k A_k exp(-ln^2(q/c_k) / (2 w_k^2)) on the grid q."""
    q = np.asarray(q, dtype=np.float64)
    out = np.zeros_like(q)
    for c, w, a in zip(centres, widths, amps):
        out += a * np.exp(-np.log(q / c) ** 2 / (2.0 * w * w))
    return out


def paper_two_bump(q) -> np.ndarray:
    """eq. (benchmark_two_bump): bumps at q = 0.3 (width 0.18) and q = 8
    (width 0.22, amplitude 0.5); used with m = 1, a = 1, q in [1e-3, 1e2]."""
    return lognormal_bumps(q, (0.3, 8.0), (0.18, 0.22), (1.0, 0.5))


def bimodal(rng, q, c=(0.05, 2.0)) -> np.ndarray:
    """Seeded bimodal f: centres c, widths U[0.3, 0.5], amplitudes U[0.1, 1]."""
    w = rng.uniform(0.3, 0.5, size=2)
    a = rng.uniform(0.1, 1.0, size=2)
    return lognormal_bumps(q, c, w, a)


def config1(seed: int = 1):
    """Single instance, N = 32, p/m in [1e-3, 10], m = 1, sigma = 1."""
    rng = np.random.default_rng(seed)
    q = log_grid(32, 1e-3, 10.0)
    return dict(q=q, mass=1.0, sigma=1.0, f0=bimodal(rng, q), n_steps=100, h=0.02)


def two_sources(q, t_scale: float = 1.0, rate: float = 0.05):
    """Two freeze-in sources: bumps at p ~ 0.05 and p ~ 2 (width 0.3), switched
    on at t = 0 and t = 3 t_scale, decaying with tau = t_scale; rate = number
    injection rate at switch-on (the shape is normalised by the consumer)."""
    shape = np.stack([lognormal_bumps(q, (0.05,), (0.3,), (1.0,)),
                      lognormal_bumps(q, (2.0,), (0.3,), (1.0,))])
    return dict(shape=shape, rate=np.array([rate, rate]),
                tau=np.array([t_scale, t_scale]), t_on=np.array([0.0, 3.0 * t_scale]))


def config2(seed: int = 2, n: int = 128):
    """Single instance N = 128 full integration with two sources, four sigmas."""
    rng = np.random.default_rng(seed)
    q = log_grid(n, 1e-3, 10.0)
    return dict(q=q, mass=1.0, sigmas=np.array(SIGMAS_CONFIG2), f0=bimodal(rng, q),
                sources=two_sources(q))


def batch_bimodal(rng, q, batch: int) -> np.ndarray:
    """[batch][n] bimodal f with random centres c1 ~ logU[0.02, 0.2],
    c2 ~ logU[0.5, 5], widths U[0.3, 0.5], amplitudes U[0.1, 1]."""
    out = np.empty((batch, q.size))
    for b in range(batch):
        c1 = np.exp(rng.uniform(np.log(0.02), np.log(0.2)))
        c2 = np.exp(rng.uniform(np.log(0.5), np.log(5.0)))
        w = rng.uniform(0.3, 0.5, size=2)
        a = rng.uniform(0.1, 1.0, size=2)
        out[b] = lognormal_bumps(q, (c1, c2), w, a)
    return out


def config3(seed: int = 3, batch: int = 512, n: int = 192):
    """B distributions sharing one N = 192 kernel, q in [1e-3, 1e2]."""
    rng = np.random.default_rng(seed)
    q = log_grid(n, 1e-3, 1e2)
    return dict(q=q, mass=1.0, f=batch_bimodal(rng, q, batch),
                sigma=np.ones(batch))


def config4(seed: int = 4, instances: int = 1024, sizes=(64, 96, 128, 192, 256)):
    """Uneven batch: N uniform over sizes, sigma log-uniform over 3 decades."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.array(sizes), size=instances)
    sig = np.exp(rng.uniform(np.log(1e-3), np.log(1.0), size=instances))
    grids = {int(n): log_grid(int(n), 1e-3, 1e2) for n in sizes}
    f = [batch_bimodal(rng, grids[int(n)], 1)[0] for n in ns]
    return dict(ns=ns, sigma=sig, grids=grids, f=f, mass=1.0)


def config5(seed: int = 5, requests: int = 2000, rate_hz: float = 200.0,
            n_min: int = 64, n_max: int = 384):
    """Poisson arrival stream of full solves: arrival times, N ~ U{n_min..n_max},
    sigma ~ logU[1e-2, 10] (3 decades), random initial bumps and source bumps."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=requests)
    arrivals = np.cumsum(gaps)
    reqs = []
    for r in range(requests):
        n = int(rng.integers(n_min, n_max + 1))
        q = log_grid(n, 1e-3, 1e2)
        sigma = float(np.exp(rng.uniform(np.log(1e-2), np.log(10.0))))
        f0 = batch_bimodal(rng, q, 1)[0]
        c = np.exp(rng.uniform(np.log(0.02), np.log(5.0), size=2))
        w = rng.uniform(0.3, 0.5, size=2)
        src = dict(shape=np.stack([lognormal_bumps(q, (c[0],), (w[0],), (1.0,)),
                                   lognormal_bumps(q, (c[1],), (w[1],), (1.0,))]),
                   rate=rng.uniform(0.01, 0.1, size=2), tau=np.array([1.0, 1.0]),
                   t_on=np.array([0.0, 3.0]))
        reqs.append(dict(arrival=float(arrivals[r]), n=n, q=q, sigma=sigma, f0=f0,
                         sources=src, mass=1.0))
    return reqs


def random_grid(rng, n: int, q_min: float = 1e-3, q_max: float = 1e2) -> np.ndarray:
    """Non-uniform ascending grid (sorted log-uniform draws), for edge cases."""
    return np.sort(np.exp(rng.uniform(np.log(q_min), np.log(q_max), size=n)))
