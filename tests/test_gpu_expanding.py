"""Expanding universe (Sec. 4, eq. numerical_evolution_loga): kx_solve_expanding
against the oracle's integration in u = ln a -- the RK4 source regime, the
switch at Gamma_2->2 / H > eps_switch (Sec. 4.2) and the adaptive Heun regime
with the kernel rebuilt at every scale factor.  FP64 path within 1e-10 (the
step controller amplifies rounding in h, as in the static-box test), FP32
path within the mixed-precision bound, comoving number conserved."""
import numpy as np
import pytest

import kx_inputs as ki
import oracle

pytestmark = pytest.mark.gpu

RD = dict(hu=[0.0, 1.0], ln_H=[0.0, -2.0])   # radiation domination: H = e^{-2u}


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2607_00755_b300 as kx
    from paper_2607_00755_b300 import build
    build.build()
    ctx = kx.Context(0)
    yield kx, ctx, torch
    ctx.close()


def case(n=24, seed=1, rate=2e-2, tau=0.3):
    q = ki.log_grid(n, 1e-3, 10.0)
    f0 = 1e-3 * ki.bimodal(np.random.default_rng(seed), q)
    src = dict(shape=ki.lognormal_bumps(q, (0.5,), (0.3,), (1.0,))[None], rate=np.array([rate]),
               tau=np.array([tau]), t_on=np.array([0.0]))
    return q, f0, src


def test_expanding_fp64_matches_oracle(env):
    """Sources, RK4 until Gamma/H > 1e-2, then Heun to u = 0.5: the same RK4
    step count and switch point, the same Heun step and reject counts, and f
    within 1e-10 of the oracle."""
    kx, ctx, torch = env
    q, f0, src = case()
    par = dict(u0=0.0, u_end=0.5, du_rk4=0.02, check_every=2, eps_switch=1e-2)
    fo, ro = oracle.solve_expanding(q, f0, oracle.M2_from_sigma(1.0, 40.0), hu=RD["hu"],
                                    hlnH=RD["ln_H"], sources=src, h0=1e-3, rtol=1e-6, atol=1e-15, **par)
    assert ro["status"] == 0 and 0.0 < ro["u_switch"] < 0.5 and ro["steps"] > 100
    fd = torch.as_tensor(f0, device="cuda")
    r = ctx.solve_expanding(q, fd, 40.0, RD["hu"], RD["ln_H"], sources=src, precision=kx.FP64,
                            h0=1e-3, rtol=1e-6, atol=1e-15, **par)
    assert r["status"] == 0 and r["u"] == 0.5
    assert r["rk4_steps"] == ro["rk4_steps"] and r["u_switch"] == ro["u_switch"]
    assert abs(r["gamma_over_H"] / ro["gamma_over_H"] - 1) < 1e-12
    assert r["steps"] == ro["steps"] and r["rejects"] == ro["rejects"]
    f = fd.cpu().numpy()
    assert np.max(np.abs(f - fo)) / np.max(fo) <= 1e-10


def test_expanding_fp32_matches_oracle_and_conserves(env):
    """The FP32 path (uncompacted FP32 tables rebuilt at each a): collisions
    from u0 (eps_switch = 0, no sources) to u = 0.3 within the mixed bound of
    the oracle, comoving number conserved to 1e-7; and with sources the same
    switch point as the oracle."""
    kx, ctx, torch = env
    q, f0, src = case(seed=2)
    hc = oracle.grid(q)["h"]
    par = dict(u0=0.0, u_end=0.3, eps_switch=0.0)
    fo, ro = oracle.solve_expanding(q, f0, oracle.M2_from_sigma(1.0, 40.0), hu=RD["hu"],
                                    hlnH=RD["ln_H"], h0=1e-3, rtol=1e-6, atol=1e-15, **par)
    fd = torch.as_tensor(f0, device="cuda")
    r = ctx.solve_expanding(q, fd, 40.0, RD["hu"], RD["ln_H"], precision=kx.FP32, h0=1e-3,
                            rtol=1e-6, atol=1e-15, **par)
    f = fd.cpu().numpy()
    assert r["status"] == 0 and r["u"] == 0.3 and r["u_switch"] == 0.0
    assert abs(r["steps"] - ro["steps"]) <= 2
    assert np.max(np.abs(f - fo)) / np.max(fo) <= 1e-5
    assert abs(np.sum(hc * f) / np.sum(hc * f0) - 1) < 1e-7
    q, f0, src = case(seed=1)
    par = dict(u0=0.0, u_end=0.3, du_rk4=0.02, check_every=2, eps_switch=1e-2)
    fo, ro = oracle.solve_expanding(q, f0, oracle.M2_from_sigma(1.0, 40.0), hu=RD["hu"],
                                    hlnH=RD["ln_H"], sources=src, h0=1e-3, **par)
    fd = torch.as_tensor(f0, device="cuda")
    r = ctx.solve_expanding(q, fd, 40.0, RD["hu"], RD["ln_H"], sources=src, precision=kx.FP32,
                            h0=1e-3, **par)
    assert 0.0 < ro["u_switch"] < 0.3
    assert r["rk4_steps"] == ro["rk4_steps"] and r["u_switch"] == ro["u_switch"]
    assert np.max(np.abs(fd.cpu().numpy() - fo)) / np.max(fo) <= 1e-5


def test_expanding_source_only_regime(env):
    """No switch (eps_switch = inf): RK4 on the sources alone, as the oracle,
    to rounding."""
    kx, ctx, torch = env
    q, f0, src = case(seed=3)
    par = dict(u0=0.0, u_end=1.0, du_rk4=0.05, check_every=4, eps_switch=np.inf)
    fo, ro = oracle.solve_expanding(q, f0, 1.0, hu=RD["hu"], hlnH=RD["ln_H"], sources=src, **par)
    for prec in (kx.FP64, kx.FP32):
        fd = torch.as_tensor(f0, device="cuda")
        r = ctx.solve_expanding(q, fd, 1.0, RD["hu"], RD["ln_H"], sources=src, precision=prec, **par)
        assert np.isnan(r["u_switch"]) and r["rk4_steps"] == ro["rk4_steps"] == 20 and r["steps"] == 0
        assert np.max(np.abs(fd.cpu().numpy() - fo)) / np.max(fo) <= 1e-13


def test_expanding_rejects_unsupported_options(env):
    kx, ctx, torch = env
    q, f0, _ = case(n=8)
    fd = torch.as_tensor(f0, device="cuda")
    with pytest.raises(kx.KxError) as ei:
        ctx.solve_expanding(q, fd, 1.0, RD["hu"], RD["ln_H"], 0.0, 0.1, precision=kx.SPLIT_TF32)
    assert ei.value.code == kx.ENOTSUP
    with pytest.raises(kx.KxError) as ei:
        ctx.solve_expanding(q, fd, 1.0, [0.0, 0.0], [0.0, -1.0], 0.0, 0.1)
    assert ei.value.code == kx.EINVAL
