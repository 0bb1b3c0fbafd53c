"""Serving (continuous batching): each request's result is bit-identical to
solving it alone with kx_solve, kernels are shared between requests on the same
grid, requests join while others run, and admission respects the budget."""
import time

import numpy as np
import pytest

import kx_inputs as ki
import oracle

pytestmark = pytest.mark.gpu

PAR = dict(rtol=1e-6, atol=1e-12, l1_tol=1e-3, check_every=5, max_attempts=200000)


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


def requests(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        n = int(rng.choice([24, 32, 40]))
        q = ki.log_grid(n, 1e-3, 10.0)
        f0 = ki.batch_bimodal(rng, q, 1)[0]
        src = ki.two_sources(q, t_scale=0.2, rate=0.02) if r % 2 else None
        out.append(dict(q=q, f0=f0, sigma=float(np.exp(rng.uniform(np.log(0.5), np.log(4.0)))),
                        src=src, t_end=float(rng.uniform(2.0, 8.0))))
    return out


@pytest.mark.parametrize("precision", [1, 2])
def test_served_results_equal_solving_alone(env, precision):
    kx, ctx, torch = env
    reqs = requests(51, 10)
    srv = kx.Server(ctx, slots_per_group=4, attempts_per_tick=4, precision=precision, **PAR)
    tickets = []
    for i, r in enumerate(reqs):
        tickets.append(srv.submit(r["q"], r["f0"], r["sigma"], sources=r["src"], t_end=r["t_end"],
                                  h0=1e-3))
        if i == 4:
            time.sleep(0.05)   # later requests arrive while earlier ones run
    served = []
    for t, r in zip(tickets, reqs):
        rc, f, res = srv.poll(t, r["q"].size, timeout=120.0)
        assert rc == kx.OK, (rc, res)
        served.append((f, res))
    st = srv.stats()
    srv.stop()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    sizes = len({r["q"].size for r in reqs})
    assert st["kernels_built"] == sizes and st["kernel_cache_hits"] == len(reqs) - sizes
    for (f, res), r in zip(served, reqs):
        k = ctx.build_kernel(r["q"], precision=precision)
        fd = torch.as_tensor(r["f0"][None], device="cuda")
        ra = ctx.solve(k, fd, r["sigma"], sources=r["src"], t_end=r["t_end"], h0=1e-3, **PAR)[0]
        np.testing.assert_array_equal(f, fd.cpu().numpy()[0])
        assert res["steps"] == ra["steps"] and res["rejects"] == ra["rejects"]
        assert res["latency_s"] > 0
        k.release()


def test_served_fp32_solve_close_to_oracle(env):
    kx, ctx, torch = env
    q = ki.log_grid(32, 1e-3, 10.0)
    f0 = ki.bimodal(np.random.default_rng(52), q)
    srv = kx.Server(ctx, slots_per_group=2, precision=kx.FP32, **PAR)
    t = srv.submit(q, f0, 2.0, t_end=1e4, h0=1e-3)
    rc, f, res = srv.poll(t, 32, timeout=120.0)
    srv.stop()
    assert rc == kx.OK and res["converged"] == 1
    W = oracle.kernel_tensor(q)
    fo, ro = oracle.solve(q, W, f0, oracle.M2_from_sigma(1.0, 2.0), t_end=1e4, h0=1e-3, **PAR)
    g = oracle.grid(q)
    assert np.sum(g["h"] * np.abs(f - fo)) / np.sum(g["h"] * fo) < 5e-3
    assert abs(np.sum(g["h"] * f) / np.sum(g["h"] * f0) - 1) < 1e-7


def test_admission_budget(env):
    kx, ctx, torch = env
    srv = kx.Server(ctx, budget_bytes=64 << 20, slots_per_group=2, precision=kx.FP32, **PAR)
    q = ki.log_grid(384, 1e-3, 1e2)
    with pytest.raises(kx.KxError) as ei:
        srv.submit(q, ki.bimodal(np.random.default_rng(1), q), 1.0, t_end=1.0)
    assert ei.value.code == kx.EADMIT
    q = ki.log_grid(24, 1e-3, 10.0)
    t = srv.submit(q, ki.bimodal(np.random.default_rng(2), q), 1.0, t_end=0.5)
    rc, f, res = srv.poll(t, 24, timeout=60.0)
    srv.stop()
    assert rc == kx.OK


def test_served_results_with_shared_contraction_grids_equal_solving_alone(env):
    """Twelve requests on twelve different grids, submitted at once: more than
    eight groups have work, so their FP32 contractions run with the shared
    (half) grid; each result is still bit-identical to kx_solve alone (whole
    GPU per launch).  A bad grid share is refused."""
    kx, ctx, torch = env
    with pytest.raises(kx.KxError):
        kx.Server(ctx, precision=kx.FP32, grid_div=17, **PAR)
    rng = np.random.default_rng(77)
    reqs = []
    for n in range(24, 48, 2):
        q = ki.log_grid(n, 1e-3, 10.0)
        reqs.append(dict(q=q, f0=ki.batch_bimodal(rng, q, 1)[0], sigma=float(rng.uniform(0.5, 2.0))))
    srv = kx.Server(ctx, slots_per_group=2, attempts_per_tick=4, precision=kx.FP32, **PAR)
    tickets = [srv.submit(r["q"], r["f0"], r["sigma"], t_end=20.0, h0=1e-3) for r in reqs]
    served = []
    for t, r in zip(tickets, reqs):
        rc, f, res = srv.poll(t, r["q"].size, timeout=300.0)
        assert rc == kx.OK, (rc, res)
        served.append((f, res))
    st = srv.stats()
    srv.stop()
    # the shared-grid graphs did run (more than eight groups had work at once)
    assert st["ticks_shared"] > 0, st
    for (f, res), r in zip(served, reqs):
        k = ctx.build_kernel(r["q"], precision=kx.FP32)
        fd = torch.as_tensor(r["f0"][None], device="cuda")
        ra = ctx.solve(k, fd, r["sigma"], t_end=20.0, h0=1e-3, **PAR)[0]
        np.testing.assert_array_equal(f, fd.cpu().numpy()[0])
        assert res["steps"] == ra["steps"] and res["rejects"] == ra["rejects"]
        k.release()
