"""Failure paths through host-side fault injection (KX_FAULT): allocation
failures, admission refusal, a non-finite staged input and an expired host
wait each return their error code, and the context keeps working afterwards.
No injected failure touches the GPU (no kernel faults or traps); the one
device wait made to expire is a self-check kernel's wait on an mbarrier that
nothing arrives on, with a limit of about 1 ms and no copy in flight."""
import time

import numpy as np
import pytest

import kx_inputs as ki

pytestmark = pytest.mark.gpu


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


def grid_and_f(n=32, B=2, seed=71):
    q = ki.log_grid(n, 1e-3, 10.0)
    return q, ki.batch_bimodal(np.random.default_rng(seed), q, B)


def test_injected_allocation_failure(env, monkeypatch):
    kx, ctx, torch = env
    q, f = grid_and_f()
    monkeypatch.setenv("KX_FAULT", "alloc")
    with pytest.raises(kx.KxError) as ei:
        ctx.build_kernel(q, precision=kx.FP32)
    assert ei.value.code == kx.ENOMEM
    monkeypatch.delenv("KX_FAULT")
    k = ctx.build_kernel(q, precision=kx.FP32)
    ref, _ = ctx.collision(k, torch.as_tensor(f, device="cuda"), 1.0)
    # a larger batch needs a larger arena: that allocation fails, the old one stays usable
    big = torch.as_tensor(np.tile(f, (1024, 1)), device="cuda")   # views above the 1 MiB first arena
    monkeypatch.setenv("KX_FAULT", "alloc")
    with pytest.raises(kx.KxError) as ei:
        ctx.collision(k, big, 1.0)
    assert ei.value.code == kx.ENOMEM
    again, _ = ctx.collision(k, torch.as_tensor(f, device="cuda"), 1.0)
    np.testing.assert_array_equal(again.cpu().numpy(), ref.cpu().numpy())
    monkeypatch.delenv("KX_FAULT")
    C, _ = ctx.collision(k, big, 1.0)
    np.testing.assert_array_equal(C.cpu().numpy()[:2], ref.cpu().numpy())
    k.release()


@pytest.mark.parametrize("precision", ["FP64", "FP32", "SPLIT_TF32"])
def test_injected_nan_input(env, monkeypatch, precision):
    kx, ctx, torch = env
    q, f = grid_and_f()
    k = ctx.build_kernel(q, precision=getattr(kx, precision))
    monkeypatch.setenv("KX_FAULT", "nan")
    C, d = ctx.collision_host(k, f, np.array([1.0, 2.0]), diag=True)
    assert d[0]["status"] == kx.ENONFINITE
    fh, res = ctx.solve_host(k, f, np.array([1.0, 2.0]), t_end=0.5, h0=1e-3)
    assert res[0]["status"] == kx.ENONFINITE and res[1]["status"] == 0
    monkeypatch.delenv("KX_FAULT")
    C2, d2 = ctx.collision_host(k, f, np.array([1.0, 2.0]), diag=True)
    assert all(x["status"] == 0 for x in d2) and np.all(np.isfinite(C2))
    np.testing.assert_array_equal(C2[1], C[1])
    k.release()


def test_injected_host_wait_timeout(env, monkeypatch):
    kx, ctx, torch = env
    q, f = grid_and_f(B=1)
    k = ctx.build_kernel(q, precision=kx.FP32)
    par = dict(t_end=5.0, h0=1e-3, rtol=1e-6, atol=1e-12)
    fd = torch.as_tensor(f, device="cuda")
    ref = ctx.solve(k, fd, 1.0, **par)[0]
    monkeypatch.setenv("KX_FAULT", "timeout")
    with pytest.raises(kx.KxError) as ei:
        ctx.solve(k, torch.as_tensor(f, device="cuda"), 1.0, **par)
    assert ei.value.code == kx.ETIMEOUT
    monkeypatch.delenv("KX_FAULT")
    fd2 = torch.as_tensor(f, device="cuda")
    res = ctx.solve(k, fd2, 1.0, **par)[0]
    assert res["status"] == 0 and res["steps"] == ref["steps"]
    np.testing.assert_array_equal(fd2.cpu().numpy(), fd.cpu().numpy())
    k.release()


def test_injected_admission_refusal(env, monkeypatch):
    kx, ctx, torch = env
    q, f = grid_and_f(B=1)
    srv = kx.Server(ctx, slots_per_group=2, precision=kx.FP32, rtol=1e-6, atol=1e-12,
                    l1_tol=0.0, max_attempts=100000)
    monkeypatch.setenv("KX_FAULT", "admit")
    with pytest.raises(kx.KxError) as ei:
        srv.submit(q, f[0], 1.0, t_end=0.5)
    assert ei.value.code == kx.EADMIT
    monkeypatch.delenv("KX_FAULT")
    t = srv.submit(q, f[0], 1.0, t_end=0.5)
    deadline = time.time() + 120
    while True:
        rc, fo, res = srv.poll(t, q.size, timeout=1.0)
        if rc != kx.PENDING or time.time() > deadline:
            break
    assert rc == kx.OK and res["status"] == 0 and np.all(np.isfinite(fo))
    srv.stop()


@pytest.mark.parametrize("precision", ["FP64", "FP32", "SPLIT_TF32"])
def test_expired_device_wait_is_reported(env, monkeypatch, precision):
    """The flag a contraction sets when one of its bounded device waits expires
    (KX_FAULT=deverr sets it from the host; no wait is made to expire here):
    kx_collision with diagnostics returns KX_ETIMEOUT and C is NaN, a solve
    stops every instance with KX_ETIMEOUT, and the next calls are clean."""
    kx, ctx, torch = env
    q, f = grid_and_f()
    k = ctx.build_kernel(q, precision=getattr(kx, precision))
    fd = torch.as_tensor(f, device="cuda")
    ref, _ = ctx.collision(k, fd, 1.0)
    monkeypatch.setenv("KX_FAULT", "deverr")
    with pytest.raises(kx.KxError) as ei:
        ctx.collision(k, fd, 1.0, diag=True)
    assert ei.value.code == kx.ETIMEOUT
    C, _ = ctx.collision(k, fd, 1.0)
    assert np.all(np.isnan(C.cpu().numpy()))
    with pytest.raises(kx.KxError) as ei:
        ctx.solve(k, torch.as_tensor(f, device="cuda"), 1.0, t_end=0.5, h0=1e-3)
    assert ei.value.code == kx.ETIMEOUT
    monkeypatch.delenv("KX_FAULT")
    C2, d2 = ctx.collision(k, fd, 1.0, diag=True)
    assert all(x["status"] == 0 for x in d2)
    np.testing.assert_array_equal(C2.cpu().numpy(), ref.cpu().numpy())
    res = ctx.solve(k, torch.as_tensor(f, device="cuda"), 1.0, t_end=0.5, h0=1e-3)
    assert all(r["status"] == 0 for r in res)
    k.release()


def test_bounded_device_wait_gives_up(env):
    """A device wait on an mbarrier that nothing arrives on gives up after its
    cycle limit (about 1 ms here) and the kernel returns: the context stays
    usable (a collision afterwards is exact)."""
    kx, ctx, torch = env
    t0 = time.time()
    assert ctx.wait_check(2_000_000) == 1
    assert time.time() - t0 < 30.0
    q, f = grid_and_f()
    k = ctx.build_kernel(q, precision=kx.FP32)
    C, d = ctx.collision(k, torch.as_tensor(f, device="cuda"), 1.0, diag=True)
    assert all(x["status"] == 0 for x in d) and np.all(np.isfinite(C.cpu().numpy()))
    k.release()
