"""kx_collision_noalloc: the collision term for callers that cannot allocate
GPU memory during the call (allocator or memory-pool callbacks, hosts that
reserved all device memory up front).  It must give kx_collision's results
while drawing its scratch from the library's fixed 8 MiB device array.

This file is collected last on purpose: a failure here does not hide the
other tests of a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

import kx_inputs as ki

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-5}


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    import paper_2607_00755_b300 as kx
    from paper_2607_00755_b300 import build
    build.build()
    ctx = kx.Context(0)
    yield kx, ctx, torch
    ctx.close()


def call_noalloc(kx, ctx, kernel, f, sigma, C, project):
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    return ctx.lib.kx_collision_noalloc(ctx.h, kernel.h, f.shape[0],
                                        ctypes.c_void_p(sig.ctypes.data),
                                        ctypes.c_void_p(f.data_ptr()),
                                        ctypes.c_void_p(C.data_ptr()), int(project))


@pytest.mark.parametrize("precision,stats", [(0, 0), (1, 0), (1, 1), (2, 0)])
def test_noalloc_matches_kx_collision_twice(env, precision, stats):
    """Two calls in a row (different inputs, so stale scratch from the first
    would show) give kx_collision's results bit for bit: the two entry points
    run the same kernels on the same inputs, only the scratch differs.  Paths:
    plain FP64, FP32 streaming (also with the Bose-Einstein factor) and the
    split-TF32 tensor-core path."""
    kx, ctx, torch = env
    n = 96
    q = ki.log_grid(n, 1e-3, 10.0)
    k = ctx.build_kernel(q, precision=precision, stats=stats)
    rng = np.random.default_rng(41)
    for call in range(2):
        B = 3 + call
        f = torch.as_tensor(ki.batch_bimodal(rng, q, B), device="cuda")
        sig = rng.uniform(0.5, 5.0, size=B)
        for project in (0, 1):
            ref, _ = ctx.collision(k, f, sig, project=bool(project))
            C = torch.full_like(f, float("nan"))
            rc = call_noalloc(kx, ctx, k, f, sig, C, project)
            assert rc == 0, ctx.lib.kx_last_error(ctx.h)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(C.cpu().numpy(), ref.cpu().numpy())
    k.release()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_noalloc_matches_oracle(env, precision):
    """The allocation-free call against the FP64 oracle (projected C of a
    bimodal batch) at the parity tolerance of each path."""
    import oracle
    kx, ctx, torch = env
    n = 40
    q = ki.log_grid(n, 1e-3, 10.0)
    f = ki.batch_bimodal(np.random.default_rng(43), q, 3)
    sig = np.array([0.7, 1.0, 3.0])
    k = ctx.build_kernel(q, precision=precision)
    C = torch.empty((3, n), dtype=torch.float64, device="cuda")
    assert call_noalloc(kx, ctx, k, torch.as_tensor(f, device="cuda"), sig, C, 1) == 0
    torch.cuda.synchronize()
    C = C.cpu().numpy()
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q)
    for b in range(3):
        Co = oracle.collision_tensor(q, W, f[b]) * oracle.M2_from_sigma(1.0, sig[b])
        Co, _ = oracle.project(g["E"], g["h"], f[b], Co)
        assert np.max(np.abs(C[b] - Co)) / np.max(np.abs(Co)) <= TOL[precision], b
    k.release()


def test_noalloc_rejects_requests_above_its_fixed_scratch(env):
    kx, ctx, torch = env
    q = ki.log_grid(512, 1e-3, 1e2)
    # the FP32 path fits 64 instances at the largest grid; the FP64 path's
    # per-chunk partials (about 0.55 MB per instance at n = 512) do not
    k = ctx.build_kernel(q, precision=kx.FP32)
    f = torch.zeros((64, 512), dtype=torch.float64, device="cuda")
    assert call_noalloc(kx, ctx, k, f, np.ones(64), torch.empty_like(f), 1) == kx.OK
    k.release()
    k = ctx.build_kernel(q, precision=kx.FP64)
    f = torch.zeros((20, 512), dtype=torch.float64, device="cuda")
    C = torch.empty_like(f)
    rc = call_noalloc(kx, ctx, k, f, np.ones(20), C, 1)
    assert rc == kx.EINVAL
    assert b"8 MiB" in ctx.lib.kx_last_error(ctx.h)
    f = torch.zeros((65, 8), dtype=torch.float64, device="cuda")
    k8 = ctx.build_kernel(ki.log_grid(8, 1e-3, 10.0), precision=kx.FP32)
    rc = call_noalloc(kx, ctx, k8, f, np.ones(65), torch.empty_like(f), 1)
    assert rc == kx.EINVAL
    k.release()
    k8.release()
