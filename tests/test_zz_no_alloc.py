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

TOL = {0: 1e-12, 1: 1e-5}


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


@pytest.mark.parametrize("precision,stats", [(0, 0), (1, 0), (1, 1)])
def test_noalloc_matches_kx_collision_twice(env, precision, stats):
    """Two calls in a row (different inputs, so stale scratch from the first
    would show) agree with kx_collision within the parity tolerance (also with
    the Bose-Einstein factor on the FP32 path)."""
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
            C = torch.empty_like(f)
            rc = call_noalloc(kx, ctx, k, f, sig, C, project)
            assert rc == 0, ctx.lib.kx_last_error(ctx.h)
            torch.cuda.synchronize()
            r, c = ref.cpu().numpy(), C.cpu().numpy()
            for b in range(B):
                err = np.max(np.abs(c[b] - r[b])) / np.max(np.abs(r[b]))
                assert err <= TOL[precision], (call, project, b, err)
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
