"""GPU: the timing entry points (kx_time_contraction, kx_time_contractions)
run the contraction through the C ABI and leave the results they time
unchanged; argument checks return KX_EINVAL."""
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


@pytest.mark.parametrize("precision", ["FP32", "FP64", "SPLIT_TF32"])
def test_rotating_timing_runs_and_leaves_results(env, precision):
    kx, ctx, torch = env
    p = getattr(kx, precision)
    q = ki.log_grid(40, 1e-3, 1e2)
    f = torch.as_tensor(ki.batch_bimodal(np.random.default_rng(5), q, 3), device="cuda")
    ks = [ctx.build_kernel(q, precision=p) for _ in range(3)]
    sig = np.ones(3)
    before, _ = ctx.collision(ks[0], f, sig)
    ms = ctx.time_contractions(ks, f, iters=4)
    ms_pdl = ctx.time_contractions(ks, f, iters=4, pdl=True)
    one = ctx.time_contraction(ks[1], f, iters=3, flush_bytes=1 << 20)
    assert 0.0 < ms < 1e3 and 0.0 < ms_pdl < 1e3 and 0.0 < one < 1e3
    after, _ = ctx.collision(ks[2], f, sig)
    np.testing.assert_array_equal(before.cpu().numpy(), after.cpu().numpy())
    for k in ks:
        k.release()


def test_rotating_timing_rejects_mixed_sizes(env):
    kx, ctx, torch = env
    k1 = ctx.build_kernel(ki.log_grid(24, 1e-3, 10.0), precision=kx.FP32)
    k2 = ctx.build_kernel(ki.log_grid(32, 1e-3, 10.0), precision=kx.FP32)
    f = torch.zeros((1, 24), dtype=torch.float64, device="cuda") + 0.5
    with pytest.raises(kx.KxError) as ei:
        ctx.time_contractions([k1, k2], f)
    assert ei.value.code == kx.EINVAL
    with pytest.raises(kx.KxError):
        ctx.time_contractions([], f)
    k1.release()
    k2.release()


@pytest.mark.parametrize("precision,stats", [("FP32", 0), ("FP64", 0), ("SPLIT_TF32", 0), ("FP32", 1)])
def test_time_collision_output_is_the_collision(env, precision, stats):
    """kx_time_collision replays the evaluation kx_collision makes: the C it
    leaves is bit-identical to kx_collision's, with and without projection."""
    kx, ctx, torch = env
    q = ki.log_grid(36, 1e-3, 1e2)
    f = torch.as_tensor(0.8 * ki.batch_bimodal(np.random.default_rng(6), q, 2), device="cuda")
    sig = np.array([1.0, 2.5])
    k = ctx.build_kernel(q, precision=getattr(kx, precision), stats=stats)
    for project in (False, True):
        ms, C = ctx.time_collision(k, f, sig, project=project, iters=3)
        ref, _ = ctx.collision(k, f, sig, project=project)
        assert 0.0 < ms < 1e3
        np.testing.assert_array_equal(C.cpu().numpy(), ref.cpu().numpy())
    k.release()
