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


def test_diagnostic_rates_and_attempt_profile(env):
    """kx_measure_peaks (FP64 and ex2 throughput), kx_measure_mma_rate (tcgen05
    issue rate) and kx_profile_attempts (per-kernel times of real attempts):
    plausible positive figures, TF32 and BF16 MMAs of one shape take the same
    cycles (the same operand bytes), the profiled attempts advance f as a solve
    does, and bad arguments are refused."""
    kx, ctx, torch = env
    fp64, ex2 = ctx.measure_peaks()
    assert 1e11 < fp64 < 1e14 and 1e12 < ex2 < 1e14
    f32c, c32 = ctx.measure_mma_rate(0, 128)
    f16c, c16 = ctx.measure_mma_rate(1, 128)
    assert 500.0 < f32c < 50000.0 and abs(f16c / f32c - 2.0) < 0.2 and abs(c16 / c32 - 1.0) < 0.1
    with pytest.raises(kx.KxError):
        ctx.measure_mma_rate(0, 100)
    q = ki.log_grid(32, 1e-3, 10.0)
    f0 = ki.batch_bimodal(np.random.default_rng(9), q, 2)
    k = ctx.build_kernel(q, precision=kx.FP32)
    fd = torch.as_tensor(f0, device="cuda")
    prof = ctx.profile_attempts(k, fd, [1.0, 2.0], attempts=20, t_end=1.0, h0=1e-3)
    assert all(0.0 < v < 1e5 for v in prof.values()) and len(prof) == 4
    assert not np.array_equal(fd.cpu().numpy(), f0)
    with pytest.raises(kx.KxError):
        ctx.profile_attempts(k, fd, [1.0, 2.0], attempts=0, t_end=1.0, h0=1e-3)
    k.release()
