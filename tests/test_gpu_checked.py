"""The bounds-checked build (libkx_check.so, compiled with -DKX_CHECK).

Its contraction and loss kernels pass their table, bracket, task, vector and
slot indices through a range check that records a failure (first site, index,
count) and substitutes index 0, so that no access leaves its array.  These
tests run the small parity cases of every path through that build: the
results must equal the oracle within the paths' tolerances and no check may
fail.  The check itself is exercised with the one-thread probe kernel, which
addresses no memory with the index.
"""
import numpy as np
import pytest

import kx_inputs as ki
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2607_00755_b300 as kx
    from paper_2607_00755_b300 import build
    build.build(check=True)
    ctx = kx.Context(0, lib=kx.load_checked_library())
    yield kx, ctx, torch
    ctx.close()


def oracle_proj(q, f, sig):
    W = oracle.kernel_tensor(q)
    g = oracle.grid(q)
    out = []
    for b in range(f.shape[0]):
        C = oracle.collision_tensor(q, W, f[b]) * oracle.M2_from_sigma(1.0, sig[b])
        out.append(oracle.project(g["E"], g["h"], f[b], C)[0])
    return np.array(out)


def test_checked_build_probe(env):
    """In range the probe returns the index and records nothing; out of range
    it returns 0 and records the site, the index and one failure; the normal
    build reports itself unchecked."""
    kx, ctx, torch = env
    st = ctx.check_status(reset=True)
    assert st["checked"]
    assert ctx.check_probe(3, 10) == 3 and ctx.check_probe(0, 1) == 0
    assert ctx.check_status()["failures"] == 0
    assert ctx.check_probe(12, 10) == 0 and ctx.check_probe(-1, 10) == 0
    st = ctx.check_status(reset=True)
    assert st["failures"] == 2 and st["first_site"] == 99 and st["first_index"] == 12
    assert ctx.check_status()["failures"] == 0
    plain = kx.Context(0)
    assert not plain.check_status()["checked"]
    assert plain.check_probe(12, 10) == 12
    plain.close()


@pytest.mark.parametrize("N", [24, 100])
def test_checked_build_parity_no_failed_check(env, N):
    """FP64, FP32 (every streaming variant) and split TF32 (exact and
    Chebyshev loss) collision terms of a small batch through the checked
    build: within the paths' tolerances of the oracle, and no failed check."""
    kx, ctx, torch = env
    q = ki.log_grid(N, 1e-3, 10.0)
    B = 4
    f = ki.batch_bimodal(np.random.default_rng(40 + N), q, B)
    sig = np.array([0.5, 1.0, 2.0, 4.0])
    ref = oracle_proj(q, f, sig)
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    ctx.check_status(reset=True)
    fd = torch.as_tensor(f, device="cuda")
    cases = [(kx.FP64, {}, None, 1e-12), (kx.SPLIT_TF32, {}, None, 1e-5),
             (kx.SPLIT_TF32, {"loss_terms": 16}, None, 1e-5)]
    cases += [(kx.FP32, {}, var, 1e-5) for var in (0, 1, 3, 4)]
    for precision, opts, var, tol in cases:
        k = ctx.build_kernel(q, precision=precision, **opts)
        if var is not None:
            ctx.set_stream_variant(N, B, var)
        C, _ = ctx.collision(k, fd, sig)
        if var is not None:
            ctx.set_stream_variant(N, B, -1)
        err = np.max(np.abs(C.cpu().numpy() - ref) / scale)
        assert err <= tol, (precision, opts, var, err)
        k.release()
    st = ctx.check_status(reset=True)
    assert st["failures"] == 0, st


def test_checked_build_solve_no_failed_check(env):
    """A short adaptive solve with sources on the FP32 path (contractions,
    stage kernels, tables) through the checked build: the same steps as the
    normal build, results equal to it bit for bit, and no failed check."""
    kx, ctx, torch = env
    c = ki.config2()
    q, f0 = c["q"], c["f0"]
    par = dict(t_end=5.0, h0=1e-3, rtol=1e-6, atol=1e-12 * float(f0.max()), l1_tol=0.0)
    ctx.check_status(reset=True)
    k = ctx.build_kernel(q, precision=kx.FP32)
    fa = torch.as_tensor(np.tile(f0, (2, 1)), device="cuda")
    ra = ctx.solve(k, fa, c["sigmas"][:2], sources=c["sources"], **par)
    k.release()
    plain = kx.Context(0)
    kp = plain.build_kernel(q, precision=kx.FP32)
    fb = torch.as_tensor(np.tile(f0, (2, 1)), device="cuda")
    rb = plain.solve(kp, fb, c["sigmas"][:2], sources=c["sources"], **par)
    kp.release()
    plain.close()
    for x, y in zip(ra, rb):
        assert x["status"] == 0 and x["steps"] == y["steps"] and x["rejects"] == y["rejects"]
    np.testing.assert_array_equal(fa.cpu().numpy(), fb.cpu().numpy())
    assert ctx.check_status(reset=True)["failures"] == 0


@pytest.mark.parametrize("loss_terms", [0, 16])
def test_checked_build_grouped_solve_no_failed_check(env, loss_terms):
    """A short grouped solve of three grids on the split path through the
    checked build (the gain GEMM's pair lists, the grids' exact loss kernels
    forked onto side streams, or the Chebyshev loss GEMM, the grouped stage):
    results bit-identical to the normal build and no failed check."""
    kx, ctx, torch = env
    rng = np.random.default_rng(120 + loss_terms)
    sizes, Bs = (24, 40, 100), (130, 3, 5)
    grids = [ki.log_grid(n, 1e-3, 1e2) for n in sizes]
    f0 = [ki.batch_bimodal(rng, q, B) for q, B in zip(grids, Bs)]
    sig = [10.0 ** rng.uniform(-1, 0.5, B) for B in Bs]
    par = dict(t_end=0.2, h0=1e-3, rtol=1e-6, atol=1e-12, l1_tol=0.0)
    ctx.check_status(reset=True)
    out = []
    plain = kx.Context(0)
    for cx in (ctx, plain):
        ks = [cx.build_kernel(q, precision=kx.SPLIT_TF32, loss_terms=loss_terms) for q in grids]
        fd = [torch.as_tensor(f, device="cuda") for f in f0]
        res = cx.solve_grouped(ks, fd, sig, **par)
        out.append(([f.cpu().numpy() for f in fd], [[(x["status"], x["steps"], x["rejects"]) for x in r] for r in res]))
        for k in ks:
            k.release()
    plain.close()
    for g in range(len(sizes)):
        np.testing.assert_array_equal(out[0][0][g], out[1][0][g])
    assert out[0][1] == out[1][1]
    assert all(s == 0 for r in out[0][1] for s, _, _ in r)
    assert ctx.check_status(reset=True)["failures"] == 0


@pytest.mark.parametrize("N", [24, 100])
def test_checked_build_quantum_split_no_failed_check(env, N):
    """The split path with Bose-Einstein factors (the quantum loss kernel's
    element, bracket and pair indices checked) through the checked build:
    within the path's tolerance of the oracle and no failed check."""
    kx, ctx, torch = env
    q = ki.log_grid(N, 1e-2, 20.0)
    B = 4
    f = 0.8 * ki.batch_bimodal(np.random.default_rng(150 + N), q, B)
    sig = np.array([0.5, 1.0, 2.0, 4.0])
    W = oracle.kernel_tensor(q)
    g = oracle.grid(q)
    ctx.check_status(reset=True)
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32, stats=1)
    C, _ = ctx.collision(k, torch.as_tensor(f, device="cuda"), sig)
    C = C.cpu().numpy()
    k.release()
    for b in range(B):
        Co = oracle.collision_tensor_stats(q, W, f[b], 1) * oracle.M2_from_sigma(1.0, sig[b])
        Co, _ = oracle.project(g["E"], g["h"], f[b], Co)
        assert np.max(np.abs(C[b] - Co)) / np.max(np.abs(Co)) <= 1e-5
    assert ctx.check_status(reset=True)["failures"] == 0
