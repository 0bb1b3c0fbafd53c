"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (max-norm relative, max_i |dC_i| / max_i |C_i|): 1e-12 for the FP64
path, 1e-5 for the FP32 streaming path; conserved moments after an FP32-path
integration to 1e-7 relative.  Integer and index data (support, bracket j_L)
are compared bit-exactly.
"""
import numpy as np
import pytest

import kx_inputs as ki
import oracle

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def kx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2607_00755_b300 as kxm
    from paper_2607_00755_b300 import build
    build.build()
    return kxm


@pytest.fixture(scope="module")
def ctx(kx):
    c = kx.Context(0)
    yield c
    c.close()


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def sym_pairs(Wo):
    """Oracle W[i, n, m] -> symmetrised pair layout S[i, (n <= m)]."""
    N = Wo.shape[0]
    iu = np.triu_indices(N)
    S = Wo + Wo.transpose(0, 2, 1)
    d = np.arange(N)
    S[:, d, d] = Wo[:, d, d]
    return S[:, iu[0], iu[1]]


def oracle_C(q, f, sigma, project, W=None):
    """Oracle C (rows [B, n]) with |M|^2 = 64 pi m^2 sigma_b."""
    f = np.atleast_2d(f)
    g = oracle.grid(q)
    if W is None:
        W = oracle.kernel_tensor(q)
    out, diags = [], []
    for b in range(f.shape[0]):
        C = oracle.collision_tensor(q, W, f[b]) * oracle.M2_from_sigma(1.0, sigma[b])
        if project:
            C, d = oracle.project(g["E"], g["h"], f[b], C)
        else:
            _, d = oracle.project(g["E"], g["h"], f[b], C)
        out.append(C)
        diags.append(d)
    return np.array(out), diags


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# --------------------------------------------------------------- kernel ----
@pytest.mark.parametrize("N,measure,grid", [(24, 0, "log"), (40, 1, "log"), (37, 0, "random")])
def test_kernel_tensor_matches_oracle(ctx, kx, N, measure, grid):
    rng = np.random.default_rng(N)
    q = ki.log_grid(N, 1e-3, 10.0) if grid == "log" else ki.random_grid(rng, N)
    k = ctx.build_kernel(q, measure=measure, precision=kx.FP64)
    g = k.grid()
    go = oracle.grid(q)
    for key in ("p", "E", "dp", "dE", "h"):
        np.testing.assert_array_equal(g[key], go[key])
    So = sym_pairs(oracle.kernel_tensor(q, measure=measure))
    jLo, omo = oracle.bracket_tensor(q)
    iu = np.triu_indices(N)
    flips = 0
    for i in range(N):
        W, jl, om = k.row(i)
        sup = jLo[i][iu] >= 0
        np.testing.assert_array_equal(W[~sup], 0.0)
        np.testing.assert_array_equal(jl[sup], jLo[i][iu][sup])
        np.testing.assert_array_equal(om[sup], omo[i][iu][sup])
        d = np.abs(W - So[i])
        flips += int(np.sum(d > 1e-12 * np.abs(So[i]) + 1e-300))
        assert np.max(d) <= 1e-13 * np.max(np.abs(So))
    assert flips == 0, f"Theta/support flips: {flips}"
    info = k.info()
    assert info["nonzero_elements"] == int(np.count_nonzero(So))


@pytest.mark.parametrize("N", [24, 70])
def test_exact_angular_kernel_matches_oracle(ctx, kx, N):
    """n_mu = 0: the closed-form N_mu -> infinity kernel (triangle overlap)
    against the oracle's exact kernel, element by element; and C on both paths."""
    q = ki.log_grid(N, 1e-3, 10.0)
    k = ctx.build_kernel(q, n_mu=0, precision=kx.FP64)
    Wo = oracle.kernel_tensor(q, angular=oracle.ANG_EXACT)
    So = sym_pairs(Wo)
    for i in range(N):
        W, _, _ = k.row(i)
        assert np.max(np.abs(W - So[i])) <= 1e-13 * np.max(np.abs(So))
    f = ki.batch_bimodal(np.random.default_rng(31), q, 2)
    Co, _ = oracle_C(q, f, [1.0, 2.0], 1, Wo)
    for prec in (kx.FP64, kx.FP32):
        kp = ctx.build_kernel(q, n_mu=0, precision=prec)
        C, _ = ctx.collision(kp, dev(f), np.array([1.0, 2.0]))
        C = C.cpu().numpy()
        for b in range(2):
            assert relerr(C[b], Co[b]) <= TOL[prec]
        kp.release()
    # the exact kernel is the limit of the GL kernels (algebraic convergence)
    Wg = sym_pairs(oracle.kernel_tensor(q, n_mu=18))
    assert np.max(np.abs(Wg - So)) < 0.05 * np.max(np.abs(So))
    k.release()


def test_build_rejects_bad_grids(ctx, kx):
    with pytest.raises(kx.KxError):
        ctx.build_kernel(np.array([1.0, 2.0, 3.0]))
    with pytest.raises(kx.KxError):
        ctx.build_kernel(np.array([1.0, 3.0, 2.0, 4.0]))
    with pytest.raises(kx.KxError):
        ctx.build_kernel(ki.log_grid(513, 1e-3, 10.0))
    with pytest.raises(kx.KxError):
        ctx.build_kernel(ki.log_grid(16, 1e-3, 10.0), mass=0.0)
    with pytest.raises(kx.KxError) as ei:
        ctx.build_kernel(ki.log_grid(16, 1e-3, 10.0), stats=1, precision=kx.SPLIT_TF32, loss_terms=16)
    assert ei.value.code == kx.ENOTSUP
    with pytest.raises(kx.KxError):
        ctx.build_kernel(ki.log_grid(16, 1e-3, 10.0), stats=2)


# ------------------------------------------------------------ collision ----
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("N", [4, 17, 64, 130, 200])
def test_collision_matches_oracle(ctx, kx, precision, N):
    rng = np.random.default_rng(100 + N)
    q = ki.log_grid(N, 1e-3, 10.0 if N < 100 else 1e2)
    f = ki.batch_bimodal(rng, q, 3)
    sigma = np.array([1.0, 0.25, 7.0])
    k = ctx.build_kernel(q, precision=precision)
    W = oracle.kernel_tensor(q)
    fd = dev(f)
    for project in (0, 1):
        C, diag = ctx.collision(k, fd, sigma, project=bool(project), diag=True)
        Co, do = oracle_C(q, f, sigma, project, W)
        C = C.cpu().numpy()
        g = oracle.grid(q)
        for b in range(3):
            assert relerr(C[b], Co[b]) <= TOL[precision], (b, relerr(C[b], Co[b]))
            assert diag[b]["status"] == 0
            if project:
                # the diagnostics are h- (and hE-) weighted ratios: their error is
                # bounded by the weighted C error, not by the max-norm one
                Craw = oracle_C(q, f[b], [sigma[b]], 0, W)[0][0]
                for key, wgt in (("eps_N_raw", g["h"]), ("eps_E_raw", g["h"] * g["E"]),
                                 ("R_N", g["h"]), ("R_E", g["h"] * g["E"])):
                    bound = 4 * np.sum(wgt * np.abs(C[b] - Co[b])) / np.sum(wgt * np.abs(Craw))
                    bound += 8 * TOL[precision] * np.max(np.abs(Craw)) * np.sum(wgt) / np.sum(wgt * np.abs(Craw))
                    assert abs(diag[b][key] - do[b][key]) <= bound + 1e-14, (key, diag[b][key], do[b][key])
                # projected moments vanish to rounding (Appendix B), amplified by the
                # condition number of the 2x2 system
                xi = np.abs(f[b]) / np.max(np.abs(f[b]))
                xi[xi <= 1e-12] = 0.0
                A = [np.sum(g["h"] * xi * g["E"] ** k) for k in range(3)]
                cond = A[0] * A[2] / (A[0] * A[2] - A[1] ** 2)
                for wgt in (g["h"], g["h"] * g["E"]):
                    assert abs(np.sum(wgt * C[b])) <= 1e-14 * cond * np.sum(wgt * np.abs(Craw))


@pytest.mark.parametrize("precision", [0, 1])
def test_collision_full_size_sampled_rows(ctx, kx, precision):
    """N = 384 and 512 (the maximum): every row on the GPU; every 8th row, both
    ends and a few random rows by the oracle's direct per-row form.  The
    tolerance scale is the largest |C| among the oracle's rows, never the GPU's
    own output (a kernel that inflated a row cannot loosen its own bound)."""
    for N in (384, 512):
        rng = np.random.default_rng(N)
        q = ki.log_grid(N, 1e-3, 1e2)
        f = ki.batch_bimodal(rng, q, 1)[0]
        k = ctx.build_kernel(q, precision=precision)
        C, _ = ctx.collision(k, dev(f[None]), 1.0, project=False)
        C = C.cpu().numpy()[0]
        assert np.all(np.isfinite(C))
        rows = np.unique(np.concatenate([np.arange(0, N, 8), [1, N // 2 + 3, N - 2, N - 1],
                                         rng.integers(0, N, 6)]))
        Co, G, L = oracle.collision_rows(q, f, rows, M2=oracle.M2_from_sigma(1.0, 1.0))
        scale = np.max(np.abs(Co))
        err = np.max(np.abs(C[rows] - Co)) / scale
        assert err <= TOL[precision], (N, err)
        # the unsampled rows cannot exceed the sampled maximum by much: the
        # operator is smooth in i (a row larger than twice the sampled maximum
        # would be a kernel fault, not physics)
        assert np.max(np.abs(C)) <= 2.0 * scale
        k.release()


@pytest.mark.parametrize("precision", [0, 1])
def test_collision_edge_cases(ctx, kx, precision):
    N = 20
    q = ki.log_grid(N, 1e-3, 10.0)
    k = ctx.build_kernel(q, precision=precision)
    g = oracle.grid(q)
    # all-zero f: C = 0, projection flagged singular
    C, d = ctx.collision(k, dev(np.zeros((1, N))), 1.0, diag=True)
    assert np.all(C.cpu().numpy() == 0.0) and d[0]["singular"] == 1
    # zeros inside the support (log floor) and a single populated bin
    f = ki.bimodal(np.random.default_rng(3), q)
    f[5:9] = 0.0
    f1 = np.zeros(N)
    f1[7] = 0.3
    for fx in (f, f1):
        C, d = ctx.collision(k, dev(fx[None]), 2.0, diag=True)
        Co, do = oracle_C(q, fx, [2.0], 1)
        assert relerr(C.cpu().numpy()[0], Co[0]) <= TOL[precision]
        assert d[0]["singular"] == do[0]["singular"]
    # Maxwell-Boltzmann fixed point (eq. app_log_interp preserves MB)
    fm = 0.4 * np.exp(-g["E"] / 0.5)
    C, d = ctx.collision(k, dev(fm[None]), 1.0, project=False, diag=True)
    _, G, _ = oracle.collision_tensor(q, oracle.kernel_tensor(q), fm, parts=True)
    assert np.max(np.abs(C.cpu().numpy())) <= (1e-13 if precision == 0 else 1e-6) * \
        oracle.M2_from_sigma(1.0, 1.0) * np.max(G)
    # non-finite input is reported
    fn = f.copy()
    fn[3] = np.nan
    _, d = ctx.collision(k, dev(fn[None]), 1.0, diag=True)
    assert d[0]["status"] == kx.ENONFINITE
    # bad sigma
    with pytest.raises(kx.KxError):
        ctx.collision(k, dev(f[None]), -1.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_collision_steep_f_on_wide_grid(ctx, kx, precision):
    """Cold, steep distributions on q in [1e-3, 1e2]: the log-linear reference of
    the FP32 path leaves deviations of several hundred (in log2 units) at the
    grid ends, so out-of-support elements see exponents beyond the float range;
    C must stay finite and within tolerance.  Inputs: the first serving-stream
    requests with N <= 120 and a cold Maxwell-Boltzmann (T = 0.05, underflowing
    to zero at high q)."""
    reqs = [r for r in ki.config5()[:40] if r["n"] <= 120][:4]
    cases = [(r["q"], r["f0"], r["sigma"]) for r in reqs]
    q = ki.log_grid(90, 1e-3, 1e2)
    E = np.sqrt(q * q + 1.0)
    cases.append((q, 0.7 * np.exp(-(E - 1.0) / 0.05) + 1e-3 * np.exp(-(E - 1.0) / 2.0), 3.0))
    for q, f, sig in cases:
        k = ctx.build_kernel(q, precision=precision)
        W = oracle.kernel_tensor(q)
        for project in (0, 1):
            C, d = ctx.collision(k, dev(f[None]), sig, project=bool(project), diag=True)
            C = C.cpu().numpy()[0]
            assert d[0]["status"] == 0 and np.all(np.isfinite(C))
            Co, _ = oracle_C(q, f, [sig], project, W)
            assert relerr(C, Co[0]) <= TOL[precision], (q.size, project, relerr(C, Co[0]))
        k.release()


@pytest.mark.parametrize("N", [48, 200])
def test_streaming_variants_are_bitwise_identical(ctx, kx, N):
    """Every streaming variant the autotuner may pick gives the same bits."""
    q = ki.log_grid(N, 1e-3, 1e2)
    f = ki.batch_bimodal(np.random.default_rng(19), q, 8)
    sig = np.linspace(0.5, 4.0, 8)
    k = ctx.build_kernel(q, precision=kx.FP32)
    variants = [0, 1, 3] + ([2] if N > 160 else [])
    out = []
    for var in variants:
        ctx.set_stream_variant(N, 8, var)
        C, _ = ctx.collision(k, dev(f), sig)
        out.append(C.cpu().numpy())
    ctx.set_stream_variant(N, 8, -1)
    for o in out[1:]:
        np.testing.assert_array_equal(o, out[0])
    with pytest.raises(kx.KxError):
        ctx.set_stream_variant(N, 1, 1)
    with pytest.raises(kx.KxError):
        ctx.set_stream_variant(N, 3, 3)
    with pytest.raises(kx.KxError):
        ctx.set_stream_variant(N, 8, 4)
    # the staged-share variant (batches of up to four): the same bits as the
    # register pipeline and as the batch of eight, instance by instance
    for Bs in (1, 2, 3, 4):
        got = []
        for var in (0, 4):
            ctx.set_stream_variant(N, Bs, var)
            C, _ = ctx.collision(k, dev(f[:Bs]), sig[:Bs])
            got.append(C.cpu().numpy())
            ctx.set_stream_variant(N, Bs, -1)
        np.testing.assert_array_equal(got[1], got[0])
        np.testing.assert_array_equal(got[1], out[0][:Bs])
    k.release()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("N", [48, 200])
def test_batch_is_bitwise_independent_of_co_scheduling(ctx, kx, precision, N):
    """Each instance's C is bit-identical alone and inside a batch."""
    q = ki.log_grid(N, 1e-3, 10.0)
    f = ki.batch_bimodal(np.random.default_rng(9), q, 6)
    sig = np.array([1.0, 2.0, 0.5, 3.0, 1.5, 0.1])
    k = ctx.build_kernel(q, precision=precision)
    Cb, _ = ctx.collision(k, dev(f), sig)
    Cb = Cb.cpu().numpy()
    for b in range(6):
        Ca, _ = ctx.collision(k, dev(f[b:b + 1]), sig[b:b + 1])
        np.testing.assert_array_equal(Ca.cpu().numpy()[0], Cb[b])
    Ch, _ = ctx.collision_host(k, f, sig)
    np.testing.assert_array_equal(Ch, Cb)


# ----------------------------------------------------------- integration ---
def test_single_heun_attempt_matches_oracle(ctx, kx):
    N = 32
    q = ki.log_grid(N, 1e-3, 10.0)
    f0 = ki.bimodal(np.random.default_rng(21), q)
    k = ctx.build_kernel(q, precision=kx.FP64)
    W = oracle.kernel_tensor(q)
    src = ki.two_sources(q)
    M2 = oracle.M2_from_sigma(1.0, 1.0)
    for h0 in (0.01, 0.5, 5.0):   # accepted, rejected by error, rejected by negativity
        fd = dev(f0[None])
        t = np.array([0.2])
        h = np.array([h0])
        res = ctx.step(k, fd, 1.0, t, h, sources=src, t_end=100.0, rtol=1e-6, atol=1e-12)
        fo, ro = oracle.solve(q, W, f0, M2, sources=src, t0=0.2, t_end=100.0, h0=h0,
                              max_attempts=1, rtol=1e-6, atol=1e-12)
        assert res[0]["steps"] == ro["steps"] and res[0]["rejects"] == ro["rejects"]
        assert abs(h[0] - ro["h"]) <= 1e-12 * ro["h"]
        assert abs(t[0] - ro["t"]) <= 1e-15 * max(1.0, ro["t"])
        assert relerr(fd.cpu().numpy()[0], fo) <= 1e-12


def test_fixed_step_solve_matches_oracle_config1(ctx, kx):
    """Configuration 1: N = 32, 100 fixed Heun steps."""
    c = ki.config1()
    q, f0 = c["q"], c["f0"]
    W = oracle.kernel_tensor(q)
    fo, ro = oracle.solve(q, W, f0, oracle.M2_from_sigma(1.0, c["sigma"]), t_end=c["n_steps"] * c["h"],
                          h0=c["h"], fixed_step=1)
    assert ro["status"] == 0 and ro["steps"] == c["n_steps"]
    g = oracle.grid(q)
    for precision in (0, 1):
        k = ctx.build_kernel(q, precision=precision)
        fd = dev(f0[None])
        res = ctx.solve(k, fd, c["sigma"], t_end=c["n_steps"] * c["h"], h0=c["h"], fixed_step=1)
        f = fd.cpu().numpy()[0]
        assert res[0]["status"] == 0 and res[0]["steps"] == c["n_steps"]
        assert relerr(f, fo) <= (1e-11 if precision == 0 else 1e-5)
        n0, n1 = np.sum(g["h"] * f0), np.sum(g["h"] * f)
        e0, e1 = np.sum(g["h"] * g["E"] * f0), np.sum(g["h"] * g["E"] * f)
        assert abs(n1 / n0 - 1) < 1e-7 and abs(e1 / e0 - 1) < 1e-7


def test_adaptive_solve_with_sources_matches_oracle(ctx, kx):
    N = 40
    q = ki.log_grid(N, 1e-3, 10.0)
    f0 = ki.bimodal(np.random.default_rng(22), q)
    src = ki.two_sources(q)
    W = oracle.kernel_tensor(q)
    par = dict(t_end=1e4, h0=1e-3, rtol=1e-6, atol=1e-12 * f0.max(), l1_tol=1e-3, check_every=5)
    fo, ro = oracle.solve(q, W, f0, oracle.M2_from_sigma(1.0, 3.0), sources=src, **par)
    assert ro["converged"] == 1
    k = ctx.build_kernel(q, precision=kx.FP64)
    fd = dev(f0[None])
    res = ctx.solve(k, fd, 3.0, sources=src, **par)[0]
    assert res["converged"] == 1 and res["status"] == 0
    assert res["steps"] == ro["steps"] and res["rejects"] == ro["rejects"]
    # the controller's err = |f_c - f_p| / (rtol |f|) is a difference of nearly
    # equal states: a 1e-16 rounding difference becomes ~1e-16/rtol = 1e-10 in err
    # and h, accumulating over the steps in t (not in f, which depends smoothly on h)
    assert abs(res["t"] / ro["t"] - 1) < 1e-9
    assert relerr(fd.cpu().numpy()[0], fo) <= 1e-10
    assert abs(res["l1_to_mb"] - ro["l1"]) < 1e-10
    # FP32 path: same physics within the mixed tolerances; moments exactly tracked
    k32 = ctx.build_kernel(q, precision=kx.FP32)
    fd32 = dev(f0[None])
    r32 = ctx.solve(k32, fd32, 3.0, sources=src, **par)[0]
    assert r32["converged"] == 1
    g = oracle.grid(q)
    f32 = fd32.cpu().numpy()[0]
    # different step sequences integrate the decaying sources with different
    # trapezoid errors (~1e-7 here), so only closeness is asserted; exact moment
    # bookkeeping is tested where the quadrature is exact (next test)
    assert np.sum(g["h"] * np.abs(f32 - fo)) / np.sum(g["h"] * fo) < 5e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_moments_conserved_through_integration(ctx, kx, precision):
    """Number and energy after an integration: without sources they stay at
    their initial values; with a constant-rate source (trapezoid exact) they
    grow by R t and R <E>_s t.  Tolerance 1e-7 (mixed path) / 1e-12 (FP64)."""
    N = 48
    q = ki.log_grid(N, 1e-3, 10.0)
    g = oracle.grid(q)
    f0 = ki.bimodal(np.random.default_rng(25), q)
    k = ctx.build_kernel(q, precision=precision)
    tol = 1e-12 if precision == 0 else 1e-7
    fd = dev(f0[None])
    r = ctx.solve(k, fd, 2.0, t_end=20.0, h0=1e-3, rtol=1e-6, atol=1e-12)[0]
    f = fd.cpu().numpy()[0]
    assert r["status"] == 0 and r["t"] == 20.0
    for w in (g["h"], g["h"] * g["E"]):
        assert abs(np.sum(w * f) / np.sum(w * f0) - 1) < tol
    shape = ki.lognormal_bumps(q, (1.0,), (0.3,), (1.0,))
    src = dict(shape=shape[None], rate=np.array([0.02]), tau=np.array([1e300]), t_on=np.array([0.0]))
    fd = dev(f0[None])
    r = ctx.solve(k, fd, 2.0, sources=src, t_end=10.0, h0=1e-3, rtol=1e-6, atol=1e-12)[0]
    f = fd.cpu().numpy()[0]
    e_s = np.sum(g["h"] * g["E"] * shape) / np.sum(g["h"] * shape)
    assert abs(np.sum(g["h"] * f) / (np.sum(g["h"] * f0) + 0.02 * 10.0) - 1) < tol
    assert abs(np.sum(g["h"] * g["E"] * f) / (np.sum(g["h"] * g["E"] * f0) + 0.02 * e_s * 10.0) - 1) < tol


def test_solve_batch_of_sigmas_matches_individual(ctx, kx):
    """Several sigmas integrated together give bit-identical results to each
    sigma alone (no cross-instance coupling)."""
    N = 32
    q = ki.log_grid(N, 1e-3, 10.0)
    f0 = ki.bimodal(np.random.default_rng(23), q)
    sig = np.array([0.5, 1.0, 4.0])
    par = dict(t_end=50.0, h0=1e-3, rtol=1e-6, atol=1e-12, l1_tol=1e-3, check_every=5)
    for precision in (0, 1):
        k = ctx.build_kernel(q, precision=precision)
        fb = dev(np.tile(f0, (3, 1)))
        rb = ctx.solve(k, fb, sig, **par)
        for b in range(3):
            fa = dev(f0[None])
            ra = ctx.solve(k, fa, sig[b], **par)[0]
            np.testing.assert_array_equal(fa.cpu().numpy()[0], fb.cpu().numpy()[b])
            assert ra["steps"] == rb[b]["steps"]
        fh, rh = ctx.solve_host(k, np.tile(f0, (3, 1)), sig, **par)
        np.testing.assert_array_equal(fh, fb.cpu().numpy())


@pytest.mark.parametrize("precision", [0, 1])
def test_concurrent_chains_equal_one_batch(ctx, kx, precision):
    """kx_solve's concurrent per-instance chains (the rule's choice for small
    FP32 batches, chains = 2 forces them on any path) give the bits of the
    one-batch solve (chains = 1): f, steps, rejects, evaluations and the MB
    fit of every instance, with per-instance sources, on device and host
    buffers alike; invalid chain settings are refused."""
    q = ki.log_grid(40, 1e-3, 10.0)
    B = 3
    f0 = ki.batch_bimodal(np.random.default_rng(66), q, B)
    sig = np.array([0.3, 1.0, 4.0])
    rng = np.random.default_rng(67)
    srcs = [dict(shape=np.stack([ki.lognormal_bumps(q, (c,), (0.3,), (1.0,)) for c in (0.05, 2.0)]),
                 rate=rng.uniform(0.01, 0.05, 2), tau=np.array([1.0, 1.0]), t_on=np.array([0.0, 1.0]))
            for _ in range(B)]
    par = dict(t_end=4.0, h0=1e-3, rtol=1e-6, atol=1e-12, l1_tol=1e-3, check_every=5)
    k = ctx.build_kernel(q, precision=precision)
    out = {}
    for ch in (1, 0, 2):
        fd = dev(f0)
        res = ctx.solve(k, fd, sig, sources=srcs, chains=ch, **par)
        out[ch] = (fd.cpu().numpy(), res)
    fh, rh = ctx.solve_host(k, f0, sig, sources=srcs, chains=2, **par)
    out["host"] = (fh, rh)
    for key in (0, 2, "host"):
        np.testing.assert_array_equal(out[key][0], out[1][0])
        for a, b in zip(out[key][1], out[1][1]):
            for fld in ("steps", "rejects", "evals", "status", "converged", "t", "h", "T_mb", "l1_to_mb"):
                assert a[fld] == b[fld], (key, fld, a[fld], b[fld])
    with pytest.raises(kx.KxError):
        ctx.solve(k, dev(f0), sig, chains=3, **par)
    k.release()


def test_mb_fit_matches_oracle(ctx, kx):
    N = 64
    q = ki.log_grid(N, 1e-3, 10.0)
    g = oracle.grid(q)
    k = ctx.build_kernel(q, precision=kx.FP64)
    fs = [0.3 * np.exp(-g["E"] / 0.7), ki.bimodal(np.random.default_rng(24), q)]
    out = ctx.mb_fit(k, dev(np.array(fs)))
    for b, f in enumerate(fs):
        r = oracle.mb_fit(g["E"], g["h"], f)
        assert abs(out[b, 0] / r["T"] - 1) < 1e-12
        assert abs(out[b, 1] - r["ln_z"]) < 1e-10
        assert abs(out[b, 2] - r["l1"]) < 1e-10 * max(1.0, r["l1"])


# ------------------------------------------------- table-driven log2 / exp ---
def test_table_log2_exp_against_cuda_and_libm(ctx, kx):
    """The stage kernels' own FP64 log2 and exp (Tang's table-driven methods)
    against CUDA's log2/exp and the host libm: absolute error within 2 ulp of
    the result's magnitude (log2), relative error within 2 ulp (exp, normal
    range), exact special cases."""
    import torch
    rng = np.random.default_rng(11)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 20000), 1.0 + rng.uniform(-1e-3, 1e-3, 2000),
                        2.0 ** np.arange(-996, 1000, 7.0), [1.0, 2.0, 0.5, 1e-300, 1.7e308]])
    out = ctx.math_check(0, torch.as_tensor(x, device="cuda")).cpu().numpy()
    ref = np.log2(x)
    tol = 2 * np.spacing(np.maximum(np.abs(ref), 1.0))
    assert np.all(np.abs(out[:, 0] - ref) <= tol)
    assert np.all(np.abs(out[:, 0] - out[:, 1]) <= tol)
    assert out[np.flatnonzero(x == 1.0)[0], 0] == 0.0
    y = np.concatenate([rng.uniform(-745, 709.7, 20000), rng.uniform(-1, 1, 2000) * 1e-3,
                        [0.0, -0.0, 1.0, -1.0, 709.78, -708.39, -745.1, -746.0, 710.0]])
    out = ctx.math_check(1, torch.as_tensor(y, device="cuda")).cpu().numpy()
    with np.errstate(over="ignore"):   # exp(710) = inf is one of the checked cases
        ref = np.exp(y)
    normal = (ref > 2.3e-308) & np.isfinite(ref)
    rel = np.abs(out[normal, 0] - ref[normal]) / ref[normal]
    assert rel.max() <= 4.5e-16, rel.max()
    sub = ref <= 2.3e-308
    assert np.all(np.abs(out[sub, 0] - ref[sub]) <= 1e-322)
    assert np.all(np.abs(out[normal, 0] - out[normal, 1]) / ref[normal] <= 4.5e-16)
    assert out[-1, 0] == np.inf and out[-2, 0] == 0.0 and out[y.size - 9, 0] == 1.0
    nan = ctx.math_check(1, torch.as_tensor(np.array([np.nan]), device="cuda")).cpu().numpy()
    assert np.isnan(nan[0, 0])


def test_lean_log2_and_conversions(ctx, kx):
    """The FP32 path's integer-pipe conversions and double-float log2 against
    numpy: float -> double exact for every class of float; double -> float
    round-to-nearest-even bit for bit in the float normal range (ties, the
    carry into the exponent, overflow to inf), zero below 2^-126; log2 of a
    normal double to 3e-14 absolute (plus the FP64 rounding of the check's
    own sum)."""
    import torch
    rng = np.random.default_rng(5)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 20000), 1.0 + rng.uniform(0, 1, 4000),
                        1.0 + np.arange(256) / 256.0, np.nextafter(1.0 + np.arange(1, 257) / 256.0, 0.0),
                        2.0 ** np.arange(-1000, 1000, 13.0), [1.0, 2.0, 0.5, 1e-300, 1.7e308]])
    out = ctx.math_check(2, torch.as_tensor(x, device="cuda")).cpu().numpy()
    ref = np.log2(x)
    assert np.all(np.abs(out[:, 0] - ref) <= 3e-14 + 2 * np.spacing(np.abs(ref))), \
        np.max(np.abs(out[:, 0] - ref))
    # double -> float: random doubles in the float range, exact ties, the largest float
    f = rng.uniform(-1, 1, 20000) * 10.0 ** rng.uniform(-37, 38, 20000)
    f = f[np.abs(f) >= 2.0 ** -125]   # (the library flushes below the float normal range)
    base = np.float32(rng.uniform(1, 2, 2000)).astype(np.float64)
    ties = base + np.spacing(np.float32(base)).astype(np.float64) / 2   # halfway between floats
    big = np.array([3.4028234663852886e38, 3.4028235677973366e38, 3.5e38, -3.5e38, np.inf, -np.inf, 0.0, -0.0])
    y = np.concatenate([f, ties, -ties, big])
    out = ctx.math_check(3, torch.as_tensor(y, device="cuda")).cpu().numpy()
    with np.errstate(over="ignore"):
        want = y.astype(np.float32).astype(np.float64)
    assert np.array_equal(out[:, 0], want)
    assert np.array_equal(np.signbit(out[:, 0]), np.signbit(want))
    tiny = np.array([1e-39, -1e-39, 1e-45, 2.0 ** -127, 1e-300])
    out = ctx.math_check(3, torch.as_tensor(tiny, device="cuda")).cpu().numpy()
    assert np.all(out[:, 0] == 0.0) and np.array_equal(np.signbit(out[:, 0]), np.signbit(tiny))
    nan = ctx.math_check(3, torch.as_tensor(np.array([np.nan]), device="cuda")).cpu().numpy()
    assert np.isnan(nan[0, 0])
    # float -> double: normals, subnormals, zeros, infinities
    z = np.concatenate([f, [1e-38, 1e-40, -1e-40, 1.4e-45, -1.4e-45, 2.0 ** -140, 0.0, -0.0, np.inf, -np.inf,
                            3.4e38]])
    out = ctx.math_check(4, torch.as_tensor(z, device="cuda")).cpu().numpy()
    assert np.array_equal(out[:, 0], out[:, 1])
    assert np.array_equal(np.signbit(out[:, 0]), np.signbit(out[:, 1]))
    assert np.array_equal(out[:, 0], z.astype(np.float32).astype(np.float64))


# ----------------------------------------------- the bench workload itself ---
def test_bench_workload_n128_four_sigmas_matches_oracle(ctx, kx):
    """The timed configuration (N = 128, q in [1e-3, 10], the four sigmas
    sharing one kernel, two sources) in the launch shape the bench uses (one
    batch of four): C of f0 on both paths against the oracle, and a short
    adaptive integration (t = 0.005, about 200 steps, sources on) against the
    oracle's."""
    c = ki.config2()
    q, sig, src = c["q"], c["sigmas"], c["sources"]
    f0 = np.tile(c["f0"], (4, 1))
    W = oracle.kernel_tensor(q)
    Co, _ = oracle_C(q, f0, sig, 1, W)
    par = dict(t_end=0.005, h0=1e-3, rtol=1e-6, atol=1e-12 * f0.max(), l1_tol=1e-3, check_every=10)
    fo = [oracle.solve(q, W, c["f0"], oracle.M2_from_sigma(1.0, s), sources=src, **par) for s in sig]
    for prec in (kx.FP64, kx.FP32):
        k = ctx.build_kernel(q, precision=prec)
        C, _ = ctx.collision(k, dev(f0), sig)
        C = C.cpu().numpy()
        for b in range(4):
            assert relerr(C[b], Co[b]) <= TOL[prec], (prec, b, relerr(C[b], Co[b]))
        fd = dev(f0)
        res = ctx.solve(k, fd, sig, sources=src, **par)
        f = fd.cpu().numpy()
        for b in range(4):
            assert res[b]["status"] == 0 and abs(res[b]["t"] - 0.005) < 1e-12
            err = relerr(f[b], fo[b][0])
            if prec == kx.FP64:
                assert res[b]["steps"] == fo[b][1]["steps"]
                assert err <= 1e-10, (b, err)
            else:
                assert err <= 1e-6, (b, err)
        k.release()


# ------------------------------------------------------- checkpoint / resume ---
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_resumes_from_the_returned_state(ctx, kx, precision):
    """A solve stopped by max_attempts returns (t, h) and leaves f on the
    device; a second solve entered with t0 = t, h0 = h continues the same
    trajectory (sources included): the plain FP64 path bit for bit, the FP32
    path within its tolerance (its tables' reference line is refitted on
    entry)."""
    N = 40
    q = ki.log_grid(N, 1e-3, 10.0)
    f0 = ki.bimodal(np.random.default_rng(61), q)
    src = ki.two_sources(q, t_scale=2.0)
    k = ctx.build_kernel(q, precision=precision)
    kw = dict(t_end=30.0, rtol=1e-6, atol=1e-12, l1_tol=0.0)
    fa = dev(f0[None])
    ra = ctx.solve(k, fa, 1.0, sources=src, h0=1e-3, **kw)[0]
    assert ra["status"] == 0 and ra["steps"] > 40
    K = (ra["steps"] + ra["rejects"]) // 2
    fb = dev(f0[None])
    r1 = ctx.solve(k, fb, 1.0, sources=src, h0=1e-3, max_attempts=K, **kw)[0]
    assert r1["status"] == kx.ENOCONV and r1["steps"] + r1["rejects"] == K and r1["t"] < kw["t_end"]
    r2 = ctx.solve(k, fb, 1.0, sources=src, t0=r1["t"], h0=r1["h"], **kw)[0]
    assert r2["status"] == 0 and r2["t"] == kw["t_end"]
    if precision == 0:
        assert r1["steps"] + r2["steps"] == ra["steps"] and r1["rejects"] + r2["rejects"] == ra["rejects"]
        np.testing.assert_array_equal(fb.cpu().numpy(), fa.cpu().numpy())
    else:
        assert abs(r1["steps"] + r2["steps"] - ra["steps"]) <= 2
        assert relerr(fb.cpu().numpy()[0], fa.cpu().numpy()[0]) <= TOL[1]
    k.release()


# ------------------------------------------------------ quantum statistics ---
@pytest.mark.parametrize("eta", [1, -1])
def test_quantum_statistics_fp64_path_matches_oracle(ctx, kx, eta):
    """Bose-Einstein / Fermi-Dirac factor (eq. Lambda_quantum) on the FP64 path:
    C raw and projected against the oracle on a bimodal f scaled to occupations
    of order one (where the factor matters), and the near-vanishing C on the
    equilibrium distribution of that statistics."""
    N = 40
    q = ki.log_grid(N, 1e-2, 20.0)
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q)
    f = 0.8 * ki.batch_bimodal(np.random.default_rng(43 + eta), q, 2)
    k = ctx.build_kernel(q, precision=kx.FP64, stats=eta)
    for project in (0, 1):
        C, _ = ctx.collision(k, dev(f), np.array([1.0, 3.0]), project=bool(project))
        C = C.cpu().numpy()
        for b, sgm in enumerate((1.0, 3.0)):
            Co = oracle.collision_tensor_stats(q, W, f[b], eta) * oracle.M2_from_sigma(1.0, sgm)
            if project:
                Co, _ = oracle.project(g["E"], g["h"], f[b], Co)
            assert relerr(C[b], Co) <= 1e-12, (project, b, relerr(C[b], Co))
    feq = 1.0 / (np.exp((g["E"] - 0.6) / 0.7) - eta)
    C, _ = ctx.collision(k, dev(feq[None]), 1.0, project=False)
    Co = oracle.collision_tensor_stats(q, W, feq, eta) * oracle.M2_from_sigma(1.0, 1.0)
    _, G, _ = oracle.collision_tensor(q, W, feq, parts=True)
    scale = oracle.M2_from_sigma(1.0, 1.0) * np.max(G)
    assert np.max(np.abs(C.cpu().numpy()[0] - Co)) <= 1e-13 * scale
    assert np.max(np.abs(Co)) < 2e-2 * scale
    k.release()


@pytest.mark.parametrize("eta", [1, -1])
def test_quantum_statistics_fp32_path_matches_oracle(ctx, kx, eta):
    """The FP32 streaming path with the Bose-Einstein / Fermi-Dirac factor
    (eq. Lambda_quantum; per element 2^a (1 - 2^d) with the line fitted to
    log2 f/(1 + eta f)): C raw and projected within the mixed-precision
    tolerance of the oracle, instances bit-identical alone and in the batch,
    and the equilibrium of that statistics near its fixed point."""
    N = 40
    q = ki.log_grid(N, 1e-2, 20.0)
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q)
    f = 0.8 * ki.batch_bimodal(np.random.default_rng(53 + eta), q, 3)
    sig = np.array([1.0, 3.0, 0.5])
    k = ctx.build_kernel(q, precision=kx.FP32, stats=eta)
    for project in (0, 1):
        C, _ = ctx.collision(k, dev(f), sig, project=bool(project))
        C = C.cpu().numpy()
        for b in range(3):
            Co = oracle.collision_tensor_stats(q, W, f[b], eta) * oracle.M2_from_sigma(1.0, sig[b])
            if project:
                Co, _ = oracle.project(g["E"], g["h"], f[b], Co)
            assert relerr(C[b], Co) <= TOL[1], (project, b, relerr(C[b], Co))
        if project:
            C1, _ = ctx.collision(k, dev(f[1:2]), sig[1:2], project=True)
            np.testing.assert_array_equal(C1.cpu().numpy()[0], C[1])
    feq = 1.0 / (np.exp((g["E"] - 0.6) / 0.7) - eta)
    C, _ = ctx.collision(k, dev(feq[None]), 1.0, project=False)
    Co = oracle.collision_tensor_stats(q, W, feq, eta) * oracle.M2_from_sigma(1.0, 1.0)
    _, G, _ = oracle.collision_tensor(q, W, feq, parts=True)
    scale = oracle.M2_from_sigma(1.0, 1.0) * np.max(G)
    assert np.max(np.abs(C.cpu().numpy()[0] - Co)) <= 1e-6 * scale
    k.release()


def test_quantum_statistics_fp32_paper_benchmark_distribution(ctx, kx):
    """The paper's runtime workload (eq. benchmark_two_bump: m = 1, a = 1,
    q in [1e-3, 1e2], N = 96, Bose-Einstein factors, no projection) on the FP32
    path against the oracle."""
    q = ki.log_grid(96, 1e-3, 1e2)
    f = ki.paper_two_bump(q)
    W = oracle.kernel_tensor(q)
    Co = oracle.collision_tensor_stats(q, W, f, 1) * oracle.M2_from_sigma(1.0, 1.0)
    for prec, tol in ((kx.FP32, TOL[1]), (kx.FP64, TOL[0])):
        k = ctx.build_kernel(q, precision=prec, stats=1)
        C, _ = ctx.collision(k, dev(f[None]), 1.0, project=False)
        assert relerr(C.cpu().numpy()[0], Co) <= tol, (prec, relerr(C.cpu().numpy()[0], Co))
        k.release()


@pytest.mark.parametrize("eta", [1, -1])
def test_quantum_statistics_fp32_fixed_step_solve(ctx, kx, eta):
    """Twenty fixed Heun steps with Bose-Einstein (Fermi-Dirac: f scaled below
    one) factors on the FP32 path against the same steps taken with the
    oracle's operator and projection; number and energy conserved to the
    mixed-precision bound."""
    c = ki.config1()
    q, f0 = c["q"], c["f0"] * (1.0 if eta == 1 else 0.5)
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q)
    M2 = oracle.M2_from_sigma(1.0, c["sigma"])
    h, steps = c["h"], 20

    def rhs(f):
        return oracle.project(g["E"], g["h"], f, oracle.collision_tensor_stats(q, W, f, eta) * M2)[0]

    fo = f0.copy()
    for _ in range(steps):
        k1 = rhs(fo)
        fp = fo + h * k1
        fo = fo + 0.5 * h * (k1 + rhs(fp))
    k = ctx.build_kernel(q, precision=kx.FP32, stats=eta)
    fd = dev(f0[None])
    res = ctx.solve(k, fd, c["sigma"], t_end=steps * h, h0=h, fixed_step=1)
    f = fd.cpu().numpy()[0]
    assert res[0]["status"] == 0 and res[0]["steps"] == steps
    assert relerr(f, fo) <= TOL[1], relerr(f, fo)
    for w in (g["h"], g["h"] * g["E"]):
        assert abs(np.sum(w * f) / np.sum(w * f0) - 1) < 1e-7
    k.release()


# ------------------------------------------------- the paper's physical sources ---
def test_solve_with_paper_sources_matches_oracle_and_cbe(ctx, kx):
    """A static box with the paper's two freeze-in terms (Sec. 2: Higgs decay at
    a bath temperature cooling with an e-folding time, and a decaying cold
    condensate binned to one cell): the FP64 solve follows the oracle's step for
    step, the number and energy it ends with are the initial ones plus the
    injected integrals (the fluid, cBE-like bookkeeping: sum_k rate_k tau_k
    (1 - exp(-(t - t_on)/tau_k)) times 1 and the row's mean energy), and the
    final Maxwell-Boltzmann temperature is the one those two moments fix."""
    N = 48
    q = ki.log_grid(N, 1e-3, 10.0)
    g = oracle.grid(q)
    f0 = ki.bimodal(np.random.default_rng(27), q)
    n0, e0 = np.sum(g["h"] * f0), np.sum(g["h"] * g["E"] * f0)
    sh, rh = kx.source_higgs_decay(q, 1.0, 5.0, 0.8, 1.0, 1.0)
    sc, rc = kx.source_condensate(q, 1.0, 3.0, 1.0, 1.0)
    tau, t_on = np.array([2.0, 1.0]), np.array([0.0, 0.5])
    # rates scaled (coupling^2 and 2 Gamma n_Phi are free) to inject 30 % and 15 % of n0
    rate = np.array([0.30 * n0 / tau[0], 0.15 * n0 / tau[1]])
    src = {"shape": np.stack([sh, sc]), "rate": rate, "tau": tau, "t_on": t_on}
    W = oracle.kernel_tensor(q)
    par = dict(t_end=1e4, h0=1e-3, rtol=1e-6, atol=1e-12 * f0.max(), l1_tol=1e-3, check_every=5)
    fo, ro = oracle.solve(q, W, f0, oracle.M2_from_sigma(1.0, 2.0), sources=src, **par)
    assert ro["converged"] == 1
    k = ctx.build_kernel(q, precision=kx.FP64)
    fd = dev(f0[None])
    res = ctx.solve(k, fd, 2.0, sources=src, **par)[0]
    f = fd.cpu().numpy()[0]
    assert res["converged"] == 1 and res["status"] == 0
    assert res["steps"] == ro["steps"] and res["rejects"] == ro["rejects"]
    assert relerr(f, fo) <= 1e-10
    # injected number and energy (trapezoid-integrated by the stepper: ~1e-7)
    inj = rate * tau * -np.expm1(-(res["t"] - t_on) / tau)
    ebar = [np.sum(g["h"] * g["E"] * s) / np.sum(g["h"] * s) for s in (sh, sc)]
    assert abs(np.sum(g["h"] * f) / (n0 + inj.sum()) - 1) < 1e-6
    assert abs(np.sum(g["h"] * g["E"] * f) / (e0 + np.dot(inj, ebar)) - 1) < 1e-6
    # the temperature the two injected moments fix: <E>_MB(T) = rho / n on the grid
    target = (e0 + np.dot(inj, ebar)) / (n0 + inj.sum())
    lo, hi = 1e-3, 1e3
    for _ in range(200):
        T = np.sqrt(lo * hi)
        w = g["h"] * np.exp(-(g["E"] - g["E"][0]) / T)
        if np.sum(w * g["E"]) / np.sum(w) < target:
            lo = T
        else:
            hi = T
    assert abs(res["T_mb"] / T - 1) < 1e-5, (res["T_mb"], T)
    k.release()
