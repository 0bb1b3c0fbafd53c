"""GPU parity of the batched split-TF32 path (tensor-core gain + exact loss)
against the FP64 oracle.  Tolerance 1e-5 max-norm relative on C (the mixed
path's bound); instances are bit-identical alone and inside a batch."""
import numpy as np
import pytest

import kx_inputs as ki
import oracle

pytestmark = pytest.mark.gpu
TOL = 1e-5


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


def oracle_rows(q, f, sigma, project):
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q)
    out = []
    for b in range(f.shape[0]):
        C = oracle.collision_tensor(q, W, f[b]) * oracle.M2_from_sigma(1.0, sigma[b])
        if project:
            C, _ = oracle.project(g["E"], g["h"], f[b], C)
        out.append(C)
    return np.array(out)


# B covers every gain-GEMM tile width: 64 (B <= 64), 128, 192, 256 and two
# column tiles (256 + 64)
@pytest.mark.parametrize("N,B", [(20, 1), (48, 3), (64, 70), (100, 5), (32, 190), (24, 256), (40, 300)])
def test_batched_collision_matches_oracle(env, N, B):
    kx, ctx, torch = env
    rng = np.random.default_rng(300 + N)
    q = ki.log_grid(N, 1e-3, 1e2)
    f = ki.batch_bimodal(rng, q, B)
    sig = rng.uniform(0.3, 3.0, size=B)
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32)
    fd = torch.as_tensor(f, device="cuda")
    for project in (0, 1):
        C, d = ctx.collision(k, fd, sig, project=bool(project), diag=True)
        C = C.cpu().numpy()
        Co = oracle_rows(q, f, sig, project)
        for b in range(B):
            err = np.max(np.abs(C[b] - Co[b])) / np.max(np.abs(Co[b]))
            assert err <= TOL, (b, err)
            assert d[b]["status"] == 0
    k.release()


@pytest.mark.parametrize("B,picks", [(67, (0, 5, 63, 64, 66)), (300, (0, 255, 256, 299))])
def test_batched_alone_equals_in_batch(env, B, picks):
    kx, ctx, torch = env
    N = 40
    q = ki.log_grid(N, 1e-3, 1e2)
    f = ki.batch_bimodal(np.random.default_rng(31), q, B)
    sig = np.linspace(0.5, 2.0, B)
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32)
    Cb, _ = ctx.collision(k, torch.as_tensor(f, device="cuda"), sig)
    Cb = Cb.cpu().numpy()
    for b in picks:
        Ca, _ = ctx.collision(k, torch.as_tensor(f[b:b + 1], device="cuda"), sig[b:b + 1])
        np.testing.assert_array_equal(Ca.cpu().numpy()[0], Cb[b])
    k.release()


def test_batched_solve_conserves_and_relaxes(env):
    kx, ctx, torch = env
    N = 48
    q = ki.log_grid(N, 1e-3, 10.0)
    g = oracle.grid(q)
    f0 = ki.batch_bimodal(np.random.default_rng(32), q, 3)
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32)
    fd = torch.as_tensor(f0, device="cuda")
    res = ctx.solve(k, fd, np.array([1.0, 2.0, 4.0]), t_end=1e4, h0=1e-3, rtol=1e-6,
                    atol=1e-12, l1_tol=1e-3, check_every=5)
    f = fd.cpu().numpy()
    W = oracle.kernel_tensor(q)
    for b in range(3):
        assert res[b]["status"] == 0 and res[b]["converged"] == 1
        for w in (g["h"], g["h"] * g["E"]):
            assert abs(np.sum(w * f[b]) / np.sum(w * f0[b]) - 1) < 1e-7
        fo, ro = oracle.solve(q, W, f0[b], oracle.M2_from_sigma(1.0, [1.0, 2.0, 4.0][b]),
                              t_end=1e4, h0=1e-3, rtol=1e-6, atol=1e-12, l1_tol=1e-3,
                              check_every=5)
        assert np.sum(g["h"] * np.abs(f[b] - fo)) / np.sum(g["h"] * fo) < 5e-3
    k.release()


def test_batched_full_size_configuration_sampled(env):
    """The batched configuration at its full size (B = 512 seeded distributions
    on one N = 192 kernel, the launch shapes the benchmark times), and the
    largest grid of the uneven batch (N = 256, 256 instances): sampled
    instances against the oracle, projected C."""
    kx, ctx, torch = env
    c = ki.config3()
    cases = [(c["q"], c["f"], c["sigma"], (0, 1, 255, 256, 511))]
    q256 = ki.log_grid(256, 1e-3, 1e2)
    rng = np.random.default_rng(404)
    cases.append((q256, ki.batch_bimodal(rng, q256, 256), rng.uniform(0.3, 3.0, 256), (0, 127, 255)))
    for q, f, sig, picks in cases:
        k = ctx.build_kernel(q, precision=kx.SPLIT_TF32)
        C, _ = ctx.collision(k, torch.as_tensor(f, device="cuda"), sig, project=True)
        C = C.cpu().numpy()
        Co = oracle_rows(q, f[list(picks)], np.asarray(sig)[list(picks)], True)
        for r, b in enumerate(picks):
            err = np.max(np.abs(C[b] - Co[r])) / np.max(np.abs(Co[r]))
            assert err <= TOL, (len(q), b, err)
        k.release()


def test_batched_fixed_step_solve_matches_oracle(env):
    """Configuration-1 style fixed-step integration on the split-TF32 path: three
    instances (N = 32, 100 Heun steps of the configuration's h) against the
    oracle's solve element by element at the mixed-precision bound, number and
    energy conserved to 1e-7 (Sec. 4.2 stepper; eq. discrete_collision_operator)."""
    kx, ctx, torch = env
    c = ki.config1()
    q = c["q"]
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q)
    f0 = np.stack([c["f0"], *ki.batch_bimodal(np.random.default_rng(33), q, 2)])
    sig = np.array([c["sigma"], 0.5 * c["sigma"], 1.5 * c["sigma"]])
    t_end = c["n_steps"] * c["h"]
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32)
    fd = torch.as_tensor(f0, device="cuda")
    res = ctx.solve(k, fd, sig, t_end=t_end, h0=c["h"], fixed_step=1)
    f = fd.cpu().numpy()
    for b in range(3):
        fo, ro = oracle.solve(q, W, f0[b], oracle.M2_from_sigma(1.0, sig[b]), t_end=t_end,
                              h0=c["h"], fixed_step=1)
        assert ro["status"] == 0 and ro["steps"] == c["n_steps"]
        assert res[b]["status"] == 0 and res[b]["steps"] == c["n_steps"]
        err = np.max(np.abs(f[b] - fo)) / np.max(np.abs(fo))
        assert err <= TOL, (b, err)
        for w in (g["h"], g["h"] * g["E"]):
            assert abs(np.sum(w * f[b]) / np.sum(w * f0[b]) - 1) < 1e-7
    k.release()


# ------------------------------------------- loss rate as a Chebyshev GEMM ---
def oracle_cheb_rows(q, f, sigma, project, K):
    """Oracle C with the loss rate's f_t in K Chebyshev terms (same truncation
    as the GPU option), and the exact oracle C beside it."""
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q)
    out, exact = [], []
    for b in range(f.shape[0]):
        M2 = oracle.M2_from_sigma(1.0, sigma[b])
        Cc = oracle.collision_chebyshev(q, W, f[b], K)[0] * M2
        Ce = oracle.collision_tensor(q, W, f[b]) * M2
        if project:
            Cc, _ = oracle.project(g["E"], g["h"], f[b], Cc)
            Ce, _ = oracle.project(g["E"], g["h"], f[b], Ce)
        out.append(Cc)
        exact.append(Ce)
    return np.array(out), np.array(exact)


# sizes cover one and two 128-row tiles of M, every instance tile width (64 ..
# 256, and 256 + 64), and K = 8 with an odd bracket count (a padded k block)
@pytest.mark.parametrize("N,B,K", [(20, 1, 16), (48, 70, 8), (65, 3, 8), (64, 130, 32),
                                   (150, 5, 16), (40, 300, 16), (33, 190, 32)])
def test_chebyshev_loss_matches_oracle(env, N, B, K):
    """loss_terms = K: the loss rate as the GEMM M (N x (N-1)K) Y against the
    oracle's Chebyshev expansion with the same K, and against the exact oracle
    (the truncation bound of these inputs is far below the tolerance)."""
    kx, ctx, torch = env
    rng = np.random.default_rng(500 + N + K)
    q = ki.log_grid(N, 1e-3, 1e2)
    f = ki.batch_bimodal(rng, q, B)
    sig = rng.uniform(0.3, 3.0, size=B)
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32, loss_terms=K)
    fd = torch.as_tensor(f, device="cuda")
    picks = sorted(set([0, B - 1, B // 2] + list(rng.integers(0, B, 3))))
    for project in (0, 1):
        C, d = ctx.collision(k, fd, sig, project=bool(project), diag=True)
        C = C.cpu().numpy()
        Cc, Ce = oracle_cheb_rows(q, f[picks], sig[picks], project, K)
        for r, b in enumerate(picks):
            scale = np.max(np.abs(Cc[r]))
            assert np.max(np.abs(C[b] - Cc[r])) / scale <= TOL, (b, project)
            assert np.max(np.abs(C[b] - Ce[r])) / np.max(np.abs(Ce[r])) <= TOL, (b, project)
            assert d[b]["status"] == 0
    k.release()


def test_chebyshev_loss_falls_back_to_the_exact_loss(env):
    """An instance with a bracket beyond the truncation bound (zeros inside the
    support: the log floor makes |d| ~ 690) takes the exact loss: its C is
    bit-identical to the exact path's; the other instances of the batch keep
    the GEMM loss and are bit-identical alone and in the batch."""
    kx, ctx, torch = env
    N = 40
    q = ki.log_grid(N, 1e-3, 10.0)
    f = ki.batch_bimodal(np.random.default_rng(61), q, 5)
    f[2, 10:14] = 0.0
    sig = np.linspace(0.5, 2.0, 5)
    kc = ctx.build_kernel(q, precision=kx.SPLIT_TF32, loss_terms=16)
    ke = ctx.build_kernel(q, precision=kx.SPLIT_TF32)
    fd = torch.as_tensor(f, device="cuda")
    Cc, _ = ctx.collision(kc, fd, sig)
    Ce, _ = ctx.collision(ke, fd, sig)
    Cc, Ce = Cc.cpu().numpy(), Ce.cpu().numpy()
    np.testing.assert_array_equal(Cc[2], Ce[2])
    assert not np.array_equal(Cc[0], Ce[0])   # the others did take the GEMM loss
    for b in (0, 2, 4):
        Ca, _ = ctx.collision(kc, torch.as_tensor(f[b:b + 1], device="cuda"), sig[b:b + 1])
        np.testing.assert_array_equal(Ca.cpu().numpy()[0], Cc[b])
    Co = oracle_rows(q, f[2:3], sig[2:3], 1)
    assert np.max(np.abs(Cc[2] - Co[0])) / np.max(np.abs(Co[0])) <= TOL
    kc.release()
    ke.release()


def test_chebyshev_loss_full_size_configuration_sampled(env):
    """The batched configuration at full size (B = 512 on one N = 192 kernel)
    with loss_terms = 16: sampled instances against the oracle."""
    kx, ctx, torch = env
    c = ki.config3()
    q, f, sig = c["q"], c["f"], c["sigma"]
    picks = (0, 1, 255, 256, 511)
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32, loss_terms=16)
    C, d = ctx.collision(k, torch.as_tensor(f, device="cuda"), sig, project=True, diag=True)
    C = C.cpu().numpy()
    Co = oracle_rows(q, f[list(picks)], np.asarray(sig)[list(picks)], True)
    for r, b in enumerate(picks):
        assert np.max(np.abs(C[b] - Co[r])) / np.max(np.abs(Co[r])) <= TOL, b
        assert d[b]["status"] == 0
    k.release()


def test_chebyshev_loss_fixed_step_solve(env):
    """Fixed-step integration with the Chebyshev loss (K = 16) against the
    oracle's solve: element-wise at the mixed bound, moments to 1e-7."""
    kx, ctx, torch = env
    c = ki.config1()
    q = c["q"]
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q)
    f0 = ki.batch_bimodal(np.random.default_rng(34), q, 3)
    sig = np.array([0.7, 1.0, 1.3]) * c["sigma"]
    t_end = c["n_steps"] * c["h"]
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32, loss_terms=16)
    fd = torch.as_tensor(f0, device="cuda")
    res = ctx.solve(k, fd, sig, t_end=t_end, h0=c["h"], fixed_step=1)
    f = fd.cpu().numpy()
    for b in range(3):
        fo, ro = oracle.solve(q, W, f0[b], oracle.M2_from_sigma(1.0, sig[b]), t_end=t_end,
                              h0=c["h"], fixed_step=1)
        assert res[b]["status"] == 0 and res[b]["steps"] == c["n_steps"]
        assert np.max(np.abs(f[b] - fo)) / np.max(np.abs(fo)) <= TOL, b
        for w in (g["h"], g["h"] * g["E"]):
            assert abs(np.sum(w * f[b]) / np.sum(w * f0[b]) - 1) < 1e-7
    k.release()


def test_chebyshev_option_is_validated(env):
    kx, ctx, torch = env
    q = ki.log_grid(16, 1e-3, 10.0)
    for prec, K, code in ((kx.FP32, 16, kx.ENOTSUP), (kx.FP64, 8, kx.ENOTSUP), (kx.SPLIT_TF32, 12, kx.EINVAL)):
        with pytest.raises(kx.KxError) as ei:
            ctx.build_kernel(q, precision=prec, loss_terms=K)
        assert ei.value.code == code


# ------------------------------------------------- uneven batch, grouped ---
@pytest.mark.parametrize("loss_terms", [0, 16])
def test_grouped_solve_equals_per_grid_solves(env, loss_terms):
    """The uneven batch as one sequence of grouped launches (three grids, two
    with more than one 128-instance tile, one with two i tiles): every
    instance bit-identical to kx_solve on its own kernel, and sampled
    instances of every grid within the mixed bound of the oracle's solve."""
    kx, ctx, torch = env
    rng = np.random.default_rng(90 + loss_terms)
    sizes, Bs = (24, 40, 260), (130, 3, 2)
    grids = [ki.log_grid(n, 1e-3, 1e2) for n in sizes]
    f0 = [ki.batch_bimodal(rng, q, B) for q, B in zip(grids, Bs)]
    sig = [10.0 ** rng.uniform(-1, 0.5, B) for B in Bs]
    ks = [ctx.build_kernel(q, precision=kx.SPLIT_TF32, loss_terms=loss_terms) for q in grids]
    par = dict(t_end=0.5, h0=1e-3, rtol=1e-6, atol=1e-12, l1_tol=0.0)
    fd = [torch.as_tensor(f, device="cuda") for f in f0]
    res = ctx.solve_grouped(ks, fd, sig, **par)
    for g in range(3):
        fa = torch.as_tensor(f0[g], device="cuda")
        ra = ctx.solve(ks[g], fa, sig[g], **par)
        np.testing.assert_array_equal(fd[g].cpu().numpy(), fa.cpu().numpy())
        for b in range(Bs[g]):
            assert res[g][b]["status"] == 0 and res[g][b]["steps"] == ra[b]["steps"]
        W = oracle.kernel_tensor(grids[g]) if sizes[g] < 200 else None
        if W is not None:
            b = Bs[g] - 1
            fo, ro = oracle.solve(grids[g], W, f0[g][b], oracle.M2_from_sigma(1.0, sig[g][b]), **par)
            err = np.max(np.abs(fd[g].cpu().numpy()[b] - fo)) / np.max(fo)
            assert err <= 1e-4, (g, err)
    for k in ks:
        k.release()


@pytest.mark.parametrize("N,B", [(96, 200), (260, 40)])
def test_split_tuning_is_result_neutral(env, N, B):
    """The split path's timed launch choices (GEMM ring depth, f' staging,
    instances per lane of the exact loss) change no bit of C: the result with
    the default rule, on the call that times the choices, and with the chosen
    ones are identical, for the exact and the Chebyshev loss; the choices are
    recorded as timed."""
    kx, ctx, torch = env
    q = ki.log_grid(N, 1e-3, 1e2)
    f = ki.batch_bimodal(np.random.default_rng(70 + N), q, B)
    sig = 10.0 ** np.random.default_rng(71).uniform(-1, 1, B)
    fd = torch.as_tensor(f, device="cuda")
    for lt in (0, 16):
        k = ctx.build_kernel(q, precision=kx.SPLIT_TF32, loss_terms=lt)
        ctx.set_split_tuning(False)
        C0 = ctx.collision(k, fd, sig)[0].cpu().numpy()
        assert ctx.split_tuning(k, B)["tuned"] == 0
        ctx.set_split_tuning(True)
        C1 = ctx.collision(k, fd, sig)[0].cpu().numpy()
        C2 = ctx.collision(k, fd, sig)[0].cpu().numpy()
        np.testing.assert_array_equal(C1, C0)
        np.testing.assert_array_equal(C2, C0)
        t = ctx.split_tuning(k, B)
        assert t["tuned"] & 1 and t["gain_S"] >= 2
        assert (t["tuned"] & 2) if lt else (t["tuned"] & 4)
        k.release()


@pytest.mark.parametrize("N", [60, 100, 192, 256, 300])
def test_gain_operand_placement_is_result_neutral(env, N):
    """The gain GEMM's generated A operand (f'_n f'_m, hi and lo) read by the
    MMAs from tensor memory or from shared memory: the same MMAs in the same
    order, so C is bit-identical; N spans the tensor-memory layouts (two
    accumulators and the A stages after them, A stages in the gaps after two
    256-column accumulators, one accumulator) and two i tiles (N = 300)."""
    kx, ctx, torch = env
    q = ki.log_grid(N, 1e-3, 1e2)
    B = 150
    f = ki.batch_bimodal(np.random.default_rng(90 + N), q, B)
    sig = 10.0 ** np.random.default_rng(91).uniform(-1, 1, B)
    fd = torch.as_tensor(f, device="cuda")
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32)
    ctx.set_split_tuning(False)
    out = {}
    try:
        for where in ("shared", "tensor"):
            ctx.set_gain_operand(where)
            out[where] = ctx.collision(k, fd, sig)[0].cpu().numpy()
            assert ctx.split_tuning(k, B)["gain_atm"] == (where == "tensor")
    finally:
        ctx.set_gain_operand("any")
        ctx.set_split_tuning(True)
    np.testing.assert_array_equal(out["tensor"], out["shared"])
    if N <= 192:
        Co = oracle_rows(q, f[:2], sig[:2], 1)
        err = np.max(np.abs(out["tensor"][:2] - Co)) / np.max(np.abs(Co))
        assert err <= TOL, err
    k.release()


@pytest.mark.parametrize("eta", [1, -1])
@pytest.mark.parametrize("N,B", [(24, 3), (40, 70), (100, 33)])
def test_quantum_statistics_split_path_matches_oracle(env, eta, N, B):
    """The split path with the Bose-Einstein / Fermi-Dirac factor (eq.
    Lambda_quantum): the gain GEMM times (1 + eta f_i) plus the exact loss
    kernel's three row sums (sum S f~, sum S f~ (f_n + f_m), sum S f~ f_n f_m);
    C raw and projected within the mixed-precision bound of the oracle on
    bimodal f of occupations of order one, instances bit-identical alone and in
    the batch, the equilibrium of the statistics near its fixed point, and the
    Chebyshev loss refused with these factors."""
    kx, ctx, torch = env
    q = ki.log_grid(N, 1e-2, 20.0)
    g = oracle.grid(q)
    W = oracle.kernel_tensor(q)
    f = 0.8 * ki.batch_bimodal(np.random.default_rng(140 + N + eta), q, B)
    sig = np.random.default_rng(141).uniform(0.3, 3.0, B)
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32, stats=eta)
    fd = torch.as_tensor(f, device="cuda")
    picks = sorted({0, B // 2, B - 1})
    for project in (0, 1):
        C = ctx.collision(k, fd, sig, project=bool(project))[0].cpu().numpy()
        for b in picks:
            Co = oracle.collision_tensor_stats(q, W, f[b], eta) * oracle.M2_from_sigma(1.0, sig[b])
            if project:
                Co, _ = oracle.project(g["E"], g["h"], f[b], Co)
            err = np.max(np.abs(C[b] - Co)) / np.max(np.abs(Co))
            assert err <= TOL, (project, b, err)
        if project:
            b = picks[-1]
            C1 = ctx.collision(k, torch.as_tensor(f[b:b + 1], device="cuda"), sig[b:b + 1], project=True)[0]
            np.testing.assert_array_equal(C1.cpu().numpy()[0], C[b])
    feq = 1.0 / (np.exp((g["E"] - 0.6) / 0.7) - eta)
    C = ctx.collision(k, torch.as_tensor(feq[None], device="cuda"), np.array([1.0]), project=False)[0]
    Co = oracle.collision_tensor_stats(q, W, feq, eta) * oracle.M2_from_sigma(1.0, 1.0)
    _, G, _ = oracle.collision_tensor(q, W, feq, parts=True)
    # the row's four sums ((1 + eta f) G, f L, f P, Q) are each up to (1 + f_max)^2
    # times the dilute gain and carry their own FP32 rounding before they cancel
    scale = oracle.M2_from_sigma(1.0, 1.0) * np.max(G) * (1.0 + np.max(np.abs(feq))) ** 2
    assert np.max(np.abs(C.cpu().numpy()[0] - Co)) <= 1e-5 * scale
    k.release()
    with pytest.raises(kx.KxError):
        ctx.build_kernel(q, precision=kx.SPLIT_TF32, stats=eta, loss_terms=16)


@pytest.mark.parametrize("eta", [1, -1])
def test_quantum_statistics_split_path_fixed_step_solve(env, eta):
    """Twenty fixed Heun steps with Bose-Einstein (Fermi-Dirac: f scaled below
    one) factors on the split path against the same steps taken with the
    oracle's operator and projection; number and energy conserved to the
    mixed-precision bound."""
    kx, ctx, torch = env
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
    k = ctx.build_kernel(q, precision=kx.SPLIT_TF32, stats=eta)
    fd = torch.as_tensor(f0[None], device="cuda")
    res = ctx.solve(k, fd, c["sigma"], t_end=steps * h, h0=h, fixed_step=1)
    f = fd.cpu().numpy()[0]
    assert res[0]["status"] == 0 and res[0]["steps"] == steps
    err = np.max(np.abs(f - fo)) / np.max(np.abs(fo))
    assert err <= TOL, err
    for w in (g["h"], g["h"] * g["E"]):
        assert abs(np.sum(w * f) / np.sum(w * f0) - 1) < 1e-7
    k.release()


def test_grouped_solve_with_quantum_statistics_equals_per_grid_solves(env):
    """Two grids with Bose-Einstein factors in one grouped solve: every
    instance bit-identical to kx_solve on its own kernel."""
    kx, ctx, torch = env
    rng = np.random.default_rng(160)
    sizes, Bs = (24, 40), (5, 3)
    grids = [ki.log_grid(n, 1e-2, 20.0) for n in sizes]
    f0 = [0.8 * ki.batch_bimodal(rng, q, B) for q, B in zip(grids, Bs)]
    sig = [10.0 ** rng.uniform(-1, 0.5, B) for B in Bs]
    ks = [ctx.build_kernel(q, precision=kx.SPLIT_TF32, stats=1) for q in grids]
    par = dict(t_end=0.3, h0=1e-3, rtol=1e-6, atol=1e-12, l1_tol=0.0)
    fd = [torch.as_tensor(f, device="cuda") for f in f0]
    res = ctx.solve_grouped(ks, fd, sig, **par)
    for g in range(len(sizes)):
        fa = torch.as_tensor(f0[g], device="cuda")
        ra = ctx.solve(ks[g], fa, sig[g], **par)
        np.testing.assert_array_equal(fd[g].cpu().numpy(), fa.cpu().numpy())
        for b in range(Bs[g]):
            assert res[g][b]["status"] == 0 and res[g][b]["steps"] == ra[b]["steps"]
    for k in ks:
        k.release()
