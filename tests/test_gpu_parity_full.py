"""GPU parity at the full sizes the bench and the large workloads run, and on caller-supplied
Jacobians.

Two kinds of comparison:
  * the context's own Jacobian (FP32 Taylor-mode recurrences) against the FP64 oracle: bounded by
    the FP32 rounding of J, so the tolerances are those of the FP32 path (1e-5 for a matvec);
  * a Jacobian handed to both sides (ngd_set_jacobian): the oracle computes J in FP64, the test
    rounds it to FP32 (a test-side operation on the oracle's output), and both sides then apply
    G = J32^T W J32 to the same inputs, so every remaining difference is the arithmetic of the
    kernels: double-float sums (~2^-48 per operation) against FP64.
Element-wise checks bound each entry by the magnitude of its own terms, (|J|^T (w |J| |v|))_k, so
that an error confined to a few entries (a wrong ragged tile, a column-split boundary) cannot hide
in a norm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gramian, mlp, nystrom, philox, solve  # noqa: E402
from paper_2505_11638_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def ngd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_11638_gb300 import build
    build.build()
    from paper_2505_11638_gb300 import ngd as _ngd
    _ngd.lib()
    return _ngd


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    return t.double().cpu().numpy()


def workload(name, n_int=None, n_bnd=None):
    wl, ths = inputs.make_workload(name, seed=0)
    pr = wl.problems[0]
    if n_int is not None:
        pr = inputs.subsample(pr, n_int, n_bnd)
    return wl, pr, ths[0]


def termwise_bound(J, w, v, mu):
    """Entry k of |J|^T (w |J| |v|) + mu |v|: the sum of the magnitudes of the terms of y_k."""
    A = np.abs(J)
    return A.T @ (w * (A @ np.abs(v))) + mu * np.abs(v)


def round32(J):
    return J.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("name,n_int,n_bnd", [("poisson10d", 1200, 300), ("heat4d", 450, 150)])
def test_two_pass_matvec_large_p(ngd, name, n_int, n_bnd):
    """p > 9216 (51073 and 133121 parameters): the stored-J matvec of an F32 context runs the row
    pass k_rowdot_df and the column pass k_coldot_df.  (i) With its own FP32 Jacobian: against the
    oracle's FP64 G at 1e-5, and every entry within 2e-5 of its term magnitude.  (ii) With the
    oracle's Jacobian rounded to FP32 given to both sides: every entry within 1e-12 of its term
    magnitude (double-float sums against FP64)."""
    wl, pr, th = workload(name, n_int, n_bnd)
    J = mlp.jacobian(pr, th)
    assert pr.p > 9216
    ctx = ngd.Context(pr, dtype="f32")
    rng = np.random.default_rng(21)
    mu = 1e-4
    v = rng.standard_normal(pr.p)
    y = host(ctx.gramian_mv(dev(th), dev(v), mu))
    y_o = gramian.gramian_mv(J, pr.w, v, mu)
    bound = termwise_bound(J, pr.w, v, mu)
    assert rel(y, y_o) <= 1e-5
    assert np.all(np.abs(y - y_o) <= 2e-5 * bound)
    J32 = round32(J)
    ctx.set_jacobian(dev(J32, torch.float32))
    for mu2 in [mu, 0.0]:
        v = rng.standard_normal(pr.p)
        y = host(ctx.gramian_mv(None, dev(v), mu2))
        y_o = gramian.gramian_mv(J32, pr.w, v, mu2)
        err = np.abs(y - y_o) / termwise_bound(J32, pr.w, v, mu2)
        assert err.max() <= 1e-12, (mu2, err.max(), int(err.argmax()))
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "df"])
def test_gramian_mm_fp64_accurate_exact_jacobian(ngd, prec):
    """Y = G V through ngd_gramian_mm in the FP64-accurate arithmetic of an F32 context (f64: the
    tensor-core digit-plane products; df: double-float on the FP32 pipes), for V and J given to
    both sides (5-D Poisson, 1500 points, ell = 130: ragged 128-wide tiles, N and p not multiples
    of the 128-row tiles or of the 256-long K-chunks): against FP64 at 1e-12 in norm, each entry
    within 1e-11 of its term magnitude; the Nystrom core V^T G V symmetric to 1e-12."""
    wl, pr, th = workload("poisson5d", 1200, 300)
    J32 = round32(mlp.jacobian(pr, th))
    ctx = ngd.Context(pr, dtype="f32")
    ctx.set_jacobian(dev(J32, torch.float32))
    ell = 130
    V = round32(nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 9, 2)))
    Y = host(ctx.gramian_mm(None, dev(V.T, torch.float32), prec)).T
    Y_o = J32.T @ (pr.w[:, None] * (J32 @ V))
    B = np.abs(J32).T @ (pr.w[:, None] * (np.abs(J32) @ np.abs(V)))
    assert rel(Y, Y_o) <= 1e-12
    assert (np.abs(Y - Y_o) / B).max() <= 1e-11
    M = V.T @ Y
    assert np.linalg.norm(M - M.T) / np.linalg.norm(M) <= 1e-12
    ctx.close()


def test_fused_pcg_headline_size_exact_jacobian(ngd):
    """The 5-D Poisson workload at its full size (N = 5000, p = 8769) and the bench's rank
    ell = 500, on the oracle's Jacobian rounded to FP32 (both sides).
    Factor: both sides factor the same Omega and Y.  lambda_hat agrees to 1e-8 on its leading part;
    P^{-1} v agrees to the rounding of the double-float factor seen through the preconditioner:
    (lam_ell + mu) / (lam + mu) has slope 1/mu near lam = 0, so an error 2^-48 |G| in the computed
    Nystrom approximation moves P^{-1} by up to ~2^-48 lambda_1 / mu (bound: 64 times that).
    pCG: the whole solve in one cooperative kernel (U staged through shared memory in chunks, row
    pass over the stored J), given the oracle's U and lambda, against FP64 pCG at 1, 2 and 3
    iterations (mu = 1e-7 resolves the system to ~1e-11 in 3).  The kernel holds U as an FP32 pair
    (48 bits) and its sums in double-float, and P^{-1} g cancels heavily here: g lies in the span
    of U to 3e-7, and (I - U U^T) g is what remains.  The reference scale of that rounding is the
    change of the FP64 oracle's own direction when U is rounded to an FP32 pair (a test-side
    operation on the oracle's U; 1.5e-8 at one iteration); the kernel's directions agree within 32
    times that (a 2^-47 relative perturbation of every matvec alone moves them by 2e-10).  To
    tolerance at mu = 1e-13 (65 iterations): the true residual under the oracle's operator."""
    wl, pr, th = workload("poisson5d")
    J32 = round32(mlp.jacobian(pr, th))
    g_o, _, _ = mlp.gradient(pr, th)
    G = J32.T @ (pr.w[:, None] * J32)
    ell = 500
    Om = round32(nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 0, 0)))
    Y = G @ Om
    U_o, lam_o, nu_o = nystrom.nystrom_factor(Om, Y, nystrom.MANTISSA_BITS["df"])
    ctx = ngd.Context(pr, dtype="f32")
    ctx.set_jacobian(dev(J32, torch.float32))
    U, lam, nu = ctx.nystrom_factor(ell, dev(Om.T, torch.float32), dev(Y.T), prec="f64")
    assert abs(nu - nu_o) <= 1e-12 * nu_o
    lam_g = host(lam)
    top = lam_o > 1e-6 * lam_o[0]
    assert rel(lam_g[top], lam_o[top]) <= 1e-8
    rng = np.random.default_rng(23)
    for mu in [1e-4, 1e-7]:
        v = rng.standard_normal(pr.p)
        z = host(ctx.precond_apply(ell, U, lam, mu, dev(v)))
        z_o = nystrom.precond_apply(U_o, lam_o, mu, v)
        assert rel(z, z_o) <= max(1e-10, 64 * 2.0 ** -48 * lam_o[0] / mu), (mu, rel(z, z_o))
    g = dev(g_o)
    U_d, lam_d = dev(U_o.T), dev(lam_o)
    mu = 1e-7
    hi = round32(U_o)
    U48 = hi + round32(U_o - hi)                 # U as the kernel holds it: an FP32 pair
    for k in [1, 2, 3]:
        d, it, rr = ctx.pcg_solve(None, g, mu, U_d, lam_d, ell, rtol=0.0, maxit=k)
        d_o, it_o, rr_o = solve.pcg(lambda v: G @ v + mu * v, g_o,
                                    lambda v: nystrom.precond_apply(U_o, lam_o, mu, v), 0.0, k)
        d_48, _, _ = solve.pcg(lambda v: G @ v + mu * v, g_o,
                               lambda v: nystrom.precond_apply(U48, lam_o, mu, v), 0.0, k)
        tol = max(1e-9, 32 * rel(d_48, d_o))
        assert it == it_o == k
        assert rel(host(d), d_o) <= tol, (k, rel(host(d), d_o), tol)
    mu = 1e-13
    d, it, rr = ctx.pcg_solve(None, g, mu, U_d, lam_d, ell, rtol=1e-6, maxit=1000)
    res = G @ host(d) + mu * host(d) - g_o
    assert rr <= 1e-6 and np.linalg.norm(res) <= 2e-6 * np.linalg.norm(g_o)
    ctx.close()


def test_ngd_step_headline_size(ngd):
    """One NGD step of the bench workload as the bench runs it (N = 5000, p = 8769, ell = 500,
    mu = 1e-7, FP64-accurate sketch, the context's own FP32 Jacobian) at fixed PCG iteration
    counts, against the oracle's FP64 step with the same Philox test matrix and the same shift
    format: loss, lambda_1, step length and update agree to the FP32 rounding of J; the direction
    solves the oracle's FP64 system to that accuracy."""
    wl, pr, th = workload("poisson5d")
    J = mlp.jacobian(pr, th)
    g_o, _, _ = mlp.gradient(pr, th)
    ctx = ngd.Context(pr, dtype="f32")
    for k in [2, 5]:
        t = dev(th)
        info = ctx.step(t, ell=500, mu=1e-7, rtol=0.0, maxit=k, seed=0, step=0, sketch="f64")
        th1_o, info_o = solve.ngd_step(pr, th, ell=500, mu=1e-7, rtol=0.0, maxit=k, seed=0, step=0,
                                       mant_bits=nystrom.MANTISSA_BITS["df"])
        assert info["pcg_iters"] == info_o.pcg_iters == k
        assert abs(info["loss_before"] - info_o.loss_before) <= 1e-5 * info_o.loss_before
        assert abs(info["lam1"] - info_o.lam1) <= 1e-5 * info_o.lam1
        assert info["alpha"] == info_o.alpha
        assert info["loss_after"] < info["loss_before"]
        upd = th - host(t)
        assert rel(upd, th - th1_o) <= 2e-3, (k, rel(upd, th - th1_o))
        d = upd / info["alpha"]
        res = J.T @ (pr.w * (J @ d)) + 1e-7 * d - g_o
        assert np.linalg.norm(res) <= 1e-3 * np.linalg.norm(g_o)
    ctx.close()


def test_fused_pcg_small_exact_jacobian_tight(ngd):
    """The fused PCG on a 1120-point subset (ell = 60, mu = 1e-5) with the oracle's Jacobian rounded
    to FP32 on both sides: the direction agrees with FP64 pCG at fixed iteration counts to 1e-8,
    three orders below the FP32-Jacobian tolerance the context's own J allows."""
    wl, pr, th = workload("poisson5d", 900, 220)
    J32 = round32(mlp.jacobian(pr, th))
    G = J32.T @ (pr.w[:, None] * J32)
    g_o, _, _ = mlp.gradient(pr, th)
    ell, mu = 60, 1e-5
    Om = nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 5, 0))
    U_o, lam_o, _ = nystrom.nystrom_factor(Om, G @ Om)
    ctx = ngd.Context(pr, dtype="f32")
    ctx.set_jacobian(dev(J32, torch.float32))
    g = dev(g_o)
    for udt in [torch.float64, torch.float32]:
        U_d = dev(U_o.T, udt)
        U_p = host(U_d).T
        for k in [1, 5, 20, 60]:
            d, it, rr = ctx.pcg_solve(None, g, mu, U_d, dev(lam_o), ell, rtol=0.0, maxit=k)
            d_o, it_o, _ = solve.pcg(lambda v: G @ v + mu * v, g_o,
                                     lambda v: nystrom.precond_apply(U_p, lam_o, mu, v), 0.0, k)
            assert it == it_o == k
            assert rel(host(d), d_o) <= 1e-8, (udt, k, rel(host(d), d_o))
    ctx.close()


@pytest.mark.parametrize("prec", ["tf32", "f64"])
def test_tensor_core_wait_timeout_recovers(ngd, prec):
    """Failure detection of the tcgen05 kernels (tf32: the rounded-operand GEMM; f64: the
    digit-plane GEMM): with a one-cycle wait limit every role's first wait runs out before its
    TMA loads land; the kernel drains what it issued, stores nothing, frees its tensor memory and
    the call reports TIMEOUT.  With the default limit restored the same context computes the same
    sketch as a fresh context."""
    wl, pr, th = workload("poisson5d", 700, 180)
    ctx = ngd.Context(pr, dtype="f32")
    t = dev(th)
    ngd.ngd_set_wait_limit(ctx.handle, 1)
    with pytest.raises(ngd.NGDError) as e:
        ctx.nystrom_sketch(t, 130, seed=3, step=1, prec=prec)
    assert e.value.name == "TIMEOUT"
    ngd.ngd_set_wait_limit(ctx.handle, 4_000_000_000)
    Om, Y = ctx.nystrom_sketch(t, 130, seed=3, step=1, prec=prec)
    ref = ngd.Context(pr, dtype="f32")
    Om2, Y2 = ref.nystrom_sketch(dev(th), 130, seed=3, step=1, prec=prec)
    assert torch.equal(Om, Om2) and torch.equal(Y, Y2)
    ref.close()
    ctx.close()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_test_matrix_single_cholesky_qr_pass(ngd, dtype, tol):
    """ell <= p / 16 (here 500 of 8769): one CholeskyQR pass orthonormalizes the Gaussian test
    matrix (condition number <= 5/3); the result is the thin QR factor of the oracle's Philox
    matrix to the working precision, and orthonormal to a few units of it."""
    wl, pr, th = workload("poisson5d", 300, 80)
    ctx = ngd.Context(pr, dtype=dtype)
    Om, Y = ctx.nystrom_sketch(dev(th), 500, seed=17, step=4, prec="f64")
    O = host(Om).T
    Om_o = nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, 500, 17, 4))
    assert rel(O, Om_o) <= tol
    assert np.abs(O.T @ O - np.eye(500)).max() <= 5 * tol
    ctx.close()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 5e-5)])
def test_matrix_free_vjp_heat_width_256(ngd, dtype, tol):
    """The matrix-free VJP (reverse of the Taylor-mode forward by layers: per-layer weight adjoints
    as GEMMs over points and channels, no Jacobian rows) on the 4-D heat network at 300 interior +
    100 boundary/initial points: FP32 with the workload's widths 256 (p = 133121), FP64 with widths
    64 (the FP64 Taylor kernels stage fewer points of a 256-wide network than they need).  With the
    stored Taylor coefficients (budget 0) and with a one-byte budget (the forward recomputed per
    chunk of points), through the autograd function and through ngd_vjp, against the oracle's VJP;
    the matrix-free Gramian matvec (JVP then this VJP) against the oracle's explicit Jacobian."""
    wl, pr, th = workload("heat4d", 300, 100)
    if dtype == "f64":
        pr, th = inputs.small_problem(pde="heat", d=4, widths=[4, 64, 64, 64, 1], n_int=300, n_bnd=100, seed=33)
    J = mlp.jacobian(pr, th)
    rng = np.random.default_rng(31)
    c = rng.standard_normal(pr.n)
    g_o = mlp.vjp(pr, th, c)
    v = rng.standard_normal(pr.p)
    y_o = gramian.gramian_mv(J, pr.w, v, 1e-3)
    for budget in [0, 1]:
        ctx = ngd.Context(pr, dtype=dtype, gv_mode="matrix_free", mem_budget=budget)
        t = dev(th).requires_grad_(True)
        r = ngd.PinnResidual.apply(t, ctx)
        (r * dev(c)).sum().backward()
        assert rel(host(t.grad), g_o) <= tol, (budget, rel(host(t.grad), g_o))
        assert rel(host(ctx.vjp(dev(th), dev(c))), g_o) <= tol
        y = host(ctx.gramian_mv(dev(th), dev(v), 1e-3))
        assert rel(y, y_o) <= (1e-10 if dtype == "f64" else 1e-5), (budget, rel(y, y_o))
        ctx.close()


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-11), ("f64", 2e-11)])
def test_gramian_full_matches_oracle(ngd, dtype, tol):
    """The explicit Gramian NGD full factors (ngd_gramian_full) on a Jacobian handed to both sides:
    the FP32 context forms it on the tensor cores from six-digit BF16 planes of the column-scaled
    J^T and (diag(w) J)^T, the FP64 context by the double-float GEMM on the lower triangle; the
    oracle computes J^T diag(w) J of the same J in FP64.  p = 1217 (10 x 13 output tiles, the last
    ragged), N = 1800 (eight K chunks of 256, the last ragged).  Each entry is bounded against
    sqrt(G_jj G_kk) (Cauchy-Schwarz: the scale of the entry's terms), the whole matrix in norm, and
    the result must be symmetric.  Bounds: the digit planes keep ~2^-46 of a column's largest
    term; the double-float GEMM holds FP64 operands as FP32 pairs (48 bits), ~2^-44 per product,
    so 1800 terms of random sign leave a few 1e-12 in the largest of 1.5e6 entries."""
    pr, th = inputs.small_problem(d=3, widths=[3, 32, 32, 1], n_int=1500, n_bnd=300, seed=97)
    assert th.size == 1217 and pr.n == 1800
    J = mlp.jacobian(pr, th)
    Jd = round32(J) if dtype == "f32" else J
    ctx = ngd.Context(pr, dtype=dtype)
    ctx.residual(dev(th))
    ctx.set_jacobian(dev(Jd, torch.float32 if dtype == "f32" else torch.float64))
    G = host(ctx.gramian_full(None))
    G_o = Jd.T @ (pr.w[:, None] * Jd)
    dg = np.sqrt(np.diag(G_o))
    err = np.abs(G - G_o) / np.maximum(np.outer(dg, dg), 1e-300)
    assert err.max() <= tol, (err.max(), np.unravel_index(int(err.argmax()), err.shape))
    assert rel(G, G_o) <= tol / 20
    assert np.array_equal(G, G.T)
    ctx.close()


@pytest.mark.parametrize("widths,n_int,n_bnd", [
    ([3, 32, 32, 1], 8000, 1800),    # p = 1217, 39 K chunks: one-chunk slices, partials reduced
    ([3, 60, 60, 1], 2400, 600),     # p = 3961, 12 K chunks: one slice, written by the GEMM itself
])
def test_gramian_full_tensor_core_layouts(ngd, widths, n_int, n_bnd):
    """The tensor-core Gramian's other two work layouts against the oracle's J^T diag(w) J of the
    same FP32-rounded J.  The GEMM runs only the output tiles that hold an entry on or below the
    diagonal.  p = 1217 with N = 9800: 76 of 130 tiles, 39 one-chunk K slices whose partials the
    reduction adds in order; p = 3961 with N = 3000: 672 of 1302 tiles, one slice of all 12 chunks
    summed by each CTA in order (double-float running sums), scaled and written by the GEMM's
    epilogue (no partials).  Bounds as in test_gramian_full_matches_oracle for the FP32 context."""
    pr, th = inputs.small_problem(d=3, widths=widths, n_int=n_int, n_bnd=n_bnd, seed=53)
    J = round32(mlp.jacobian(pr, th))
    ctx = ngd.Context(pr, dtype="f32")
    ctx.residual(dev(th))
    ctx.set_jacobian(dev(J, torch.float32))
    G = host(ctx.gramian_full(None))
    G_o = J.T @ (pr.w[:, None] * J)
    dg = np.sqrt(np.diag(G_o))
    err = np.abs(G - G_o) / np.maximum(np.outer(dg, dg), 1e-300)
    assert err.max() <= 1e-11, (err.max(), np.unravel_index(int(err.argmax()), err.shape))
    assert rel(G, G_o) <= 5e-13
    assert np.array_equal(G, G.T)
    ctx.close()


def test_factor_wide_core_matches_oracle(ngd):
    """The FP64-accurate factor of an FP32 context at l = 700: its core is wide enough that the
    compact-WY back-transform passes the rows of each block of reflectors through shared memory in
    two chunks (the l = 500 core of the bench fits in one), the double-float tridiagonalization
    holds five columns of B^T B per block, and the tensor-core products cut K = p into 35 chunks
    over 8 x 8 lower tiles.  Eigenvalues and the preconditioner apply against the oracle's factor of
    the same FP32-rounded Omega and FP64 Y (double-float shift), as in
    test_factor_and_preconditioner_match_oracle[f32-f64]."""
    wl, pr, th = workload("poisson5d", 600, 150)
    ell = 700
    J = mlp.jacobian(pr, th)
    Om_o = nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 11, 0))
    ctx = ngd.Context(pr, dtype="f32")
    Om_d = torch.tensor(Om_o.T.copy(), dtype=torch.float32, device="cuda")
    Om_r = host(Om_d).T
    Y_r = J.T @ (pr.w[:, None] * (J @ Om_r))
    Y_d = torch.tensor(Y_r.T.copy(), dtype=torch.float64, device="cuda")
    U, lam, nu = ctx.nystrom_factor(ell, Om_d, Y_d, prec="f64")
    U_o, lam_o, nu_o = nystrom.nystrom_factor(Om_r, host(Y_d).T, nystrom.MANTISSA_BITS["df"])
    assert abs(nu - nu_o) <= 1e-12 * nu_o
    lam_g = host(lam)
    top = lam_o > 1e-6 * lam_o[0]
    assert np.all(np.diff(lam_g) <= 0)
    assert rel(lam_g[top], lam_o[top]) <= 1e-8
    mu = 1e-4
    rng = np.random.default_rng(5)
    for _ in range(2):
        v = rng.standard_normal(pr.p)
        z = host(ctx.precond_apply(ell, U, lam, mu, dev(v)))
        z_o = nystrom.precond_apply(U_o, lam_o, mu, v)
        assert rel(z, z_o) <= 1e-8
    ctx.close()


def test_ngd_full_step_fp32_tensor_core_cholesky(ngd):
    """NGD full in an FP32 context at p = 1217: the blocked Cholesky of G + mu I (256-column
    diagonal blocks, a ragged last one of 193) with its trailing updates on the digit-plane
    tensor-core GEMM (panel rows split into six digits, lower tiles, the product subtracted by the
    GEMM's epilogue).  The step's direction solves (G + mu I) d = g, with the context's own G at
    theta (ngd_gramian_full, pinned against the oracle by the test_gramian_full tests) and its own
    gradient, to a backward error of 1e-10, and the step decreases the loss."""
    pr, th = inputs.small_problem(d=3, widths=[3, 32, 32, 1], n_int=1500, n_bnd=300, seed=97)
    assert th.size == 1217
    ctx = ngd.Context(pr, dtype="f32")
    t = dev(th)
    G = host(ctx.gramian_full(t))
    g, _, _ = ctx.gradient(t)
    g = host(g)
    info = ctx.step(t, precond="full", ell=1, mu=1e-6, seed=3, step=0, sketch="f64")
    assert info["loss_after"] < info["loss_before"] and info["alpha"] > 0
    d = (th - host(t)) / info["alpha"]
    res = G @ d + info["mu"] * d - g
    assert np.linalg.norm(res) <= 1e-10 * (np.linalg.norm(G, 2) * np.linalg.norm(d) + np.linalg.norm(g))
    ctx.close()
