"""GPU parity: every step of the hot path through the C ABI against the FP64 oracle.

Tolerances (relative 2-norm unless noted):
  FP64 path: residual/gradient/JVP/VJP 1e-11, Gramian matvec 1e-10 (the stated target),
             preconditioned direction 1e-6 at a fixed iteration count.
  FP32 path: residual/JVP/VJP 2e-5 (FP32 Taylor recurrences over <= 5 layers), Gramian matvec
             1e-5 (the stated target), Omega 1e-6.
  TF32 / BF16 sketch: 5e-3 / 4e-2 (operand rounding 2^-10 / 2^-8, error grows like sqrt(K) u).
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


def dev(x):
    return torch.tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def host(t):
    return t.double().cpu().numpy()


SMALL = [
    dict(pde="poisson", d=2, widths=[2, 7, 5, 1], n_int=37, n_bnd=11),     # ragged tiles, odd widths
    dict(pde="poisson", d=3, widths=[3, 16, 16, 16, 1], n_int=50, n_bnd=0),  # interior only
    dict(pde="poisson", d=2, widths=[2, 8, 1], n_int=0, n_bnd=9),            # boundary only, one hidden layer
    dict(pde="heat", d=4, widths=[4, 12, 9, 1], n_int=29, n_bnd=13),
    dict(pde="poisson", d=10, widths=[10, 20, 20, 1], n_int=21, n_bnd=5),    # 12 Taylor channels
    dict(pde="poisson", d=2, widths=[2, 3, 1], n_int=1, n_bnd=0),            # a single point
]


def small(case, seed=0):
    c = dict(case)
    pde = c.pop("pde")
    return inputs.small_problem(pde=pde, seed=seed, **c)


@pytest.mark.parametrize("case", range(len(SMALL)))
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_residual_gradient_jvp_vjp_small(ngd, case, dtype):
    pr, th = small(SMALL[case], seed=case)
    ctx = ngd.Context(pr, dtype=dtype)
    t = dev(th)
    r, loss = ctx.residual(t)
    r_o, L_o = mlp.residual(pr, th)
    tol = 1e-11 if dtype == "f64" else 2e-5
    assert rel(host(r), r_o) <= tol
    assert abs(loss - L_o) <= tol * max(abs(L_o), 1e-300)
    g, r2, loss2 = ctx.gradient(t)
    g_o = mlp.vjp(pr, th, pr.w * r_o)
    assert rel(host(g), g_o) <= (1e-11 if dtype == "f64" else 5e-5)
    rng = np.random.default_rng(case)
    v = rng.standard_normal(pr.p)
    c = rng.standard_normal(pr.n)
    assert rel(host(ctx.jvp(t, dev(v))), mlp.jvp(pr, th, v)) <= tol
    assert rel(host(ctx.vjp(t, dev(c))), mlp.vjp(pr, th, c)) <= (1e-11 if dtype == "f64" else 5e-5)
    ctx.close()


@pytest.mark.parametrize("case", [0, 3, 4])
@pytest.mark.parametrize("dtype,mode", [("f64", "stored"), ("f64", "matrix_free"), ("f32", "stored"),
                                        ("f32", "matrix_free")])
def test_gramian_mv_small(ngd, case, dtype, mode):
    pr, th = small(SMALL[case], seed=10 + case)
    ctx = ngd.Context(pr, dtype=dtype, gv_mode=mode)
    v = np.random.default_rng(1).standard_normal(pr.p)
    y = host(ctx.gramian_mv(dev(th), dev(v), 1e-3))
    y_o = gramian.gramian_mv(mlp.jacobian(pr, th), pr.w, v, 1e-3)
    assert rel(y, y_o) <= (1e-10 if dtype == "f64" else 1e-5)
    ctx.close()


def _workload(name, n_int=None, n_bnd=None):
    wl, ths = inputs.make_workload(name, seed=0)
    pr = wl.problems[0]
    if n_int is not None:
        pr = inputs.subsample(pr, n_int, n_bnd)
    return wl, pr, ths[0]


@pytest.mark.parametrize("name,dtype", [("poisson2d", "f64"), ("poisson5d", "f32")])
def test_gramian_mv_full_size(ngd, name, dtype):
    """The matvec at the full point sets of the two smaller workloads, J formed explicitly by the oracle."""
    wl, pr, th = _workload(name)
    ctx = ngd.Context(pr, dtype=dtype)
    rng = np.random.default_rng(2)
    J = mlp.jacobian(pr, th)
    for mu in [wl.mu, 0.0]:
        v = rng.standard_normal(pr.p)
        y = host(ctx.gramian_mv(dev(th) if mu == wl.mu else None, dev(v), mu))
        y_o = gramian.gramian_mv(J, pr.w, v, mu)
        assert rel(y, y_o) <= (1e-10 if dtype == "f64" else 1e-5), (name, mu)
    ctx.close()


@pytest.mark.parametrize("name", ["poisson10d", "heat4d"])
def test_large_workloads_sampled(ngd, name):
    """At the full sizes of the two large workloads: residuals and J rows on sampled points
    (the oracle evaluates those points one block at a time) and exact identities of the matvec."""
    wl, pr, th = _workload(name)
    ctx = ngd.Context(pr, dtype="f32")
    t = dev(th)
    r, loss = ctx.residual(t)
    rows = np.concatenate([np.arange(0, pr.n_int, pr.n_int // 40), pr.n_int + np.arange(0, pr.n_bnd, pr.n_bnd // 10),
                           [pr.n - 1]])
    sub = inputs.Problem(pr.name, pr.pde, pr.widths, pr.X[rows], pr.w[rows], pr.target[rows],
                         int(np.sum(rows < pr.n_int)), int(np.sum(rows >= pr.n_int)), pr.kappa, pr.freq)
    r_o, _ = mlp.residual(sub, th)
    assert rel(host(r)[rows], r_o) <= 2e-5
    rng = np.random.default_rng(3)
    v = rng.standard_normal(pr.p)
    jv = host(ctx.jvp(t, dev(v)))
    assert rel(jv[rows], mlp.jacobian(sub, th) @ v) <= 2e-5
    # Gramian identities at full size: v^T (G + mu I) v = sum_r w_r (J v)_r^2 + mu |v|^2, symmetry
    u = rng.standard_normal(pr.p)
    Gv = host(ctx.gramian_mv(t, dev(v), 1e-4))
    Gu = host(ctx.gramian_mv(None, dev(u), 1e-4))
    assert abs(v @ Gv - (np.sum(pr.w * jv * jv) + 1e-4 * v @ v)) <= 1e-5 * abs(v @ Gv)
    assert abs(u @ Gv - v @ Gu) <= 1e-5 * np.sqrt(abs(u @ Gu) * abs(v @ Gv))
    ctx.close()


def test_test_matrix_matches_oracle_philox(ngd):
    pr, th = small(SMALL[0], seed=20)
    for dtype, tol in [("f64", 1e-12), ("f32", 2e-6)]:
        ctx = ngd.Context(pr, dtype=dtype)
        ell = 9
        Om, Y = ctx.nystrom_sketch(dev(th), ell, seed=123456789012, step=5, prec=dtype)
        Om_o = nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 123456789012, 5))
        assert rel(host(Om).T, Om_o) <= tol, dtype
        ctx.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5), ("tf32", 5e-3), ("bf16", 4e-2)])
def test_sketch_matches_oracle(ngd, prec, tol):
    wl, pr, th = _workload("poisson5d", 700, 180) if prec != "f64" else _workload("poisson2d")
    dtype = "f64" if prec == "f64" else "f32"
    ctx = ngd.Context(pr, dtype=dtype)
    ell = 130 if prec != "f64" else 100      # not a multiple of the 128-wide tensor-core tile
    Om, Y = ctx.nystrom_sketch(dev(th), ell, seed=3, step=1, prec=prec)
    J = mlp.jacobian(pr, th)
    Om_o = nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 3, 1))
    Y_o = J.T @ (pr.w[:, None] * (J @ Om_o))
    assert rel(host(Y).T, Y_o) <= tol
    ctx.close()


@pytest.mark.parametrize("prec,sym_tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_sketch_core_symmetry_fp32_context(ngd, prec, sym_tol):
    """In an FP32 context the double-float sketch keeps Omega^T Y = Omega^T G Omega symmetric far
    below FP32 rounding: G = J^T W J of the stored FP32 Jacobian is an exactly symmetric operator.
    The FP32 pair carries 48 significant bits; its low word is summed in FP32 over the K = N
    products, so the error grows like K u32^2 (~1e-13 relative at N = 1120; FP64 BLAS: ~1e-15).
    FP32 arithmetic breaks the symmetry at its own rounding level."""
    wl, pr, th = _workload("poisson5d", 900, 220)
    ctx = ngd.Context(pr, dtype="f32")
    Om, Y = ctx.nystrom_sketch(dev(th), 96, seed=4, step=0, prec=prec)
    O, Yh = host(Om).T, host(Y).T
    M = O.T @ Yh
    assert np.linalg.norm(M - M.T) / np.linalg.norm(M) <= sym_tol
    J = mlp.jacobian(pr, th)
    assert rel(Yh, J.T @ (pr.w[:, None] * (J @ O))) <= 1e-5      # against the FP64 oracle Jacobian
    ctx.close()


@pytest.mark.parametrize("dtype,prec", [("f64", "f64"), ("f32", "f32"), ("f32", "f64")])
def test_factor_and_preconditioner_match_oracle(ngd, dtype, prec):
    wl, pr, th = _workload("poisson2d") if dtype == "f64" else _workload("poisson5d", 600, 150)
    ell = 60
    J = mlp.jacobian(pr, th)
    Om_o = nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 11, 0))
    Y_o = J.T @ (pr.w[:, None] * (J @ Om_o))
    ctx = ngd.Context(pr, dtype=dtype)
    wd = torch.float64 if dtype == "f64" else torch.float32
    Om_d = torch.tensor(Om_o.T.copy(), dtype=wd, device="cuda")
    # Y is float64 for the FP64-accurate factor; the oracle's Y is exact for the rounded Omega
    Om_r = host(Om_d).T
    Y_r = J.T @ (pr.w[:, None] * (J @ Om_r))
    Y_d = torch.tensor(Y_r.T.copy(), dtype=torch.float64 if prec == "f64" else wd, device="cuda")
    U, lam, nu = ctx.nystrom_factor(ell, Om_d, Y_d, prec=prec)
    # the oracle factors the same (rounded) inputs
    # an FP64-accurate factor in an FP32 context runs in double-float (48-bit spacing)
    mb = nystrom.MANTISSA_BITS["df" if (prec == "f64" and dtype == "f32") else prec]
    U_o, lam_o, nu_o = nystrom.nystrom_factor(Om_r, host(Y_d).T, mb)
    assert abs(nu - nu_o) <= 1e-12 * nu_o
    lam_g = host(lam)
    top = lam_o > 1e-6 * lam_o[0]
    assert np.all(np.diff(lam_g) <= 0)
    assert rel(lam_g[top], lam_o[top]) <= (1e-8 if prec == "f64" else 1e-4)
    mu = 1e-6 if dtype == "f64" else 1e-4
    rng = np.random.default_rng(4)
    for _ in range(3):
        v = rng.standard_normal(pr.p)
        z = host(ctx.precond_apply(ell, U, lam, mu, dev(v)))
        z_o = nystrom.precond_apply(U_o, lam_o, mu, v)
        # U is FP64 after an FP64-accurate factor; an F32 factor stores U in FP32
        assert rel(z, z_o) <= (1e-8 if prec == "f64" else 2e-3)
    # the preconditioner apply itself on identical factors is exact up to rounding
    U64 = torch.tensor(U_o.T.copy(), dtype=wd, device="cuda")
    z = host(ctx.precond_apply(ell, U64, dev(lam_o), mu, dev(v)))
    z_o = nystrom.precond_apply(host(U64).T, lam_o, mu, v)
    assert rel(z, z_o) <= 1e-12    # FP64 arithmetic, or double-float accumulation over FP32 U
    ctx.close()


@pytest.mark.parametrize("dtype,prec", [("f64", "f64"), ("f32", "f32"), ("f32", "f64")])
def test_factor_eigen_edge_sizes(ngd, dtype, prec):
    """The l x l eigen-solver at sizes that hit its edge cases: l = 1, 2 (no Householder step),
    3, around the 32-wide tiles of the tridiagonal reduction and, for FP32 contexts, around
    multiples of 16; an FP32 context's FP64-accurate factor (double-float reduction) to 1e-8."""
    pr, th = small(SMALL[3], seed=31)          # heat, p = 4*12+12+12*9+9+9+1 = 187
    J = mlp.jacobian(pr, th)
    G = J.T @ (pr.w[:, None] * J)
    ctx = ngd.Context(pr, dtype=dtype)
    wd = torch.float64 if dtype == "f64" else torch.float32
    yd = torch.float64 if prec == "f64" else wd
    # an FP64-accurate factor in an FP32 context runs in double-float (48-bit spacing)
    mb = nystrom.MANTISSA_BITS["df" if (prec == "f64" and dtype == "f32") else prec]
    tight = prec == "f64"
    rng = np.random.default_rng(8)
    sizes = [1, 2, 3, 31, 32, 33, 64, 65, 97] if dtype == "f64" else [1, 2, 3, 15, 16, 17, 31, 32, 33, 47, 64, 65, 97]
    for ell in sizes:
        Om = nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 17, ell))
        Om_d = torch.tensor(np.ascontiguousarray(Om.T), dtype=wd, device="cuda")
        Y_d = torch.tensor(np.ascontiguousarray((G @ host(Om_d).T).T), dtype=yd, device="cuda")
        # G has rank 42 here (42 residual rows), so for l > 42 the core's smallest eigenvalues
        # are the shift itself; as in the step, a core that the shifted Cholesky finds
        # indefinite is retried with 8x the shift (the oracle then factors with the same shift)
        for scale in [1.0, 8.0, 64.0, 512.0]:
            try:
                U, lam, nu = ctx.nystrom_factor(ell, Om_d, Y_d, prec=prec, shift_scale=scale)
                break
            except ngd.NGDError as err:
                assert "NOT_SPD" in str(err) and scale < 512.0, (ell, scale)
        U_o, lam_o, nu_o = nystrom.nystrom_factor(host(Om_d).T, host(Y_d).T, mb, shift_scale=scale)
        lam_g = host(lam)
        top = lam_o > 1e-6 * lam_o[0]
        assert rel(lam_g[top], lam_o[top]) <= (1e-8 if tight else 1e-4), ell
        Ug = host(U).T[:, top]     # columns below the core's noise floor are only an orthonormal completion
        assert np.abs(Ug.T @ Ug - np.eye(int(top.sum()))).max() <= (1e-10 if tight else 2e-5), ell
        v = rng.standard_normal(pr.p)
        mu = 1e-5
        z = host(ctx.precond_apply(ell, U, lam, mu, dev(v)))
        assert rel(z, nystrom.precond_apply(U_o, lam_o, mu, v)) <= (1e-8 if tight else 2e-3), ell
    ctx.close()


def test_factor_reports_not_spd(ngd):
    pr, th = small(SMALL[0], seed=30)
    ctx = ngd.Context(pr, dtype="f64")
    ell = 6
    Om = nystrom.thin_qr(np.random.default_rng(0).standard_normal((pr.p, ell)))
    Om_d = dev(Om.T.copy())
    with pytest.raises(ngd.NGDError) as e:
        ctx.nystrom_factor(ell, Om_d, dev(-5.0 * Om.T), prec="f64")   # Omega^T Y_nu = -5 I + nu I
    assert e.value.name == "NOT_SPD"
    ctx.close()


def test_pcg_matches_oracle_at_fixed_iterations(ngd):
    wl, pr, th = _workload("poisson2d")
    J = mlp.jacobian(pr, th)
    G = gramian.gramian(J, pr.w)
    g_o, _, _ = mlp.gradient(pr, th)
    ell, mu = 100, 1e-6
    Om_o = nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 5, 0))
    U_o, lam_o, _ = nystrom.nystrom_factor(Om_o, G @ Om_o)
    ctx = ngd.Context(pr, dtype="f64")
    t = dev(th)
    g, _, _ = ctx.gradient(t)
    U_d = dev(U_o.T.copy())
    for k in [1, 3, 10]:
        d, it, rr = ctx.pcg_solve(None, g, mu, U_d, dev(lam_o), ell, rtol=0.0, maxit=k)
        d_o, it_o, rr_o = solve.pcg(lambda v: G @ v + mu * v, g_o, lambda v: nystrom.precond_apply(U_o, lam_o, mu, v),
                                    0.0, k)
        assert it == it_o == k
        assert rel(host(d), d_o) <= 1e-8, k
        assert abs(rr - rr_o) <= 1e-6 * rr_o + 1e-8   # relres is relative to ||g||; rounding floor ~1e-9
    # to tolerance: the true residual of the GPU direction, measured with the oracle's G
    d, it, rr = ctx.pcg_solve(None, g, mu, U_d, dev(lam_o), ell, rtol=1e-10, maxit=2000)
    res = (G + mu * np.eye(pr.p)) @ host(d) - g_o
    assert rr <= 1e-10 and np.linalg.norm(res) <= 1e-8 * np.linalg.norm(g_o)
    # unpreconditioned CG runs more iterations to the same tolerance
    d2, it2, rr2 = ctx.pcg_solve(None, g, mu, None, None, 0, rtol=1e-10, maxit=5000)
    assert it2 > it
    ctx.close()


def test_pcg_matrix_free_matches_oracle_at_fixed_iterations(ngd):
    """PCG with the matrix-free Gramian (JVP then VJP per product; the iterations replayed from a
    captured CUDA graph two at a time): at 1, 3 and 6 iterations (stops inside and at the end of a
    replayed chunk) the iterates are the FP64 oracle's; a second solve with the same inputs (a
    new output buffer, so a new capture) returns the same direction bit for bit."""
    wl, pr, th = _workload("poisson2d")
    J = mlp.jacobian(pr, th)
    G = gramian.gramian(J, pr.w)
    g_o, _, _ = mlp.gradient(pr, th)
    ell, mu = 60, 1e-5
    Om_o = nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 6, 0))
    U_o, lam_o, _ = nystrom.nystrom_factor(Om_o, G @ Om_o)
    ctx = ngd.Context(pr, dtype="f64", gv_mode="matrix_free")
    t = dev(th)
    g, _, _ = ctx.gradient(t)
    U_d = dev(U_o.T.copy())
    lam_d = dev(lam_o)
    for k in [1, 3, 6]:
        d, it, rr = ctx.pcg_solve(None, g, mu, U_d, lam_d, ell, rtol=0.0, maxit=k)
        d_o, it_o, rr_o = solve.pcg(lambda v: G @ v + mu * v, g_o, lambda v: nystrom.precond_apply(U_o, lam_o, mu, v),
                                    0.0, k)
        assert it == it_o == k
        assert rel(host(d), d_o) <= 1e-8, k
    d1, it1, rr1 = ctx.pcg_solve(None, g, mu, U_d, lam_d, ell, rtol=1e-9, maxit=500)
    d2, it2, rr2 = ctx.pcg_solve(None, g, mu, U_d, lam_d, ell, rtol=1e-9, maxit=500)
    assert rr1 <= 1e-9 and it1 == it2 and rr1 == rr2
    assert np.array_equal(host(d1), host(d2))
    res = (G + mu * np.eye(pr.p)) @ host(d1) - g_o
    assert np.linalg.norm(res) <= 1e-7 * np.linalg.norm(g_o)
    ctx.close()


def test_fp32_matvec_symmetry_and_linearity(ngd):
    """The FP32-context matvec (one pass over the stored FP32 Jacobian, double-float sums): for
    that J, G = J^T W J is exactly symmetric and linear, so u.(Gv) = v.(Gu) and G(u + 2v) =
    Gu + 2Gv hold to the pair's ~48-bit precision; FP32 sums would break both at ~1e-7."""
    wl, pr, th = _workload("poisson5d")
    ctx = ngd.Context(pr, dtype="f32")
    rng = np.random.default_rng(12)
    u, v = rng.standard_normal(pr.p), rng.standard_normal(pr.p)
    Gu = host(ctx.gramian_mv(dev(th), dev(u), 0.0))
    Gv = host(ctx.gramian_mv(None, dev(v), 0.0))
    Guv = host(ctx.gramian_mv(None, dev(u + 2.0 * v), 0.0))
    assert abs(u @ Gv - v @ Gu) <= 1e-11 * np.linalg.norm(u) * np.linalg.norm(Gv)
    assert rel(Guv, Gu + 2.0 * Gv) <= 1e-11
    assert v @ Gv > 0.0
    ctx.close()


@pytest.mark.parametrize("precond", ["f64", "f32", "none"])
def test_pcg_fp32_context(ngd, precond):
    """PCG in an FP32 context (the whole solve in one cooperative kernel).  To rtol 1e-8: the
    true residual of the returned direction, measured with the context's own matvec, meets the
    tolerance; iterations and direction agree with the FP64 oracle on the FP64 Jacobian up to
    the FP32 Jacobian's rounding (~2e-4 in d at mu = 1e-5, a few iterations)."""
    wl, pr, th = _workload("poisson5d", 900, 220)
    J = mlp.jacobian(pr, th)
    G = gramian.gramian(J, pr.w)
    g_o, _, _ = mlp.gradient(pr, th)
    ell, mu = 60, 1e-5
    Om = nystrom.thin_qr(philox.gaussian_test_matrix(pr.p, ell, 5, 0))
    U_o, lam_o, _ = nystrom.nystrom_factor(Om, G @ Om)
    ctx = ngd.Context(pr, dtype="f32")
    g, _, _ = ctx.gradient(dev(th))
    if precond == "none":
        d, it, rr = ctx.pcg_solve(None, g, mu, None, None, 0, rtol=1e-8, maxit=3000)
        Pinv = None
    else:
        wd = torch.float64 if precond == "f64" else torch.float32
        U_d = torch.tensor(np.ascontiguousarray(U_o.T), dtype=wd, device="cuda")
        d, it, rr = ctx.pcg_solve(None, g, mu, U_d, dev(lam_o), ell, rtol=1e-8, maxit=3000)
        U_p = host(U_d).T

        def Pinv(v):
            return nystrom.precond_apply(U_p, lam_o, mu, v)
    d_o, it_o, rr_o = solve.pcg(lambda v: G @ v + mu * v, g_o, Pinv, 1e-8, 3000)
    assert rr <= 1e-8
    res = host(ctx.gramian_mv(None, d, mu)) - host(g)
    assert np.linalg.norm(res) <= 1e-7 * np.linalg.norm(host(g))
    # unpreconditioned CG runs ~250 iterations here, where rounding alone moves the count by ~10%
    assert abs(it - it_o) <= max(3, (0.25 if precond == "none" else 0.1) * it_o), (it, it_o)
    assert rel(host(d), d_o) <= 2e-3
    # a fixed iteration count stops there exactly
    d3, it3, rr3 = ctx.pcg_solve(None, g, mu, None, None, 0, rtol=0.0, maxit=3)
    assert it3 == 3 and rr3 > 0.0
    ctx.close()


def test_ngd_step_matches_oracle_fp64(ngd):
    wl, pr, th = _workload("poisson2d")
    ctx = ngd.Context(pr, dtype="f64")
    t = dev(th)
    info = ctx.step(t, ell=wl.ell, mu=wl.mu, rtol=wl.rtol, maxit=1000, seed=0, step=0, sketch="f64")
    th1_o, info_o = solve.ngd_step(pr, th, ell=wl.ell, mu=wl.mu, rtol=0.0, maxit=info["pcg_iters"], seed=0, step=0)
    assert info["loss_after"] < info["loss_before"]
    assert abs(info["loss_before"] - info_o.loss_before) <= 1e-12 * info_o.loss_before
    assert abs(info["lam1"] - info_o.lam1) <= 1e-9 * info_o.lam1
    assert info["alpha"] == info_o.alpha
    assert rel(host(t) - th, th1_o - th) <= 1e-6
    assert info["relres"] <= wl.rtol
    ctx.close()


@pytest.mark.parametrize("dtype,packing", [("f64", None), ("f32", 1), ("f32", 2), ("f32", 0)])
def test_batch_step_matches_oracle(ngd, dtype, packing):
    """Batching form: problems of uneven sizes (and different source frequencies) stepped by one
    ngd_batch_step; problem i uses Philox key seed + i.  Each problem's step matches the oracle's
    step on that problem (FP64: to the PCG direction tolerance; FP32: the FP64-accurate sketch).
    FP32 solves run one per launch (packing 1), two per cooperative launch on block groups of
    their own (packing 2: two launches for three problems), or with the packing tuned on the
    step (packing 0)."""
    probs, thetas = [], []
    for i, (n_int, n_bnd, k) in enumerate([(600, 150, 1.0), (1100, 275, 3.0), (350, 87, 2.0)]):
        pr, th = inputs.small_problem(d=3, widths=[3, 24, 24, 1], n_int=n_int, n_bnd=n_bnd, seed=40 + i, freq=k)
        probs.append(pr)
        thetas.append(th)
    batch = ngd.Batch(probs, dtype=dtype)
    if packing is not None:
        batch.set_packing(packing)
    ts = [dev(th) for th in thetas]
    ell, mu, rtol = 60, 1e-6, (1e-10 if dtype == "f64" else 1e-7)
    infos = batch.step(ts, ell=ell, mu=mu, rtol=rtol, maxit=2000, seed=7, step=3, sketch="f64")
    assert len(infos) == 3
    if packing == 2:
        assert batch.solve_launches == 2 and batch.packing == 2
    if packing == 0:
        assert batch.packing in (1, 2, 4, 8)          # tuned on this step
    for i, (pr, th, info) in enumerate(zip(probs, thetas, infos)):
        th1_o, info_o = solve.ngd_step(pr, th, ell=ell, mu=mu, rtol=0.0, maxit=info["pcg_iters"], seed=7 + i, step=3)
        assert info["relres"] <= rtol, i
        assert info["loss_after"] < info["loss_before"], i
        if dtype == "f64":
            assert abs(info["lam1"] - info_o.lam1) <= 1e-9 * info_o.lam1, i
            assert info["alpha"] == info_o.alpha, i
            assert rel(host(ts[i]) - th, th1_o - th) <= 1e-6, i
        else:
            # FP32 residuals and Jacobian: the direction agrees to the FP32 rounding of J
            assert abs(info["lam1"] - info_o.lam1) <= 1e-4 * info_o.lam1, i
            assert rel(host(ts[i]) - th, th1_o - th) <= 5e-3, i
    batch.close()


def test_ngd_step_fp32_paths(ngd):
    """FP32 path: the FP64-accurate (double-float) and F32 sketches converge to rtol; TF32 / BF16
    sketches need a shift of their own eps, which truncates the captured spectrum (more PCG
    iterations, never a failure)."""
    wl, pr, th = _workload("poisson5d", 1200, 300)
    J = mlp.jacobian(pr, th)
    g_o = mlp.vjp(pr, th, pr.w * mlp.residual(pr, th)[0])
    iters = {}
    for sketch in ["f64", "df", "f32", "tf32", "bf16"]:
        ctx = ngd.Context(pr, dtype="f32")
        t = dev(th)
        info = ctx.step(t, ell=200, mu=1e-7, rtol=1e-6, maxit=600, seed=1, step=0, sketch=sketch)
        iters[sketch] = info["pcg_iters"]
        assert info["loss_after"] < info["loss_before"], sketch
        if sketch in ("f32", "f64", "df"):
            assert info["relres"] <= 1e-6
            # the direction solves the oracle's FP64 system to the accuracy of the FP32 operator
            d = (th - host(t)) / info["alpha"]
            res = J.T @ (pr.w * (J @ d)) + 1e-7 * d - g_o
            assert np.linalg.norm(res) <= 1e-3 * np.linalg.norm(g_o)
        ctx.close()
    assert iters["f64"] <= iters["f32"] <= iters["tf32"] and iters["f32"] <= iters["bf16"], iters
    # the two FP64-accurate forms (tensor-core digit planes, double-float) need the same iterations
    assert abs(iters["f64"] - iters["df"]) <= max(1, 0.02 * iters["df"]), iters


def test_heuristic_mu(ngd):
    pr, th = small(SMALL[0], seed=40)
    ctx = ngd.Context(pr, dtype="f64")
    info = ctx.step(dev(th), ell=20, mu=None, rtol=1e-8, maxit=500, seed=2, step=3, sketch="f64")
    assert info["mu"] == pytest.approx(10 * 2.0 ** -52 * info["lam1"], rel=1e-12)
    ctx.close()


def test_autograd_function_store_and_recompute(ngd):
    pr, th = small(SMALL[3], seed=50)
    for budget in [0, 1]:          # 0: unlimited (matrix-free keeps the tape); 1 byte: recompute
        ctx = ngd.Context(pr, dtype="f64", gv_mode="matrix_free", mem_budget=budget)
        t = dev(th).requires_grad_(True)
        r = ngd.PinnResidual.apply(t, ctx)
        c = torch.randn(pr.n, dtype=torch.float64, device="cuda")
        (r * c).sum().backward()
        assert rel(host(t.grad), mlp.vjp(pr, th, host(c))) <= 1e-11
        ctx.close()


def test_nonfinite_and_invalid(ngd):
    pr, th = small(SMALL[0], seed=60)
    ctx = ngd.Context(pr, dtype="f64")
    with pytest.raises(ngd.NGDError) as e:
        ctx.nystrom_sketch(dev(th), pr.p + 1, prec="f64")
    assert e.value.name == "INVALID_ARG"
    bad = th.copy()
    bad[3] = np.nan
    g, _, _ = ctx.gradient(dev(bad))
    with pytest.raises(ngd.NGDError) as e:
        ctx.pcg_solve(None, g, 1e-3, None, None, 0, rtol=1e-8, maxit=10)
    assert e.value.name == "NONFINITE"
    ctx.close()


@pytest.mark.parametrize("case", [0, 3, 4])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_eval_channels_match_oracle_forward(ngd, case, dtype):
    """ngd_eval: u, grad u and Delta u at the context's points against the oracle's hand-derived
    forward Laplacian (FP64 path 1e-11, FP32 path 2e-5)."""
    pr, th = small(SMALL[case], seed=60 + case)
    ctx = ngd.Context(pr, dtype=dtype)
    out = host(ctx.eval(dev(th)))
    u, gu, lu, _ = mlp.taylor_forward(th, pr.widths, pr.X, mlp.spatial_mask(pr.pde, pr.d))
    ref = np.concatenate([u[:, None], gu, lu[:, None]], axis=1)
    tol = 1e-11 if dtype == "f64" else 2e-5
    assert out.shape == ref.shape
    for c in range(ref.shape[1]):
        assert rel(out[:, c], ref[:, c]) <= tol, c
    ctx.close()


def _guarded_rank(lam, mu, ell, ell_max, delta, band=1e-6):
    """Alg. 4's rank from the oracle's spectrum, or None when an eigenvalue lies within `band`
    (relative) of 10 mu, where the two sides' last bits may legitimately decide differently."""
    lam = np.asarray(lam)
    if np.any(np.abs(lam - 10.0 * mu) <= band * 10.0 * mu):
        return None
    return nystrom.next_rank(lam, mu, ell, ell_max, delta)


def test_step_adaptive_damping_and_rank_match_oracle(ngd):
    """One step with the damping of Sec. 5 (mu = max(gamma eps lambda_1, 1e-4 L^2)) and Alg. 4's
    rank update: mu, ell_next and the update agree with the oracle step (same Omega stream, same
    PCG iteration count)."""
    pr, th = small(SMALL[0], seed=71)
    ctx = ngd.Context(pr, dtype="f64")
    t = dev(th)
    ell, ell_max, delta = 12, 30, 6
    info = ctx.step(t, ell=ell, mu=None, mu_loss_coef=1e-4, ell_max=ell_max, ell_delta=delta, rtol=1e-10,
                    maxit=500, seed=5, step=2, sketch="f64")
    th1_o, info_o, parts = solve.ngd_step(pr, th, ell=ell, mu=None, rtol=0.0, maxit=info["pcg_iters"], seed=5, step=2,
                                          mu_loss_coef=1e-4, ell_max=ell_max, ell_delta=delta, return_parts=True)
    assert info["mu"] == pytest.approx(max(10 * 2.0 ** -52 * info["lam1"], 1e-4 * info["loss_before"] ** 2), rel=1e-14)
    assert info["mu"] == pytest.approx(info_o.mu, rel=1e-10)
    want = _guarded_rank(parts["lam"], info_o.mu, ell, ell_max, delta)
    if want is not None:
        assert info["ell_next"] == want == info_o.ell_next
    assert rel(host(t) - th, th1_o - th) <= 1e-6
    ctx.close()


def test_nystrom_ngd_run_matches_oracle(ngd):
    """Four NystromNGD steps (adaptive damping and rank, Alg. 4 with Sec. 5) from the same theta:
    the GPU's rank sequence is the oracle's, and the parameters after the run agree (the oracle
    replays the GPU's PCG iteration counts)."""
    pr, th = small(SMALL[1], seed=72)
    ctx = ngd.Context(pr, dtype="f64")
    t = dev(th)
    ell, ells, iters = 6, [], []
    for k in range(4):
        ells.append(ell)
        info = ctx.step(t, ell=ell, mu=None, mu_loss_coef=1e-4, ell_max=24, ell_delta=6, rtol=1e-10, maxit=500,
                        seed=9, step=k, sketch="f64")
        iters.append(info["pcg_iters"])
        ell = info["ell_next"]
    th_o, infos_o, ells_o = solve.nystrom_ngd(pr, th, steps=4, ell0=6, ell_max=24, ell_delta=6, seed=9,
                                              mu_loss_coef=1e-4, pcg_iters=iters)
    assert ells == ells_o
    assert rel(host(t) - th, th_o - th) <= 1e-6
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("mode", ["stored", "matrix_free"])
def test_gramian_diag_matches_oracle(ngd, dtype, mode):
    """ngd_gramian_diag against diag(J^T W J) of the oracle's Jacobian (FP64 1e-12, FP32 2e-5)."""
    pr, th = small(SMALL[0], seed=80)
    ctx = ngd.Context(pr, dtype=dtype, gv_mode=mode)
    d = host(ctx.gramian_diag(dev(th)))
    d_o = gramian.gramian_diag(mlp.jacobian(pr, th), pr.w)
    assert rel(d, d_o) <= (1e-12 if dtype == "f64" else 2e-5)
    ctx.close()


@pytest.mark.parametrize("dtype,prec", [("f64", "f64"), ("f32", "f64"), ("f32", "f32")])
def test_sampled_sketch_matches_oracle(ngd, dtype, prec):
    """The sampling test matrix: the sampled indices are the oracle's exponential race on the same
    FP64 diagonal (bit-exact integers), Omega = I[:, S], and Y = G[:, S]."""
    pr, th = small(SMALL[1], seed=81)
    ctx = ngd.Context(pr, dtype=dtype)
    ell = 15
    idx, Om, Y = ctx.nystrom_sketch_sampled(dev(th), ell, seed=6, step=4, prec=prec)
    d_gpu = host(ctx.gramian_diag(None))
    S = nystrom.sampling_indices(d_gpu, ell, seed=6, step=4)
    assert [int(i) for i in idx.cpu().tolist()] == [int(i) for i in S]
    assert np.array_equal(host(Om).reshape(ell, -1).T, nystrom.selection_matrix(S, pr.p))
    G = gramian.gramian(mlp.jacobian(pr, th), pr.w)
    Yg = host(Y).reshape(ell, -1).T
    assert rel(Yg, G[:, S]) <= (1e-10 if dtype == "f64" else 1e-5)
    ctx.close()


def test_ngd_step_sampling_test_matrix_matches_oracle(ngd):
    """One NystromNGD Sampling step: the same S, factor, PCG (same iteration count) and update as
    the oracle."""
    pr, th = small(SMALL[0], seed=82)
    ctx = ngd.Context(pr, dtype="f64")
    t = dev(th)
    info = ctx.step(t, ell=14, mu=1e-6, rtol=1e-10, maxit=500, seed=3, step=2, sketch="f64", test_matrix="sampling")
    th1_o, info_o = solve.ngd_step(pr, th, ell=14, mu=1e-6, rtol=0.0, maxit=info["pcg_iters"], seed=3, step=2,
                                   test_matrix="sampling")
    assert info["loss_after"] < info["loss_before"]
    assert abs(info["lam1"] - info_o.lam1) <= 1e-9 * info_o.lam1
    assert rel(host(t) - th, th1_o - th) <= 1e-6
    ctx.close()


def test_sampling_rejects_too_few_positive_diagonal_entries(ngd):
    """A one-point problem has a rank-one G: asking for more columns than diag G has positive
    entries is an error reported through the status word (no GPU fault)."""
    pr, th = small(SMALL[5], seed=83)             # a single point
    ctx = ngd.Context(pr, dtype="f64")
    ell = min(pr.p, 2048)
    d = host(ctx.gramian_diag(dev(th)))
    npos = int(np.sum(d > 0))
    if npos >= ell:
        pytest.skip("every diagonal entry is positive")
    with pytest.raises(ngd.NGDError) as e:
        ctx.nystrom_sketch_sampled(dev(th), ell, seed=1, step=0)
    assert e.value.name == "INVALID_ARG"
    ctx.close()


@pytest.mark.parametrize("mu", [1e-6, None])
def test_rpchol_step_matches_oracle(ngd, mu):
    """One RPCholNGD step (Alg. 5): the power-method lambda_1, mu, the rank block RPCholesky finds
    (same pivot races on the FP64 residual diagonal) and the update agree with the oracle step at
    the GPU's PCG iteration count."""
    pr, th = small(SMALL[0], seed=90)
    ctx = ngd.Context(pr, dtype="f64")
    t = dev(th)
    kw = dict(ell=24, rpchol_block=6, mu=mu, mu_loss_coef=1e-4 if mu is None else 0.0)
    info = ctx.step(t, precond="rpchol", rtol=1e-10, maxit=500, seed=4, step=1, sketch="f64", **kw)
    th1_o, info_o = solve.ngd_step(pr, th, rtol=0.0, maxit=info["pcg_iters"], seed=4, step=1, precond="rpchol", **kw)
    assert info["loss_after"] < info["loss_before"]
    assert info["lam1"] == pytest.approx(info_o.lam1, rel=1e-10)
    assert info["mu"] == pytest.approx(info_o.mu, rel=1e-10)
    assert info["ell_next"] == info_o.ell_next
    assert rel(host(t) - th, th1_o - th) <= 1e-6
    ctx.close()


def test_rpchol_step_fp32_context(ngd):
    """RPCholNGD in an FP32 context (FP64-accurate columns of G and FP64 F): the step solves to the
    requested tolerance, decreases the loss and finds the oracle's rank within one block."""
    pr, th = inputs.small_problem(d=3, widths=[3, 24, 24, 1], n_int=600, n_bnd=150, seed=91)
    ctx = ngd.Context(pr, dtype="f32")
    t = dev(th)
    info = ctx.step(t, precond="rpchol", ell=60, rpchol_block=10, mu=1e-6, rtol=1e-7, maxit=2000, seed=2, step=0,
                    sketch="f64")
    _, info_o = solve.ngd_step(pr, th, ell=60, rpchol_block=10, mu=1e-6, rtol=1e-7, maxit=2000, seed=2, step=0,
                               precond="rpchol")
    assert info["relres"] <= 1e-7
    assert info["loss_after"] < info["loss_before"]
    assert info["lam1"] == pytest.approx(info_o.lam1, rel=1e-4)
    assert abs(info["ell_next"] - info_o.ell_next) <= 10
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_ngd_full_step_matches_oracle(ngd, dtype):
    """NGD full (Alg. 2): the explicit Gramian, the power-method lambda_1, mu, the FP64 Cholesky and
    two triangular solves give the oracle's direct direction.  FP64: the direction tolerance 1e-6
    (the Gramian is formed to ~2^-48 and kappa(G + mu I) ~ 1e8 here), and the GPU direction solves
    the oracle's system to a backward error of 1e-12; FP32 context: the FP32 rounding of J, 5e-3."""
    pr, th = inputs.small_problem(d=3, widths=[3, 20, 20, 1], n_int=500, n_bnd=120, seed=95)
    ctx = ngd.Context(pr, dtype=dtype)
    t = dev(th)
    info = ctx.step(t, precond="full", ell=1, mu=1e-6, seed=3, step=0, sketch="f64")
    th1_o, info_o, parts = solve.ngd_step(pr, th, ell=1, mu=1e-6, rtol=0.0, maxit=1, seed=3, step=0, precond="full",
                                          return_parts=True)
    assert info["pcg_iters"] == 0
    assert info["loss_after"] < info["loss_before"]
    assert info["lam1"] == pytest.approx(info_o.lam1, rel=1e-10 if dtype == "f64" else 1e-4)
    assert rel(host(t) - th, th1_o - th) <= (1e-6 if dtype == "f64" else 5e-3)
    if dtype == "f64" and info["alpha"] > 0:
        d_gpu = (th - host(t)) / info["alpha"]
        G, g = parts["G"], parts["g"]
        res = G @ d_gpu + 1e-6 * d_gpu - g
        assert np.linalg.norm(res) <= 1e-12 * (np.linalg.norm(G, 2) * np.linalg.norm(d_gpu) + np.linalg.norm(g))
    ctx.close()


def test_ngd_full_step_blocked_cholesky(ngd):
    """NGD full at p = 1217: the blocked Cholesky (diagonal blocks of 256 and a ragged last one of
    193, panel solves, lower-triangle trailing updates) and an even leading dimension 1220 give the
    oracle's direction; the GPU direction solves the oracle's system to a backward error of 1e-12."""
    pr, th = inputs.small_problem(d=3, widths=[3, 32, 32, 1], n_int=1500, n_bnd=300, seed=97)
    assert th.size == 1217
    ctx = ngd.Context(pr, dtype="f64")
    t = dev(th)
    info = ctx.step(t, precond="full", ell=1, mu=1e-6, seed=3, step=0, sketch="f64")
    th1_o, info_o, parts = solve.ngd_step(pr, th, ell=1, mu=1e-6, rtol=0.0, maxit=1, seed=3, step=0, precond="full",
                                          return_parts=True)
    assert info["loss_after"] < info["loss_before"]
    assert info["alpha"] == info_o.alpha
    assert rel(host(t) - th, th1_o - th) <= 1e-6
    d_gpu = (th - host(t)) / info["alpha"]
    G, g = parts["G"], parts["g"]
    res = G @ d_gpu + 1e-6 * d_gpu - g
    assert np.linalg.norm(res) <= 1e-12 * (np.linalg.norm(G, 2) * np.linalg.norm(d_gpu) + np.linalg.norm(g))
    ctx.close()


def test_ngd_full_blocked_cholesky_retries(ngd):
    """NGD full at p = 1217 with N = 600 rows (G of rank <= 600) and mu = 1e-16, far below the
    rounding of the formed G: the blocked Cholesky meets a non-positive pivot, the lower triangle
    is rebuilt from the upper one (leading dimension 1220) and the factorization retried with
    8 mu, 64 mu, ...  The damping used is mu times a power of 8, and the direction solves
    (G + mu_used I) d = g to a backward error of the Cholesky's precision."""
    pr, th = inputs.small_problem(d=3, widths=[3, 32, 32, 1], n_int=500, n_bnd=100, seed=98)
    assert th.size == 1217
    mu0 = 1e-16
    ctx = ngd.Context(pr, dtype="f64")
    t = dev(th)
    info = ctx.step(t, precond="full", ell=1, mu=mu0, seed=4, step=0, sketch="f64", armijo_max=60)
    k = np.log(info["mu"] / mu0) / np.log(8.0)
    assert 1 <= round(k) <= 5 and abs(k - round(k)) < 1e-9
    _, _, parts = solve.ngd_step(pr, th, ell=1, mu=mu0, rtol=0.0, maxit=1, seed=4, step=0, precond="full",
                                 return_parts=True)
    if info["alpha"] > 0:
        d_gpu = (th - host(t)) / info["alpha"]
        G, g = parts["G"], parts["g"]
        res = G @ d_gpu + info["mu"] * d_gpu - g
        assert np.linalg.norm(res) <= 1e-9 * (np.linalg.norm(G, 2) * np.linalg.norm(d_gpu) + np.linalg.norm(g))
    ctx.close()


def test_ngd_full_step_adaptive_damping(ngd):
    """NGD full with mu = max(10 eps lambda_1, 1e-4 L^2): mu from the power method and the loss."""
    pr, th = small(SMALL[0], seed=96)
    ctx = ngd.Context(pr, dtype="f64")
    info = ctx.step(dev(th), precond="full", ell=1, mu=None, mu_loss_coef=1e-4, seed=1, step=2, sketch="f64")
    assert info["mu"] == pytest.approx(max(10 * 2.0 ** -52 * info["lam1"], 1e-4 * info["loss_before"] ** 2),
                                       rel=1e-14)
    ctx.close()
