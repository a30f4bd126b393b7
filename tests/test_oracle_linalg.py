"""Pins for oracle/gramian.py, oracle/nystrom.py, oracle/solve.py and oracle/philox.py (no GPU)."""
import os

import numpy as np
import pytest
import scipy.stats

from oracle import gramian, mlp, nystrom, philox, solve
from paper_2505_11638_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small(seed=0, n_int=16, n_bnd=6, widths=None, d=2):
    pr, theta = inputs.small_problem(d=d, widths=widths, n_int=n_int, n_bnd=n_bnd, seed=seed)
    J = mlp.jacobian(pr, theta)
    return pr, theta, J


# ----------------------------------------------------------------------------- Gramian
def test_gramian_brute_force_symmetric_psd_trace():
    pr, theta, J = _small(seed=1, n_int=8, n_bnd=3, widths=[2, 4, 3, 1])
    G = gramian.gramian(J, pr.w)
    # brute force entry by entry (Thm. 1: G_ij = sum_r w_r dr_r/dtheta_i dr_r/dtheta_j)
    Gb = np.zeros_like(G)
    for i in range(pr.p):
        for j in range(pr.p):
            Gb[i, j] = sum(pr.w[r] * J[r, i] * J[r, j] for r in range(pr.n))
    np.testing.assert_allclose(G, Gb, rtol=1e-13, atol=1e-16)
    assert np.abs(G - G.T).max() <= 1e-15 * np.abs(G).max()
    ev = np.linalg.eigvalsh(G)
    assert ev[0] >= -1e-12 * ev[-1]
    # rank <= number of points
    assert np.sum(ev > 1e-10 * ev[-1]) <= pr.n
    # trace and diagonal: Eq. gram_diagonal
    assert np.trace(G) == pytest.approx(sum(pr.w[r] * J[r] @ J[r] for r in range(pr.n)), rel=1e-13)
    np.testing.assert_allclose(gramian.gramian_diag(J, pr.w), np.diag(G), rtol=1e-13)


def test_gramian_mv_matches_explicit_and_blocked():
    pr, theta, J = _small(seed=2)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(pr.p)
    G = gramian.gramian(J, pr.w)
    y = gramian.gramian_mv(J, pr.w, v, 1e-3)
    np.testing.assert_allclose(y, G @ v + 1e-3 * v, rtol=1e-12, atol=1e-14)
    yb = gramian.gramian_mv_blocked(lambda rows: mlp.jacobian(pr, theta, rows), pr.n, pr.w, v, 1e-3, block=5)
    np.testing.assert_allclose(yb, y, rtol=1e-12, atol=1e-14)
    # matrix-free form by JVP then VJP (Thm. 1 consequence)
    ymf = mlp.vjp(pr, theta, pr.w * mlp.jvp(pr, theta, v)) + 1e-3 * v
    np.testing.assert_allclose(ymf, y, rtol=1e-11, atol=1e-14)


def test_direct_direction_residual():
    pr, theta, J = _small(seed=3)
    G = gramian.gramian(J, pr.w)
    g = mlp.gradient(pr, theta)[0]
    mu = 1e-6
    d = gramian.direct_direction(G, g, mu)
    res = (G + mu * np.eye(pr.p)) @ d - g
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(g)


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = philox.philox4x32_10(np.array([v[0:4]], dtype=np.uint32), np.array([v[4:6]], dtype=np.uint32))
        assert out[0].tolist() == v[6:10]


def test_uniform52_and_box_muller():
    u = philox.uniform52(np.array([0, 0xFFFFFFFF], dtype=np.uint32), np.array([0, 0xFFFFFFFF], dtype=np.uint32))
    assert u[0] == 0.5 * 2.0 ** -52 and u[1] == 1.0 - 0.5 * 2.0 ** -52
    assert 0.0 < u[0] < u[1] < 1.0
    # resolution: consecutive codes differ by exactly 2^-52
    v = philox.uniform52(np.array([7, 7], dtype=np.uint32), np.array([0, 1 << 12], dtype=np.uint32))
    assert v[1] - v[0] == 2.0 ** -52
    rng = np.random.default_rng(0)
    u1, u2 = rng.uniform(1e-12, 1, 1000), rng.uniform(0, 1, 1000)
    z0, z1 = philox.box_muller(u1, u2)
    # invert the polar map: u1 = exp(-(z0^2 + z1^2)/2), 2 pi u2 = atan2(z1, z0) mod 2 pi
    np.testing.assert_allclose(np.exp(-(z0 ** 2 + z1 ** 2) / 2), u1, rtol=1e-10)
    np.testing.assert_allclose(np.mod(np.arctan2(z1, z0), 2 * np.pi), 2 * np.pi * u2, rtol=1e-9, atol=1e-9)


def test_gaussian_test_matrix_distribution_and_layout():
    Om = philox.gaussian_test_matrix(4001, 50, seed=12345, step=7)
    assert Om.shape == (4001, 50)
    x = Om.ravel()
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01
    assert scipy.stats.kstest(x, "norm").pvalue > 1e-3
    # independent streams for other seeds / steps; identical for the same counters
    assert not np.allclose(Om, philox.gaussian_test_matrix(4001, 50, seed=12345, step=8))
    assert not np.allclose(Om, philox.gaussian_test_matrix(4001, 50, seed=12346, step=7))
    np.testing.assert_array_equal(Om[:, :20], philox.gaussian_test_matrix(4001, 20, seed=12345, step=7))
    np.testing.assert_array_equal(Om[:4000], philox.gaussian_test_matrix(4000, 50, seed=12345, step=7))
    # rows 2m and 2m+1 come from one block: counter (m, j, step, 0), key (seed, 0)
    blk = philox.philox4x32_10(np.array([[3, 5, 7, 0]], dtype=np.uint32), np.array([[12345, 0]], dtype=np.uint32))[0]
    z0, z1 = philox.box_muller(philox.uniform52(blk[0], blk[1]), philox.uniform52(blk[2], blk[3]))
    assert Om[6, 5] == z0 and Om[7, 5] == z1


# ----------------------------------------------------------------------------- Nystrom
def _psd(p, rank, rng, decay=0.5):
    Q = np.linalg.qr(rng.standard_normal((p, rank)))[0]
    lam = decay ** np.arange(rank)
    return (Q * lam) @ Q.T


def test_thin_qr_unique():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 9))
    Q = nystrom.thin_qr(A)
    np.testing.assert_allclose(Q.T @ Q, np.eye(9), atol=1e-14)
    R = Q.T @ A
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(np.tril(R, -1), 0, atol=1e-13)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)


def test_nystrom_exact_when_rank_below_ell():
    """With ell >= rank G the Nystrom approximation reproduces G."""
    pr, theta, J = _small(seed=4, n_int=14, n_bnd=6, widths=[2, 6, 5, 1])   # N=20, p=59
    G = gramian.gramian(J, pr.w)
    Om = philox.gaussian_test_matrix(pr.p, 30, seed=1, step=0)
    _, _, U, lam, nu = nystrom.randomized_nystrom(lambda V: G @ V, Om)
    Gh = nystrom.nystrom_matrix(U, lam)
    assert np.linalg.norm(Gh - G, 2) <= 1e-10 * np.linalg.norm(G, 2)
    np.testing.assert_allclose(U.T @ U, np.eye(30), atol=1e-12)
    assert np.all(np.diff(lam) <= 0)


def test_nystrom_matches_definition_and_bounds():
    """Eq. nystrom_approx: G_hat = (G Om)(Om^T G Om)^+ (G Om)^T; G - G_hat is PSD; lambda_hat_i <= lambda_i."""
    rng = np.random.default_rng(5)
    p, ell = 60, 12
    G = _psd(p, 40, rng, decay=0.7)
    Om = rng.standard_normal((p, ell))
    _, _, U, lam, nu = nystrom.randomized_nystrom(lambda V: G @ V, Om)
    Gh = nystrom.nystrom_matrix(U, lam)
    Y = G @ Om
    Gdef = Y @ np.linalg.pinv(Om.T @ Y) @ Y.T
    assert np.linalg.norm(Gh - Gdef, 2) <= 1e-10 * np.linalg.norm(G, 2)
    assert np.linalg.eigvalsh(G - Gh)[0] >= -1e-12 * np.linalg.norm(G, 2)
    lam_true = np.sort(np.linalg.eigvalsh(G))[::-1][:ell]
    assert np.all(lam <= lam_true * (1 + 1e-10) + 1e-14)


def test_nystrom_invariant_under_right_multiplication():
    rng = np.random.default_rng(6)
    p, ell = 50, 10
    G = _psd(p, 30, rng, decay=0.6)
    Om = rng.standard_normal((p, ell))
    R = rng.standard_normal((ell, ell)) + 3 * np.eye(ell)
    G1 = nystrom.nystrom_matrix(*nystrom.randomized_nystrom(lambda V: G @ V, Om)[2:4])
    G2 = nystrom.nystrom_matrix(*nystrom.randomized_nystrom(lambda V: G @ V, Om @ R)[2:4])
    assert np.linalg.norm(G1 - G2, 2) <= 1e-10 * np.linalg.norm(G, 2)


def test_shift_is_spacing_in_the_sketch_precision():
    for x in [1.0, 3.7, 1e-3, 123456.0, 9.6951]:
        assert nystrom.shift(x) == np.spacing(x)                          # FP64: MATLAB eps(x)
        assert nystrom.shift(x, 23) == float(np.spacing(np.float32(x)))   # FP32: eps(single(x))
        assert nystrom.shift(x, 52) == 2.0 ** (np.floor(np.log2(x)) - 52)
    assert nystrom.shift(8.0, 10) == 8.0 * 2.0 ** -10                       # TF32 spacing at 8
    assert nystrom.shift(3.0, 7) == 2.0 * 2.0 ** -7                         # BF16 spacing at 3


def test_preconditioner_exact_nystrom_gives_mu_identity():
    """If G_hat = G (ell > rank) then lambda_ell = 0 and P^{-1}(G + mu I) = mu I."""
    rng = np.random.default_rng(7)
    p = 40
    G = _psd(p, 8, rng, decay=0.5)
    _, _, U, lam, nu = nystrom.randomized_nystrom(lambda V: G @ V, rng.standard_normal((p, 12)))
    assert lam[-1] == 0.0
    mu = 1e-3
    M = np.column_stack([nystrom.precond_apply(U, lam, mu, e) for e in np.eye(p)])
    np.testing.assert_allclose(M @ (G + mu * np.eye(p)), mu * np.eye(p), atol=1e-10)
    # P^{-1} is symmetric positive definite
    assert np.abs(M - M.T).max() < 1e-12
    assert np.linalg.eigvalsh(M)[0] > 0


# ----------------------------------------------------------------------------- PCG / Armijo / step
def test_pcg_reaches_direct_solution():
    pr, theta, J = _small(seed=8, n_int=30, n_bnd=8)
    G = gramian.gramian(J, pr.w)
    g = mlp.gradient(pr, theta)[0]
    mu = 1e-4
    dstar = gramian.direct_direction(G, g, mu)
    x, it, rr = solve.pcg(lambda v: G @ v + mu * v, g, None, 1e-13, 2000)
    assert rr <= 1e-13
    assert np.linalg.norm(x - dstar) <= 1e-8 * np.linalg.norm(dstar)
    _, _, U, lam, _ = nystrom.randomized_nystrom(lambda V: G @ V, philox.gaussian_test_matrix(pr.p, 20, 3, 0))
    x2, it2, rr2 = solve.pcg(lambda v: G @ v + mu * v, g, lambda v: nystrom.precond_apply(U, lam, mu, v), 1e-13, 2000)
    assert np.linalg.norm(x2 - dstar) <= 1e-8 * np.linalg.norm(dstar)
    assert it2 < it


def test_cg_finite_termination_low_rank():
    """G + mu I with rank G = r has at most r + 1 distinct eigenvalues: CG ends in <= r + 1 steps."""
    rng = np.random.default_rng(9)
    p, r = 30, 4
    G = _psd(p, r, rng, decay=0.5)
    g = rng.standard_normal(p)
    x, it, rr = solve.pcg(lambda v: G @ v + 0.1 * v, g, None, 1e-10, 100)
    assert it <= r + 1 and rr <= 1e-10


def test_cg_energy_error_monotone():
    rng = np.random.default_rng(10)
    p = 25
    A = _psd(p, p, rng, decay=0.8) + 1e-2 * np.eye(p)
    g = rng.standard_normal(p)
    xs = np.linalg.solve(A, g)
    errs = []
    for k in range(1, 15):
        x, _, _ = solve.pcg(lambda v: A @ v, g, None, 0.0, k)
        e = x - xs
        errs.append(e @ A @ e)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))


def test_pcg_one_iteration_with_exact_nystrom():
    rng = np.random.default_rng(11)
    p = 40
    G = _psd(p, 6, rng, decay=0.5)
    _, _, U, lam, _ = nystrom.randomized_nystrom(lambda V: G @ V, rng.standard_normal((p, 10)))
    g = rng.standard_normal(p)
    mu = 1e-3
    x, it, rr = solve.pcg(lambda v: G @ v + mu * v, g, lambda v: nystrom.precond_apply(U, lam, mu, v), 1e-10, 50)
    assert it == 1
    np.testing.assert_allclose(x, np.linalg.solve(G + mu * np.eye(p), g), rtol=1e-8)


def test_pcg_breakdown_detected():
    with pytest.raises(solve.Breakdown):
        solve.pcg(lambda v: -v, np.ones(3), None, 1e-8, 10)


def test_armijo_backtracking_exact_alpha():
    loss = lambda th: 0.5 * float(th @ th)
    th = np.array([1.0, -2.0, 0.5])
    g = th.copy()
    a, L, n = solve.armijo(loss, th, g, g, loss(th))
    assert a == 1.0 and L == 0.0 and n == 1
    a, L, n = solve.armijo(loss, th, 3 * g, g, loss(th))       # alpha = 1 overshoots to -2 theta
    assert a == 0.5 and n == 2 and L == pytest.approx(loss(-0.5 * th))
    a, L, n = solve.armijo(lambda t: np.nan, th, g, g, 1.0, max_trials=4)
    assert a == 0.0 and n == 4


def test_ngd_step_decreases_loss_and_matches_direct():
    pr, theta = inputs.small_problem(d=2, n_int=40, n_bnd=12, seed=12)
    th1, info, parts = solve.ngd_step(pr, theta, ell=30, mu=1e-6, rtol=1e-12, maxit=500, seed=5, step=0,
                                      return_parts=True)
    assert info.loss_after < info.loss_before
    G = gramian.gramian(parts["J"], pr.w)
    dstar = gramian.direct_direction(G, parts["g"], 1e-6)
    assert np.linalg.norm(parts["d"] - dstar) <= 1e-6 * np.linalg.norm(dstar)
    # the heuristic mu of Alg. 4
    _, info2 = solve.ngd_step(pr, theta, ell=30, mu=None, rtol=1e-8, maxit=100, seed=5, step=0)
    assert info2.mu == pytest.approx(10 * 2.0 ** -52 * info2.lam1)


# ---------------------------------------------------------------------------- NystromNGD control (Alg. 4, Sec. 5)
def test_next_rank_rule_on_constructed_spectra():
    """Alg. 4's rank update, worked by hand on spectra whose crossing of 10 mu is placed."""
    mu = 0.01                                            # 10 mu = 0.1
    # lambda_hat_ell above 10 mu: grow by delta, capped by ell_max
    assert nystrom.next_rank([10.0, 5.0, 2.0, 1.0], mu, 4, 30, 20) == 24
    assert nystrom.next_rank([10.0, 5.0, 2.0, 1.0], mu, 4, 10, 20) == 10
    assert nystrom.next_rank([10.0, 5.0, 2.0, 1.0], mu, 4, 4, 20) == 4
    # decay reached: one past the first (1-based) index below 10 mu
    assert nystrom.next_rank([10.0, 5.0, 0.05, 0.01], mu, 4, 30, 20) == 4      # i = 3
    assert nystrom.next_rank([10.0, 0.05, 0.01, 0.0], mu, 4, 30, 20) == 3      # i = 2
    assert nystrom.next_rank([0.09, 0.05, 0.01, 0.0], mu, 4, 30, 20) == 2      # i = 1
    lam = np.concatenate([np.full(7, 3.0), np.full(3, 1e-9)])
    assert nystrom.next_rank(lam, mu, 10, 30, 20) == 9                         # i = 8
    assert nystrom.next_rank(lam, mu, 10, 5, 20) == 5                          # capped
    # lambda_hat_ell exactly 10 mu: no index is below it, the rank stays (reading)
    assert nystrom.next_rank([1.0, 0.5, 0.1], mu, 3, 30, 20) == 3
    # 0.1 is not below 10 mu, 0.0999 is
    assert nystrom.next_rank([1.0, 0.1, 0.0999], mu, 3, 30, 20) == 4


def test_adaptive_damping_is_the_larger_of_the_two_rules():
    eps = 2.0 ** -52
    assert nystrom.mu_adaptive(1e3, 1e-6, gamma=10.0, coef=1e-4) == 10.0 * eps * 1e3   # late: Alg. 4 value
    assert nystrom.mu_adaptive(1e3, 2.0, gamma=10.0, coef=1e-4) == 4e-4                # early: 1e-4 L^2
    assert nystrom.mu_adaptive(0.0, 0.0) == 0.0


def test_nystrom_ngd_grows_the_rank_then_caps_it_and_decreases_the_loss():
    pr, th = inputs.small_problem(d=2, widths=[2, 6, 5, 1], n_int=30, n_bnd=10, seed=3)
    theta, infos, ells = solve.nystrom_ngd(pr, th, steps=5, ell0=4, ell_max=14, ell_delta=4, rtol=1e-10,
                                           maxit=400, seed=1, mu_loss_coef=1e-4)
    for k, info in enumerate(infos):
        expect_grow = info.lam_ell > 10.0 * info.mu
        if expect_grow:
            assert info.ell_next == min(ells[k] + 4, 14)
        else:
            assert info.ell_next <= ells[k] + 1
        assert info.mu >= 1e-4 * info.loss_before ** 2 * (1 - 1e-15)
        assert info.loss_after <= info.loss_before
        if k + 1 < len(ells):
            assert ells[k + 1] == info.ell_next
    assert ells[0] == 4 and max(ells) <= 14
    assert infos[-1].loss_after < infos[0].loss_before


# ---------------------------------------------------------------------------- sampling test matrix (Sec. 3, Sec. 5)
def test_sampling_takes_the_only_positive_entries_and_rejects_too_few():
    d = np.array([0.0, 2.0, 0.0, 5.0, -1.0, 1e-300])
    assert list(nystrom.sampling_indices(d, 3, seed=4, step=1)) == [1, 3, 5]
    with pytest.raises(ValueError):
        nystrom.sampling_indices(d, 4, seed=4, step=1)


def test_sampling_matches_sequential_draws_without_replacement():
    """Inclusion frequencies of the exponential race against the exact probabilities of drawing two
    indices one after another proportionally to the weights among those left (brute force)."""
    wts = np.array([4.0, 3.0, 2.0, 1.0])
    W = wts.sum()
    pair = {}
    for i in range(4):
        for j in range(4):
            if i != j:
                key = tuple(sorted((i, j)))
                pair[key] = pair.get(key, 0.0) + wts[i] / W * wts[j] / (W - wts[i])
    n = 6000
    counts = {}
    for seed in range(n):
        key = tuple(int(x) for x in nystrom.sampling_indices(wts, 2, seed=seed, step=3))
        counts[key] = counts.get(key, 0) + 1
    assert set(counts) <= set(pair)
    for key, pr in pair.items():
        f = counts.get(key, 0) / n
        assert abs(f - pr) <= 4.5 * np.sqrt(pr * (1 - pr) / n), (key, f, pr)


def test_sampled_nystrom_is_the_column_nystrom_approximation():
    """With Omega = I[:, S], App. A reproduces Eq. nystrom_approx: G[:, S] G[S, S]^{-1} G[S, :]."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((40, 25))
    G = A.T @ A / 40.0
    S = nystrom.sampling_indices(np.diag(G), 8, seed=2, step=0)
    Om = nystrom.selection_matrix(S, 25)
    assert np.array_equal(np.abs(nystrom.thin_qr(Om)), Om)            # already orthonormal
    U, lam, nu = nystrom.nystrom_factor(Om, G @ Om)
    Ghat = nystrom.nystrom_matrix(U, lam)
    ref = G[:, S] @ np.linalg.solve(G[np.ix_(S, S)], G[S, :])
    assert np.linalg.norm(Ghat - ref) <= 1e-9 * np.linalg.norm(ref)


def test_ngd_step_with_sampling_test_matrix_decreases_the_loss():
    pr, th = inputs.small_problem(d=2, widths=[2, 6, 5, 1], n_int=30, n_bnd=10, seed=5)
    th1, info = solve.ngd_step(pr, th, ell=12, mu=None, rtol=1e-10, maxit=400, seed=3, step=1,
                               test_matrix="sampling")
    assert info.loss_after < info.loss_before


# ---------------------------------------------------------------------------- RPCholesky (Sec. 3, App. B, Alg. 5)
def _decaying_psd(p=30, n=60, rate=3.0, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, p)) * np.exp(-np.arange(p) / rate)[None, :]
    return A.T @ A / n


def test_rpcholesky_is_the_nystrom_approximation_of_its_pivots():
    """F F^T = G[:, S] G[S, S]^{-1} G[S, :] (RPCholesky equals Nystrom with the pivot columns),
    and the residual diagonal sums to the trace-norm error tr(G - F F^T)."""
    G = _decaying_psd()
    F, piv = nystrom.rpcholesky_block(lambda S: G[:, S], np.diag(G), 5, 3, 0.0, 3, 1)
    S = np.array(piv)
    ref = G[:, S] @ np.linalg.solve(G[np.ix_(S, S)], G[S, :])
    assert np.linalg.norm(F @ F.T - ref) <= 1e-9 * np.linalg.norm(G)
    d = np.maximum(np.diag(G) - np.sum(F * F, axis=1), 0.0)
    assert abs(d.sum() - np.trace(G - F @ F.T)) <= 1e-12 * np.trace(G)


def test_rpcholesky_is_exact_on_a_low_rank_matrix():
    rng = np.random.default_rng(4)
    B = rng.standard_normal((25, 6))
    G = B @ B.T
    F, piv = nystrom.rpcholesky_block(lambda S: G[:, S], np.diag(G), 4, 10, 1e-10 * np.trace(G), 5, 0)
    # a round of 4 pivots can overshoot rank 6 by columns of rounding size; it stops right after
    assert 6 <= F.shape[1] <= 6 + 3
    assert np.linalg.norm(G - F @ F.T) <= 1e-10 * np.linalg.norm(G)
    assert np.linalg.matrix_rank(F, tol=1e-6 * np.linalg.norm(F)) == 6


def test_rpcholesky_pivots_are_drawn_proportionally_to_the_diagonal():
    """The first sample of the first round follows d / sum(d) (one race per sample)."""
    d = np.array([1.0, 2.0, 3.0, 4.0])
    n = 5000
    hits = np.zeros(4)
    for seed in range(n):
        u = philox.rpchol_uniforms(4, 1, 0, seed, 2)[:, 0]
        hits[int(np.argmin(-np.log(u) / d))] += 1
    pr = d / d.sum()
    assert np.all(np.abs(hits / n - pr) <= 4.5 * np.sqrt(pr * (1 - pr) / n))


def test_rpchol_preconditioner_is_the_inverse_of_ffT_plus_mu():
    rng = np.random.default_rng(6)
    F = rng.standard_normal((20, 7))
    mu = 0.3
    v = rng.standard_normal(20)
    z = nystrom.rpchol_precond_apply(F, mu, v)
    assert np.linalg.norm(z - np.linalg.solve(F @ F.T + mu * np.eye(20), v)) <= 1e-12 * np.linalg.norm(z)
    U, s, _ = np.linalg.svd(F, full_matrices=False)         # Eq. rpchol_svdprecond
    z2 = (v - U @ (U.T @ v)) / mu + U @ ((U.T @ v) / (s * s + mu))
    assert np.linalg.norm(z - z2) <= 1e-12 * np.linalg.norm(z)
    assert np.array_equal(nystrom.rpchol_precond_apply(np.zeros((20, 0)), mu, v), v / mu)


def test_power_method_estimate_with_a_spectral_gap():
    """Four matrix-vector products: the estimate is the Rayleigh quotient of G^3 v0, in closed form
    sum c_i^2 lambda_i^7 / sum c_i^2 lambda_i^6 (c = Q^T v0), and with lambda_2 / lambda_1 = 0.05
    it is within ~0.05^6 of lambda_1."""
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    lam = np.concatenate([[10.0, 0.5], np.linspace(0.4, 0.01, 10)])
    G = (Q * lam) @ Q.T
    v0 = philox.power_start(12, 3, 0)
    est = nystrom.power_lambda1(lambda v: G @ v, v0, 4)
    c2 = (Q.T @ v0) ** 2
    assert abs(est - np.sum(c2 * lam ** 7) / np.sum(c2 * lam ** 6)) <= 1e-13 * 10.0
    assert abs(est - 10.0) <= 1e-5 * 10.0


def test_rpchol_ngd_step_decreases_the_loss():
    pr, th = inputs.small_problem(d=2, widths=[2, 6, 5, 1], n_int=30, n_bnd=10, seed=7)
    th1, info = solve.ngd_step(pr, th, ell=20, mu=None, rtol=1e-10, maxit=400, seed=2, step=0, precond="rpchol",
                               rpchol_block=5, mu_loss_coef=1e-4)
    assert info.loss_after < info.loss_before
    assert 1 <= info.ell_next <= 20


def test_ngd_full_step_solves_the_damped_system():
    """NGD full (Alg. 2): the direction solves (G + mu I) d = g to rounding, with mu from the power
    method, and the step decreases the loss."""
    pr, th = inputs.small_problem(d=2, widths=[2, 6, 5, 1], n_int=30, n_bnd=10, seed=8)
    th1, info, parts = solve.ngd_step(pr, th, ell=1, mu=None, rtol=0.0, maxit=1, seed=1, step=0, precond="full",
                                      return_parts=True)
    G, g, d = parts["G"], parts["g"], parts["d"]
    assert info.mu == pytest.approx(10 * 2.0 ** -52 * info.lam1, rel=1e-15)
    assert info.lam1 <= np.linalg.eigvalsh(G)[-1] * (1 + 1e-12)
    res = G @ d + info.mu * d - g
    assert np.linalg.norm(res) <= 1e-6 * np.linalg.norm(g)
    assert info.loss_after < info.loss_before
