"""Pins for oracle/mlp.py: closed forms and finite differences (no GPU)."""
import math

import numpy as np
import pytest

from oracle import mlp
from paper_2505_11638_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _fd_laplacian(fn, X, h, dims):
    lap = np.zeros(X.shape[0])
    f0 = fn(X)
    for k in dims:
        e = np.zeros(X.shape[1])
        e[k] = h
        lap += (fn(X + e) - 2.0 * f0 + fn(X - e)) / (h * h)
    return lap


def _fd_grad(fn, X, h):
    g = np.zeros_like(X)
    for k in range(X.shape[1]):
        e = np.zeros(X.shape[1])
        e[k] = h
        g[:, k] = (fn(X + e) - fn(X - e)) / (2 * h)
    return g


def test_param_counts_match_configs():
    # p = sum_l (n_l n_{l-1} + n_l) (Sec. 2.3) for the five workload networks.
    assert mlp.num_params([2, 32, 32, 1]) == 1185
    assert mlp.num_params([5, 64, 64, 64, 1]) == 8769
    assert mlp.num_params([10, 128, 128, 128, 128, 1]) == 51073
    assert mlp.num_params([4, 256, 256, 256, 1]) == 133121
    assert mlp.num_params([3, 64, 64, 64, 1]) == 8641


@pytest.mark.parametrize("name", ["poisson2d", "poisson5d", "heat4d"])
def test_manufactured_source_matches_pde(name):
    """f (and g) of the generators solve the PDE: -Delta u* = f, u*_t = kappa Delta u*."""
    wl, _ = inputs.make_workload(name, seed=3)
    pr = wl.problems[0]
    X = pr.X[:200]
    h = 1e-4
    fn = lambda x: inputs.u_star(pr, x)
    if pr.pde == "poisson":
        lap = _fd_laplacian(fn, X, h, range(pr.d))
        np.testing.assert_allclose(-lap, pr.target[:200], rtol=1e-5, atol=1e-6)
    else:
        lap = _fd_laplacian(fn, X, h, range(1, 4))
        ut = _fd_grad(fn, X, 1e-6)[:, 0]
        np.testing.assert_allclose(ut - pr.kappa * lap, 0.0, atol=1e-6)
    # boundary values are u* itself, and boundary points lie on a face
    xb = pr.X[pr.n_int:]
    np.testing.assert_allclose(pr.target[pr.n_int:], inputs.u_star(pr, xb), rtol=0, atol=0)
    sp = xb[:, 1:] if pr.pde == "heat" else xb
    on_face = np.any((sp == 0.0) | (sp == 1.0), axis=1)
    if pr.pde == "heat":
        on_face |= xb[:, 0] == 0.0
    assert on_face.all()


def test_one_hidden_layer_closed_form():
    """Special case with a closed form: u = sum_j c_j tanh(w_j.x + b_j) + c0 gives
    grad u = sum_j c_j tanh'(a_j) w_j and Delta u = sum_j c_j tanh''(a_j) ||w_j||^2."""
    rng = np.random.default_rng(1)
    d, n = 3, 7
    widths = [d, n, 1]
    theta = rng.standard_normal(mlp.num_params(widths))
    (W1, b1), (W2, b2) = mlp.unpack(theta, widths)
    X = rng.uniform(0, 1, size=(11, d))
    u, gu, lu, _ = mlp.taylor_forward(theta, widths, X, np.ones(d, bool))
    a = X @ W1.T + b1
    t = np.tanh(a)
    d1 = 1 - t ** 2
    d2 = -2 * t * d1
    np.testing.assert_allclose(u, t @ W2[0] + b2[0], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(gu, (d1 * W2[0]) @ W1, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(lu, (d2 * W2[0]) @ np.sum(W1 ** 2, axis=1), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("pde", ["poisson", "heat"])
def test_forward_laplacian_vs_finite_differences(pde):
    pr, theta = inputs.small_problem(pde=pde, d=3, n_int=16, n_bnd=4, seed=2)
    spatial = mlp.spatial_mask(pde, pr.d)
    u, gu, lu, _ = mlp.taylor_forward(theta, pr.widths, pr.X, spatial)
    fn = lambda x: mlp.network_value(theta, pr.widths, x)
    np.testing.assert_allclose(u, fn(pr.X), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(gu, _fd_grad(fn, pr.X, 1e-6), rtol=1e-6, atol=1e-8)
    lap = _fd_laplacian(fn, pr.X, 1e-4, np.nonzero(spatial)[0])
    np.testing.assert_allclose(lu, lap, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("pde", ["poisson", "heat"])
def test_residual_definition(pde):
    pr, theta = inputs.small_problem(pde=pde, d=2 if pde == "poisson" else 4, seed=4)
    r, L = mlp.residual(pr, theta)
    fn = lambda x: mlp.network_value(theta, pr.widths, x)
    ni = pr.n_int
    if pde == "poisson":
        lap = _fd_laplacian(fn, pr.X[:ni], 1e-4, range(pr.d))
        np.testing.assert_allclose(r[:ni], lap + pr.target[:ni], rtol=1e-5, atol=1e-5)
    else:
        lap = _fd_laplacian(fn, pr.X[:ni], 1e-4, range(1, 4))
        ut = _fd_grad(fn, pr.X[:ni], 1e-6)[:, 0]
        np.testing.assert_allclose(r[:ni], ut - pr.kappa * lap - pr.target[:ni], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(r[ni:], fn(pr.X[ni:]) - pr.target[ni:], rtol=1e-14, atol=1e-14)
    assert L == pytest.approx(0.5 * sum(pr.w[i] * r[i] ** 2 for i in range(r.size)), rel=1e-14)


@pytest.mark.parametrize("pde", ["poisson", "heat"])
def test_jacobian_vs_finite_differences(pde):
    pr, theta = inputs.small_problem(pde=pde, d=3 if pde == "poisson" else 4, n_int=10, n_bnd=4, seed=5)
    J = mlp.jacobian(pr, theta)
    assert J.shape == (pr.n, pr.p)
    rng = np.random.default_rng(0)
    h = 1e-6
    cols = rng.choice(pr.p, size=min(pr.p, 100), replace=False)
    for j in cols:
        e = np.zeros(pr.p)
        e[j] = h
        fd = (mlp.residual(pr, theta + e)[0] - mlp.residual(pr, theta - e)[0]) / (2 * h)
        np.testing.assert_allclose(J[:, j], fd, rtol=1e-6, atol=1e-7 * (1 + np.abs(fd).max()))
    for _ in range(8):
        v = rng.standard_normal(pr.p)
        fd = (mlp.residual(pr, theta + h * v)[0] - mlp.residual(pr, theta - h * v)[0]) / (2 * h)
        np.testing.assert_allclose(J @ v, fd, rtol=1e-6, atol=1e-7 * (1 + np.abs(fd).max()))


def test_gradient_vs_finite_differences():
    pr, theta = inputs.small_problem(d=2, n_int=20, n_bnd=6, seed=6)
    g, r, L = mlp.gradient(pr, theta)
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(8):
        v = rng.standard_normal(pr.p)
        fd = (mlp.residual(pr, theta + h * v)[1] - mlp.residual(pr, theta - h * v)[1]) / (2 * h)
        assert g @ v == pytest.approx(fd, rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("pde", ["poisson", "heat"])
def test_jvp_vjp_adjoint_and_fd(pde):
    pr, theta = inputs.small_problem(pde=pde, d=3 if pde == "poisson" else 4, seed=7)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(pr.p)
    c = rng.standard_normal(pr.n)
    Jv = mlp.jvp(pr, theta, v)
    JTc = mlp.vjp(pr, theta, c)
    lhs, rhs = Jv @ c, v @ JTc
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0) * 10
    h = 1e-6
    fd = (mlp.residual(pr, theta + h * v)[0] - mlp.residual(pr, theta - h * v)[0]) / (2 * h)
    np.testing.assert_allclose(Jv, fd, rtol=1e-6, atol=1e-7 * (1 + np.abs(fd).max()))
    J = mlp.jacobian(pr, theta)
    np.testing.assert_allclose(J @ v, Jv, rtol=1e-12, atol=1e-12 * np.abs(Jv).max())
    np.testing.assert_allclose(J.T @ c, JTc, rtol=1e-12, atol=1e-12 * np.abs(JTc).max())


def test_jacobian_row_subsets_agree():
    pr, theta = inputs.small_problem(d=2, n_int=12, n_bnd=5, seed=8)
    J = mlp.jacobian(pr, theta)
    rows = np.array([0, 3, 11, 12, 16])
    np.testing.assert_allclose(mlp.jacobian(pr, theta, rows), J[rows], rtol=0, atol=0)


def test_theta_layout_row_major():
    """The flat index of W_l(i, j) is off_l + i n_in + j, then b_l (Sec. 2.3 stacking)."""
    widths = [2, 3, 1]
    theta = np.arange(mlp.num_params(widths), dtype=float)
    (W1, b1), (W2, b2) = mlp.unpack(theta, widths)
    assert W1[1, 0] == 2 and W1[2, 1] == 5 and b1.tolist() == [6, 7, 8]
    assert W2.tolist() == [[9, 10, 11]] and b2.tolist() == [12]


@pytest.mark.parametrize("name", ["poisson3d", "heat4d"])
def test_grad_u_star_matches_central_differences(name):
    """The manufactured solution's gradient (used for H1 errors) against central differences."""
    wl, _ = inputs.make_workload(name, seed=0)
    pr = wl.problems[0]
    x = inputs.eval_points(pr, 64, seed=1)
    g = inputs.grad_u_star(pr, x)
    h = 1e-6
    for i in range(pr.d):
        e = np.zeros(pr.d)
        e[i] = h
        fd = (inputs.u_star(pr, x + e) - inputs.u_star(pr, x - e)) / (2 * h)
        np.testing.assert_allclose(g[:, i], fd, rtol=1e-7, atol=1e-8)
