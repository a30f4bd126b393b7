"""Oracle: tanh MLP, forward-Laplacian residual, Jacobian rows, JVP and VJP (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Network (Sec. 2.3): x_0 = x, x_l = tanh(W_l x_{l-1} + b_l) for the L hidden
layers, u = W_{L+1} x_L + b_{L+1}; theta = [W_1, b_1, ..., W_{L+1}, b_{L+1}] with
each W_l stored row-major (n_l x n_{l-1}).

Residuals (Sec. 2.2.1 and Sec. 5.1, Eq. energy_poisson): the least-squares energy
E = 1/2 ||F(u) - f||^2 + 1/2 ||u - g||^2 discretised by Monte-Carlo quadrature,
L(theta) = 1/2 sum_r w_r r_r^2 with
    Poisson interior   r = Delta u + f          (the paper's sign, Eq. energy_poisson)
    heat interior      r = u_t - kappa Delta u - f   (f = 0 for the manufactured u*)
    boundary/initial   r = u - g.
Each r_r is linear in the output "channels" (u, grad u, Delta u) of one point, so
the Jacobian J[r, :] = grad_theta r_r is the Jacobian of Thm. 1 with the
stop-gradient metric: phi = 1 and F_u linear (Remark metrics_examples; the PINN
metric of Eq. metric_poisson is Gauss-Newton on r).

Taylor mode (derived by hand, not by an AD tool).  Every point carries the
channels c = (value, d gradient entries, Laplacian).  Through a hidden layer,
with a = W x + b, t = tanh a, s1 = 1 - t^2 = tanh', s2 = -2 t s1 = tanh'',
s3 = -2 s1 (1 - 3 t^2) = tanh''', and q = sum_{k spatial} (grad_k a)^2:
    x' = t,   grad x' = s1 grad a,   Delta x' = s1 Delta a + s2 q.
For the heat equation coordinate 0 is time: its gradient channel is carried
(u_t is needed) but excluded from q (the Laplacian is spatial only).
"""
from __future__ import annotations

import numpy as np

POISSON = "poisson"
HEAT = "heat"


# ----------------------------------------------------------------------------- layout
def layer_shapes(widths):
    return [(widths[i + 1], widths[i]) for i in range(len(widths) - 1)]


def num_params(widths) -> int:
    return int(sum(o * i + o for o, i in layer_shapes(widths)))


def unpack(theta, widths):
    """theta -> [(W_l, b_l)], W_l row-major (n_out x n_in) then b_l (Sec. 2.3)."""
    out, off = [], 0
    for n_out, n_in in layer_shapes(widths):
        W = theta[off:off + n_out * n_in].reshape(n_out, n_in)
        off += n_out * n_in
        b = theta[off:off + n_out]
        off += n_out
        out.append((W, b))
    assert off == theta.size, "theta has the wrong length for these widths"
    return out


def spatial_mask(pde: str, d: int) -> np.ndarray:
    """Which gradient channels enter the Laplacian: all for Poisson, 1..3 for heat (t first)."""
    m = np.ones(d, dtype=bool)
    if pde == HEAT:
        m[0] = False
    return m


# ----------------------------------------------------------------------------- forward
def taylor_forward(theta, widths, X, spatial):
    """Forward Laplacian of u_theta at the points X (N, d).

    Returns u (N,), grad u (N, d), Delta u (N,) and the per-layer cache that the
    reverse pass needs.  Gradient arrays are laid out (N, d, n).
    """
    layers = unpack(theta, widths)
    N, d = X.shape
    x = X.copy()
    gx = np.broadcast_to(np.eye(d)[None, :, :], (N, d, d)).copy()   # grad of x_0 = identity
    lx = np.zeros((N, d))                                             # Delta of x_0 = 0
    cache = []
    n_hidden = len(layers) - 1
    for l, (W, b) in enumerate(layers):
        a = x @ W.T + b
        ga = gx @ W.T
        la = lx @ W.T
        if l < n_hidden:
            t = np.tanh(a)
            s1 = 1.0 - t * t
            s2 = -2.0 * t * s1
            s3 = -2.0 * s1 * (1.0 - 3.0 * t * t)
            q = np.sum(ga[:, spatial, :] ** 2, axis=1)
            cache.append(dict(x=x, gx=gx, lx=lx, ga=ga, la=la, s1=s1, s2=s2, s3=s3, q=q))
            x, gx, lx = t, s1[:, None, :] * ga, s1 * la + s2 * q
        else:
            cache.append(dict(x=x, gx=gx, lx=lx))
            return a[:, 0], ga[:, :, 0], la[:, 0], cache
    raise AssertionError("unreachable")


def _channels_to_residual(problem, u, gu, lu):
    """r from the output channels (Sec. 2.2.1 energies; see the module docstring)."""
    ni = problem.n_int
    r = np.empty_like(u)
    if problem.pde == POISSON:
        r[:ni] = lu[:ni] + problem.target[:ni]
    else:
        r[:ni] = gu[:ni, 0] - problem.kappa * lu[:ni] - problem.target[:ni]
    r[ni:] = u[ni:] - problem.target[ni:]
    return r


def residual(problem, theta):
    """Residual vector r (N,) and loss L = 1/2 sum_r w_r r_r^2."""
    spatial = spatial_mask(problem.pde, problem.X.shape[1])
    u, gu, lu, _ = taylor_forward(theta, problem.widths, problem.X, spatial)
    r = _channels_to_residual(problem, u, gu, lu)
    return r, 0.5 * float(np.sum(problem.w * r * r))


def network_value(theta, widths, X):
    """u_theta(X) only (plain forward, for error metrics)."""
    x = X
    layers = unpack(theta, widths)
    for l, (W, b) in enumerate(layers):
        x = x @ W.T + b
        if l < len(layers) - 1:
            x = np.tanh(x)
    return x[:, 0]


# ----------------------------------------------------------------------------- reverse
def _output_seeds(problem, rows, scale):
    """Cotangents of the output channels (u, grad u, Delta u) that give scale * r."""
    d = problem.X.shape[1]
    n = rows.size
    su, sg, sl = np.zeros(n), np.zeros((n, d)), np.zeros(n)
    interior = rows < problem.n_int
    if problem.pde == POISSON:
        sl[interior] = 1.0
    else:
        sg[interior, 0] = 1.0
        sl[interior] = -problem.kappa
    su[~interior] = 1.0
    return su * scale, sg * scale[:, None], sl * scale


def _reverse(problem, theta, rows, scale):
    """Per-layer adjoints (abar, grad abar, Delta abar) of a = W x + b for each point.

    Adjoint of a tanh layer (transpose of the Taylor-mode forward, by hand):
        abar      = s1 xbar' + s2 sum_k grad_k a grad_k xbar' + (s2 Delta a + s3 q) Deltaxbar'
        grad_k abar = s1 grad_k xbar' + 2 s2 grad_k a Deltaxbar'   (second term spatial k only)
        Delta abar  = s1 Deltaxbar'
    and of a linear layer: (xbar, grad xbar, Delta xbar) = W^T (abar, grad abar, Delta abar).
    """
    spatial = spatial_mask(problem.pde, problem.X.shape[1])
    X = problem.X[rows]
    _, _, _, cache = taylor_forward(theta, problem.widths, X, spatial)
    layers = unpack(theta, problem.widths)
    su, sg, sl = _output_seeds(problem, rows, scale)
    abar, gabar, labar = su[:, None], sg[:, :, None], sl[:, None]
    adjoints = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        adjoints[l] = (abar, gabar, labar)
        if l == 0:
            break
        W = layers[l][0]
        xbar, gxbar, lxbar = abar @ W, gabar @ W, labar @ W
        c = cache[l - 1]
        sp = spatial[None, :, None]
        abar = (c["s1"] * xbar + c["s2"] * np.sum(c["ga"] * gxbar, axis=1)
                + (c["s2"] * c["la"] + c["s3"] * c["q"]) * lxbar)
        gabar = c["s1"][:, None, :] * gxbar + np.where(sp, 2.0 * c["s2"][:, None, :] * c["ga"] * lxbar[:, None, :], 0.0)
        labar = c["s1"] * lxbar
    return cache, adjoints


def jacobian(problem, theta, rows=None):
    """Explicit Jacobian rows J[r, :] = grad_theta r_r for the given rows (all by default).

    For W_l the entry of point r is sum over channels c of Abar_l[c, i] X_{l-1}[c, j]
    (value, gradient and Laplacian channels); for b_l it is abar_l[i].
    """
    rows = np.arange(problem.X.shape[0]) if rows is None else np.asarray(rows)
    cache, adj = _reverse(problem, theta, rows, np.ones(rows.size))
    blocks = []
    for l, (abar, gabar, labar) in enumerate(adj):
        c = cache[l]
        JW = (np.einsum("ni,nj->nij", abar, c["x"]) + np.einsum("nki,nkj->nij", gabar, c["gx"])
              + np.einsum("ni,nj->nij", labar, c["lx"]))
        blocks.append(JW.reshape(rows.size, -1))
        blocks.append(abar)
    return np.concatenate(blocks, axis=1)


def vjp(problem, theta, cot):
    """J^T cot for a cotangent cot (N,), by the reverse pass summed over points."""
    rows = np.arange(problem.X.shape[0])
    cache, adj = _reverse(problem, theta, rows, np.asarray(cot, dtype=np.float64))
    parts = []
    for l, (abar, gabar, labar) in enumerate(adj):
        c = cache[l]
        W_bar = abar.T @ c["x"] + np.einsum("nki,nkj->ij", gabar, c["gx"]) + labar.T @ c["lx"]
        parts.append(W_bar.ravel())
        parts.append(abar.sum(axis=0))
    return np.concatenate(parts)


def gradient(problem, theta):
    """grad L = J^T (w * r) (the gradient of Alg. 1), with r and L."""
    r, L = residual(problem, theta)
    return vjp(problem, theta, problem.w * r), r, L


def jvp(problem, theta, v):
    """J v by forward-mode tangents of the Taylor-mode forward (independent of the reverse pass).

    Tangent rules through a tanh layer, with adot = Wdot x + W xdot + bdot etc.:
        xdot'       = s1 adot
        grad xdot'  = s2 adot grad a + s1 grad adot
        Delta xdot' = s1 Delta adot + s2 adot Delta a + 2 s2 sum_{k sp} grad_k a grad_k adot + s3 adot q
    """
    spatial = spatial_mask(problem.pde, problem.X.shape[1])
    layers = unpack(theta, problem.widths)
    dlayers = unpack(np.asarray(v, dtype=np.float64), problem.widths)
    X = problem.X
    N, d = X.shape
    x, xd = X.copy(), np.zeros_like(X)
    gx = np.broadcast_to(np.eye(d)[None], (N, d, d)).copy()
    gxd = np.zeros_like(gx)
    lx, lxd = np.zeros((N, d)), np.zeros((N, d))
    n_hidden = len(layers) - 1
    for l, ((W, b), (Wd, bd)) in enumerate(zip(layers, dlayers)):
        a, ad = x @ W.T + b, x @ Wd.T + xd @ W.T + bd
        ga, gad = gx @ W.T, gx @ Wd.T + gxd @ W.T
        la, lad = lx @ W.T, lx @ Wd.T + lxd @ W.T
        if l == n_hidden:
            u_d, gu_d, lu_d = ad[:, 0], gad[:, :, 0], lad[:, 0]
            break
        t = np.tanh(a)
        s1 = 1.0 - t * t
        s2 = -2.0 * t * s1
        s3 = -2.0 * s1 * (1.0 - 3.0 * t * t)
        q = np.sum(ga[:, spatial, :] ** 2, axis=1)
        qd = 2.0 * np.sum(ga[:, spatial, :] * gad[:, spatial, :], axis=1)
        x, xd = t, s1 * ad
        gx, gxd = s1[:, None, :] * ga, s2[:, None, :] * ad[:, None, :] * ga + s1[:, None, :] * gad
        lx, lxd = s1 * la + s2 * q, s1 * lad + s2 * ad * la + s2 * qd + s3 * ad * q
    out = np.empty(N)
    ni = problem.n_int
    if problem.pde == POISSON:
        out[:ni] = lu_d[:ni]
    else:
        out[:ni] = gu_d[:ni, 0] - problem.kappa * lu_d[:ni]
    out[ni:] = u_d[ni:]
    return out
