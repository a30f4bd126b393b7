"""Oracle: preconditioned CG, Armijo backtracking and one Nystrom-preconditioned NGD step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper solves (G + mu I) d = grad L with pCG (Sec. 4, Alg. 3) but prints no
pCG pseudocode; this is textbook preconditioned CG (Hestenes-Stiefel, Saad
Alg. 9.1) with x_0 = 0:
    r_0 = g, z_0 = P^{-1} r_0, p_0 = z_0
    repeat: q = A p; alpha = r^T z / p^T q; x += alpha p; r -= alpha q;
            stop when ||r|| <= rtol ||g|| or maxit iterations are done;
            z = P^{-1} r; beta = r_new^T z_new / r^T z; p = z + beta p.
The recurrence residual is the one tested (reading: the paper fixes only maxit).

Armijo (Sec. 4.4 "Algorithmic details", Alg. 1): alpha = 1, accept when
L(theta - alpha d) <= L(theta) - c1 alpha g^T d, else alpha <- rho alpha; the
constants are not printed (reading: c1 = 1e-4, rho = 1/2, at most 30 trials,
non-finite losses rejected, alpha = 0 if no trial is accepted).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import gramian as _gram
from . import mlp as _mlp
from . import nystrom as _nys
from . import philox as _philox


# Shift multipliers tried in turn when Omega^T Y_nu is not positive definite (reading: the paper
# fixes nu = eps(||Y||_F) and is silent on failures; the noise of a sketch summed over thousands
# of terms can exceed one spacing, so the shift grows by 8x up to 8^5).
SHIFT_SCALES = (1.0, 8.0, 64.0, 512.0, 4096.0, 32768.0)


class Breakdown(RuntimeError):
    """p^T (G + mu I) p <= 0 inside CG."""


def pcg(A, g, Pinv, rtol: float, maxit: int):
    """Returns (x, iterations, final recurrence relres ||r_k|| / ||g||)."""
    g = np.asarray(g, dtype=np.float64)
    x = np.zeros_like(g)
    gnorm = float(np.linalg.norm(g))
    if gnorm == 0.0 or maxit <= 0:
        return x, 0, 0.0 if gnorm == 0.0 else 1.0
    r = g.copy()
    z = Pinv(r) if Pinv is not None else r.copy()
    p = z.copy()
    rz = float(r @ z)
    for k in range(1, maxit + 1):
        q = A(p)
        pq = float(p @ q)
        if not pq > 0.0:
            raise Breakdown(f"p^T A p = {pq} at iteration {k}")
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        rn = float(np.linalg.norm(r))
        if rn <= rtol * gnorm or k == maxit:
            return x, k, rn / gnorm
        z = Pinv(r) if Pinv is not None else r.copy()
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    raise AssertionError("unreachable")


def armijo(loss_fn, theta, d, g, L0, c1=1e-4, rho=0.5, max_trials=30):
    """Backtracking along alpha -> theta - alpha d.  Returns (alpha, L(theta - alpha d), trials)."""
    slope = float(g @ d)
    alpha = 1.0
    for i in range(max_trials):
        L = loss_fn(theta - alpha * d)
        if np.isfinite(L) and L <= L0 - c1 * alpha * slope:
            return alpha, float(L), i + 1
        alpha *= rho
    return 0.0, float(L0), max_trials


@dataclass
class StepInfo:
    loss_before: float
    loss_after: float
    alpha: float
    mu: float
    lam1: float
    lam_ell: float
    nu: float
    pcg_iters: int
    relres: float
    armijo_trials: int
    ell_next: int = 0


def ngd_step(problem, theta, ell, mu, rtol, maxit, seed, step, mant_bits=52, gamma=10.0,
             c1=1e-4, rho=0.5, max_trials=30, return_parts=False, mu_loss_coef=0.0, ell_max=0, ell_delta=20,
             test_matrix="gaussian", precond="nystrom", rpchol_block=20):
    """One Nystrom-preconditioned matrix-free NGD step (Alg. 1 + Alg. 3 + Alg. 4).

    mu=None selects mu = gamma eps lambda_hat_1 (Alg. 4), raised to mu_loss_coef L(theta)^2 when
    mu_loss_coef > 0 (the damping of Sec. 5).  maxit caps pCG; rtol=0 runs exactly maxit
    iterations (for comparisons at a fixed iteration count).  ell_max > 0 applies the rank rule
    of Alg. 4 to the returned info.ell_next (otherwise ell_next = ell).  test_matrix "sampling"
    draws Omega = I[:, S] with S sampled proportionally to diag G (Sec. 3 and Sec. 5).
    precond "full" takes the direction of NGD full instead (Alg. 2): the explicit G, lambda_1 by four
    power-method steps, mu, Cholesky of G + mu I and two triangular solves (no pCG, ell unused).
    precond "rpchol" builds the RPCholNGD preconditioner instead (Alg. 5): diag G, lambda_1 by four
    power-method steps, mu, block RPCholesky of rank at most ell (blocks of rpchol_block, stopping
    when the trace of the residual is below mu p), P^{-1} by Woodbury (Eq. rpchol_precond);
    info.ell_next is then the rank found.
    """
    if precond == "rpchol":
        return _rpchol_step(problem, theta, ell, mu, rtol, maxit, seed, step, gamma, c1, rho, max_trials,
                            return_parts, mu_loss_coef, rpchol_block)
    if precond == "full":
        return _full_step(problem, theta, mu, seed, step, gamma, c1, rho, max_trials, return_parts, mu_loss_coef)
    g, r, L0 = _mlp.gradient(problem, theta)                       # Alg. 1: gradient
    J = _mlp.jacobian(problem, theta)                              # 'precompute Jacobian only'
    w = problem.w

    def G_apply(V):
        return J.T @ (w[:, None] * (J @ V)) if V.ndim == 2 else _gram.gramian_mv(J, w, V)

    if test_matrix == "sampling":
        S = _nys.sampling_indices(_gram.gramian_diag(J, w), ell, seed, step)
        Omega = _nys.selection_matrix(S, J.shape[1])                # columns of the identity
    else:
        Omega_raw = _philox.gaussian_test_matrix(J.shape[1], ell, seed, step)
        Omega = _nys.thin_qr(Omega_raw)                            # Alg. 4: randomized Nystrom (App. A)
    Y = G_apply(Omega)
    for scale in SHIFT_SCALES:          # a non-positive-definite core is retried with a larger shift
        try:
            U, lam, nu = _nys.nystrom_factor(Omega, Y, mant_bits, scale)
            break
        except np.linalg.LinAlgError:
            if scale == SHIFT_SCALES[-1]:
                raise
    if mu is not None:
        mu_eff = float(mu)
    elif mu_loss_coef > 0.0:
        mu_eff = _nys.mu_adaptive(lam[0], L0, gamma, mu_loss_coef)  # Sec. 5 damping
    else:
        mu_eff = _nys.mu_from_lambda1(lam[0], gamma)                 # Alg. 4: damping

    def A(v):
        return _gram.gramian_mv(J, w, v, mu_eff)

    def Pinv(v):
        return _nys.precond_apply(U, lam, mu_eff, v)

    d, iters, relres = pcg(A, g, Pinv, rtol, maxit)                # Alg. 3: direction by pCG

    def loss_fn(th):
        return _mlp.residual(problem, th)[1]

    alpha, L1, trials = armijo(loss_fn, theta, d, g, L0, c1, rho, max_trials)   # Alg. 1: line search
    ell_next = _nys.next_rank(lam, mu_eff, ell, ell_max, ell_delta) if ell_max > 0 else ell   # Alg. 4
    info = StepInfo(L0, L1, alpha, mu_eff, float(lam[0]), float(lam[-1]), nu, iters, relres, trials, ell_next)
    theta_new = theta - alpha * d                                   # Alg. 1: update
    if return_parts:
        return theta_new, info, dict(g=g, r=r, J=J, Omega=Omega, Y=Y, U=U, lam=lam, d=d)
    return theta_new, info


def nystrom_ngd(problem, theta0, steps, ell0, ell_max, ell_delta=20, rtol=1e-6, maxit=20, seed=0,
                gamma=10.0, mu_loss_coef=1e-4, mant_bits=52, pcg_iters=None):
    """NystromNGD over several steps (Alg. 1 with Alg. 3 and Alg. 4): adaptive damping and rank.

    Step k draws its test matrix from the Philox counter (seed, k) with rank ell_k, and
    ell_{k+1} = info.ell_next.  pcg_iters (a list) replays fixed iteration counts (rtol 0)
    instead of the rtol stop, for comparisons at equal iteration counts.
    Returns (theta, [StepInfo per step], [ell per step]).
    """
    theta = np.asarray(theta0, dtype=np.float64).copy()
    ell = int(ell0)
    infos, ells = [], []
    for k in range(steps):
        it_rtol, it_max = (0.0, int(pcg_iters[k])) if pcg_iters is not None else (rtol, maxit)
        theta, info = ngd_step(problem, theta, ell, None, it_rtol, it_max, seed, k, mant_bits=mant_bits,
                               gamma=gamma, mu_loss_coef=mu_loss_coef, ell_max=ell_max, ell_delta=ell_delta)
        infos.append(info)
        ells.append(ell)
        ell = info.ell_next
    return theta, infos, ells


def _rpchol_step(problem, theta, ell, mu, rtol, maxit, seed, step, gamma, c1, rho, max_trials, return_parts,
                 mu_loss_coef, b):
    """One RPCholNGD step (Alg. 1 with Alg. 3 and Alg. 5)."""
    g, r, L0 = _mlp.gradient(problem, theta)                       # Alg. 1: gradient
    J = _mlp.jacobian(problem, theta)
    w = problem.w
    p = J.shape[1]

    def G_apply(v):
        return _gram.gramian_mv(J, w, v)

    def G_cols(S):
        return J.T @ (w[:, None] * J[:, S])

    d0 = _gram.gramian_diag(J, w)                                   # Alg. 5: diagonal
    lam1 = _nys.power_lambda1(G_apply, _philox.power_start(p, seed, step), 4)   # Alg. 5: power method
    if mu is not None:
        mu_eff = float(mu)
    elif mu_loss_coef > 0.0:
        mu_eff = _nys.mu_adaptive(lam1, L0, gamma, mu_loss_coef)
    else:
        mu_eff = _nys.mu_from_lambda1(lam1, gamma)
    F, piv = _nys.rpcholesky_block(G_cols, d0, b, ell // b, mu_eff * p, seed, step)   # Alg. 5: RPCholesky

    def A(v):
        return _gram.gramian_mv(J, w, v, mu_eff)

    def Pinv(v):
        return _nys.rpchol_precond_apply(F, mu_eff, v)

    d, iters, relres = pcg(A, g, Pinv, rtol, maxit)                # Alg. 3: direction by pCG

    def loss_fn(th):
        return _mlp.residual(problem, th)[1]

    alpha, L1, trials = armijo(loss_fn, theta, d, g, L0, c1, rho, max_trials)   # Alg. 1: line search
    sig2 = np.linalg.svd(F, compute_uv=False) ** 2 if F.shape[1] else np.zeros(0)
    info = StepInfo(L0, L1, alpha, mu_eff, lam1, float(sig2[-1]) if sig2.size else 0.0, 0.0, iters, relres,
                    trials, F.shape[1])
    theta_new = theta - alpha * d                                   # Alg. 1: update
    if return_parts:
        return theta_new, info, dict(g=g, r=r, J=J, F=F, piv=piv, d=d, d0=d0)
    return theta_new, info


def _full_step(problem, theta, mu, seed, step, gamma, c1, rho, max_trials, return_parts, mu_loss_coef):
    """One step of NGD full (Alg. 1 with Alg. 2): direction d = (G + mu I)^{-1} g by Cholesky."""
    g, r, L0 = _mlp.gradient(problem, theta)                       # Alg. 1: gradient
    J = _mlp.jacobian(problem, theta)
    G = _gram.gramian(J, problem.w)                                 # Alg. 2: full Gramian
    lam1 = _nys.power_lambda1(lambda v: G @ v, _philox.power_start(G.shape[0], seed, step), 4)
    if mu is not None:
        mu_eff = float(mu)
    elif mu_loss_coef > 0.0:
        mu_eff = _nys.mu_adaptive(lam1, L0, gamma, mu_loss_coef)
    else:
        mu_eff = _nys.mu_from_lambda1(lam1, gamma)
    for scale in SHIFT_SCALES:          # a numerically indefinite G + mu I is retried with 8 mu, ...
        try:
            d = _gram.direct_direction(G, g, mu_eff)                # Alg. 2: Cholesky, two solves
            break
        except np.linalg.LinAlgError:
            if scale == SHIFT_SCALES[-1]:
                raise
            mu_eff *= 8.0

    def loss_fn(th):
        return _mlp.residual(problem, th)[1]

    alpha, L1, trials = armijo(loss_fn, theta, d, g, L0, c1, rho, max_trials)   # Alg. 1: line search
    info = StepInfo(L0, L1, alpha, mu_eff, lam1, 0.0, 0.0, 0, 0.0, trials, 0)
    theta_new = theta - alpha * d                                   # Alg. 1: update
    if return_parts:
        return theta_new, info, dict(g=g, r=r, J=J, G=G, d=d)
    return theta_new, info
