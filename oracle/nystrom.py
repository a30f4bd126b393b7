"""Oracle: randomized Nystrom approximation (App. A) and the Nystrom preconditioner (Alg. 4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

App. A, Alg. randomized_nystrom, in the paper's order:
    Omega = randn(p, ell);  Omega = qr(Omega, 0);  Y = G Omega;
    nu = eps(norm(Y, 'fro'));  Y_nu = Y + nu Omega;  C = chol(Omega^T Y_nu);
    B = Y_nu / C;  [U, Sigma, ~] = svd(B, 0);  Lambda = max(0, Sigma^2 - nu I).
Readings where the paper is silent (shared with the CUDA side):
  * qr is the thin QR normalised so that R has a positive diagonal (unique).
  * eps(x) is MATLAB's spacing at x in the precision Y was computed in: for a number
    format with m explicit mantissa bits, eps_m(x) = 2^(floor(log2 x) - m).  m = 52 (FP64)
    is the paper's algorithm; a sketch computed in double-float (pairs of FP32, 48 bits,
    "df"), FP32 (m = 23), TF32 (m = 10) or BF16 (m = 7) takes its own spacing, which keeps
    Omega^T Y_nu positive definite despite the rounding of Y (as eps(single(x)) would in
    MATLAB).
  * chol reads the symmetric part (Omega^T Y_nu + Y_nu^T Omega)/2 and returns the
    upper factor C with C^T C = that matrix (MATLAB's chol reads one triangle; the
    two agree in exact arithmetic).
Sampling test matrix (Sec. 3: columns of the identity; Sec. 5: drawn with probabilities
proportional to diag G): ell distinct indices drawn one after another, each with probability
proportional to diag G among the indices not yet drawn (reading: without replacement, since a
repeated column adds nothing to Omega).  Realised as an exponential race (Efraimidis & Spirakis,
2006): the ell smallest keys -ln(u_j) / (diag G)_j, ties to the smaller index, with u_j from
philox.sampling_uniforms; Omega = I[:, S] with S increasing.
Preconditioner, Alg. 4 (scaled form of Eq. nystrom_inverse):
    P^{-1} v = (lambda_ell + mu) U (Lambda + mu I)^{-1} U^T v + (I - U U^T) v.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import philox as _philox

EPS64 = 2.0 ** -52


def thin_qr(Omega):
    """Thin QR with a positive diagonal in R; returns Q (App. A, second step)."""
    Q, R = np.linalg.qr(Omega, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


MANTISSA_BITS = {"f64": 52, "df": 48, "f32": 23, "tf32": 10, "bf16": 7}


def shift(normY: float, mant_bits: int = 52) -> float:
    """nu = eps(||Y||_F) in a format with mant_bits explicit mantissa bits (reading above)."""
    if not normY > 0.0:
        return 0.0
    return float(np.ldexp(1.0, int(np.floor(np.log2(normY))) - mant_bits))


def nystrom_factor(Omega, Y, mant_bits: int = 52, shift_scale: float = 1.0):
    """Steps 4-9 of App. A given the orthonormal test matrix and Y = G Omega.

    mant_bits selects the precision whose eps gives the shift; shift_scale multiplies it (the
    step retries a non-positive-definite core with 8x and 64x).  Returns U (p, ell),
    lambda_hat (ell, descending) and the shift nu.  Raises numpy.linalg.LinAlgError if
    Omega^T Y_nu is not positive definite.
    """
    nu = shift_scale * shift(np.linalg.norm(Y, "fro"), mant_bits)
    Ynu = Y + nu * Omega
    M = Omega.T @ Ynu
    M = 0.5 * (M + M.T)
    C = np.linalg.cholesky(M).T                      # upper, C^T C = M
    B = scipy.linalg.solve_triangular(C, Ynu.T, trans="T", lower=False).T   # B C = Y_nu
    U, S, _ = np.linalg.svd(B, full_matrices=False)
    lam = np.maximum(0.0, S * S - nu)
    return U, lam, nu


def randomized_nystrom(G_apply, Omega_raw, mant_bits: int = 52):
    """The whole of App. A: orthonormalise, sketch Y = G Omega, factor."""
    Omega = thin_qr(Omega_raw)
    Y = G_apply(Omega)
    U, lam, nu = nystrom_factor(Omega, Y, mant_bits)
    return Omega, Y, U, lam, nu


def sampling_indices(diag, ell: int, seed: int, step: int) -> np.ndarray:
    """S: ell distinct indices, increasing, sampled proportionally to diag (see the module notes).
    Indices with diag <= 0 are never drawn; raises ValueError if fewer than ell are positive."""
    diag = np.asarray(diag, dtype=np.float64)
    pos = (diag > 0.0) & np.isfinite(diag)
    if int(pos.sum()) < ell:
        raise ValueError("fewer positive diagonal entries than the sample size")
    u = _philox.sampling_uniforms(diag.size, seed, step)
    keys = np.full(diag.size, np.inf)
    keys[pos] = -np.log(u[pos]) / diag[pos]
    order = np.lexsort((np.arange(diag.size), keys))     # by key, then by index
    return np.sort(order[:ell])


def selection_matrix(idx, p: int) -> np.ndarray:
    """Omega = I[:, idx] (p, ell)."""
    Om = np.zeros((p, len(idx)))
    Om[np.asarray(idx), np.arange(len(idx))] = 1.0
    return Om


def nystrom_matrix(U, lam):
    """G_hat = U diag(lambda_hat) U^T (only for small checks)."""
    return (U * lam[None, :]) @ U.T


def precond_apply(U, lam, mu, v):
    """P^{-1} v in the scaled form of Alg. 4."""
    Utv = U.T @ v
    return (lam[-1] + mu) * (U @ (Utv / (lam + mu))) + (v - U @ Utv)


def mu_from_lambda1(lam1: float, gamma: float = 10.0, eps: float = EPS64) -> float:
    """mu = gamma * eps_mach * lambda_hat_1 (Sec. 4.3 and Alg. 4)."""
    return gamma * eps * lam1


def mu_adaptive(lam1: float, loss: float, gamma: float = 10.0, coef: float = 1e-4, eps: float = EPS64) -> float:
    """The damping of the paper's experiments (Sec. 5): the larger of the Alg. 4 value and
    coef L(theta)^2, which regularises more strongly while the loss is large."""
    return max(mu_from_lambda1(lam1, gamma, eps), coef * loss * loss)


def next_rank(lam, mu: float, ell: int, ell_max: int, delta: int) -> int:
    """Rank of the next sketch (the rank update of Alg. 4), with the paper's 1-based index i.

    lambda_hat_ell > 10 mu: the approximation has not reached the decay yet, grow by delta up
    to ell_max.  Otherwise shrink to one past the first eigenvalue below 10 mu,
    min(min{i : lambda_hat_i < 10 mu} + 1, ell_max).  Reading where the paper is silent: when
    lambda_hat_ell equals 10 mu exactly no index qualifies, and the rank stays ell.
    """
    lam = np.asarray(lam, dtype=np.float64)
    assert lam.shape == (ell,)
    if lam[ell - 1] > 10.0 * mu:
        return min(ell + delta, ell_max)
    below = [i for i in range(1, ell + 1) if lam[i - 1] < 10.0 * mu]
    if not below:
        return ell
    return min(below[0] + 1, ell_max)


# ----------------------------------------------------------------------------- RPCholesky (Sec. 3, App. B)
# Block RPCholesky (the paper's block variant, after Epperly et al.): rounds of b pivots sampled
# i.i.d. proportionally to the residual diagonal d, then the residual block
#     C = G[:, S'] - F F[S', :]^T,  R = chol(C[S', S']),  new columns of F = C R^{-1},
#     d <- d - squared row norms of the new columns,
# stopping when sum(d) < eps or after t rounds.  Readings (the paper is silent):
#   * sample k of round i is the winner of an exponential race, argmin_j -ln(u_jk) / d_j, with u_jk
#     from Philox at counter (j, 2^30 + i b + k, step) (philox.rpchol_uniforms); the b winners are
#     made unique (S' increasing);
#   * d is clamped at 0 after each round and set to 0 on the pivots (their residual is zero);
#   * a round whose pivot block C[S', S'] is not numerically positive definite ends the
#     factorization with the columns found so far.
def rpcholesky_block(G_cols, d0, b: int, t: int, eps: float, seed: int, step: int):
    """F (p, r) with G ~ F F^T, and the pivots in selection order.  G_cols(S) returns G[:, S]."""
    d = np.maximum(np.asarray(d0, dtype=np.float64).copy(), 0.0)
    p = d.size
    cols, piv = [], []
    F = np.zeros((p, 0))
    for i in range(t):
        if not d.sum() >= eps or not np.any(d > 0.0):
            break
        u = _philox.rpchol_uniforms(p, b, i, seed, step)          # (p, b)
        keys = np.full((p, b), np.inf)
        pos = d > 0.0
        keys[pos, :] = -np.log(u[pos, :]) / d[pos, None]
        S = np.unique(np.argmin(keys, axis=0))
        C = G_cols(S) - F @ F[S, :].T
        try:
            L = np.linalg.cholesky(0.5 * (C[S, :] + C[S, :].T))
        except np.linalg.LinAlgError:
            break
        Fn = scipy.linalg.solve_triangular(L, C.T, lower=True).T    # C L^{-T} = C R^{-1}, R = L^T
        F = np.concatenate([F, Fn], axis=1)
        piv.extend(int(s) for s in S)
        d = np.maximum(d - np.sum(Fn * Fn, axis=1), 0.0)
        d[S] = 0.0
        if d.sum() < eps:
            break
    return F, piv


def rpchol_precond_apply(F, mu, v):
    """P^{-1} v for P = F F^T + mu I by the Woodbury identity with F^T F + mu I = R^T R
    (Eq. rpchol_precond): mu^{-1} (v - F R^{-1} R^{-T} F^T v)."""
    r = F.shape[1]
    if r == 0:
        return np.asarray(v, dtype=np.float64) / mu
    R = np.linalg.cholesky(F.T @ F + mu * np.eye(r)).T
    t = scipy.linalg.solve_triangular(R, scipy.linalg.solve_triangular(R, F.T @ v, trans="T"))
    return (v - F @ t) / mu


def power_lambda1(G_apply, v0, iters: int = 4) -> float:
    """lambda_1 of G by the power method (Alg. 5): v <- G v / ||G v|| from v0, the estimate the
    Rayleigh quotient v^T G v of the last step."""
    v = np.asarray(v0, dtype=np.float64) / np.linalg.norm(v0)
    lam = 0.0
    for _ in range(iters):
        w = G_apply(v)
        lam = float(v @ w)
        v = w / np.linalg.norm(w)
    return lam
