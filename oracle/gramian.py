"""Oracle: the Gramian of Thm. 1, its matvec and diagonal, and the direct damped solve.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Thm. 1 (Eq. G_matrixfree): with quadrature weights w_r (and phi = 1 for the PINN
metric), G = J^T diag(w) J, where J is the Jacobian of the residual rows.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def gramian(J, w):
    """Explicit G = J^T diag(w) J (Eq. G_matrixfree; the 'precompute Gramian' strategy)."""
    return J.T @ (w[:, None] * J)


def gramian_mv(J, w, v, mu=0.0):
    """(G + mu I) v = J^T (w * (J v)) + mu v ('precompute Jacobian only', Sec. 4.1.2)."""
    return J.T @ (w * (J @ v)) + mu * v


def gramian_mv_blocked(jac_rows, n, w, v, mu=0.0, block=2048):
    """(G + mu I) v with the Jacobian formed one point block at a time (Eq. G_matrixfree_batch).

    ``jac_rows(rows)`` returns J[rows, :].
    """
    y = mu * np.asarray(v, dtype=np.float64)
    for s in range(0, n, block):
        rows = np.arange(s, min(n, s + block))
        Jb = jac_rows(rows)
        y = y + Jb.T @ (w[rows] * (Jb @ v))
    return y


def gramian_diag(J, w):
    """diag(G) = sum_r w_r (grad_theta r_r)^2 elementwise (Eq. gram_diagonal)."""
    return np.einsum("r,rj,rj->j", w, J, J)


def direct_direction(G, g, mu):
    """d = (G + mu I)^{-1} g by Cholesky and two triangular solves (Alg. 2, fixed mu)."""
    c = scipy.linalg.cho_factor(G + mu * np.eye(G.shape[0]), lower=False)
    return scipy.linalg.cho_solve(c, g)
