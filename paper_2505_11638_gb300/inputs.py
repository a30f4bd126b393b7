"""Seeded synthetic PINN problems shaped like the paper's workloads.

This module only *draws data*: collocation points, quadrature weights, the
manufactured solution's source and boundary values, and an initial parameter
vector.  It holds none of the method's arithmetic (no network evaluation, no
Jacobian, no Gramian, no solver), so both the FP64 oracle (through the tests)
and the CUDA library can consume the same arrays.

Workloads (the paper uses Monte-Carlo quadrature: points drawn uniformly once
and kept fixed for the run, Sec. 5 "Discretization and sampling strategies"):

* ``poisson2d``   -Delta u = f on [0,1]^2, u* = sin(pi x) sin(pi y), MLP 2-32-32-1,
                   900 interior + 120 boundary points, FP64, mu = 1e-6, ell = 100.
* ``poisson5d``   [0,1]^5, u* = prod sin(pi x_i), MLP 5-64-64-64-1, 4000 + 1000
                   points, FP32 activations, mu = 1e-7, ell = 500.
* ``poisson10d``  [0,1]^10, u* = prod sin(pi x_i / 2), MLP 10-128x4-1,
                   16384 + 4096 points, ell = 1000.
* ``heat4d``      u_t = kappa Delta u on [0,1]^3 x [0,1] (coordinate 0 is t),
                   kappa = 0.1, u* = exp(-3 kappa pi^2 t) prod sin(pi x_i),
                   MLP 4-256-256-256-1, 32768 interior + 8192 boundary/initial.
* ``batch64``     64 independent Poisson problems on [0,1]^3 with
                   u*_j = prod sin(k_j pi x_i), k_j in {1..4}, MLP 3-64x3-1,
                   N_int,j uniform in [1000, 8000], N_bnd,j = floor(N_int,j / 4).
* ``poisson3d``   [0,1]^3, u* = prod sin(pi x_i), MLP 3-64-64-64-1 (p = 8641), 10000 interior +
                   1000 boundary points: the paper's 3-D Poisson PINN, trained by NystromNGD
                   (adaptive rank from 20 up to 500, adaptive damping, pCG capped at 20 iterations).

Layout conventions (shared with the C ABI):
  X       (N, d) float64, row-major, interior rows first, then boundary rows.
  w       (N,)  float64 quadrature weights, uniform 1/N (N = interior + boundary).
  target  (N,)  float64: the source f at interior rows, the Dirichlet value g at
                boundary rows.
  theta   (p,)  float64: layer by layer, W_l row-major (n_l x n_{l-1}) then b_l
                (Sec. 2.3 stacks theta = [W_1, b_1, ..., W_{L+1}, b_{L+1}]).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

POISSON = "poisson"
HEAT = "heat"


@dataclass
class Problem:
    """One PINN problem instance: network shape, PDE, and its collocation data."""
    name: str
    pde: str
    widths: List[int]
    X: np.ndarray
    w: np.ndarray
    target: np.ndarray
    n_int: int
    n_bnd: int
    kappa: float = 0.0
    freq: float = 1.0          # k in u* = prod sin(k pi x_i) (Poisson)
    extra: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.widths[0]

    @property
    def n(self) -> int:
        return self.n_int + self.n_bnd

    @property
    def p(self) -> int:
        return num_params(self.widths)


@dataclass
class Workload:
    """A named workload: problem(s) plus the solver settings the config fixes."""
    name: str
    problems: List[Problem]
    dtype: str            # "f64" | "f32": working precision of activations / J
    ell: int
    mu: float | None      # None: mu = gamma * eps * lambda_hat_1 (Alg. 4)
    rtol: float
    steps: int
    sketch: str           # "f64" | "f32" | "tf32" | "bf16"


def num_params(widths) -> int:
    return int(sum(widths[i + 1] * widths[i] + widths[i + 1] for i in range(len(widths) - 1)))


def glorot_theta(widths, rng: np.random.Generator) -> np.ndarray:
    """Glorot/Xavier-uniform weights U(+-sqrt(6/(n_in+n_out))), zero biases."""
    parts = []
    for i in range(len(widths) - 1):
        n_in, n_out = widths[i], widths[i + 1]
        a = math.sqrt(6.0 / (n_in + n_out))
        parts.append(rng.uniform(-a, a, size=(n_out, n_in)).ravel())
        parts.append(np.zeros(n_out))
    return np.concatenate(parts).astype(np.float64)


def _boundary_box(rng, n, d, lo=0.0, hi=1.0):
    """Uniform on the boundary of [lo,hi]^d: a face uniformly among the 2d faces,
    then a uniform point on that face."""
    x = rng.uniform(lo, hi, size=(n, d))
    face = rng.integers(0, 2 * d, size=n)
    axis = face // 2
    side = np.where(face % 2 == 0, lo, hi)
    x[np.arange(n), axis] = side
    return x


def _sin_product(x, k):
    return np.prod(np.sin(k * math.pi * x), axis=1)


def poisson_problem(name, d, widths, n_int, n_bnd, rng, freq=1.0) -> Problem:
    """-Delta u = f on [0,1]^d with u* = prod_i sin(freq pi x_i).

    The closed form -Delta u* = d (freq pi)^2 u* gives f; g = u* on the boundary.
    """
    assert widths[0] == d and widths[-1] == 1
    xi = rng.uniform(0.0, 1.0, size=(n_int, d))
    xb = _boundary_box(rng, n_bnd, d)
    X = np.concatenate([xi, xb], axis=0)
    f = d * (freq * math.pi) ** 2 * _sin_product(xi, freq)
    g = _sin_product(xb, freq)
    n = n_int + n_bnd
    return Problem(name=name, pde=POISSON, widths=list(widths), X=X, w=np.full(n, 1.0 / n),
                   target=np.concatenate([f, g]), n_int=n_int, n_bnd=n_bnd, freq=freq)


def heat_problem(name, widths, n_int, n_bnd, kappa, rng) -> Problem:
    """u_t = kappa Delta u on [0,1]^3 x [0,1] with u* = exp(-3 kappa pi^2 t) prod sin(pi x_i).

    Coordinate 0 is t.  u* solves the equation exactly, so the interior source is 0.
    Boundary rows: 3/4 on the lateral faces (x_i in {0,1}, t uniform), 1/4 on the
    initial slice t = 0; g = u* there.
    """
    assert widths[0] == 4 and widths[-1] == 1
    ds = 3
    xi = rng.uniform(0.0, 1.0, size=(n_int, 4))
    n_lat = (3 * n_bnd) // 4
    n_ini = n_bnd - n_lat
    lat = np.empty((n_lat, 4))
    lat[:, 0] = rng.uniform(0.0, 1.0, size=n_lat)
    lat[:, 1:] = _boundary_box(rng, n_lat, ds)
    ini = np.empty((n_ini, 4))
    ini[:, 0] = 0.0
    ini[:, 1:] = rng.uniform(0.0, 1.0, size=(n_ini, ds))
    xb = np.concatenate([lat, ini], axis=0)
    X = np.concatenate([xi, xb], axis=0)

    def u_star(x):
        return np.exp(-3.0 * kappa * math.pi ** 2 * x[:, 0]) * _sin_product(x[:, 1:], 1.0)

    n = n_int + n_bnd
    return Problem(name=name, pde=HEAT, widths=list(widths), X=X, w=np.full(n, 1.0 / n),
                   target=np.concatenate([np.zeros(n_int), u_star(xb)]), n_int=n_int, n_bnd=n_bnd,
                   kappa=kappa)


def u_star(problem: Problem, x: np.ndarray) -> np.ndarray:
    """The manufactured solution of ``problem`` at points x (n, d)."""
    if problem.pde == POISSON:
        return _sin_product(x, problem.freq)
    return np.exp(-3.0 * problem.kappa * math.pi ** 2 * x[:, 0]) * _sin_product(x[:, 1:], 1.0)


def grad_u_star(problem: Problem, x: np.ndarray) -> np.ndarray:
    """First derivatives (n, d) of the manufactured solution of ``problem`` at points x (n, d)."""
    if problem.pde == POISSON:
        k = problem.freq * math.pi
        s, c = np.sin(k * x), np.cos(k * x)
        out = np.empty_like(x)
        for i in range(x.shape[1]):
            out[:, i] = k * c[:, i] * np.prod(np.delete(s, i, axis=1), axis=1)
        return out
    kappa = problem.kappa
    e = np.exp(-3.0 * kappa * math.pi ** 2 * x[:, 0])
    s, c = np.sin(math.pi * x[:, 1:]), np.cos(math.pi * x[:, 1:])
    out = np.empty_like(x)
    out[:, 0] = -3.0 * kappa * math.pi ** 2 * e * np.prod(s, axis=1)
    for i in range(3):
        out[:, 1 + i] = math.pi * e * c[:, i] * np.prod(np.delete(s, i, axis=1), axis=1)
    return out


def eval_points(problem: Problem, n_eval: int, seed: int) -> np.ndarray:
    """Independent interior points for error evaluation (10x the training set in the paper)."""
    rng = np.random.default_rng(seed + 7919)
    return rng.uniform(0.0, 1.0, size=(n_eval, problem.d))


WORKLOADS = ("poisson2d", "poisson5d", "poisson10d", "heat4d", "batch64", "poisson3d")


def make_workload(name: str, seed: int = 0) -> tuple[Workload, list[np.ndarray]]:
    """Build a named workload.  Returns (workload, [theta_0 per problem]).

    Per-workload seed = master seed + workload index, one PCG64 stream for points
    and initial parameters.
    """
    idx = WORKLOADS.index(name)
    rng = np.random.default_rng(seed + idx)
    if name == "poisson2d":
        widths = [2, 32, 32, 1]
        prob = poisson_problem(name, 2, widths, 900, 120, rng)
        wl = Workload(name, [prob], "f64", ell=100, mu=1e-6, rtol=1e-10, steps=1, sketch="f64")
    elif name == "poisson5d":
        widths = [5, 64, 64, 64, 1]
        prob = poisson_problem(name, 5, widths, 4000, 1000, rng)
        wl = Workload(name, [prob], "f32", ell=500, mu=1e-7, rtol=1e-6, steps=50, sketch="tf32")
    elif name == "poisson10d":
        widths = [10, 128, 128, 128, 128, 1]
        prob = poisson_problem(name, 10, widths, 16384, 4096, rng, freq=0.5)
        wl = Workload(name, [prob], "f32", ell=1000, mu=None, rtol=1e-6, steps=50, sketch="bf16")
    elif name == "heat4d":
        widths = [4, 256, 256, 256, 1]
        prob = heat_problem(name, widths, 32768, 8192, 0.1, rng)
        wl = Workload(name, [prob], "f32", ell=200, mu=None, rtol=1e-6, steps=1, sketch="tf32")
    elif name == "batch64":
        widths = [3, 64, 64, 64, 1]
        probs = []
        for j in range(64):
            n_int = int(rng.integers(1000, 8001))
            k = int(rng.integers(1, 5))
            probs.append(poisson_problem(f"{name}[{j}]", 3, widths, n_int, n_int // 4, rng, freq=float(k)))
        wl = Workload(name, probs, "f32", ell=200, mu=None, rtol=1e-6, steps=1, sketch="f64")
    elif name == "poisson3d":
        # the paper's 3-D Poisson PINN (MLP 3-64-64-64-1, 10k interior + 1k boundary points),
        # trained by NystromNGD: adaptive rank up to 500 in steps of 20, pCG capped at 20 iterations
        widths = [3, 64, 64, 64, 1]
        prob = poisson_problem(name, 3, widths, 10000, 1000, rng)
        wl = Workload(name, [prob], "f32", ell=20, mu=None, rtol=1e-10, steps=200, sketch="f64")
    else:  # pragma: no cover
        raise KeyError(name)
    thetas = [glorot_theta(pr.widths, rng) for pr in wl.problems]
    return wl, thetas


def small_problem(pde: str = POISSON, d: int = 2, widths=None, n_int: int = 24, n_bnd: int = 8,
                  seed: int = 0, kappa: float = 0.1, freq: float = 1.0):
    """A tiny problem for exhaustive oracle checks and parity tests with ragged tails."""
    rng = np.random.default_rng(10_000 + seed)
    if pde == POISSON:
        widths = widths or [d, 6, 5, 1]
        prob = poisson_problem("small", d, widths, n_int, n_bnd, rng, freq=freq)
    else:
        widths = widths or [4, 6, 5, 1]
        prob = heat_problem("small-heat", widths, n_int, n_bnd, kappa, rng)
    theta = glorot_theta(prob.widths, rng)
    # Non-zero biases make every term of the Taylor recurrences show up in the checks.
    theta = theta + 0.1 * rng.standard_normal(theta.shape)
    return prob, theta


def subsample(problem: Problem, n_int: int, n_bnd: int) -> Problem:
    """The first n_int interior and first n_bnd boundary rows of ``problem``
    (uniform weights renormalised to the new point count)."""
    ii = np.arange(min(n_int, problem.n_int))
    bb = problem.n_int + np.arange(min(n_bnd, problem.n_bnd))
    rows = np.concatenate([ii, bb])
    n = rows.size
    return Problem(name=problem.name + "-sub", pde=problem.pde, widths=problem.widths,
                   X=problem.X[rows].copy(), w=np.full(n, 1.0 / n), target=problem.target[rows].copy(),
                   n_int=ii.size, n_bnd=bb.size, kappa=problem.kappa, freq=problem.freq)
