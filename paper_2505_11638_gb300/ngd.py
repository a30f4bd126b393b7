"""Thin Python binding of libngd (include/ngd.h).

Argument marshalling only: every step of the hot path runs in the CUDA kernels of
``libngd.so``.  Device memory and streams come from PyTorch; each call enqueues on
``torch.cuda.current_stream()``.  The module-level functions carry the C names
(``ngd_residual``, ``ngd_gramian_mv``, ``ngd_nystrom_sketch``, ``ngd_nystrom_factor``,
``ngd_pcg_solve``, ``ngd_step``, ...); ``Context`` wraps them for convenience and
``PinnResidual`` exposes the residual kernel and its hand-written reverse as a
``torch.autograd.Function``.

There is no fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libngd.so")

NGD_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_SPD", 5: "BREAKDOWN", 6: "MAXIT",
                7: "NONFINITE", 8: "TIMEOUT", 9: "UNSUPPORTED"}
DTYPES = {"f64": 0, "f32": 1}
SKETCH = {"f64": 0, "f32": 1, "tf32": 2, "bf16": 3, "df": 4}
TEST_MATRIX = {"gaussian": 0, "sampling": 1}
PRECOND = {"nystrom": 0, "rpchol": 1, "full": 2}
PDES = {"poisson": 0, "heat": 1}
GV_MODES = {"auto": 0, "stored": 1, "matrix_free": 2}


class NGDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))


class ProblemDesc(ctypes.Structure):
    _fields_ = [("pde", ctypes.c_int), ("kappa", ctypes.c_double), ("n_layers", ctypes.c_int),
                ("widths", ctypes.POINTER(ctypes.c_int)), ("n_int", ctypes.c_int64), ("n_bnd", ctypes.c_int64),
                ("X", ctypes.c_void_p), ("w", ctypes.c_void_p), ("target", ctypes.c_void_p),
                ("dtype", ctypes.c_int), ("gv_mode", ctypes.c_int), ("mem_budget", ctypes.c_size_t),
                ("stream", ctypes.c_void_p)]


class StepOpts(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_int), ("mu", ctypes.c_double), ("gamma", ctypes.c_double),
                ("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("sketch", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("step", ctypes.c_uint64), ("armijo_c1", ctypes.c_double),
                ("armijo_rho", ctypes.c_double), ("armijo_max", ctypes.c_int), ("mu_loss_coef", ctypes.c_double),
                ("ell_max", ctypes.c_int), ("ell_delta", ctypes.c_int), ("test_matrix", ctypes.c_int),
                ("precond", ctypes.c_int), ("rpchol_block", ctypes.c_int)]


class StepInfo(ctypes.Structure):
    _fields_ = [("loss_before", ctypes.c_double), ("loss_after", ctypes.c_double), ("alpha", ctypes.c_double),
                ("mu", ctypes.c_double), ("lam1", ctypes.c_double), ("lam_ell", ctypes.c_double),
                ("nu", ctypes.c_double), ("relres", ctypes.c_double), ("pcg_iters", ctypes.c_int),
                ("armijo_trials", ctypes.c_int), ("shift_retries", ctypes.c_int), ("status", ctypes.c_int),
                ("ms_linearize", ctypes.c_double), ("ms_sketch", ctypes.c_double), ("ms_factor", ctypes.c_double),
                ("ms_pcg", ctypes.c_double), ("ms_linesearch", ctypes.c_double), ("ell_next", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_U64 = ctypes.c_uint64

_SIGS = {
    "ngd_create": ([ctypes.POINTER(ProblemDesc), ctypes.POINTER(_P)], _I),
    "ngd_destroy": ([_P], None),
    "ngd_last_error": ([_P], ctypes.c_char_p),
    "ngd_num_params": ([_P], ctypes.c_int64),
    "ngd_num_points": ([_P], ctypes.c_int64),
    "ngd_set_stream": ([_P, _P], _I),
    "ngd_set_wait_limit": ([_P, ctypes.c_int64], _I),
    "ngd_residual": ([_P, _P, _P, ctypes.POINTER(_D)], _I),
    "ngd_eval": ([_P, _P, _P], _I),
    "ngd_jvp": ([_P, _P, _P, _P], _I),
    "ngd_vjp": ([_P, _P, _P, _P], _I),
    "ngd_gradient": ([_P, _P, _P, _P, ctypes.POINTER(_D)], _I),
    "ngd_gramian_mv": ([_P, _P, _P, _D, _P], _I),
    "ngd_set_jacobian": ([_P, _P, ctypes.c_int64], _I),
    "ngd_gramian_mm": ([_P, _P, _I, _P, ctypes.c_int64, _I, _P, ctypes.c_int64], _I),
    "ngd_nystrom_sketch": ([_P, _P, _I, _U64, _U64, _I, _P, _P], _I),
    "ngd_nystrom_sketch_sampled": ([_P, _P, _I, _U64, _U64, _I, _P, _P, _P], _I),
    "ngd_gramian_diag": ([_P, _P, _P], _I),
    "ngd_gramian_full": ([_P, _P, _P, ctypes.c_int64], _I),
    "ngd_nystrom_factor": ([_P, _I, _P, _P, _I, _D, _P, _P, ctypes.POINTER(_D)], _I),
    "ngd_precond_apply": ([_P, _I, _P, _I, _P, _D, _P, _P], _I),
    "ngd_pcg_solve": ([_P, _P, _P, _D, _P, _I, _P, _I, _D, _I, _P, ctypes.POINTER(_I), ctypes.POINTER(_D)], _I),
    "ngd_step": ([_P, _P, ctypes.POINTER(StepOpts), ctypes.POINTER(StepInfo)], _I),
    "ngd_default_step_opts": ([ctypes.POINTER(StepOpts)], None),
    "ngd_kernel_launches": ([], ctypes.c_uint64),
    "ngd_precond_apply_noalloc": ([_I, ctypes.c_int64, _I, _P, ctypes.c_int64, _P, _D, _P, _P, _P], _I),
    "ngd_batch_create": ([_P, _I, ctypes.POINTER(_P)], _I),
    "ngd_batch_destroy": ([_P], None),
    "ngd_batch_size": ([_P], _I),
    "ngd_batch_context": ([_P, _I], _P),
    "ngd_batch_last_error": ([_P], ctypes.c_char_p),
    "ngd_batch_step": ([_P, _P, ctypes.POINTER(StepOpts), _P], _I),
    "ngd_batch_set_packing": ([_P, _I], _I),
    "ngd_batch_packing": ([_P], _I),
    "ngd_batch_solve_launches": ([_P], _I),
}


def lib():
    """Load libngd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2505_11638_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(handle, name)
            fn.argtypes = args
            fn.restype = res
        _lib = handle
    return _lib


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(ctx_handle, status):
    if status != NGD_OK:
        msg = lib().ngd_last_error(ctx_handle) if ctx_handle else b""
        raise NGDError(status, (msg or b"").decode())


def _need(t: torch.Tensor, dtype, numel, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    return t


# ---------------------------------------------------------------- C-named entry points
def ngd_create(desc: ProblemDesc):
    h = ctypes.c_void_p()
    _check(None, lib().ngd_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def ngd_destroy(h):
    lib().ngd_destroy(h)


def ngd_set_wait_limit(h, cycles):
    _check(h, lib().ngd_set_wait_limit(h, int(cycles)))


def ngd_residual(h, theta, r, want_loss=True):
    lib().ngd_set_stream(h, _stream())
    loss = ctypes.c_double(0.0)
    _check(h, lib().ngd_residual(h, _ptr(theta), _ptr(r), ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def ngd_eval(h, theta, out):
    lib().ngd_set_stream(h, _stream())
    _check(h, lib().ngd_eval(h, _ptr(theta), _ptr(out)))


def ngd_jvp(h, theta, v, out):
    lib().ngd_set_stream(h, _stream())
    _check(h, lib().ngd_jvp(h, _ptr(theta), _ptr(v), _ptr(out)))


def ngd_vjp(h, theta, cot, out):
    lib().ngd_set_stream(h, _stream())
    _check(h, lib().ngd_vjp(h, _ptr(theta), _ptr(cot), _ptr(out)))


def ngd_gradient(h, theta, g, r=None, want_loss=True):
    lib().ngd_set_stream(h, _stream())
    loss = ctypes.c_double(0.0)
    _check(h, lib().ngd_gradient(h, _ptr(theta), _ptr(g), _ptr(r), ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def ngd_gramian_mv(h, theta, v, mu, y):
    lib().ngd_set_stream(h, _stream())
    _check(h, lib().ngd_gramian_mv(h, _ptr(theta), _ptr(v), float(mu), _ptr(y)))


def ngd_set_jacobian(h, J, ldJ):
    lib().ngd_set_stream(h, _stream())
    _check(h, lib().ngd_set_jacobian(h, _ptr(J), int(ldJ)))


def ngd_gramian_mm(h, theta, ell, V, ldV, prec, Y, ldY):
    lib().ngd_set_stream(h, _stream())
    _check(h, lib().ngd_gramian_mm(h, _ptr(theta), int(ell), _ptr(V), int(ldV), SKETCH[prec], _ptr(Y), int(ldY)))


def ngd_nystrom_sketch(h, theta, ell, seed, step, prec, Omega, Y):
    lib().ngd_set_stream(h, _stream())
    _check(h, lib().ngd_nystrom_sketch(h, _ptr(theta), int(ell), int(seed), int(step), SKETCH[prec], _ptr(Omega),
                                       _ptr(Y)))


def ngd_nystrom_sketch_sampled(h, theta, ell, seed, step, prec, idx, Omega, Y):
    lib().ngd_set_stream(h, _stream())
    _check(h, lib().ngd_nystrom_sketch_sampled(h, _ptr(theta), int(ell), int(seed), int(step), SKETCH[prec],
                                               _ptr(idx), _ptr(Omega), _ptr(Y)))


def ngd_gramian_full(h, theta, G, ldG):
    """G (p x p column-major, ldG) = J^T diag(w) J at the linearization."""
    _check(h, lib().ngd_gramian_full(h, _ptr(theta), _ptr(G), int(ldG)))


def ngd_gramian_diag(h, theta, d):
    lib().ngd_set_stream(h, _stream())
    _check(h, lib().ngd_gramian_diag(h, _ptr(theta), _ptr(d)))


def ngd_nystrom_factor(h, ell, Omega, Y, prec, shift_scale, U, lam):
    lib().ngd_set_stream(h, _stream())
    nu = ctypes.c_double(0.0)
    _check(h, lib().ngd_nystrom_factor(h, int(ell), _ptr(Omega), _ptr(Y), SKETCH[prec], float(shift_scale), _ptr(U),
                                       _ptr(lam), ctypes.byref(nu)))
    return nu.value


def _u_dtype(U):
    return DTYPES["f64"] if U is None or U.dtype == torch.float64 else DTYPES["f32"]


def ngd_precond_apply(h, ell, U, lam, mu, v, z):
    lib().ngd_set_stream(h, _stream())
    _check(h, lib().ngd_precond_apply(h, int(ell), _ptr(U), _u_dtype(U), _ptr(lam), float(mu), _ptr(v), _ptr(z)))


def ngd_pcg_solve(h, theta, g, mu, U, lam, ell, rtol, maxit, d):
    lib().ngd_set_stream(h, _stream())
    iters = ctypes.c_int(0)
    relres = ctypes.c_double(0.0)
    _check(h, lib().ngd_pcg_solve(h, _ptr(theta), _ptr(g), float(mu), _ptr(U), _u_dtype(U), _ptr(lam), int(ell),
                                  float(rtol), int(maxit), _ptr(d), ctypes.byref(iters), ctypes.byref(relres)))
    return iters.value, relres.value


def ngd_step(h, theta, opts: StepOpts):
    lib().ngd_set_stream(h, _stream())
    info = StepInfo()
    _check(h, lib().ngd_step(h, _ptr(theta), ctypes.byref(opts), ctypes.byref(info)))
    return info


def ngd_kernel_launches() -> int:
    return int(lib().ngd_kernel_launches())


def ngd_default_step_opts() -> StepOpts:
    o = StepOpts()
    lib().ngd_default_step_opts(ctypes.byref(o))
    return o


# ---------------------------------------------------------------- convenience wrapper
class Context:
    """One PINN problem on the current CUDA device (see ``ngd_problem_desc``)."""

    def __init__(self, problem, dtype: str = "f64", gv_mode: str = "auto", mem_budget: int = 0,
                 device: str | torch.device = "cuda"):
        dev = torch.device(device)
        self.problem = problem
        self.dtype = dtype
        self.wdtype = torch.float64 if dtype == "f64" else torch.float32
        self.X = torch.as_tensor(problem.X, dtype=torch.float64, device=dev).contiguous()
        self.w = torch.as_tensor(problem.w, dtype=torch.float64, device=dev).contiguous()
        self.target = torch.as_tensor(problem.target, dtype=torch.float64, device=dev).contiguous()
        self._widths = (ctypes.c_int * len(problem.widths))(*problem.widths)
        desc = ProblemDesc(pde=PDES[problem.pde], kappa=float(getattr(problem, "kappa", 0.0)),
                           n_layers=len(problem.widths) - 1, widths=self._widths, n_int=int(problem.n_int),
                           n_bnd=int(problem.n_bnd), X=self.X.data_ptr(), w=self.w.data_ptr(),
                           target=self.target.data_ptr(), dtype=DTYPES[dtype], gv_mode=GV_MODES[gv_mode],
                           mem_budget=int(mem_budget), stream=torch.cuda.current_stream(dev).cuda_stream)
        self.handle = ngd_create(desc)
        self.device = dev
        self.p = int(lib().ngd_num_params(self.handle))
        self.N = int(lib().ngd_num_points(self.handle))
        self.version = 0

    def close(self):
        if getattr(self, "handle", None):
            ngd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, n, dtype=torch.float64):
        return torch.empty(n, dtype=dtype, device=self.device)

    def residual(self, theta):
        _need(theta, torch.float64, self.p, "theta")
        r = self._vec(self.N)
        loss = ngd_residual(self.handle, theta, r)
        self.version += 1
        return r, loss

    def eval(self, theta):
        """(N, d + 2) float64: u, grad u (d) and Delta u of the network at the context's points."""
        _need(theta, torch.float64, self.p, "theta")
        out = torch.empty(self.N, self.problem.widths[0] + 2, dtype=torch.float64, device=self.device)
        ngd_eval(self.handle, theta, out)
        self.version += 1
        return out

    def jvp(self, theta, v):
        _need(v, torch.float64, self.p, "v")
        out = self._vec(self.N)
        ngd_jvp(self.handle, theta, v, out)
        self.version += 1
        return out

    def vjp(self, theta, cot):
        _need(cot, torch.float64, self.N, "cot")
        out = self._vec(self.p)
        ngd_vjp(self.handle, theta, cot, out)
        return out

    def gradient(self, theta):
        _need(theta, torch.float64, self.p, "theta")
        g, r = self._vec(self.p), self._vec(self.N)
        loss = ngd_gradient(self.handle, theta, g, r)
        self.version += 1
        return g, r, loss

    def gramian_mv(self, theta, v, mu):
        _need(v, torch.float64, self.p, "v")
        y = self._vec(self.p)
        ngd_gramian_mv(self.handle, theta, v, mu, y)
        if theta is not None:
            self.version += 1
        return y

    def set_jacobian(self, J):
        """Replace the stored Jacobian by J, an (N, p) CUDA tensor of the context dtype (row-major)."""
        if not isinstance(J, torch.Tensor) or not J.is_cuda or J.dtype != self.wdtype or J.dim() != 2 \
                or J.shape[0] != self.N or J.shape[1] != self.p or J.stride(1) != 1:
            raise ValueError(f"J: expected an ({self.N}, {self.p}) CUDA {self.wdtype} tensor with unit column stride")
        ngd_set_jacobian(self.handle, J, J.stride(0))
        self.version += 1

    def gramian_mm(self, theta, V, prec="f64"):
        """Y = G V for V an (ell, p) tensor of the context dtype (column-major p x ell); Y likewise,
        float64 when prec is "f64"."""
        _need(V, self.wdtype, None, "V")
        if V.dim() != 2 or V.shape[1] != self.p:
            raise ValueError(f"V: expected shape (ell, {self.p})")
        ell = V.shape[0]
        Y = torch.empty((ell, self.p), dtype=torch.float64 if prec in ("f64", "df") else self.wdtype,
                        device=self.device)
        ngd_gramian_mm(self.handle, theta, ell, V, self.p, prec, Y, self.p)
        if theta is not None:
            self.version += 1
        return Y

    def nystrom_sketch(self, theta, ell, seed=0, step=0, prec="f64"):
        Om = torch.empty((ell, self.p), dtype=self.wdtype, device=self.device)   # column-major p x ell
        Y = torch.empty((ell, self.p), dtype=torch.float64 if prec in ("f64", "df") else self.wdtype, device=self.device)
        ngd_nystrom_sketch(self.handle, theta, ell, seed, step, prec, Om, Y)
        if theta is not None:
            self.version += 1
        return Om, Y

    def nystrom_sketch_sampled(self, theta, ell, seed=0, step=0, prec="f64"):
        """The sampling test matrix: returns (idx, Omega, Y), idx the sampled parameter indices."""
        idx = torch.empty(ell, dtype=torch.int32, device=self.device)
        Om = torch.empty((ell, self.p), dtype=self.wdtype, device=self.device)
        Y = torch.empty((ell, self.p), dtype=torch.float64 if prec in ("f64", "df") else self.wdtype, device=self.device)
        ngd_nystrom_sketch_sampled(self.handle, theta, ell, seed, step, prec, idx, Om, Y)
        if theta is not None:
            self.version += 1
        return idx, Om, Y

    def gramian_full(self, theta):
        """The explicit Gramian as a (p, p) float64 CUDA tensor (symmetric)."""
        G = torch.empty((self.p, self.p), dtype=torch.float64, device=self.device)
        ngd_gramian_full(self.handle, theta, G, self.p)
        if theta is not None:
            self.version += 1
        return G

    def gramian_diag(self, theta):
        d = self._vec(self.p)
        ngd_gramian_diag(self.handle, theta, d)
        if theta is not None:
            self.version += 1
        return d

    def nystrom_factor(self, ell, Omega, Y, prec="f64", shift_scale=1.0):
        _need(Omega, self.wdtype, self.p * ell, "Omega")
        _need(Y, torch.float64 if prec in ("f64", "df") else self.wdtype, self.p * ell, "Y")
        U = torch.empty((ell, self.p), dtype=torch.float64 if prec in ("f64", "df") else self.wdtype, device=self.device)
        lam = self._vec(ell)
        nu = ngd_nystrom_factor(self.handle, ell, Omega, Y, prec, shift_scale, U, lam)
        return U, lam, nu

    def precond_apply(self, ell, U, lam, mu, v):
        z = self._vec(self.p)
        ngd_precond_apply(self.handle, ell, U, lam, mu, v, z)
        return z

    def pcg_solve(self, theta, g, mu, U=None, lam=None, ell=0, rtol=1e-6, maxit=500):
        d = self._vec(self.p)
        iters, relres = ngd_pcg_solve(self.handle, theta, g, mu, U, lam, ell if U is not None else 0, rtol, maxit, d)
        if theta is not None:
            self.version += 1
        return d, iters, relres

    def step(self, theta, **kw):
        o = ngd_default_step_opts()
        if self.dtype == "f64":
            o.sketch = SKETCH["f64"]
        for k, v in kw.items():
            if k == "sketch":
                v = SKETCH[v]
            if k == "test_matrix":
                v = TEST_MATRIX[v]
            if k == "precond":
                v = PRECOND[v]
            if k == "mu" and v is None:
                v = 0.0
            setattr(o, k, v)
        info = ngd_step(self.handle, theta, o)
        self.version += 1
        return info.as_dict()


class PinnResidual(torch.autograd.Function):
    """r(theta) by the forward-Laplacian kernel; backward by the hand-written reverse kernel.

    The reverse reuses the Taylor coefficients the forward stored when the context's memory
    budget allowed it and nothing else ran on the context in between; otherwise it recomputes
    them from theta.
    """

    @staticmethod
    def forward(ctx, theta: torch.Tensor, ngd: Context):
        r, _ = ngd.residual(theta)
        ctx.ngd = ngd
        ctx.version = ngd.version
        ctx.save_for_backward(theta)
        return r

    @staticmethod
    def backward(ctx, grad_r):
        (theta,) = ctx.saved_tensors
        ngd: Context = ctx.ngd
        reuse = ngd.version == ctx.version
        g = ngd.vjp(None if reuse else theta, grad_r.contiguous().to(torch.float64))
        return g, None


class Batch:
    """Many independent problems stepped together (``ngd_batch_*``): one context per problem,
    all on the current stream; ``step`` runs one NGD step for every problem."""

    def __init__(self, problems, dtype: str = "f32", device: str | torch.device = "cuda"):
        dev = torch.device(device)
        self.device = dev
        self.dtype = dtype
        self._keep = []
        n = len(problems)
        descs = (ProblemDesc * n)()
        for i, pr in enumerate(problems):
            X = torch.as_tensor(pr.X, dtype=torch.float64, device=dev).contiguous()
            w = torch.as_tensor(pr.w, dtype=torch.float64, device=dev).contiguous()
            tg = torch.as_tensor(pr.target, dtype=torch.float64, device=dev).contiguous()
            widths = (ctypes.c_int * len(pr.widths))(*pr.widths)
            self._keep += [X, w, tg, widths]
            descs[i] = ProblemDesc(pde=PDES[pr.pde], kappa=float(getattr(pr, "kappa", 0.0)),
                                   n_layers=len(pr.widths) - 1, widths=widths, n_int=int(pr.n_int),
                                   n_bnd=int(pr.n_bnd), X=X.data_ptr(), w=w.data_ptr(), target=tg.data_ptr(),
                                   dtype=DTYPES[dtype], gv_mode=GV_MODES["auto"], mem_budget=0,
                                   stream=torch.cuda.current_stream(dev).cuda_stream)
        h = ctypes.c_void_p()
        st = lib().ngd_batch_create(descs, n, ctypes.byref(h))
        if st != NGD_OK:
            raise NGDError(st, "ngd_batch_create failed")
        self.handle = h
        self.n = n
        self.p = [int(lib().ngd_num_params(lib().ngd_batch_context(h, i))) for i in range(n)]

    def close(self):
        if getattr(self, "handle", None):
            lib().ngd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_packing(self, solves_per_launch: int):
        """Solves per cooperative launch (0: tune on the next step, 1: one per launch)."""
        st = lib().ngd_batch_set_packing(self.handle, int(solves_per_launch))
        if st != NGD_OK:
            raise NGDError(st, "ngd_batch_set_packing")

    @property
    def packing(self) -> int:
        return int(lib().ngd_batch_packing(self.handle))

    @property
    def solve_launches(self) -> int:
        return int(lib().ngd_batch_solve_launches(self.handle))

    def step(self, thetas, **kw):
        """thetas: list of float64 device tensors (one per problem), updated in place."""
        assert len(thetas) == self.n
        for th, p in zip(thetas, self.p):
            _need(th, torch.float64, p, "theta")
        o = ngd_default_step_opts()
        for k, v in kw.items():
            if k == "sketch":
                v = SKETCH[v]
            if k == "mu" and v is None:
                v = 0.0
            setattr(o, k, v)
        ptrs = (ctypes.c_void_p * self.n)(*[th.data_ptr() for th in thetas])
        infos = (StepInfo * self.n)()
        st = lib().ngd_batch_step(self.handle, ptrs, ctypes.byref(o), infos)
        if st != NGD_OK:
            msg = lib().ngd_batch_last_error(self.handle).decode()
            raise NGDError(st, msg)
        return [infos[i].as_dict() for i in range(self.n)]
