"""The allocation-free preconditioner apply (ngd_precond_apply_noalloc).

It serves callers that cannot call cudaMalloc (device memory owned by their own pool
allocator, or loops that cannot accept the synchronisation a cudaMalloc may imply).  Here it
is called through the C ABI and compared with the context-based ngd_precond_apply on two
calls in a row; the file sorts last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import nystrom  # noqa: E402
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


def _call(ngd, dtype, p, ell, U, lam, mu, v, z, ldU=None):
    return ngd.lib().ngd_precond_apply_noalloc(ngd.DTYPES[dtype], p, ell, ctypes.c_void_p(U.data_ptr()),
                                               p if ldU is None else ldU,
                                               ctypes.c_void_p(lam.data_ptr()), float(mu),
                                               ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_context_apply_on_two_calls(ngd, dtype):
    pr, _ = inputs.small_problem(d=3, widths=[3, 16, 16, 1], n_int=30, n_bnd=8, seed=99)
    ctx = ngd.Context(pr, dtype=dtype)
    wd = torch.float64 if dtype == "f64" else torch.float32
    rng = np.random.default_rng(5)
    free_between = []
    for call, (ell, mu) in enumerate([(37, 1e-4), (11, 3e-2)]):
        Q = np.linalg.qr(rng.standard_normal((pr.p, ell)))[0]
        lam = np.sort(rng.uniform(1e-3, 10.0, ell))[::-1].copy()
        U = torch.tensor(np.ascontiguousarray(Q.T), dtype=wd, device="cuda")      # p x ell column-major
        lam_d = torch.tensor(lam, device="cuda")
        v = torch.tensor(rng.standard_normal(pr.p), device="cuda")
        z_ref = ctx.precond_apply(ell, U, lam_d, mu, v)
        z = torch.full((pr.p,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _call(ngd, dtype, pr.p, ell, U, lam_d, mu, v, z) == 0
        torch.cuda.synchronize()
        free_between.append((free0, torch.cuda.mem_get_info()[0]))
        err = float(torch.linalg.norm(z - z_ref) / torch.linalg.norm(z_ref))
        assert err <= 1e-12, (call, err)
    # the second call (the array already set up) allocates nothing on the device
    assert free_between[1][0] == free_between[1][1]
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(ngd):
    p, ell = 1500, 1025
    U = torch.zeros((ell, p), dtype=torch.float64, device="cuda")
    lam = torch.ones(ell, dtype=torch.float64, device="cuda")
    v = torch.ones(p, dtype=torch.float64, device="cuda")
    z = torch.zeros(p, dtype=torch.float64, device="cuda")
    assert _call(ngd, "f64", p, ell, U, lam, 1e-3, v, z) == 9      # NGD_ERR_UNSUPPORTED
    assert _call(ngd, "f64", p, 0, U, lam, 1e-3, v, z) == 1        # NGD_ERR_INVALID_ARG
    assert _call(ngd, "f64", p, 10, U, lam, 1e-3, v, v) == 1       # aliased v, z


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_at_its_maximum_rank_with_padded_columns(ngd, dtype):
    """ell = NGD_NOALLOC_MAX_ELL (the whole scratch array; the largest dynamic shared memory the
    apply takes) with a leading dimension ldU = p + 8: against the FP64 oracle of Alg. 4 on the
    same (rounded) U, and against the context apply on a contiguous copy."""
    pr, _ = inputs.small_problem(d=3, widths=[3, 32, 32, 1], n_int=40, n_bnd=10, seed=98)
    p, ell, ldU = pr.p, 1024, pr.p + 8
    assert p >= ell
    wd = torch.float64 if dtype == "f64" else torch.float32
    rng = np.random.default_rng(6)
    Q = np.linalg.qr(rng.standard_normal((p, ell)))[0]
    lam = np.sort(rng.uniform(1e-3, 10.0, ell))[::-1].copy()
    Upad = torch.full((ell, ldU), float("nan"), dtype=wd, device="cuda")   # padding never read
    Upad[:, :p] = torch.tensor(Q.T, dtype=wd, device="cuda")
    U_r = Upad[:, :p].double().cpu().numpy().T                                # the rounded U both sides use
    lam_d = torch.tensor(lam, device="cuda")
    ctx = ngd.Context(pr, dtype=dtype)
    for call, mu in enumerate([1e-4, 2e-2]):
        v_h = rng.standard_normal(p)
        v = torch.tensor(v_h, device="cuda")
        z = torch.full((p,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(ngd, dtype, p, ell, Upad, lam_d, mu, v, z, ldU=ldU) == 0
        torch.cuda.synchronize()
        z_o = nystrom.precond_apply(U_r, lam, mu, v_h)
        z_h = z.cpu().numpy()
        assert np.linalg.norm(z_h - z_o) <= 1e-12 * np.linalg.norm(z_o), call
        z_ref = ctx.precond_apply(ell, Upad[:, :p].contiguous(), lam_d, mu, v)
        assert float(torch.linalg.norm(z - z_ref) / torch.linalg.norm(z_ref)) <= 1e-12, call
    ctx.close()
