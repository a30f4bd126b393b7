"""The C-ABI library builds, loads and exports every entry point include/ngd.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ngd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2505_11638_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ngd_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ngd_residual", "ngd_gramian_mv", "ngd_nystrom_sketch", "ngd_nystrom_factor", "ngd_pcg_solve",
                     "ngd_step", "ngd_create", "ngd_destroy", "ngd_jvp", "ngd_vjp"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header():
    from paper_2505_11638_gb300 import ngd

    assert set(declared_functions()) <= set(ngd._SIGS)


def test_default_options_host_only(lib):
    from paper_2505_11638_gb300 import ngd

    o = ngd.ngd_default_step_opts()
    assert o.ell == 100 and o.gamma == 10.0 and o.armijo_c1 == 1e-4 and o.armijo_rho == 0.5 and o.armijo_max == 30


def test_create_rejects_bad_descriptions_before_touching_the_gpu(lib):
    from paper_2505_11638_gb300 import ngd

    widths = (ctypes.c_int * 4)(2, 8, 8, 2)          # output width must be 1
    d = ngd.ProblemDesc(pde=0, kappa=0.0, n_layers=3, widths=widths, n_int=4, n_bnd=2, X=16, w=16, target=16,
                        dtype=0, gv_mode=0, mem_budget=0, stream=None)
    h = ctypes.c_void_p()
    assert ngd.lib().ngd_create(ctypes.byref(d), ctypes.byref(h)) == 1
    widths2 = (ctypes.c_int * 4)(2, 8, 8, 1)
    for bad in [dict(n_layers=1), dict(n_int=0, n_bnd=0), dict(pde=7), dict(dtype=5), dict(X=None)]:
        kw = dict(pde=0, kappa=0.0, n_layers=3, widths=widths2, n_int=4, n_bnd=2, X=16, w=16, target=16, dtype=0,
                  gv_mode=0, mem_budget=0, stream=None)
        kw.update(bad)
        d = ngd.ProblemDesc(**kw)
        assert ngd.lib().ngd_create(ctypes.byref(d), ctypes.byref(h)) == 1, bad
    assert ngd.lib().ngd_last_error(None) == b"null context"


def _c_layout(struct: str, fields):
    """sizeof and offsetof of a struct of include/ngd.h, from a C program compiled with gcc."""
    import shutil
    import subprocess
    import tempfile

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    body = "\n".join(f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    src = ("#include <stddef.h>\n#include <stdio.h>\n#include \"ngd.h\"\n"
           f"int main(void) {{\n  printf(\"%zu\\n\", sizeof({struct}));\n{body}\n  return 0;\n}}\n")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run([cc, "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("cname,pyname", [("ngd_step_opts", "StepOpts"), ("ngd_step_info", "StepInfo"),
                                          ("ngd_problem_desc", "ProblemDesc")])
def test_binding_structs_match_the_header_layout(cname, pyname):
    from paper_2505_11638_gb300 import ngd

    cls = getattr(ngd, pyname)
    fields = [f for f, _ in cls._fields_]
    size, offsets = _c_layout(cname, fields)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offsets


def test_default_step_opts_fill_the_adaptive_fields(lib):
    from paper_2505_11638_gb300 import ngd

    o = ngd.ngd_default_step_opts()
    assert o.mu_loss_coef == 0.0 and o.ell_max == 0 and o.ell_delta == 20
