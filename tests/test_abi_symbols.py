"""The C ABI library loads without a GPU and exports every symbol include/gpnufft.h declares.

Also checks that the ctypes mirrors of gp_plan_opts / gp_plan_info have the
C layout (sizes and field offsets compiled from the header with gcc).
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpnufft.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char\s*\*|const char\s*\*)\s*\*?\s*(gp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03608_gb300 import abi
    return abi


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("gp_plan", "gp_matvec", "gp_cg_solve", "gp_cg_solve_refined", "gp_posterior_mean",
                 "gp_plan_info_get", "gp_destroy", "gp_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(so, name), name
    assert sorted(declared_functions()) == sorted(lib.EXPORTED)


def test_version_and_error_strings_without_gpu(lib):
    assert "sm_103a" in lib.gp_version()
    assert lib.LIB.gp_last_error() == b""


def test_null_arguments_are_rejected_without_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    st = lib.LIB.gp_plan(ctypes.byref(h), None, 10, 1, None, None, 1.5, 1e-6, None, None)
    assert st == lib.GP_EINVAL and h.value is None
    assert b"null" in lib.LIB.gp_last_error()
    st = lib.LIB.gp_matvec(None, None, None, 1, 0.0, None)
    assert st == lib.GP_EINVAL
    lib.LIB.gp_destroy(None)


def test_struct_layout_matches_header(lib, tmp_path):
    # every field of the ctypes mirrors, at the offset gcc gives the header's field
    fields = [(sname, f[0]) for sname in ("gp_plan_opts", "gp_plan_info") for f in getattr(lib, sname)._fields_]
    body = "".join("  F(%s, %s)\n" % sf for sf in fields)
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "gpnufft.h"
#define F(S, m) printf("%s.%s %zu\n", #S, #m, offsetof(S, m));
int main(void) {
  printf("gp_plan_opts %zu\n", sizeof(gp_plan_opts));
  printf("gp_plan_info %zu\n", sizeof(gp_plan_info));
''' + body + r'''
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)], text=True).split("\n") if line)
    assert int(out["gp_plan_opts"]) == ctypes.sizeof(lib.gp_plan_opts)
    assert int(out["gp_plan_info"]) == ctypes.sizeof(lib.gp_plan_info)
    assert len(out) == 2 + len(fields)
    for key, val in out.items():
        if "." in key:
            s, m = key.split(".")
            assert getattr(getattr(lib, s), m).offset == int(val), key


def test_every_entry_point_refuses_a_null_plan(lib):
    L = lib.LIB
    calls = {
        "gp_matvec": lambda: L.gp_matvec(None, None, None, 1, 0.0, None),
        "gp_cg_solve": lambda: L.gp_cg_solve(None, None, None, 1, 0.0, 1e-6, 10, None, None, None),
        "gp_cg_solve_refined": lambda: L.gp_cg_solve_refined(None, None, None, None, 1, 0.0, 1e-8, 1e-4, 5, 10,
                                                             None, None, None),
        "gp_posterior_mean": lambda: L.gp_posterior_mean(None, None, None, 1, None, None, None, None),
        "gp_posterior_mean_noalloc": lambda: L.gp_posterior_mean_noalloc(None, None, None, 1, None, None, None, None),
        "gp_posterior_variance": lambda: L.gp_posterior_variance(None, None, 1, 0.1, 1e-6, 10, None, None, None),
        "gp_profile_enable": lambda: L.gp_profile_enable(None, 1),
        "gp_profile_read": lambda: L.gp_profile_read(None, None, None),
        "gp_profile_read_rows": lambda: L.gp_profile_read_rows(None, None),
        "gp_plan_info_get": lambda: L.gp_plan_info_get(None, None),
    }
    plan_taking = [n for n in declared_functions() if n not in
                   ("gp_plan", "gp_plan_opts_default", "gp_plan_params", "gp_tile_candidates", "gp_destroy",
                    "gp_last_error", "gp_version")]
    assert sorted(calls) == sorted(plan_taking)
    for name, call in calls.items():
        assert call() == lib.GP_EINVAL, name
        assert L.gp_last_error() == b"null plan", name


def test_plan_arguments_are_checked_before_any_device_work(lib):
    h = ctypes.c_void_p()
    x = (ctypes.c_double * 4)(0.1, 0.2, 0.3, 0.4)
    one = (ctypes.c_double * 4)(1, 1, 1, 1)
    o = lib.default_opts()
    bad = [
        (x, 4, 4, one, one, 1.5, 1e-6, o, "d must be"),
        (x, 0, 1, one, one, 1.5, 1e-6, o, "N must be"),
        (x, 4, 1, one, one, -1.0, 1e-6, o, "nu must be"),
        (x, 4, 1, one, one, 1.5, 0.5, o, "eps must be"),
        (x, 4, 1, one, one, 1.5, 0.0, o, "eps must be"),
        (x, 4, 1, one, one, 1.5, 1e-6, lib.default_opts(precision=7), "precision"),
        (x, 4, 1, one, one, 1.5, 1e-6, lib.default_opts(max_rhs=5000), "max_rhs"),
        (x, 4, 1, one, one, 1.5, 1e-6, lib.default_opts(autotune=9), "autotune"),
    ]
    for pts, n, d, fa, fb, nu, eps, opts, msg in bad:
        st = _plan_call(lib, h, pts, n, d, fa, fb, nu, eps, opts)
        assert st == lib.GP_EINVAL, msg
        assert msg.encode() in lib.LIB.gp_last_error(), (msg, lib.LIB.gp_last_error())
        assert h.value is None


def _plan_call(lib, h, pts, n, d, fa, fb, nu, eps, opts):
    return lib.LIB.gp_plan(ctypes.byref(h), pts, n, d, fa, fb, nu, eps, ctypes.byref(opts), None)


def test_no_cpu_fallback_without_a_gpu(lib):
    # the product path has no host implementation: without a CUDA device a plan cannot
    # be built, and the call says why
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import numpy as np
    import paper_2407_03608_gb300 as gpn
    with pytest.raises(gpn.GPError) as e:
        gpn.Plan(np.linspace(0, 1, 50).reshape(-1, 1), np.ones(50), np.full(50, 0.05), nu=1.5, eps=1e-4)
    assert e.value.status == lib.GP_ECUDA


def test_importing_without_the_built_library_raises(tmp_path):
    # a copy of the package's Python files with no _build directory: the import fails
    # loudly instead of falling back to anything
    import shutil
    import sys
    pkg = os.path.join(ROOT, "paper_2407_03608_gb300")
    dst = tmp_path / "paper_2407_03608_gb300"
    dst.mkdir()
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            shutil.copy(os.path.join(pkg, f), dst / f)
    r = subprocess.run([sys.executable, "-c", "import paper_2407_03608_gb300"], cwd=str(tmp_path),
                       capture_output=True, text=True, env=dict(os.environ, PYTHONPATH=str(tmp_path)))
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libgpnufft.so is not built" in r.stderr
