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
