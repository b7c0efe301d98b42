"""The C-ABI library builds, loads and exports every symbol include/amg.h
declares; the binding declares the same set.  No compute call (no GPU here)."""
import os
import re

import pytest
from ctypes import sizeof as C_sizeof

from paper_1907_04417_gb300 import amg, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "amg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(amg_[a-z_]+)\s*\(", src))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return amg.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"amg_setup_from_aggregates", "amg_solve", "amg_solve_batched", "amg_adjoint"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(amg.SIGNATURES), names ^ set(amg.SIGNATURES)


def test_default_options_and_struct_layout(lib):
    o = amg.opts()
    assert o.tol_svd == 0.1 and o.pre == 1 and o.post == 1 and o.cycle_precision == 64
    assert o.rtol == 1e-8 and o.maxit == 1000
    assert amg.amg_opts.rtol.offset == 24 and amg.amg_info.relres.offset == 16
    # the variant switches default to the l1-Jacobi V-cycle
    assert o.smoother == amg.SMOOTHER_L1JACOBI and o.cycle == amg.CYCLE_V
    assert amg.amg_opts.cycle.offset == 56 and C_sizeof(amg.amg_opts) == 64


def test_null_arguments_rejected_without_gpu(lib):
    import ctypes
    assert lib.amg_solve(None, None, None, 1, None, None, None) == amg.AMG_ERR_INVALID_ARG
    assert "non-null" in amg.last_error()
    assert lib.amg_setup_from_aggregates(None, 0, None, None, None, 1, None, None, None) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_hierarchy_info(None, None) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_level_colours(None, 0, None, None) == amg.AMG_ERR_INVALID_ARG
    out = ctypes.c_void_p()
    assert lib.amg_setup_from_aggregates(None, 0, None, None, None, 1, None, None, ctypes.byref(out)) != amg.AMG_OK


def test_bootstrap_test_rejects_bad_arguments_without_gpu(lib):
    import ctypes
    hp = (ctypes.c_void_p * 1)(None)
    assert lib.amg_bootstrap_test(None, 1, None, 1, 1, 1, None, None, None, None) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_bootstrap_test(hp, 0, None, 1, 1, 1, None, None, None, None) == amg.AMG_ERR_INVALID_ARG
    x = (ctypes.c_double * 4)()
    assert lib.amg_bootstrap_test(hp, 1, x, 1, 1, 1, None, None, None, None) == amg.AMG_ERR_INVALID_ARG
    assert "hierarchy" in amg.last_error()


def test_header_is_plain_c_and_links_from_c(lib, tmp_path):
    """include/amg.h compiles as strict C99, and a C program links against
    the library and calls the entry points that need no GPU."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only", "-x", "c",
                        os.path.join(inc, "amg.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    src = tmp_path / "use_amg.c"
    src.write_text(
        '#include <stdio.h>\n#include "amg.h"\n'
        "int main(void) {\n"
        "  amg_opts o; amg_hier_info hi; int32_t nc = 0;\n"
        "  amg_default_opts(&o);\n"
        "  amg_status s1 = amg_hierarchy_info(NULL, &hi);\n"
        "  amg_status s2 = amg_level_colours(NULL, 0, NULL, &nc);\n"
        '  printf("%d %d %d %d %d %d %s\\n", o.pre, o.post, o.cycle_precision, o.smoother, o.cycle,\n'
        "         (int)(s1 == AMG_ERR_INVALID_ARG && s2 == AMG_ERR_INVALID_ARG), amg_last_error());\n"
        "  return 0;\n}\n")
    exe = tmp_path / "use_amg"
    libdir = os.path.dirname(amg.LIB_PATH)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", str(src), "-I", inc, "-L", libdir, "-lamg_gb300",
                        f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    fields = r.stdout.split()
    assert fields[:6] == ["1", "1", "64", "0", "0", "1"], r.stdout


def test_static_bases_refusals_leave_their_reason(lib):
    """The allocation-free entry point records why it refused (argument
    checks run before any CUDA call), and a later refusal replaces the
    message of an earlier one."""
    assert lib.amg_solve(None, None, None, 1, None, None, None) == amg.AMG_ERR_INVALID_ARG
    assert "non-null" in amg.last_error()
    assert lib.amg_local_bases_static(None, 0, None, 1, 1, 0.1, None, None, None) == amg.AMG_ERR_INVALID_ARG
    assert "m must be in [1, 16]" in amg.last_error()
    assert lib.amg_local_bases_static(None, 4, None, 0, 1, 0.1, None, None, None) == amg.AMG_ERR_INVALID_ARG
    assert "nagg and nf must be positive" in amg.last_error()
    big = (1 << 17) // 4 + 1
    assert lib.amg_local_bases_static(None, 4, None, 1, big, 0.1, None, None, None) == amg.AMG_ERR_INVALID_ARG
    assert "work area" in amg.last_error()
    assert lib.amg_local_bases_static(None, 4, None, 1, 16, -1.0, None, None, None) == amg.AMG_ERR_INVALID_ARG
    assert "tol" in amg.last_error()
