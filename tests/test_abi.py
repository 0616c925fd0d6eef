"""The C-ABI library builds, loads and exports every entry point that
include/lsr.h declares; host-side argument checks. CPU only (no compute call)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1801_01572_gb300 import _build
    return _build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "lsr.h")).read()
    return sorted(set(re.findall(r"^LSR_API\s+[^;(]*?\b(lsr_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_binding_functions():
    import paper_1801_01572_gb300 as pkg
    assert _declared() == sorted(pkg.ABI_FUNCTIONS)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lsr_\w+)$", out, flags=re.M))
    missing = [f for f in _declared() if f not in exported]
    assert not missing, missing
    # nothing else of the implementation leaks out of the library
    assert exported == set(_declared())


def test_library_loads_and_binds(libpath):
    import paper_1801_01572_gb300 as pkg
    L = pkg.lib()
    for name in pkg.ABI_FUNCTIONS:
        assert getattr(L, name) is not None


def test_defaults_and_error_strings(libpath):
    import paper_1801_01572_gb300 as pkg
    p = pkg.default_params()
    assert abs(p.r_normal - 0.05) < 1e-7 and abs(p.r_feature - 0.125) < 1e-7
    assert abs(p.eps_inlier - 0.0375) < 1e-7 and abs(p.tau - 0.9) < 1e-7
    assert p.n_hypotheses == 4_000_000 and p.match_precision == pkg.MATCH_FP32
    L = pkg.lib()
    for code in (0, -1, -2, -3, -4, -5):
        assert L.lsr_error_string(code)
    assert L.lsr_last_error(None) == b"null context"


def test_null_and_invalid_arguments_without_device(libpath):
    import paper_1801_01572_gb300 as pkg
    L = pkg.lib()
    # NULL context is rejected before any device work
    assert L.lsr_register_pair(None, None, 0, None, 0, None, None, None) == pkg.LSR_E_STATE
    assert L.lsr_destroy(None) == pkg.LSR_OK
    assert L.lsr_create(None, None, 0, None) == pkg.LSR_E_ARG
    bad = pkg.default_params(tau=1.5)
    h = C.c_void_p()
    assert L.lsr_create(C.byref(h), C.byref(bad), 0, None) == pkg.LSR_E_ARG
    bad = pkg.default_params(n_hypotheses=0)
    assert L.lsr_create(C.byref(h), C.byref(bad), 0, None) == pkg.LSR_E_ARG


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1801_01572_gb300.lsr as m
    monkeypatch.setattr(m, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(m, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        m.lib()


def test_header_is_plain_c(tmp_path):
    """include/lsr.h compiles as C99 and as C++ on its own: plain pointers and
    sizes, no C++ or framework types in the boundary."""
    src = tmp_path / "use.c"
    src.write_text('#include "lsr.h"\nint main(void) {\n  lsr_params p;\n  lsr_default_params(&p);\n'
                   '  return p.n_hypotheses > 0 ? 0 : 1;\n}\n')
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src)], check=True)
    subprocess.run(["g++", "-x", "c++", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src)], check=True)


def test_next_row_entry_points_reject_a_null_context(libpath):
    import paper_1801_01572_gb300 as pkg
    L = pkg.lib()
    assert L.lsr_information_matrix(None, None, 0, None, 0, None, C.c_float(0.05), None, None) == pkg.LSR_E_STATE
    assert L.lsr_voxel_downsample(None, None, 0, C.c_float(0.05), None, 0, None) == pkg.LSR_E_STATE
    assert L.lsr_surfel_correct(None, 0, None, None, None, None, 0, None, None, None, None, None, None, None,
                                None) == pkg.LSR_E_STATE
