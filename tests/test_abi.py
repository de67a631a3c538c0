"""The C-ABI library builds, loads without a GPU, and exports every symbol that
include/sylv.h declares; the binding's struct layouts match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_10574_gb300 import build, sylv
    build.build()
    return sylv.load()


def _header_functions():
    src = open(os.path.join(ROOT, "include", "sylv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sylv_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _header_functions()
    assert "sylv_tri_solve" in names and "sylv_tri_solve_backward" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1905_10574_gb300 import sylv
    assert sorted(sylv.SIGNATURES) == _header_functions()


def test_struct_layouts():
    from paper_1905_10574_gb300 import sylv
    # offsets implied by the C declarations (natural alignment)
    assert ctypes.sizeof(sylv.sylv_opts) == 80
    assert sylv.sylv_opts.omega.offset == 16 and sylv.sylv_opts.timeout_ms.offset == 40
    assert sylv.sylv_opts.workspace_bytes.offset == 64
    assert ctypes.sizeof(sylv.sylv_result) == 40
    assert sylv.sylv_result.info.offset == 16 and sylv.sylv_result.min_tile_exp.offset == 36


def test_host_side_argument_errors(lib):
    """Invalid arguments are rejected on the host before any GPU work (no device needed)."""
    from paper_1905_10574_gb300 import sylv
    assert sylv.sylv_tri_solve(-1, 4, 0, 1, 0, 4, 0, 1)[0] == -1
    assert sylv.sylv_tri_solve(4, 4, 1, 2, 1, 4, 1, 4)[0] == -4  # lda < m
    assert sylv.sylv_tri_solve(4, 4, 1, 4, 1, 4, 1, 4, tile=1)[0] == -9
    o = sylv.sylv_default_opts()
    o.precision = 7
    assert sylv.sylv_tri_solve_ex(4, 4, 1, 4, 1, 4, 1, 4, o) == sylv.SYLV_ERR_UNSUPPORTED
    assert sylv.sylv_error_string(sylv.SYLV_ERR_TIMEOUT).startswith("a device-side wait")
    assert "sm_103a" in sylv.sylv_version()


def test_workspace_size_monotone(lib):
    from paper_1905_10574_gb300 import sylv
    o = sylv.sylv_default_opts()
    a = sylv.sylv_workspace_size(256, 256, o)
    b = sylv.sylv_workspace_size(1024, 1024, o)
    assert 0 < a < b
    o.precision = sylv.SYLV_FP32_REFINE
    assert sylv.sylv_workspace_size(256, 256, o) > a
    assert sylv.sylv_workspace_size(0, 5, o) == 0


def test_library_links_no_blas(lib):
    """Every product on the solver's path runs in the library's own kernels: the
    shared library needs no BLAS library (its dynamic section lists none)."""
    import shutil
    import subprocess
    from paper_1905_10574_gb300 import build
    if not shutil.which("readelf"):
        pytest.skip("readelf not available")
    out = subprocess.run(["readelf", "-d", build.LIB], capture_output=True, text=True, check=True).stdout
    needed = [ln for ln in out.splitlines() if "NEEDED" in ln]
    assert needed and not any("blas" in ln.lower() for ln in needed), needed
