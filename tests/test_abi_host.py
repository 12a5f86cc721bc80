"""Host-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/gigalens.h declares; the Python binding
covers the same names. No kernel is launched."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gigalens.h")


def declared_functions():
    with open(HEADER) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|size_t|long long|const char\s*\*)\s*\**\s*(gl_\w+)\s*\(", src, flags=re.M)
    assert names, "no declarations parsed"
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2202_07663_gb300 import build
    build.build()
    from paper_2202_07663_gb300 import abi
    return abi.lib_handle()


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_header():
    from paper_2202_07663_gb300 import abi
    assert sorted(abi.SIGNATURES) == declared_functions()


def test_error_strings_without_gpu(lib):
    from paper_2202_07663_gb300 import abi
    assert lib.gl_error_string(0) == b"GL_OK"
    assert lib.gl_error_string(-1) == b"GL_ERR_INVALID_ARG"
    assert lib.gl_error_string(-6) == b"GL_ERR_UNSUPPORTED"
    assert lib.gl_kernel_name(abi.GL_K_RAY_ADJ) == b"k_ray_adj"
    # argument validation happens before any device call
    assert lib.gl_system_create(None, None, None, 0.0, 1, 1, None, 1, 1.0, 1, 1.0, None) == -1
    assert lib.gl_loglik(None, None, 1, None, None, None) == -1


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2202_07663_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "gl_oracle" not in text, f
    # and the oracle never includes the CUDA sources
    osrc = open(os.path.join(ROOT, "oracle", "gl_oracle.cpp")).read()
    assert "gl_device" not in osrc and "gigalens.h" not in osrc
