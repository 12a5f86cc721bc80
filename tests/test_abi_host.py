"""Host-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/gigalens.h declares; the Python binding
covers the same names; the header is plain C and a C program links against
the library. No kernel is launched."""
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


def test_kernel_kinds_mirror_header(lib):
    """The instrumentation kinds: the header's enum, the binding's constants
    and the library's names agree, one name per kind."""
    from paper_2202_07663_gb300 import abi
    text = _read(HEADER)
    kinds = dict(re.findall(r"(GL_K_\w+)\s*=\s*(\d+)", text))
    n = int(re.search(r"#define GL_KERNEL_KINDS (\d+)", text).group(1))
    assert n == abi.GL_KERNEL_KINDS and sorted(int(v) for v in kinds.values()) == list(range(n))
    for name, value in kinds.items():
        assert getattr(abi, name) == int(value), name
    names = [lib.gl_kernel_name(i) for i in range(n)]
    assert len(set(names)) == n and b"unknown" not in names
    assert lib.gl_kernel_name(abi.GL_K_ORDER) == b"k_order"
    assert lib.gl_kernel_name(n) == b"unknown"


def test_error_codes_mirror_header():
    from paper_2202_07663_gb300 import abi
    codes = dict(re.findall(r"(GL_(?:OK|ERR_\w+))\s*=\s*(-?\d+)", _read(HEADER)))
    assert len(codes) == 7
    for name, value in codes.items():
        assert getattr(abi, name) == int(value), name


# calls that accept NULL (destroy), only read state, or take no pointer
NULL_TOLERANT = {"gl_system_destroy", "gl_batcher_destroy", "gl_profile_read", "gl_error_string",
                 "gl_last_error_message", "gl_kernel_name", "gl_launch_count", "gl_profile_enable",
                 "gl_profile_reset", "gl_vi_param_count", "gl_vi_workspace_bytes", "gl_system_scratch_bytes",
                 "gl_system_resident_bytes", "gl_system_scratch_held", "gl_batcher_segment_bytes",
                 "gl_profile_select"}


@pytest.mark.parametrize("name", [n for n in declared_functions() if n not in NULL_TOLERANT])
def test_null_pointers_are_refused_before_any_launch(lib, name):
    """Each call that takes pointers returns GL_ERR_INVALID_ARG, with a
    message, for NULL ones at size 1, and launches nothing: the checks come
    before any device work (this runs without a GPU)."""
    import ctypes
    from paper_2202_07663_gb300 import abi
    args, _ = abi.SIGNATURES[name]
    vals = [1 if a in (ctypes.c_int, ctypes.c_size_t) else 1.0 if a in (ctypes.c_double, ctypes.c_float) else None
            for a in args]
    n0 = lib.gl_launch_count()
    assert getattr(lib, name)(*vals) == abi.GL_ERR_INVALID_ARG
    assert lib.gl_last_error_message().startswith(b"null")
    assert lib.gl_launch_count() == n0


def test_chained_leapfrog_refuses_aliased_state(lib):
    """gl_hmc_leapfrog_whitened_chain reads z before overwriting it lane by
    lane, so x, p, z and grad_theta must be distinct; the check runs before
    any launch (the pointers below are never dereferenced)."""
    import ctypes
    from paper_2202_07663_gb300 import abi, map as gmap
    table = gmap.prior_table()   # held: the call reads it on the host
    prior = ctypes.addressof(table)
    a, b, c, d, m = 0x1000, 0x2000, 0x3000, 0x4000, 0x5000
    n0 = lib.gl_launch_count()
    for x, p, z, g in ((a, b, a, c), (a, b, b, c), (a, a, b, c), (a, b, c, c), (a, c, b, c), (c, b, d, c)):
        assert lib.gl_hmc_leapfrog_whitened_chain(4, x, p, z, g, m, 0.1, None, 1.0, m, m, prior, m,
                                                  None) == abi.GL_ERR_INVALID_ARG
        assert b"alias" in lib.gl_last_error_message()
    assert lib.gl_hmc_leapfrog_whitened_chain(4, a, b, c, d, m, float("nan"), None, 1.0, m, m, prior, m,
                                              None) == abi.GL_ERR_INVALID_ARG
    assert lib.gl_hmc_leapfrog_whitened_chain(-1, a, b, c, d, m, 0.1, None, 1.0, m, m, prior, m,
                                              None) == abi.GL_ERR_INVALID_ARG
    assert lib.gl_hmc_leapfrog_whitened_chain(0, a, b, c, d, m, 0.1, None, 1.0, m, m, prior, m, None) == abi.GL_OK
    assert lib.gl_launch_count() == n0


def _read(path):
    with open(path) as f:
        return f.read()


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2202_07663_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = _read(os.path.join(dirpath, f))
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "gl_oracle" not in text, f
    # and the oracle never includes the CUDA sources
    osrc = _read(os.path.join(ROOT, "oracle", "gl_oracle.cpp"))
    assert "gl_device" not in osrc and "gigalens.h" not in osrc


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: without the built CUDA library every call raises."""
    from paper_2202_07663_gb300 import abi
    monkeypatch.setattr(abi, "_lib", None)
    monkeypatch.setattr(abi, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libgigalens.so"))
    with pytest.raises(RuntimeError, match="not built"):
        abi.lib_handle()


def test_benchmark_without_a_gpu_exits_nonzero():
    """The benchmark's own arm has no host path: on a machine without a GPU it
    stops with an error instead of timing anything."""
    import subprocess
    import sys
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = subprocess.run([sys.executable, "bench.py", "--steps", "1", "--warmup", "3", "--no-workloads",
                        "--no-cpu-baseline"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/gigalens.h compiles as strict C99 and as C++; a C program that
    takes the address of every declared call links against the library and
    runs its GPU-free calls."""
    import shutil
    import subprocess
    from paper_2202_07663_gb300 import abi
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    names = declared_functions()
    src = tmp_path / "abi_probe.c"
    src.write_text('#include <stdio.h>\n#include "gigalens.h"\n'
                   "typedef void (*fn_t)(void);\n"
                   "static fn_t table[] = {" + ", ".join("(fn_t)%s" % n for n in names) + "};\n"
                   "int main(void) {\n"
                   "  printf(\"%d %s %s\\n\", (int)(sizeof table / sizeof table[0]), gl_error_string(GL_ERR_INVALID_ARG),"
                   " gl_kernel_name(GL_K_RAY_ADJ));\n"
                   "  return gl_loglik(NULL, NULL, 1, NULL, NULL, NULL) == GL_ERR_INVALID_ARG ? 0 : 1;\n}\n")
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(abi.LIB_PATH)
    exe = tmp_path / "abi_probe"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-Wno-cast-function-type",
                    "-I", inc, str(src), "-o", str(exe), "-L", libdir, "-lgigalens", "-Wl,-rpath," + libdir],
                   check=True, capture_output=True, text=True)
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c++",
                    "-I", inc, "-"], input='#include "gigalens.h"\n', check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == [str(len(names)), "GL_ERR_INVALID_ARG", "k_ray_adj"]
