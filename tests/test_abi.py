"""The C-ABI library loads and exports every entry point its headers declare
(no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^(?!\s*(?:typedef|#))[^;{}()]*?\b(sbc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_headers_declare_entry_points():
    names = declared_functions()
    for must in ("sbc_graph_create", "sbc_count", "sbc_last_error"):
        assert must in names


@pytest.mark.parametrize("name", declared_functions())
def test_symbol_exported(lib, name):
    assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_version_and_error_without_gpu(lib):
    lib.sbc_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.sbc_version()
    lib.sbc_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.sbc_last_error(), bytes)


def test_invalid_arguments_rejected_on_host(lib):
    # argument checks that happen before any CUDA call
    lib.sbc_count.restype = ctypes.c_int
    lib.sbc_count.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                              ctypes.c_void_p]
    assert lib.sbc_count(None, 3, 3, None, None) == 1  # SBC_E_INVAL
    lib.sbc_set_allocator.restype = ctypes.c_int
    lib.sbc_set_allocator.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.sbc_set_allocator(ctypes.c_void_p(1), None, None) == 1
    assert lib.sbc_set_allocator(None, None, None) == 0


def test_autotune_rejects_empty_batch_on_host(lib):
    lib.sbc_autotune.restype = ctypes.c_int
    lib.sbc_autotune.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    out = (ctypes.c_int32 * 4)()
    assert lib.sbc_autotune(None, 0, 3, 3, 0, out, None) == 1  # SBC_E_INVAL
    assert lib.sbc_autotune(None, 0, 3, 3, 0, None, None) == 1


def test_plain_c_client(lib, tmp_path):
    """sbc.h compiles as C and a C program linked against libsbc.so runs the
    host-side paths (argument and graph errors, a local graph)."""
    import subprocess

    path = lib._name
    exe = str(tmp_path / "abi_client")
    libdir = os.path.dirname(path)
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "abi_client.c"), "-o", exe,
                           path, f"-Wl,-rpath,{libdir}"])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "ok"
