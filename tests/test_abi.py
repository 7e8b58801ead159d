"""The C-ABI library loads and exports every entry point include/nlem.h declares (CPU only:
no compute calls), and the binding refuses to run without the library."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nlem.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def lib():
    from paper_1501_03879_gb300 import build as pkg_build
    path = pkg_build.build()
    return ctypes.CDLL(path)


def test_header_parsed():
    names = declared_functions()
    for must in ("em_solve", "em_solve_batch", "nlem_denoise", "nlem_ctx_create", "nlem_last_error"):
        assert must in names


def test_every_declared_symbol_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu(lib):
    lib.nlem_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.nlem_version()
    lib.nlem_last_error.restype = ctypes.c_char_p
    assert lib.nlem_last_error() is not None


def test_options_default(lib):
    from paper_1501_03879_gb300._binding import _Options
    o = _Options()
    o.tol = 3.0
    lib.nlem_options_default(ctypes.byref(o))
    assert o.tol == 0.0 and o.check_every == 1 and o.precision == 0 and o.init == 0


def test_null_ctx_is_invalid(lib):
    # argument validation happens before any device call
    lib.em_solve_batch.restype = ctypes.c_int
    from paper_1501_03879_gb300._binding import _Box
    rc = lib.em_solve_batch(None, None, None, ctypes.c_longlong(1), 3, 2, _Box(0.0, 1.0), ctypes.c_float(1.0), 5,
                            None, None, None, None, None, None, None, None)
    assert rc == -1
    lib.nlem_last_error.restype = ctypes.c_char_p
    assert b"ctx" in lib.nlem_last_error()
