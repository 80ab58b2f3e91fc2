"""The C ABI library loads and exports every function include/fh.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fh_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1004_1122_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declarations_present():
    names = _declared()
    assert "fh_create" in names and "fh_apply" in names and "fh_solve" in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1004_1122_gb300 import fh

    assert sorted(fh.EXPORTS) == _declared()


def test_status_strings_without_gpu(lib):
    lib.fh_status_string.restype = ctypes.c_char_p
    lib.fh_status_string.argtypes = [ctypes.c_int]
    assert lib.fh_status_string(0) == b"FH_OK"
    assert lib.fh_status_string(2) == b"FH_ERR_EVEN_N"
    assert lib.fh_status_string(99) == b"FH_UNKNOWN"


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    """Argument validation happens on the host first: short axes, bad d, null pointers."""
    lib.fh_create.restype = ctypes.c_int
    ctx = ctypes.c_void_p()
    N = (ctypes.c_int * 2)(8, 9)
    L = (ctypes.c_double * 4)(1, 0, 0, 1)
    ph = (ctypes.c_uint8 * 72)()
    N2 = (ctypes.c_int * 2)(2, 9)
    rc = lib.fh_create(ctypes.byref(ctx), 2, N2, None, ph, 0, 1, L, None, 0, None)
    assert rc == 1  # FH_ERR_ARG: an axis below 3 nodes
    rc = lib.fh_create(ctypes.byref(ctx), 4, N, None, ph, 0, 1, L, None, 0, None)
    assert rc == 1  # FH_ERR_ARG
    rc = lib.fh_create(None, 2, N, None, ph, 0, 1, L, None, 0, None)
    assert rc == 1
    assert not ctx.value


def test_wait_limit_is_validated_on_the_host(lib):
    lib.fh_set_wait_limit.restype = ctypes.c_int
    lib.fh_set_wait_limit.argtypes = [ctypes.c_double]
    assert lib.fh_set_wait_limit(-1.0) == 1      # FH_ERR_ARG
    assert lib.fh_set_wait_limit(float("nan")) == 1
    assert lib.fh_set_wait_limit(0.5) == 0
    assert lib.fh_set_wait_limit(0.0) == 0        # back to the default
