"""The C-ABI library loads and exports every entry point include/gp.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "gp.h")).read()
    return re.findall(r"^\s*(?:gp_status|int|long long|const char\*)\s+(gp_\w+)\s*\(", hdr, re.M)


@pytest.fixture(scope="module")
def lib():
    from paper_2003_03590_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_abi():
    names = _declared()
    for must in ("gp_plan_create", "gp_plan_destroy", "gp_init_srp", "gp_init_rvr", "gp_step",
                 "gp_diagnostics", "gp_adjoint_step", "gp_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2003_03590_gb300 import _lib
    assert set(_declared()) == set(_lib.SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.gp_status_string.restype = ctypes.c_char_p
    assert lib.gp_status_string(0) == b"GP_OK"
    assert lib.gp_status_string(2) == b"GP_ERR_UNSUPPORTED_SIZE"
    # invalid arguments are rejected on the host before any CUDA call
    from paper_2003_03590_gb300 import _lib
    L = _lib.load()
    out = ctypes.c_void_p()
    fp = _lib.FieldParams(n=10, xi=0.1, alpha=0.0, beta=0.0, dt=0.01, precision=0, split=0, nonlin_minus_one=1)
    assert L.gp_plan_create(ctypes.byref(fp), 1, None, ctypes.byref(out)) == 2   # N = 10 unsupported
    fp.n = 16
    fp.dt = float("nan")
    assert L.gp_plan_create(ctypes.byref(fp), 1, None, ctypes.byref(out)) == 1
    assert L.gp_plan_create(None, 1, None, ctypes.byref(out)) == 1
    assert not out.value


def test_product_path_fails_loudly_without_the_library(tmp_path, monkeypatch):
    from paper_2003_03590_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()
