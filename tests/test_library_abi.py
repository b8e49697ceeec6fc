"""The C-ABI library loads and exports every symbol include/cps.h declares
(no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "cps.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cps_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2309_03543_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("cps_create", "cps_assemble", "cps_solve", "cps_solve_batch", "cps_adjoint",
                 "cps_set_precond", "cps_last_error", "cps_sys_free"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_declares_every_symbol(lib):
    from paper_2309_03543_gb300 import _cps
    assert sorted(_cps.SIGNATURES) == declared_symbols()


def test_null_handles_are_rejected_without_a_gpu(lib):
    lib.cps_solve.restype = ctypes.c_int
    lib.cps_sys_free.restype = ctypes.c_int
    assert lib.cps_sys_free(None) == -1
    assert lib.cps_destroy(None) == -1
    out = ctypes.c_void_p()
    # no device in this container: create must fail cleanly, not crash
    rc = lib.cps_create(ctypes.byref(out), 0)
    assert rc in (0, -1, -9)
