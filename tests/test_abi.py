"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol include/hg.h declares.
No compute call is made here (there is no GPU on the build host)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hg_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1602_05700_gb300.builder import build
    return build()


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    declared = _declared()
    assert {"hg_init_grid", "hg_set_density", "hg_step", "hg_accel", "hg_get_phi", "hg_free"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_debug_variant_exports_the_same_symbols():
    """The HG_DEBUG library is the same ABI with index checks compiled in; without a GPU only its exports and its
    own answer to hg_is_debug_build are checkable."""
    from paper_1602_05700_gb300.builder import build
    D = ctypes.CDLL(build(debug=True))
    missing = [n for n in sorted(_declared()) if not hasattr(D, n)]
    assert not missing, f"declared but not exported by the debug build: {missing}"
    assert D.hg_is_debug_build() == 1


def test_binding_covers_every_declared_symbol():
    from paper_1602_05700_gb300 import _lib
    assert _declared() == set(_lib.SIGNATURES)


def test_release_library_reports_release(lib_path):
    assert ctypes.CDLL(lib_path).hg_is_debug_build() == 0


def test_last_error_is_empty_string_initially(lib_path):
    from paper_1602_05700_gb300 import _lib
    assert _lib.lib().hg_last_error() == b""


def test_invalid_arguments_rejected_on_host(lib_path):
    """Argument checks run before any device call, so they are testable without a GPU."""
    from paper_1602_05700_gb300 import _lib
    L = _lib.lib()
    h = ctypes.c_void_p()
    org = (ctypes.c_double * 3)(-0.5, -0.5, -0.5)
    assert L.hg_init_grid(ctypes.byref(h), 0, 8, 8, 0.1, org, 1.0, 1.0, 0.01, 0, 2, 0, None) == _lib.HG_ERR_ARG
    assert h.value is None
    assert L.hg_init_grid(ctypes.byref(h), 8, 8, 8, 0.1, org, 1.0, 1.0, 0.01, 7, 2, 0, None) == _lib.HG_ERR_ARG
    assert L.hg_init_grid(ctypes.byref(h), 8, 8, 8, 0.1, org, 1.0, 1.0, 0.01, 0, 9, 0, None) == _lib.HG_ERR_ARG
    assert L.hg_init_grid(ctypes.byref(h), 8, 8, 8, 0.1, org, 1.0, 1.0, 0.01, 0, 1, 99, None) == _lib.HG_ERR_ARG
    # nu sqrt(3) = 1.0 * 0.06 / 0.1 * 1.732 > 1
    assert L.hg_init_grid(ctypes.byref(h), 8, 8, 8, 0.1, org, 1.0, 1.0, 0.06, 0, 2, 0, None) == _lib.HG_ERR_CFL
    assert b"unstable" in L.hg_last_error()
    assert L.hg_step(None, 1) == _lib.HG_ERR_ARG
    L.hg_free(None)


def test_hydro_invalid_arguments_rejected_on_host(lib_path):
    from paper_1602_05700_gb300 import _lib
    L = _lib.lib()
    h = ctypes.c_void_p()
    assert L.hg_hydro_init(ctypes.byref(h), 0, 8, 8, 0.1, 5.0 / 3.0, 0.0, 0.0, 0, None) == _lib.HG_ERR_ARG
    assert h.value is None
    assert L.hg_hydro_init(ctypes.byref(h), 8, 8, 8, 0.1, 1.0, 0.0, 0.0, 0, None) == _lib.HG_ERR_ARG
    assert L.hg_hydro_init(ctypes.byref(h), 8, 8, 8, -0.1, 5.0 / 3.0, 0.0, 0.0, 0, None) == _lib.HG_ERR_ARG
    assert L.hg_hydro_init(ctypes.byref(h), 8, 8, 8, 0.1, 5.0 / 3.0, -1.0, 0.0, 0, None) == _lib.HG_ERR_ARG
    assert L.hg_hydro_init(ctypes.byref(h), 8, 8, 8, 0.1, 5.0 / 3.0, 0.0, 0.0, 5, None) == _lib.HG_ERR_ARG
    assert L.hg_hydro_step(None, None, 0.1, 1) == _lib.HG_ERR_ARG
    assert L.hg_hydro_virial(None, None, None) == _lib.HG_ERR_ARG
