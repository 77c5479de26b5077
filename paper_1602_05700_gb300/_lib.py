"""ctypes declarations of the C ABI in include/hg.h and include/hg_hydro.h (argument marshalling only).

The library is loaded from paper_1602_05700_gb300/_build/libhypergrav.so, or from its checked variant
_build/libhypergrav_debug.so when the environment sets HG_DEBUG=1 (the same ABI, with index checks before the
sub-step kernels' stores).  There is no other implementation: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
DEBUG = os.environ.get("HG_DEBUG", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "_build", "libhypergrav_debug.so" if DEBUG else "libhypergrav.so")

HG_OK = 0
HG_ERR_ARG = -1
HG_ERR_CFL = -2
HG_ERR_CUDA = -3
HG_ERR_NONFINITE = -4
HG_ERR_TIMEOUT = -5
HG_ERR_STATE = -6
HG_ERR_BOUNDS = -7

HG_PREC_F32K = 0
HG_PREC_F64 = 1
HG_DT_F32 = 0
HG_DT_F64 = 1
HG_BC_DIRICHLET_ANALYTIC = 0
HG_BC_DIRICHLET_MULTIPOLE = 1
HG_BC_ROBIN = 2
HG_BC_PERIODIC = 3
HG_MAX_LMAX = 8
HG_MAX_TEMPORAL_DEPTH = 8


class hg_stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("residual_rms", ctypes.c_double), ("residual_max", ctypes.c_double),
                ("change_rel", ctypes.c_double), ("phi_max", ctypes.c_double), ("step", ctypes.c_longlong),
                ("nonfinite", ctypes.c_int)]


class HGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hg error {code}: {msg}")
        self.code = code


_V = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_P = ctypes.POINTER

# name -> (restype, argtypes); the exported symbols of include/hg.h and include/hg_hydro.h
SIGNATURES = {
    "hg_init_grid": (_I, [_P(_V), _I, _I, _I, _D, _P(_D), _D, _D, _D, _I, _I, _I, _V]),
    "hg_set_density": (_I, [_V, _V, _I, _I]),
    "hg_set_phi": (_I, [_V, _V, _V, _I, _I]),
    "hg_step": (_I, [_V, _I]),
    "hg_set_temporal_depth": (_I, [_V, _I]),
    "hg_set_temporal_exact": (_I, [_V, _I]),
    "hg_set_block_depth": (_I, [_V, _I]),
    "hg_accel": (_I, [_V, _V, _V, _V, _I]),
    "hg_get_phi": (_I, [_V, _V, _I, _I]),
    "hg_get_phi_ghosted": (_I, [_V, _P(_D)]),
    "hg_get_stats": (_I, [_V, _P(hg_stats)]),
    "hg_get_moments": (_I, [_V, _P(_D)]),
    "hg_compare": (_I, [_V, _V, _I, _P(_D)]),
    "hg_state_bytes": (ctypes.c_size_t, [_V]),
    "hg_save_state": (_I, [_V, _V, _I]),
    "hg_load_state": (_I, [_V, _V, _I]),
    "hg_adjoint_reset": (_I, [_V]),
    "hg_adjoint_inject": (_I, [_V, _V, _I, _I]),
    "hg_adjoint_step": (_I, [_V, _I]),
    "hg_adjoint_grad": (_I, [_V, _V, _I, _I]),
    "hg_adjoint": (_I, [_V, _V, _I, _V, _I, _I]),
    "hg_profile": (_I, [_V, _I]),
    "hg_profile_read": (_I, [_V, _P(_D), _P(ctypes.c_longlong), _P(ctypes.c_longlong)]),
    "hg_io_step": (_I, [_V, _V, _I, _I, _V, _V, _V, _I]),
    "hg_io_wait": (_I, [_V, _I]),
    "hg_check_bounded_wait": (_I, [_V]),
    "hg_sync": (_I, [_V]),
    "hg_free": (None, [_V]),
    "hg_batch_create": (_I, [_P(_V), _I, _P(_V)]),
    "hg_batch_step": (_I, [_V, _I]),
    "hg_batch_info": (_I, [_V, _P(_I), _P(ctypes.c_longlong)]),
    "hg_batch_tuning": (_I, [_V, _P(_I)]),
    "hg_batch_set_split": (_I, [_V, _I]),
    "hg_batch_free": (None, [_V]),
    "hg_moments_noalloc": (_I, [_V, _I, _I, _I, _I, _D, _P(_D), _I, _V, _I, _V]),
    "hg_probe_rate": (_I, [_I, _P(_D), _P(_D)]),
    "hg_init_slab": (_I, [_P(_V), _I, _I, _I, _D, _P(_D), _D, _D, _D, _I, _I, _I, _V, _I]),
    "hg_set_z_interface": (_I, [_V, _I, _I]),
    "hg_plane_bytes": (ctypes.c_size_t, [_V]),
    "hg_get_plane": (_I, [_V, _I, _V, _I]),
    "hg_put_ghost_plane": (_I, [_V, _I, _V, _I]),
    "hg_set_boundary_moments": (_I, [_V, _P(_D)]),
    "hg_last_error": (ctypes.c_char_p, []),
    # include/hg_hydro.h
    "hg_hydro_init": (_I, [_P(_V), _I, _I, _I, _D, _D, _D, _D, _I, _V]),
    "hg_hydro_set_primitive": (_I, [_V, _V, _I, _I]),
    "hg_hydro_set_state": (_I, [_V, _V, _I, _I]),
    "hg_hydro_get_state": (_I, [_V, _V, _I, _I]),
    "hg_hydro_max_speed": (_I, [_V, _P(_D)]),
    "hg_hydro_step": (_I, [_V, _V, _D, _I]),
    "hg_hydro_virial": (_I, [_V, _V, _P(_D)]),
    "hg_hydro_launches": (_I, [_V, _P(ctypes.c_longlong)]),
    "hg_hydro_profile": (_I, [_V, _I]),
    "hg_hydro_profile_read": (_I, [_V, _P(_D), _P(ctypes.c_longlong)]),
    "hg_hydro_free": (None, [_V]),
    "hg_check_bounds": (_I, [_V]),
    "hg_is_debug_build": (_I, []),
}

_lib = None


def lib():
    """The loaded library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run paper_1602_05700_gb300.build() "
                               "(debug=True for the HG_DEBUG variant, or __graft_entry__.build()) first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != HG_OK:
        raise HGError(rc, lib().hg_last_error().decode())
