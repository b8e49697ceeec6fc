"""ctypes declarations of the C ABI in include/cps.h (libcps.so).

Loading fails loudly when the CUDA library has not been built: there is no
CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcps.so")

OK = 0
ERR_ARG = -1
ERR_NONMANIFOLD = -2
ERR_NONDELAUNAY = -3
ERR_ORIENTATION = -4
ERR_NOT_SPD = -5
ERR_NOT_CONVERGED = -6
ERR_SINGULAR = -7
ERR_NOMEM = -8
ERR_CUDA = -9
ERR_TIMEOUT = -10

KIND_CP2, KIND_CP1_X, KIND_CP1_Y = 0, 1, 2
PER_VERTEX, PER_CELL, PER_CELL_LOGK = 0, 1, 2
PC_JACOBI, PC_IC0, PC_REDUCED = 1, 2, 3
FP64, MIXED = 0, 1
PATH_AUTO, PATH_STREAM, PATH_CLUSTER, PATH_PERSISTENT, PATH_STREAM_L2, PATH_PERSISTENT_L2 = (
    0, 1, 2, 3, 4, 5)
PATH_CLUSTER_1RED = 6
PATH_CLUSTER_PIPE = 11
PATH_CLUSTER_SSTEP2, PATH_CLUSTER_SSTEP3 = 12, 13
PATH_STREAM_1RED, PATH_STREAM_1RED_L2 = 7, 8
PATH_PERSISTENT_1RED, PATH_PERSISTENT_1RED_L2 = 9, 10
BATCH_ONE_LAUNCH, BATCH_GRAPH = 0, 1
CP1_ONE_LAUNCH, CP1_HOST = 0, 1

ERROR_NAMES = {
    ERR_ARG: "CPS_ERR_ARG", ERR_NONMANIFOLD: "CPS_ERR_NONMANIFOLD",
    ERR_NONDELAUNAY: "CPS_ERR_NONDELAUNAY", ERR_ORIENTATION: "CPS_ERR_ORIENTATION",
    ERR_NOT_SPD: "CPS_ERR_NOT_SPD", ERR_NOT_CONVERGED: "CPS_ERR_NOT_CONVERGED",
    ERR_SINGULAR: "CPS_ERR_SINGULAR", ERR_NOMEM: "CPS_ERR_NOMEM", ERR_CUDA: "CPS_ERR_CUDA",
    ERR_TIMEOUT: "CPS_ERR_TIMEOUT",
}

# Every symbol include/cps.h declares, with (restype, argtypes).
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("rel_res", ctypes.c_double),
                ("status", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("launches", ctypes.c_int64)]


class Cp1Stats(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int64), ("solve_iters", ctypes.c_int64),
                ("err", ctypes.c_double), ("rel_res_max", ctypes.c_double)]


SIGNATURES = {
    "cps_create": (_I, [ctypes.POINTER(_P), _I]),
    "cps_destroy": (_I, [_P]),
    "cps_last_error": (ctypes.c_char_p, [_P]),
    "cps_assemble": (_I, [_P, _P, _I64, _P, _I64, _P, _I64, _P, _P, _I, _I, _D, _D,
                          ctypes.POINTER(_P), _P]),
    "cps_set_precond": (_I, [_P, _I, _P]),
    "cps_sys_free": (_I, [_P]),
    "cps_sys_info": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                          ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_I64)]),
    "cps_export_matrix": (_I, [_P, _P, _P, _P, _P]),
    "cps_solve": (_I, [_P, _P, _P, _D, _I64, _I, ctypes.POINTER(Stats), _P]),
    "cps_solve_batch": (_I, [_P, _I, _P, _P, _D, _I64, _I, ctypes.POINTER(Stats), _P]),
    "cps_adjoint": (_I, [_P, _P, _P, _P, _P, _P, _D, _I64, ctypes.POINTER(Stats), _P]),
    "cps_matvec": (_I, [_P, _P, _P, _P]),
    "cps_cp2_setup": (_I, [_P, _P, _P, _P, _P, _P]),
    "cps_cp2_kernel_times": (_I, [_P, _P]),
    "cps_cp1_setup": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "cps_cp1_step": (_I, [_P, _P, _P, _P, _D, _I64, _D, _I64, _I, ctypes.POINTER(Cp1Stats),
                          _P]),
    "cps_cp2_step": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _D, _I64, _I, ctypes.POINTER(Stats),
                          _P]),
    "cps_get_tuning": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "cps_get_gear_shape": (_I, [_P, _P, _P, _P]),
    "cps_set_solver_path": (_I, [_P, _I]),
    "cps_set_batch_path": (_I, [_P, _I]),
    "cps_set_cp1_path": (_I, [_P, _I]),
    "cps_set_kernel_shapes": (_I, [_P, _I, _P, _P, _P]),
    "cps_test_inject": (_I, [_P, _I]),
    "cps_solve_ell_noalloc": (_I, [_I64, _P, _P, _P, _P, _P, _D, _I64, ctypes.POINTER(Stats),
                                   _P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libcps.so and declare every C-ABI symbol.  Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
