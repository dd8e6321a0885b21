"""ctypes binding of the oracle's C kernels (test infrastructure only)."""
import ctypes
import numpy as np

from . import build as _build

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_L = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _lib.or_cell_matrices.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D,
                                          ctypes.c_int, _D, ctypes.c_int, _I, _D]
        _lib.or_cell_mass.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D]
        _lib.or_cell_rhs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D,
                                     ctypes.c_int, _D, ctypes.c_int, _D, _D]
        _lib.or_cell_qpoints.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D]
        _lib.or_l2_error_sq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D, ctypes.c_int]
        _lib.or_l2_error_sq.restype = ctypes.c_double
        _lib.or_csr_spmv.argtypes = [ctypes.c_int64, _L, _L, _D, _D, _D]
    return _lib


def dp(a):
    return a.ctypes.data_as(_D)


def ip(a):
    return a.ctypes.data_as(_I)


def lp(a):
    return a.ctypes.data_as(_L)


def f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)
