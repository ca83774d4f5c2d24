"""Build and load the C part of the oracle (liboracle.so, built in-tree).

Test infrastructure only: imported by tests, the smoke check and the CPU
baseline leg of the benchmark, never by the product library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O3, OpenMP, portable flags)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_D = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            ci = C.c_int
            L.orc_abi_version.restype = ci
            L.orc_set_threads.argtypes = [ci]
            L.orc_set_threads.restype = ci
            L.orc_healpix_geom.argtypes = [ci, _D, _D, _I64, _D, _I64]
            L.orc_gl_geom.argtypes = [ci, _D, _D, _D]
            L.orc_lambda.argtypes = [ci, ci, C.c_double, C.c_double, _D]
            L.orc_lambda_spin2.argtypes = [ci, ci, C.c_double, C.c_double, _D, _D]
            geo = [ci, _D, _D, _I64, _D, _I64, ci]
            L.orc_alm2map.argtypes = geo + [_D, _D]
            L.orc_alm2map_adjoint.argtypes = geo + [_D, _D]
            L.orc_alm2map_adjoint_m.argtypes = geo + [_D, _D, ci, C.c_void_p]
            L.orc_alm2map_spin2.argtypes = geo + [_D, _D, _D, _D]
            L.orc_alm2map_spin2_adjoint_m.argtypes = geo + [_D, _D, _D, _D, ci, C.c_void_p]
            L.orc_diag_ringsum.argtypes = [ci, _D, _D, ci, ci, _D, _D]
            for f in ("orc_healpix_geom", "orc_gl_geom", "orc_lambda", "orc_lambda_spin2",
                      "orc_alm2map", "orc_alm2map_adjoint", "orc_alm2map_adjoint_m",
                      "orc_alm2map_spin2", "orc_alm2map_spin2_adjoint_m", "orc_diag_ringsum"):
                getattr(L, f).restype = None
            _lib = L
    return _lib
