"""ctypes binding of the C ABI declared in include/shtg.h (argument
marshalling only; every computation runs in libshtg.so)."""
from __future__ import annotations

import ctypes as C
import os
import threading

_lock = threading.Lock()
_lib = None

SHTG_OK = 0
ERRORS = {-1: "SHTG_ERR_ARG", -2: "SHTG_ERR_CUDA", -3: "SHTG_ERR_NOT_CONVERGED",
          -4: "SHTG_ERR_TIMEOUT", -5: "SHTG_ERR_NONFINITE", -6: "SHTG_ERR_NOT_SPD",
          -7: "SHTG_ERR_NOMEM"}
GEOM_HEALPIX, GEOM_GAUSS = 0, 1
FP64, FP32, TC32, DF64 = 0, 1, 2, 3
ARITH_DEFAULT, ARITH_FP64, ARITH_DF64 = 0, 1, 2
SPIN0, SPIN2, BLOCK_SOLVER = 1, 2, 4
CG_FP64, CG_MIXED, CG_MIXED_TC, CG_BLOCK = 0, 1, 2, 3
HOST_INPUTS = 1
PROFILE = 2
NO_GRAPHS = 4
SPLIT_RHS = 8
GROUPED = 16
GRAD_COMPONENTS = 1
PRECOND_NONE, PRECOND_DIAG, PRECOND_LOWL, PRECOND_AZIM = 0, 1, 2, 3

# every symbol include/shtg.h declares
SYMBOLS = ("shtg_plan_create", "shtg_plan_destroy", "shtg_plan_get_info",
           "shtg_last_error_string", "shtg_version", "shtg_alm2map", "shtg_alm2map_adjoint",
           "shtg_alm2map_vjp",
           "shtg_map2alm", "shtg_cg_sample", "shtg_cg_sample_chains", "shtg_apply_operator",
           "shtg_logpost_grad", "shtg_probe_fma_peak", "shtg_fluctuation_rescale",
           "shtg_joint_log_target", "shtg_joint_acceptance", "shtg_logpost_grad_binned",
           "shtg_lowl_block", "shtg_precond_apply")


class PlanInfo(C.Structure):
    _fields_ = [("geom", C.c_int), ("nside", C.c_int), ("nring", C.c_int), ("lmax", C.c_int),
                ("max_batch", C.c_int), ("flags", C.c_int), ("npix", C.c_int64),
                ("nalm", C.c_int64), ("device_bytes", C.c_int64)]


class Problem(C.Structure):
    _fields_ = [("ncomp", C.c_int), ("nbatch", C.c_int), ("cl", C.c_void_p), ("bl", C.c_void_p),
                ("ninv", C.c_void_p), ("d", C.c_void_p), ("w1", C.c_void_p), ("w2", C.c_void_p),
                ("cl_scale", C.c_void_p)]


class CGOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int), ("mode", C.c_int),
                ("precond", C.c_int), ("reliable_delta", C.c_double), ("fp64_arith", C.c_int),
                ("check_every", C.c_int), ("flags", C.c_int), ("lowl_lmax", C.c_int),
                ("block_lmax", C.c_int)]


class CGStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer_steps", C.c_int), ("fp64_matvecs", C.c_int),
                ("converged", C.c_int), ("rel_residual", C.c_double), ("ms_setup", C.c_double),
                ("ms_rhs", C.c_double), ("ms_solve", C.c_double), ("ms_total", C.c_double),
                ("launches", C.c_longlong), ("kernel_ms", C.c_double * 8),
                ("kernel_launches", C.c_int * 8)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if k.startswith("kernel_") else v
        return out


class ShtgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "libshtg.so")


def load(build_if_missing: bool = True):
    """Load libshtg.so (building it in-tree first if it is missing or stale).
    Raises if the library cannot be built or loaded: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if build_if_missing and not _build.up_to_date():
            _build.build()
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run paper_2306_15511_gb300.build")
        L = C.CDLL(path)
        vp, ci, cd = C.c_void_p, C.c_int, C.c_double
        L.shtg_plan_create.argtypes = [ci, ci, ci, ci, ci, ci, C.POINTER(vp)]
        L.shtg_plan_destroy.argtypes = [vp]
        L.shtg_plan_get_info.argtypes = [vp, C.POINTER(PlanInfo)]
        L.shtg_last_error_string.restype = C.c_char_p
        L.shtg_alm2map.argtypes = [vp, ci, ci, vp, vp, ci, vp]
        L.shtg_alm2map_adjoint.argtypes = [vp, ci, ci, vp, vp, ci, vp]
        L.shtg_alm2map_vjp.argtypes = [vp, ci, ci, vp, vp, ci, vp]
        L.shtg_map2alm.argtypes = [vp, ci, ci, vp, vp, ci, ci, vp]
        L.shtg_cg_sample.argtypes = [vp, C.POINTER(Problem), vp, C.POINTER(CGOpts),
                                     C.POINTER(CGStats), vp]
        L.shtg_apply_operator.argtypes = [vp, C.POINTER(Problem), vp, vp, vp]
        L.shtg_logpost_grad.argtypes = [vp, vp, vp, vp, vp, vp, ci, vp, vp, ci, C.POINTER(cd),
                                        vp, vp, vp]
        L.shtg_probe_fma_peak.argtypes = [ci, C.POINTER(ci), C.POINTER(cd), vp]
        L.shtg_fluctuation_rescale.argtypes = [vp, ci, vp, vp, vp, vp, ci, vp]
        L.shtg_joint_log_target.argtypes = [vp, C.POINTER(Problem), ci, vp, vp, vp, vp]
        L.shtg_joint_acceptance.argtypes = [cd, cd, cd, cd, C.POINTER(cd)]
        L.shtg_lowl_block.argtypes = [vp, C.POINTER(Problem), ci, vp, vp, C.POINTER(ci), vp]
        L.shtg_precond_apply.argtypes = [vp, C.POINTER(Problem), C.POINTER(CGOpts), vp, vp, vp]
        L.shtg_logpost_grad_binned.argtypes = [vp, vp, vp, vp, vp, vp, ci, vp, vp, vp, ci, C.POINTER(cd),
                                               vp, vp, vp]
        for s in SYMBOLS:
            if s != "shtg_last_error_string":
                getattr(L, s).restype = ci
        _lib = L
        return _lib


def check(rc: int, allow=()):
    if rc != SHTG_OK and rc not in allow:
        raise ShtgError(rc, load().shtg_last_error_string().decode())
    return rc
