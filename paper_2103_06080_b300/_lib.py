"""ctypes binding of libkzk.so (the C ABI declared in include/kzk.h).

Argument marshalling only: every step of the propagator runs in the CUDA
library.  If the shared object is missing this module raises; there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkzk.so")

KZK_OK, KZK_ERR_ARG, KZK_ERR_SIZE, KZK_ERR_CFL, KZK_ERR_NONFINITE, KZK_ERR_CUDA, KZK_ERR_TIMEOUT, \
    KZK_ERR_OOM, KZK_ERR_STATE = range(9)
KZK_FP64, KZK_FP32 = 0, 1
STATUS_NAMES = ["KZK_OK", "KZK_ERR_ARG", "KZK_ERR_SIZE", "KZK_ERR_CFL", "KZK_ERR_NONFINITE",
                "KZK_ERR_CUDA", "KZK_ERR_TIMEOUT", "KZK_ERR_OOM", "KZK_ERR_STATE"]


class KzkGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("tau_min", ctypes.c_double), ("tau_max", ctypes.c_double),
                ("y_min", ctypes.c_double), ("y_max", ctypes.c_double),
                ("prec", ctypes.c_int32)]


class KzkCoeffs(ctypes.Structure):
    _fields_ = [("B", ctypes.c_double), ("A", ctypes.c_double),
                ("diffraction", ctypes.c_double), ("reg_eps", ctypes.c_double),
                ("weno_eps", ctypes.c_double), ("lf_umax", ctypes.c_double),
                ("B_prof", ctypes.c_double * 4), ("A_prof", ctypes.c_double * 4),
                ("has_profile", ctypes.c_int32), ("n_relax", ctypes.c_int32),
                ("relax_C", ctypes.c_double * 2), ("relax_theta", ctypes.c_double * 2),
                ("method", ctypes.c_int32)]


class KzkMedium(ctypes.Structure):
    _fields_ = [("n_modes", ctypes.c_int32), ("klam", ctypes.POINTER(ctypes.c_double)),
                ("theta", ctypes.POINTER(ctypes.c_double)), ("phase", ctypes.POINTER(ctypes.c_double)),
                ("amp", ctypes.POINTER(ctypes.c_double))]


class KzkOptions(ctypes.Structure):
    _fields_ = [("row_kernel", ctypes.c_int32), ("col_kernel", ctypes.c_int32),
                ("fp32_state", ctypes.c_int32), ("transforms", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("graph", ctypes.c_int32)]


# kzk_options values (include/kzk.h), by option
KZK_AUTO = 0
OPTION_VALUES = {
    "row_kernel": {"auto": 0, "pair": 1, "single": 2},
    "col_kernel": {"auto": 0, "pair": 1, "tma": 2, "tile": 3},
    "fp32_state": {"auto": 0, "compensated": 1, "plain": 2},
    "transforms": {"auto": 0, "mixed": 1},
    "graph": {"auto": 0, "on": 1, "off": 2},
}


class KzkDiag(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("energy", ctypes.c_double),
                ("max_abs", ctypes.c_double), ("nonfinite", ctypes.c_double),
                ("run_max_abs", ctypes.c_double), ("run_nonfinite", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: float(getattr(self, k)) for k, _ in self._fields_}


class KzkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_LIB = None

# (name, restype, argtypes) of every exported function of include/kzk.h
_VP = ctypes.c_void_p
_SIGS = [
    ("kzk_plan_create", ctypes.c_int, [ctypes.POINTER(KzkGrid), ctypes.POINTER(KzkCoeffs), ctypes.c_double,
                                       ctypes.c_int32, ctypes.POINTER(_VP)]),
    ("kzk_plan_create_ex", ctypes.c_int, [ctypes.POINTER(KzkGrid), ctypes.POINTER(KzkCoeffs), ctypes.c_double,
                                          ctypes.c_int32, ctypes.POINTER(KzkOptions), ctypes.POINTER(_VP)]),
    ("kzk_plan_info", ctypes.c_int, [_VP, ctypes.POINTER(KzkOptions)]),
    ("kzk_advance", ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_double, _VP, ctypes.POINTER(KzkDiag)]),
    ("kzk_diag_history", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, _VP]),
    ("kzk_rhs", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, _VP]),
    ("kzk_step_stages", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_double, _VP]),
    ("kzk_tau_fft", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP]),
    ("kzk_get_tables", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
    ("kzk_adjoint", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_double, ctypes.c_int32, _VP]),
    ("kzk_plan_destroy", ctypes.c_int, [_VP]),
    ("kzk_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("kzk_last_error", ctypes.c_char_p, []),
    ("kzk_launch_count", ctypes.c_int64, []),
    ("kzk_kernel_times", ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_double, _VP,
                                        ctypes.POINTER(ctypes.c_double)]),
    ("kzk_alu_peak", ctypes.c_int, [ctypes.c_int32, _VP, ctypes.POINTER(ctypes.c_double)]),
    ("kzk_tile_copy_rate", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP,
                                          ctypes.POINTER(ctypes.c_double)]),
    ("kzk_advance_checkpointed", ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_double, ctypes.c_int32, _VP]),
    ("kzk_adjoint_checkpointed", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("kzk_plan_create_batched", ctypes.c_int, [ctypes.POINTER(KzkGrid), ctypes.POINTER(KzkCoeffs),
                                               ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(_VP)]),
    ("kzk_plan_create_batched_ex", ctypes.c_int, [ctypes.POINTER(KzkGrid), ctypes.POINTER(KzkCoeffs),
                                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.POINTER(KzkOptions), ctypes.POINTER(_VP)]),
    ("kzk_advance_batched", ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.c_int64, ctypes.c_double, _VP,
                                           ctypes.POINTER(KzkDiag)]),
    ("kzk_batch_info", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int64)]),
    ("kzk_batch_test_barrier", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int64]),
    ("kzk_rhs_noalloc", ctypes.c_int, [ctypes.POINTER(KzkGrid), ctypes.POINTER(KzkCoeffs), ctypes.c_int32,
                                       _VP, _VP, ctypes.c_double, _VP]),
    ("kzk_plan_set_medium", ctypes.c_int, [_VP, ctypes.POINTER(KzkMedium)]),
    ("kzk_medium_eval", ctypes.c_int, [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), _VP]),
]

NOALLOC_MAX_POINTS = 1 << 18
KZK_BATCH_AUTOTUNE = 1
KZK_BATCH_STREAMS = 2
KZK_BATCH_PERSISTENT = 4
KZK_COPY_STRIP = 0
KZK_COPY_CONTIGUOUS = 1
KZK_EXPRK22 = 0
KZK_EXPEULER = 1


def lib():
    """Load libkzk.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                               f"g.build()'` (nvcc, sm_103a); there is no non-CUDA path")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def check(status: int) -> None:
    if status != KZK_OK:
        raise KzkError(status, lib().kzk_last_error().decode())


def exported_names() -> list:
    return [s[0] for s in _SIGS]
