"""ctypes declarations of the C ABI in include/qb.h and include/qb_diag.h
(argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

QB_OK, QB_EINVAL, QB_ENOMEM, QB_ECUDA, QB_ETIMEOUT, QB_EINTERNAL, QB_EUNSUPPORTED = range(7)
QB_MAX_MODES = 16
QB_TILE_SHAPES = 5
QB_CROSSED, QB_AT_START, QB_NOT_CROSSED = 0, 1, 2
QB_LOSS_Q, QB_LOSS_PO = 0, 1

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_i64_p = ctypes.POINTER(ctypes.c_int64)


class QbModel(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("w", _c_double_p), ("L", _c_double_p), ("exact_momentum", ctypes.c_int)]


MX = QB_MAX_MODES


class QbObs(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double),
        ("norm", ctypes.c_double),
        ("N", ctypes.c_double),
        ("H", ctypes.c_double),
        ("n_tot", ctypes.c_double),
        ("Q", ctypes.c_double),
        ("lam_p", ctypes.c_double),
        ("PO", ctypes.c_double),
        ("gap", ctypes.c_double),
        ("Vminus_p", ctypes.c_double),
        ("a", ctypes.c_double * (2 * MX)),
        ("Mij", ctypes.c_double * (2 * MX * MX)),
        ("aa", ctypes.c_double * (2 * MX * MX)),
        ("xi", ctypes.c_double * (2 * MX)),
        ("eig", ctypes.c_double * MX),
        ("Vminus", ctypes.c_double * MX),
    ]


# name -> (restype, argtypes); must list every function include/*.h declares
SIGNATURES = {
    "qb_last_error": (ctypes.c_char_p, []),
    "qb_sector_build": (ctypes.c_int, [ctypes.POINTER(QbModel), ctypes.c_int, ctypes.c_int, _c_int_p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "qb_space_free": (None, [ctypes.c_void_p]),
    "qb_space_info": (ctypes.c_int, [ctypes.c_void_p, _c_i64_p, _c_int_p, _c_i64_p]),
    "qb_space_sectors": (ctypes.c_int, [ctypes.c_void_p, _c_int_p, _c_int_p, _c_i64_p, _c_i64_p]),
    "qb_space_basis": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "qb_space_rank": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "qb_space_terms": (ctypes.c_int, [ctypes.c_void_p, _c_i64_p, _c_i64_p, ctypes.c_void_p]),
    "qb_init_number": (ctypes.c_int, [ctypes.c_void_p, _c_int_p, ctypes.c_void_p, ctypes.c_void_p]),
    "qb_init_coherent": (ctypes.c_int, [ctypes.c_void_p, _c_double_p, ctypes.c_void_p, _c_double_p, ctypes.c_void_p]),
    "qb_init_field_number": (ctypes.c_int, [ctypes.c_void_p, _c_double_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "qb_workspace_bytes": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int]),
    "qb_hpsi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "qb_evolve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "qb_space_set_resident_max": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "qb_space_set_order": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "qb_space_set_tile_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "qb_evolve_plain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "qb_evolve_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, _c_double_p, ctypes.c_double,
                                       ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "qb_observables": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(QbObs), ctypes.c_void_p]),
    "qb_observables_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(QbObs),
                                              ctypes.c_void_p]),
    "qb_evolve_observe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int64,
                                         ctypes.c_int, ctypes.POINTER(QbObs), ctypes.c_void_p, ctypes.c_void_p]),
    "qb_adjoint_workspace_bytes": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]),
    "qb_adjoint": (ctypes.c_int, [ctypes.c_void_p, _c_double_p, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                  ctypes.c_int, ctypes.c_int, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                  ctypes.c_void_p, ctypes.c_void_p]),
    "qb_adjoint_couplings": (ctypes.c_int, [ctypes.c_void_p, _c_double_p, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_int, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                    _c_double_p, ctypes.c_void_p, ctypes.c_void_p]),
    "qb_breaktime": (ctypes.c_int, [_c_double_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, _c_double_p,
                                    _c_int_p]),
    "qb_squeezing": (ctypes.c_int, [_c_double_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, _c_double_p,
                                     _c_int_p, _c_double_p, _c_double_p]),
    "qb_interaction_per_occupation": (ctypes.c_int, [ctypes.POINTER(QbModel), _c_double_p, _c_double_p]),
    "qb_fit": (ctypes.c_int, [_c_double_p, _c_double_p, ctypes.c_int, ctypes.c_int, _c_double_p, _c_double_p]),
    "qb_meanfield": (ctypes.c_int, [ctypes.POINTER(QbModel), _c_double_p, ctypes.c_double, ctypes.c_int64,
                                    ctypes.c_int, _c_double_p]),
    # include/qb_diag.h
    "qb_space_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_int_p, ctypes.c_void_p]),
    "qb_measure_fp64_fma": (ctypes.c_int, [ctypes.c_int, _c_double_p, ctypes.c_void_p]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Loads libqb.so, building it in-tree first if it is missing or stale.
    Raises if the CUDA library cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libqb.so missing at {path}")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class QbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qb error {code}: {msg}")
        self.code = code


def check(code: int) -> None:
    if code != QB_OK:
        msg = lib().qb_last_error()
        raise QbError(code, msg.decode() if msg else "")
