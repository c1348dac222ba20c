"""ctypes view of the C ABI declared in include/dcg.h (argument marshalling only).

Loading fails loudly when libdcg.so has not been built: there is no fallback
implementation behind this module.
"""

from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdcg.so")

DCG_OK = 0
DCG_MAX_RHS = 32  # include/dcg.h
STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARG", 2: "NOMEM", 3: "CUDA", 4: "BREAKDOWN",
    5: "SUBSPACE_SINGULAR", 6: "MAXITER", 7: "TIMEOUT", 8: "STATE", 9: "UNSUPPORTED",
    10: "STAGNATION",
}
WINDOW = {"first": 0, "last": 1}
SELECT = {"largest": 0, "smallest": 1}
EXTRACTION = {"harmonic": 0, "ritz": 1}
FG_FORM = {"explicit": 0, "sparse": 1}
XFORMAT = {"fp32": 0, "bf16": 1, "tf32": 2}


class DcgConfig(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("k", ctypes.c_int32),
        ("ell", ctypes.c_int32),
        ("window", ctypes.c_int32),
        ("select", ctypes.c_int32),
        ("refine_every", ctypes.c_int32),
        ("max_iter", ctypes.c_int32),
        ("warm_start", ctypes.c_int32),
        ("reproject", ctypes.c_int32),
        ("record_history", ctypes.c_int32),
        ("host_loop", ctypes.c_int32),
        ("extraction", ctypes.c_int32),
        ("fg_form", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 4),
        ("tol", ctypes.c_double),
    ]


class DcgSolveInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("iters", ctypes.c_int32),
        ("matvecs_loop", ctypes.c_int32),
        ("matvecs_setup", ctypes.c_int32),
        ("matvecs_check", ctypes.c_int32),
        ("k_used", ctypes.c_int32),
        ("stored", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("relres_recursive", ctypes.c_double),
        ("relres_true", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("ms_setup", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PD = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); mirrors include/dcg.h
SIGNATURES = {
    "dcg_status_string": (ctypes.c_char_p, [_I32]),
    "dcg_last_error": (ctypes.c_char_p, [_P]),
    "dcg_create": (_I32, [ctypes.POINTER(DcgConfig), _P, ctypes.POINTER(_P)]),
    "dcg_destroy": (_I32, [_P]),
    "dcg_set_operator_dense": (_I32, [_P, _P, _I64]),
    "dcg_set_operator_dense_sym": (_I32, [_P, _P, _I64]),
    "dcg_set_operator_rbf": (_I32, [_P, _P, _I32, _I32, _D, _D, _D]),
    "dcg_set_rbf_params": (_I32, [_P, _D, _D, _D]),
    "dcg_form_rbf_dense": (_I32, [_P, _I64, _I32, _D, _D, _D, _P, _I64, _P]),
    "dcg_solve": (_I32, [_P, _P, _P, ctypes.POINTER(DcgSolveInfo)]),
    "dcg_solve_multi": (_I32, [_P, _I32, _P, _P, ctypes.POINTER(DcgSolveInfo)]),
    "dcg_update_subspace": (_I32, [_P, _PI32]),
    "dcg_update_subspace_async": (_I32, [_P]),
    "dcg_get_ritz_values": (_I32, [_P, _PD, _I32, _PI32]),
    "dcg_get_pencil": (_I32, [_P, _PD, _PD, _I32, _PI32]),
    "dcg_get_pencil_form": (_I32, [_P, _PI32]),
    "dcg_set_subspace": (_I32, [_P, _P, _I32]),
    "dcg_get_subspace": (_I32, [_P, _P, _PI32]),
    "dcg_get_history": (_I32, [_P, _PD, _I32, _PI32]),
    "dcg_matvec": (_I32, [_P, _P, _P, _PD]),
    "dcg_rbf_dtheta": (_I32, [_P, _P, _P, _I32, _PD]),
    "dcg_matvec_dense_noalloc": (_I32, [_P, _I64, _I64, _P, _P, _P, _P]),
    "dcg_residual": (_I32, [_P, _P, _P, _P, _PD, _PD]),
    "dcg_apply_block": (_I32, [_P, _P, _I32, _P]),
    "dcg_sync": (_I32, [_P]),
    "dcg_debug_arm_barrier_timeout": (_I32, [_P, _I32]),
    "dcg_measure_ex2_rate": (_I32, [_P, _PD, _PD]),
    "dcg_laplace_system": (_I32, [_P, _P, _I64, _P, _P, _P, _I64, _P, _P, _P]),
    "dcg_laplace_update": (_I32, [_P, _P, _I64, _P, _P, _P, _P, _P, _P, _PD]),
}

_lib = None


def load(path: str | None = None):
    """Loads libdcg.so (once) and declares every entry point's signature."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            f"{p} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class DcgError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"dcg status {STATUS_NAMES.get(status, status)}: {message}")


def check(status: int, ctx=None, what: str = ""):
    if status != DCG_OK:
        lib = load()
        msg = lib.dcg_last_error(ctx)
        msg = msg.decode() if msg else ""
        raise DcgError(status, f"{what}: {msg}" if what else msg)
