"""ctypes binding of libspmc.so (include/spmc.h): argument marshalling only.

Every step of the method runs in the CUDA library.  There is no CPU fallback:
if the shared library is missing or cannot be loaded, importing this module
raises.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspmc.so")

SPMC_OK, SPMC_ERR_INVALID, SPMC_ERR_UNSUPPORTED, SPMC_ERR_CUDA, SPMC_ERR_OOM, SPMC_ERR_TIMEOUT, \
    SPMC_ERR_NONFINITE = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "UNSUPPORTED", 3: "CUDA", 4: "OOM", 5: "TIMEOUT", 6: "NONFINITE"}
TIME_LGL, TIME_RADAU_LEFT, TIME_CHEB = 0, 1, 2
BASIS_JACOBI, BASIS_CHEB = 0, 1
FP64, MIXED = 0, 1
F_POLY3, F_SIN = 0, 1
EX_NONE, EX_SIN, EX_COSHALF, EX_POLY, EX_COSTHIRD, EX_SINPLUS, EX_FRAC_SIN, EX_FRAC_POLY = range(8)
BC_ZERO, BC_LIFT, BC_RAW = 0, 1, 2
EST_RESIDUAL, EST_DIRECT = 0, 1
U0_NODAL, U0_PHI_COEF = 0, 1
SPMC_SWEEP_EVENTS, SPMC_SWEEP_COHORT, SPMC_SWEEP_EVENTS_ALU = 0, 1, 2
WALK_BALLS, WALK_FIXED, WALK_STABLE = 0, 1, 2
ACCEL_NONE, ACCEL_AITKEN = 0, 1


class PlanDesc(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n_space", C.c_int), ("time_family", C.c_int), ("max_intervals", C.c_int),
        ("max_degree", C.c_int), ("M", C.c_longlong), ("K", C.c_int), ("tol", C.c_double),
        ("n_ref", C.c_int), ("n_sub", C.c_int), ("shell", C.c_double), ("max_steps", C.c_int),
        ("kappa", C.c_double), ("seed", C.c_ulonglong), ("precision", C.c_int), ("batch", C.c_int),
        ("walk_mode", C.c_int), ("estimator", C.c_int), ("alpha", C.c_double), ("basis", C.c_int),
    ]


class Problem(C.Structure):
    _fields_ = [
        ("n_intervals", C.c_int), ("t_breaks", C.POINTER(C.c_double)), ("degrees", C.POINTER(C.c_int)),
        ("f_kind", C.c_int), ("f_coef", C.c_double * 4), ("f_scale", C.c_double),
        ("ex_kind", C.c_int), ("ex_beta", C.c_double), ("u0_kind", C.c_int), ("n_coef", C.c_int),
        ("u0", C.POINTER(C.c_double)), ("bc_kind", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [("node_samples", C.c_longlong), ("points", C.c_longlong), ("capped", C.c_longlong),
                ("iterations_run", C.c_int), ("last_max_eps", C.c_double),
                ("sweep_launches", C.c_longlong), ("sweep_ms", C.c_double),
                ("walk_ms", C.c_double), ("eval_ms", C.c_double), ("eval_launches", C.c_longlong),
                ("fill_ms", C.c_double), ("workspace_bytes", C.c_longlong), ("graph_launches", C.c_longlong)]


# The C-ABI entry points and their signatures, as declared in include/spmc.h.
_PLAN = C.c_void_p
_SIGNATURES = {
    "spmc_plan": (C.c_int, [C.POINTER(PlanDesc), C.POINTER(_PLAN)]),
    "spmc_set_problem": (C.c_int, [_PLAN, C.c_int, C.POINTER(Problem)]),
    "spmc_solution_layout": (C.c_int, [_PLAN, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "spmc_solve": (C.c_int, [_PLAN, C.c_void_p, C.c_void_p]),
    "spmc_begin_interval": (C.c_int, [_PLAN, C.c_void_p, C.c_int]),
    "spmc_iterate": (C.c_int, [_PLAN, C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "spmc_get_nodes": (C.c_int, [_PLAN, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "spmc_get_solution": (C.c_int, [_PLAN, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "spmc_set_nodes": (C.c_int, [_PLAN, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "spmc_iterate_static": (C.c_int, [_PLAN, C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "spmc_grad": (C.c_int, [_PLAN, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "spmc_set_timing": (C.c_int, [_PLAN, C.c_int]),
    "spmc_set_graphs": (C.c_int, [_PLAN, C.c_int]),
    "spmc_set_acceleration": (C.c_int, [_PLAN, C.c_int]),
    "spmc_round_nodes": (C.c_int, [_PLAN, C.c_int, C.POINTER(C.c_longlong)]),
    "spmc_iterate_shard": (C.c_int, [_PLAN, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "spmc_apply_eps": (C.c_int, [_PLAN, C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_double)]),
    "spmc_set_sweep": (C.c_int, [_PLAN, C.c_int, C.c_longlong]),
    "spmc_autotune": (C.c_int, [_PLAN, C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "spmc_space_nodes": (C.c_int, [_PLAN, C.POINTER(C.c_double)]),
    "spmc_get_stats": (C.c_int, [_PLAN, C.POINTER(Stats)]),
    "spmc_last_error": (C.c_char_p, [_PLAN]),
    "spmc_destroy": (None, [_PLAN]),
    "spmc_version": (C.c_char_p, []),
}


def exported_symbols():
    return list(_SIGNATURES)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class SpmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"spmc status {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, plan=None):
    if status != SPMC_OK:
        msg = lib.spmc_last_error(plan).decode() if plan else ""
        raise SpmcError(status, msg)
