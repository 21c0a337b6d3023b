"""ctypes declarations of the libstm C-ABI (include/stm.h). Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libstm.so")

STM_OK, STM_ERR_INVALID_ARG, STM_ERR_CUDA, STM_ERR_OOM = 0, 1, 2, 3
STM_ERR_SINGULAR_CELL, STM_ERR_NOT_CONVERGED, STM_ERR_NONFINITE, STM_ERR_STATE = 4, 5, 6, 7
STATUS_NAMES = {0: "STM_OK", 1: "STM_ERR_INVALID_ARG", 2: "STM_ERR_CUDA", 3: "STM_ERR_OOM",
                4: "STM_ERR_SINGULAR_CELL", 5: "STM_ERR_NOT_CONVERGED", 6: "STM_ERR_NONFINITE",
                7: "STM_ERR_STATE"}
PRECISION = {"f64": 0, "f32": 1, "bf16": 2}
SMOOTHER = {"additive": 0, "coloured": 1, "overwrite": 2}
KCLASS = {"vanka_local": 0, "jacobian_spmv": 1, "vanka_combine": 2, "transfer": 3, "coarse": 4, "krylov": 5, "defect_f32": 6, "round_f32": 7}


class StmParams(C.Structure):
    _fields_ = [("dim", C.c_int), ("k", C.c_int), ("n_levels", C.c_int), ("coarse_cells", C.c_int * 3),
                ("length", C.c_double * 3), ("obstacle_lo", C.c_int * 3), ("obstacle_hi", C.c_int * 3),
                ("tau", C.c_double), ("nu", C.c_double), ("gamma1", C.c_double), ("gamma2", C.c_double),
                ("inv_precision", C.c_int), ("smoother", C.c_int), ("omega", C.c_double),
                ("nu1", C.c_int), ("nu2", C.c_int), ("defect_precision", C.c_int)]


class GmresOpts(C.Structure):
    _fields_ = [("restart", C.c_int), ("max_iter", C.c_int), ("transpose", C.c_int), ("use_x0", C.c_int),
                ("rtol", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("rel_res_true", C.c_double), ("rel_res_est", C.c_double),
                ("history", C.POINTER(C.c_double)), ("n_history", C.c_int), ("ms_total", C.c_double),
                ("graphs", C.c_int)]


NEWTON_MAX_STEPS = 32  # STM_NEWTON_MAX_STEPS


class NewtonOpts(C.Structure):
    _fields_ = [("max_newton", C.c_int), ("max_halvings", C.c_int), ("abs_tol", C.c_double),
                ("reduction", C.c_double)]


class NewtonInfo(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("gmres_iters", C.c_int), ("converged", C.c_int), ("n_res", C.c_int),
                ("res", C.c_double * (NEWTON_MAX_STEPS + 1)), ("lam", C.c_double * NEWTON_MAX_STEPS),
                ("gmres_step", C.c_int * NEWTON_MAX_STEPS)]


_P, _D, _I, _L, _V = C.c_void_p, C.c_double, C.c_int, C.c_longlong, C.c_void_p
_LP = C.POINTER(C.c_longlong)
_IP = C.POINTER(C.c_int)
_DP = C.POINTER(C.c_double)

SIGNATURES = {
    "stm_build_hierarchy": ([C.POINTER(StmParams), C.POINTER(_P)], _I),
    "stm_sizes": ([_P, _I, _LP, _LP, _IP, _LP], _I),
    "stm_dof_lattice_index": ([_P, _I, _LP], _I),
    "stm_assemble_jacobian": ([_P, _P, _D, _P], _I),
    "stm_factor_cells": ([_P, _P, _IP, _LP], _I),
    "stm_spmv": ([_P, _I, _P, _P, _I, _P], _I),
    "stm_defect": ([_P, _I, _P, _P, _P, _I, _P], _I),
    "stm_vanka_sweep": ([_P, _I, _P, _P, _I, _P], _I),
    "stm_restrict": ([_P, _I, _P, _P, _P], _I),
    "stm_prolongate_add": ([_P, _I, _P, _P, _P], _I),
    "stm_coarse_solve": ([_P, _P, _P, _I, _P], _I),
    "stm_vcycle": ([_P, _P, _P, _I, _P], _I),
    "stm_gmres_solve": ([_P, _P, _P, C.POINTER(GmresOpts), C.POINTER(SolveInfo), _P], _I),
    "stm_gmres_solve_host": ([_P, _DP, _DP, C.POINTER(GmresOpts), C.POINTER(SolveInfo), _P], _I),
    "stm_assemble_rhs": ([_P, _D, _D, _I, _P, _P], _I),
    "stm_assemble_load": ([_P, _D, _D, _P, _P, _P], _I),
    "stm_adjoint_gradient": ([_P, _D, _D, _P, _P, C.POINTER(GmresOpts), C.POINTER(SolveInfo), _P, _DP, _DP, _P], _I),
    "stm_newton_solve": ([_P, _D, _D, _P, _P, C.POINTER(NewtonOpts), C.POINTER(GmresOpts), C.POINTER(NewtonInfo),
                          _P], _I),
    "stm_functional_weights": ([_P, _IP, _IP, _P, _P], _I),
    "stm_jacobian_dnu_apply": ([_P, _P, _P, _P], _I),
    "stm_dot": ([_P, _P, _P, _L, _DP, _P], _I),
    "stm_vanka_sweep_multi": ([_P, _I, _I, _P, _P, _P], _I),
    "stm_gmres_solve_multi": ([_P, _I, _P, _P, C.POINTER(GmresOpts), C.POINTER(SolveInfo), _P], _I),
    "stm_vanka_sweep_fused": ([_P, _I, _I, _P, _P, _I, _P, _P, _P], _I),
    "stm_copy_jacobian": ([_P, _I, _LP, _IP, _DP], _I),
    "stm_copy_cell_inverses": ([_P, _I, _DP], _I),
    "stm_vanka_apply_noalloc": ([_L, _I, _L, _P, _P, _P, _P, _D, _P], _I),
    "stm_profile_enable": ([_P, _I], _I),
    "stm_profile_read": ([_P, _I, _I, _DP, _LP, _DP], _I),
    "stm_kernel_launches": ([], C.c_longlong),
    "stm_measure_fp64_peak": ([_DP, _P], _I),
    "stm_selftest_bounded_wait": ([_IP, _DP, _P], _I),
    "stm_destroy": ([_P], None),
    "stm_last_error": ([], C.c_char_p),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libstm.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libstm.so not found at {path}: run __graft_entry__.build() "
                           "(python -m paper_2107_10561_gb300.build) first")
    lib = C.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


class StmError(RuntimeError):
    def __init__(self, status, where, msg):
        self.status = status
        self.status_name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.status_name}: {msg}")


def check(status, where):
    if status != STM_OK:
        msg = load().stm_last_error()
        raise StmError(status, where, msg.decode() if msg else "")
