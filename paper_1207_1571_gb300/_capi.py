"""ctypes declarations of the ``libfvgb`` C ABI (``include/fvgb.h``).

Argument marshalling only: every function here forwards to the CUDA library
with the same name.  The structures mirror the header field by field."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfvgb.so")

FV_OK, FV_E_INVALID, FV_E_CUDA, FV_E_NOMEM, FV_E_NOT_CONVERGED, FV_E_DIVERGED, \
    FV_E_TIMEOUT, FV_E_UNSUPPORTED = range(8)
STATUS_NAMES = {0: "FV_OK", 1: "FV_E_INVALID", 2: "FV_E_CUDA", 3: "FV_E_NOMEM",
                4: "FV_E_NOT_CONVERGED", 5: "FV_E_DIVERGED", 6: "FV_E_TIMEOUT",
                7: "FV_E_UNSUPPORTED"}
FV_PATCH_WALL, FV_PATCH_INLET, FV_PATCH_OUTLET, FV_PATCH_EMPTY = range(4)
FV_PREC_FP64, FV_PREC_MIXED = 0, 1
FV_PSOLVER_JACOBI, FV_PSOLVER_AMG = 0, 1
FV_MAX_CORR = 8

EXPORTS = [
    "fv_mesh_create", "fv_mesh_destroy", "fv_mesh_plan", "fv_mesh_cell_order",
    "fv_mesh_face_order", "fv_mesh_info", "fv_mesh_addressing", "fv_case_create",
    "fv_case_destroy", "fv_case_set_fields", "fv_case_get_fields", "fv_case_set_fields_host",
    "fv_case_get_fields_host", "fv_patch_set_value", "fv_patch_set_face_values", "fv_piso_step",
    "fv_simple_iter", "fv_piso_run_graph", "fv_pcg_solve", "fv_bicgstab_solve", "fv_gauss_grad",
    "fv_ldu_matvec", "fv_last_error", "fv_set_barrier_spin_limit", "fv_case_memory",
    "fv_profile_enable", "fv_profile_read", "fv_case_last_stats", "fv_pcg_solve_noalloc",
    "fv_pcg_solve_mixed", "fv_batch_create", "fv_batch_destroy", "fv_batch_piso_step",
    "fv_batch_run_graph", "fv_batch_get_fields", "fv_batch_schedule_info", "fv_batch_set_schedule",
    "fv_batch_autotune", "fv_ellj_build_host", "fv_ellj_create", "fv_ellj_destroy", "fv_ellj_info",
    "fv_ellj_from_ldu", "fv_ellj_spmv", "fv_pcg_solve_amg", "fv_amg_info",
    "fv_case_set_pressure_solver", "fv_amg_coarsen_host", "fv_pcg_solve_amg_mixed",
]
PROF_STAGES = ["momentum", "bicgstab", "hbya", "pressure", "pcg", "correct", "other"]


class fv_patch(C.Structure):
    _fields_ = [("type", C.c_int32), ("start", C.c_int32), ("size", C.c_int32),
                ("pad_", C.c_int32), ("u", C.c_double * 3), ("p", C.c_double)]


class fv_mesh_desc(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("n_internal_faces", C.c_int32),
                ("n_boundary_faces", C.c_int32), ("n_patches", C.c_int32),
                ("owner", C.c_void_p), ("neighbour", C.c_void_p), ("Sf", C.c_void_p),
                ("Cf", C.c_void_p), ("C", C.c_void_p), ("V", C.c_void_p),
                ("patches", C.POINTER(fv_patch)), ("renumber", C.c_int32), ("pad_", C.c_int32)]


class fv_solve_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("res0", C.c_double),
                ("res", C.c_double), ("outer", C.c_int32), ("pad_", C.c_int32)]


class fv_step_stats(C.Structure):
    _fields_ = [("u", fv_solve_stats * 3), ("p", fv_solve_stats * FV_MAX_CORR),
                ("n_p", C.c_int32), ("status", C.c_int32), ("init_res_max", C.c_double)]


class fv_piso_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("n_corr", C.c_int32), ("p_maxit", C.c_int32),
                ("p_tol", C.c_double), ("u_tol", C.c_double), ("u_maxit", C.c_int32),
                ("p_ref_cell", C.c_int32), ("p_ref_value", C.c_double),
                ("n_nonorth", C.c_int32), ("pad_", C.c_int32)]


class fv_simple_params(C.Structure):
    _fields_ = [("alpha_u", C.c_double), ("alpha_p", C.c_double), ("p_tol", C.c_double),
                ("p_reltol", C.c_double), ("u_tol", C.c_double), ("u_reltol", C.c_double),
                ("p_maxit", C.c_int32), ("u_maxit", C.c_int32), ("p_ref_cell", C.c_int32),
                ("n_nonorth", C.c_int32), ("p_ref_value", C.c_double)]


class fv_pcg_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("reltol", C.c_double), ("maxit", C.c_int32),
                ("pad_", C.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built (there is no
    fallback of any kind)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfvgb.so not found at {path}: build it with "
                           "paper_1207_1571_gb300.build.build()")
    L = C.CDLL(path)
    vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
    P = C.POINTER
    sig = {
        "fv_mesh_create": [P(fv_mesh_desc), vp, P(vp)],
        "fv_mesh_destroy": [vp],
        "fv_mesh_plan": [P(fv_mesh_desc), vp, vp, vp],
        "fv_mesh_cell_order": [vp, vp],
        "fv_mesh_face_order": [vp, vp, vp],
        "fv_mesh_info": [vp, vp],
        "fv_mesh_addressing": [vp, vp, vp],
        "fv_case_create": [vp, dbl, i32, P(vp)],
        "fv_case_destroy": [vp],
        "fv_case_set_fields": [vp, vp, vp, vp, i32],
        "fv_case_get_fields": [vp, vp, vp, vp, i32],
        "fv_case_set_fields_host": [vp, vp, vp, vp, i32],
        "fv_case_get_fields_host": [vp, vp, vp, vp, i32],
        "fv_patch_set_value": [vp, i32, vp, dbl],
        "fv_patch_set_face_values": [vp, i32, vp, vp],
        "fv_piso_step": [vp, P(fv_piso_params), P(fv_step_stats)],
        "fv_simple_iter": [vp, P(fv_simple_params), P(fv_step_stats)],
        "fv_piso_run_graph": [vp, P(fv_piso_params), i32, P(fv_step_stats)],
        "fv_pcg_solve": [vp, vp, vp, vp, vp, P(fv_pcg_params), P(fv_solve_stats)],
        "fv_pcg_solve_noalloc": [vp, vp, vp, vp, vp, P(fv_pcg_params), P(fv_solve_stats)],
        "fv_pcg_solve_mixed": [vp, vp, vp, vp, vp, P(fv_pcg_params), P(fv_solve_stats)],
        "fv_batch_create": [vp, i32, vp, vp, i32, vp, P(vp)],
        "fv_batch_destroy": [vp],
        "fv_batch_piso_step": [vp, P(fv_piso_params), vp],
        "fv_batch_run_graph": [vp, P(fv_piso_params), i32, vp],
        "fv_batch_get_fields": [vp, i32, vp, vp, vp],
        "fv_batch_schedule_info": [i32, vp],
        "fv_batch_set_schedule": [vp, i32],
        "fv_batch_autotune": [vp, P(fv_piso_params), vp, vp],
        "fv_bicgstab_solve": [vp, vp, vp, vp, vp, vp, P(fv_pcg_params), P(fv_solve_stats)],
        "fv_gauss_grad": [vp, vp, vp, vp],
        "fv_ldu_matvec": [vp, vp, vp, vp, vp, vp],
        "fv_ellj_build_host": [i32, vp, vp, i32, vp, vp, vp, vp, vp, vp],
        "fv_ellj_create": [vp, i32, P(vp)],
        "fv_ellj_destroy": [vp],
        "fv_ellj_info": [vp, vp, vp],
        "fv_ellj_from_ldu": [vp, vp, vp, vp, vp, vp],
        "fv_ellj_spmv": [vp, vp, vp, vp, vp, i32],
        "fv_pcg_solve_amg": [vp, vp, vp, vp, vp, P(fv_pcg_params), P(fv_solve_stats)],
        "fv_amg_info": [vp, vp, vp],
        "fv_pcg_solve_amg_mixed": [vp, vp, vp, vp, vp, P(fv_pcg_params), P(fv_solve_stats)],
        "fv_case_set_pressure_solver": [vp, i32],
        "fv_amg_coarsen_host": [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp],
        "fv_set_barrier_spin_limit": [C.c_int64],
        "fv_case_memory": [vp, P(C.c_int64)],
        "fv_profile_enable": [i32],
        "fv_profile_read": [vp, vp, i32],
        "fv_case_last_stats": [vp, P(fv_step_stats)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.fv_last_error.argtypes = []
    L.fv_last_error.restype = C.c_char_p
    _lib = L
    return L


class FvError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().fv_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str, allow=()):
    if status != FV_OK and status not in allow:
        raise FvError(status, where)
    return status
