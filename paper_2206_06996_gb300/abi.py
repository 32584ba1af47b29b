"""ctypes declarations of the C ABI in include/scr_gb300.h."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

SCR_OK, SCR_INVALID_ARG, SCR_CUDA_ERROR, SCR_NOT_CONVERGED, SCR_DEVICE_TIMEOUT, SCR_SINGULAR = range(6)
SCR_FP64, SCR_MIXED = 0, 1
SCR_PC_SCR, SCR_PC_SIMPLE, SCR_PC_SIMPLEC = 0, 1, 2
SCR_HIER_A, SCR_HIER_SHAT, SCR_HIER_MESH = 0, 1, 2
SCR_EXPORT_OPERATOR, SCR_EXPORT_PROLONGATOR, SCR_EXPORT_AGGREGATES, SCR_EXPORT_ROOTS = 0, 1, 2, 3
SCR_EXPORT_BLOCK_B, SCR_EXPORT_BLOCK_C, SCR_EXPORT_BLOCK_D = 4, 5, 6

STATUS_NAMES = {0: "SCR_OK", 1: "SCR_INVALID_ARG", 2: "SCR_CUDA_ERROR", 3: "SCR_NOT_CONVERGED",
                4: "SCR_DEVICE_TIMEOUT", 5: "SCR_SINGULAR"}


class ScrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Opts(C.Structure):
    _fields_ = [
        ("rtol", C.c_double), ("max_it", C.c_int), ("restart", C.c_int),
        ("rtol_A", C.c_double), ("rtol_S", C.c_double), ("rtol_I", C.c_double),
        ("max_A", C.c_int), ("max_S", C.c_int), ("max_I", C.c_int), ("restart_inner", C.c_int),
        ("precision", C.c_int), ("precond", C.c_int),
        ("amg_theta", C.c_double), ("amg_max_levels", C.c_int), ("amg_coarse_size", C.c_int),
        ("amg_nu", C.c_int), ("amg_trunc", C.c_double), ("amg_pmax", C.c_int), ("autotune", C.c_int),
        ("amg_smoother", C.c_int), ("amg_degree", C.c_int), ("spmv_group", C.c_int),
        ("sell", C.c_int), ("vec", C.c_int), ("inner_vcycles", C.c_int), ("inter_vcycles", C.c_int),
        ("newton", C.c_int), ("pdl", C.c_int), ("tangent_resetup", C.c_int),
        ("mapped_scalars", C.c_int),
        ("l2_prefetch", C.c_int), ("amg_coarse_bf16", C.c_int), ("cuda_graphs", C.c_int),
        ("graph_krylov", C.c_int), ("nrhs", C.c_int),
        ("mm_rtol", C.c_double), ("mm_max_it", C.c_int), ("verbose", C.c_int),
    ]


class Mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("n_elem", C.c_int), ("n_p", C.c_int), ("xyz", C.c_void_p),
                ("ien", C.c_void_p), ("pien", C.c_void_p), ("etype", C.c_void_p), ("dir_v", C.c_void_p)]


class Physics(C.Structure):
    _fields_ = [("rho_f", C.c_double), ("mu_f", C.c_double), ("rho_s", C.c_double), ("E_s", C.c_double),
                ("nu_s", C.c_double), ("dt", C.c_double), ("rho_inf", C.c_double), ("c_m_solid", C.c_double),
                ("c_c_solid", C.c_double)]


class Bsr(C.Structure):
    _fields_ = [("nb_rows", C.c_int), ("nb_cols", C.c_int), ("br", C.c_int), ("bc", C.c_int),
                ("nnzb", C.c_int), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p)]


class BsrOut(C.Structure):
    _fields_ = [("nb_rows", C.c_int), ("nb_cols", C.c_int), ("br", C.c_int), ("bc", C.c_int),
                ("nnzb", C.c_int), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [
        ("outer_iters", C.c_int), ("a_solves", C.c_int), ("a_iters", C.c_int), ("s_iters", C.c_int),
        ("i_iters", C.c_int), ("vcycles_A", C.c_int), ("vcycles_S", C.c_int), ("vcycles_M", C.c_int),
        ("mm_iters", C.c_int), ("rel_res", C.c_double), ("mm_rel_res", C.c_double),
        ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("mm_setup_ms", C.c_double),
        ("mm_solve_ms", C.c_double), ("kernel_launches", C.c_longlong), ("spmv_bytes", C.c_longlong),
        ("levels_A", C.c_int), ("levels_S", C.c_int), ("levels_M", C.c_int), ("syncs", C.c_int),
        ("kernel_A", C.c_int), ("kernel_Shat", C.c_int), ("pc_graph_runs", C.c_int),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class KProf(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("timed", C.c_longlong), ("ms", C.c_double),
                ("bytes", C.c_double), ("flops", C.c_double)]


SCR_PROF_SPMV_A, SCR_PROF_BLOCK_OP = 0, 1

EXPORTED = [
    "scr_default_opts", "scr_create", "scr_destroy", "scr_setup", "scr_solve", "scr_iters",
    "scr_residual", "scr_get_stats", "mm_setup", "mm_solve", "mm_iters", "scr_last_error",
    "scr_apply_op", "scr_apply_pc", "scr_apply_schur", "scr_amg_apply", "scr_amg_levels",
    "scr_export", "scr_bsr_spmv", "scr_profile_begin", "scr_profile_end", "scr_bsr_spmv_noalloc",
    "scr_setup_batch", "scr_solve_batch", "scr_batch_residuals", "scr_tune_save", "scr_tune_load",
    "scr_solve_multi", "scr_set_outlets", "scr_assembly_setup", "scr_assemble_residual",
    "scr_corrector", "scr_mesh_coupling", "scr_corrector_ale", "scr_assemble_tangent", "scr_update_values",
]

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False):
    """Load the built library (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise ImportError(f"CUDA library {_build.LIB} is not built; run __graft_entry__.build()")
        _build.build()
    L = C.CDLL(_build.LIB)
    P, V = C.POINTER, C.c_void_p
    L.scr_default_opts.argtypes = [P(Opts)]
    L.scr_create.argtypes = [P(V), P(Opts), V]
    L.scr_destroy.argtypes = [V]
    L.scr_setup.argtypes = [V, P(Bsr), P(Bsr), P(Bsr), P(Bsr), C.c_int]
    L.scr_update_values.argtypes = [V, P(Bsr), P(Bsr), P(Bsr), P(Bsr), C.c_int]
    L.scr_solve.argtypes = [V, V, V, C.c_int]
    L.scr_iters.argtypes = [V, P(C.c_int), P(C.c_int)]
    L.scr_residual.argtypes = [V, P(C.c_double)]
    L.scr_get_stats.argtypes = [V, P(Stats)]
    L.mm_setup.argtypes = [V, P(Bsr), C.c_int]
    L.mm_solve.argtypes = [V, V, V, C.c_int]
    L.mm_iters.argtypes = [V, P(C.c_int), P(C.c_double)]
    L.scr_last_error.restype = C.c_char_p
    L.scr_apply_op.argtypes = [V, V, V]
    L.scr_apply_pc.argtypes = [V, V, V]
    L.scr_apply_schur.argtypes = [V, V, V]
    L.scr_amg_apply.argtypes = [V, C.c_int, V, V]
    L.scr_amg_levels.argtypes = [V, C.c_int, P(C.c_int)]
    L.scr_export.argtypes = [V, C.c_int, C.c_int, C.c_int, P(BsrOut)]
    L.scr_bsr_spmv.argtypes = [P(Bsr), V, V, V]
    L.scr_bsr_spmv_noalloc.argtypes = [P(Bsr), V, V, V]
    L.scr_setup_batch.argtypes = [V, C.c_int, P(Bsr), P(Bsr), P(Bsr), P(Bsr), C.c_int]
    L.scr_solve_batch.argtypes = [V, P(V), P(V), C.c_int]
    L.scr_batch_residuals.argtypes = [V, P(C.c_double)]
    L.scr_profile_begin.argtypes = [V, C.c_int, C.c_int]
    L.scr_profile_end.argtypes = [V, P(KProf)]
    for name in EXPORTED:
        getattr(L, name)
        if name != "scr_last_error":
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(status: int, allow=(SCR_OK,)) -> int:
    if status not in allow:
        msg = load_library().scr_last_error().decode(errors="replace")
        raise ScrError(status, msg)
    return status
