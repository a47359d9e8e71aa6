"""ctypes declarations of the C ABI in ``include/pod_cg.h`` (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import _build

STATUS_NAMES = {0: "ok", 1: "arg", 2: "not_spd", 3: "breakdown", 4: "maxit", 5: "nonfinite",
                6: "cuda", 7: "timeout", 8: "oom", 9: "state"}

# every function the header declares (checked by the symbol-export test)
EXPORTS = ["pod_cg_config_default", "pod_cg_create", "pod_cg_destroy", "pod_cg_last_error",
           "pod_cg_add_snapshots", "pod_cg_clear_snapshots", "pod_cg_set_output_functionals", "pod_cg_solve", "pod_cg_solve_adjoint",
           "pod_cg_get_basis", "pod_cg_get_stage3_basis", "pod_cg_time_kernels", "pod_cg_tuning", "pod_cg_proj_tuning", "pod_cg_spmv", "pod_cg_spmm", "pod_cg_gram_workspace", "pod_cg_gram_workspace_for", "pod_cg_gram", "pod_cg_gram_noalloc", "pod_cg_debug_wait_timeout",
           "pod_cg_gram_tc_workspace", "pod_cg_gram_tc", "pod_cg_diffusion_assemble",
           "pod_cg_diffusion_theta_grad", "pod_cg_batch_create", "pod_cg_batch_solve", "pod_cg_batch_info",
           "pod_cg_batch_last_error", "pod_cg_batch_destroy", "pod_cg_batch_tiles", "pod_cg_batch_set_tiles",
           "pod_cg_pod", "pod_cg_set_krylov", "pod_cg_krylov_state", "pod_cg_krylov_coords",
           "pod_cg_krylov_compress", "pod_cg_w_tuning"]


class Config(ctypes.Structure):
    _fields_ = [("w_max", ctypes.c_int), ("s_max", ctypes.c_int), ("energy", ctypes.c_double),
                ("rank_tol", ctypes.c_double), ("k_max", ctypes.c_int), ("max_refine", ctypes.c_int),
                ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double), ("use_tc_gram", ctypes.c_int),
                ("cond_diag", ctypes.c_int), ("keep_factors", ctypes.c_int), ("loop_mode", ctypes.c_int),
                ("proj_form", ctypes.c_int), ("spmv_lanes", ctypes.c_int), ("three_stage", ctypes.c_int),
                ("y_max", ctypes.c_int), ("energy_y", ctypes.c_double), ("tol_stage2", ctypes.c_double),
                ("tol_inner", ctypes.c_double), ("bsr", ctypes.c_int), ("pod_metric", ctypes.c_int),
                ("w_select", ctypes.c_int)]


class KrylovConfig(ctypes.Structure):
    _fields_ = [("y_threshold", ctypes.c_int), ("y_keep", ctypes.c_int), ("w_keep", ctypes.c_int),
                ("nu", ctypes.c_double), ("weights", ctypes.c_int), ("p_cap", ctypes.c_int), ("frozen", ctypes.c_int)]


class CSRStruct(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class BatchSeq(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nnz", ctypes.c_int64), ("p", ctypes.c_int), ("w_max", ctypes.c_int),
                ("s_max", ctypes.c_int), ("tol", ctypes.c_double), ("energy", ctypes.c_double),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("x", ctypes.c_void_p)]


class BatchSysStat(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("refinements", ctypes.c_int),
                ("w", ctypes.c_int), ("final_relres", ctypes.c_double), ("stage1_relres", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("refinements", ctypes.c_int),
                ("w", ctypes.c_int), ("s", ctypes.c_int), ("chol_failed", ctypes.c_int),
                ("system_id", ctypes.c_int), ("spmv_count", ctypes.c_int),
                ("launches", ctypes.c_int), ("y", ctypes.c_int), ("stage2_iters", ctypes.c_int),
                ("inner_iters", ctypes.c_int),
                ("stage1_relres", ctypes.c_double), ("final_relres", ctypes.c_double),
                ("cond_gram", ctypes.c_double), ("ms_pod", ctypes.c_float), ("ms_stage1", ctypes.c_float),
                ("ms_stage2", ctypes.c_float), ("ms_stage3", ctypes.c_float), ("gram_tc", ctypes.c_int),
                ("ms_loop", ctypes.c_float)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["status"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the built library. Fails loudly when it has not been built: there is no
    fallback implementation."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(p)
    vp, ci, cd, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    P = ctypes.POINTER
    L.pod_cg_config_default.argtypes = [P(Config)]
    L.pod_cg_create.argtypes = [ci, P(Config), vp, P(vp)]
    L.pod_cg_destroy.argtypes = [vp]
    L.pod_cg_last_error.argtypes = [vp]
    L.pod_cg_last_error.restype = ctypes.c_char_p
    L.pod_cg_add_snapshots.argtypes = [vp, vp, ci]
    L.pod_cg_clear_snapshots.argtypes = [vp]
    L.pod_cg_set_output_functionals.argtypes = [vp, vp, ci]
    L.pod_cg_solve.argtypes = [vp, P(CSRStruct), vp, cd, vp, P(Stats)]
    L.pod_cg_solve_adjoint.argtypes = [vp, ci, P(CSRStruct), vp, cd, vp, P(Stats)]
    L.pod_cg_get_basis.argtypes = [vp, vp, P(ci)]
    L.pod_cg_get_stage3_basis.argtypes = [vp, vp, vp, P(ci)]
    L.pod_cg_time_kernels.argtypes = [vp, P(CSRStruct), vp, ci, P(ctypes.c_float)]
    L.pod_cg_tuning.argtypes = [vp, P(ci), P(ctypes.c_float)]
    L.pod_cg_proj_tuning.argtypes = [vp, P(ci), P(ctypes.c_float)]
    L.pod_cg_spmv.argtypes = [P(CSRStruct), vp, vp, vp]
    L.pod_cg_spmm.argtypes = [P(CSRStruct), vp, ci, vp, vp]
    L.pod_cg_gram_workspace.argtypes = [ci, ci, ci]
    L.pod_cg_gram_workspace.restype = sz
    L.pod_cg_gram_workspace_for.argtypes = [ci, ci, ci, ci]
    L.pod_cg_gram_workspace_for.restype = sz
    L.pod_cg_gram.argtypes = [ci, vp, ci, vp, ci, vp, vp, sz, vp]
    L.pod_cg_gram_noalloc.argtypes = [ci, vp, ci, vp, ci, vp, vp]
    L.pod_cg_debug_wait_timeout.argtypes = [ci, ctypes.c_longlong]
    L.pod_cg_gram_tc_workspace.argtypes = [ci, ci, ci]
    L.pod_cg_gram_tc_workspace.restype = sz
    L.pod_cg_gram_tc.argtypes = [ci, ci, vp, ci, vp, ci, vp, vp, vp, sz, vp]
    L.pod_cg_diffusion_assemble.argtypes = [ci, ci, ci, vp, vp, vp, vp, vp]
    L.pod_cg_diffusion_theta_grad.argtypes = [ci, ci, ci, vp, ci, vp, vp, vp, vp]
    L.pod_cg_batch_create.argtypes = [P(BatchSeq), ci, P(Config), ci, vp, P(vp)]
    L.pod_cg_batch_solve.argtypes = [vp, P(BatchSysStat), P(ctypes.c_float)]
    L.pod_cg_batch_info.argtypes = [vp, P(ci), P(ci), P(ctypes.c_float)]
    L.pod_cg_batch_last_error.argtypes = [vp]
    L.pod_cg_batch_last_error.restype = ctypes.c_char_p
    L.pod_cg_batch_destroy.argtypes = [vp]
    L.pod_cg_batch_tiles.argtypes = [vp, P(ci), P(ci), P(ctypes.c_float)]
    L.pod_cg_batch_set_tiles.argtypes = [vp, P(ci), P(ci)]
    L.pod_cg_pod.argtypes = [ci, ci, vp, cd, cd, ci, vp, vp, P(ci), vp, sz, vp]
    L.pod_cg_set_krylov.argtypes = [vp, P(KrylovConfig)]
    L.pod_cg_krylov_state.argtypes = [vp, P(ci), P(ci), P(ci), vp, P(ci)]
    L.pod_cg_krylov_coords.argtypes = [vp, P(CSRStruct), vp, vp, vp]
    L.pod_cg_krylov_compress.argtypes = [vp, P(CSRStruct), vp, ci, ci]
    L.pod_cg_w_tuning.argtypes = [vp, P(ci), P(ci), P(ctypes.c_float)]
    for name in EXPORTS:
        if name not in ("pod_cg_last_error", "pod_cg_gram_workspace", "pod_cg_gram_workspace_for",
                        "pod_cg_gram_tc_workspace",
                        "pod_cg_batch_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _LIB = L
    return L
