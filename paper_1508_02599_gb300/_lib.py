"""ctypes binding of libfeti.so (argument marshalling only; see include/feti.h)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfeti.so")

FETI_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "PARTITION", 3: "ELEMENT_INVERTED", 4: "LOCAL_SINGULAR",
                5: "KERNEL_DETECT", 6: "BREAKDOWN", 7: "NOT_CONVERGED", 8: "NEWTON_DIVERGED", 9: "TIMEOUT",
                10: "OOM", 11: "CUDA", 12: "STATE", 13: "IO"}

LINEAR_ISO, HGO_TWO_FIBRE, LINEAR_ISO_P0 = 0, 1, 2
CLASSICAL, ALL_FLOATING = 0, 1
PREC_IDENTITY, PREC_LUMPED, PREC_DIRICHLET = 0, 1, 2
FP64, MIXED, MIXED_F32FACTOR = 0, 1, 2

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class FetiMesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("coords", _dp), ("n_tets", C.c_int32), ("tets", _ip),
                ("part", _ip), ("n_parts", C.c_int32), ("nodes_per_tet", C.c_int32)]


class FetiMaterial(C.Structure):
    _fields_ = [("kind", C.c_int32), ("E", C.c_double), ("nu", C.c_double), ("c", C.c_double),
                ("k1", C.c_double), ("k2", C.c_double), ("kappa", C.c_double), ("fibres", _dp)]


class FetiBC(C.Structure):
    _fields_ = [("n_dir", C.c_int32), ("dir_dof", _ip), ("dir_val", _dp),
                ("n_press", C.c_int32), ("press_tri", _ip), ("press_owner", _ip), ("pressure", C.c_double),
                ("n_trac", C.c_int32), ("trac_tri", _ip), ("trac_owner", _ip), ("traction", C.c_double * 3)]


class FetiOptions(C.Structure):
    _fields_ = [("method", C.c_int32), ("precond", C.c_int32), ("precision", C.c_int32), ("tol", C.c_double),
                ("maxit", C.c_int32), ("chunk", C.c_int32), ("follower", C.c_int32),
                ("n_load_steps", C.c_int32), ("newton_tol", C.c_double), ("newton_maxit", C.c_int32),
                ("inner_tol", C.c_double), ("max_outer", C.c_int32), ("no_tensor_cores", C.c_int32),
                ("per_subdomain", C.c_int32), ("symmetric", C.c_int32), ("spin_timeout_ns", C.c_uint64),
                ("coarse_form", C.c_int32), ("local_form", C.c_int32), ("workspace_mb", C.c_int32)]


class FetiCheckpointInfo(C.Structure):
    _fields_ = [("n_dofs", C.c_int64), ("step", C.c_int32), ("n_load_steps", C.c_int32), ("tau", C.c_double)]


class FetiReport(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("rel_residual", C.c_double),
                ("cond_est", C.c_double), ("t_setup_ms", C.c_double), ("t_pcg_ms", C.c_double),
                ("t_total_ms", C.c_double), ("n_lambda", C.c_int64), ("coarse_dim", C.c_int64),
                ("newton_iters", C.c_int32), ("newton_rel_res", C.c_double), ("outer_iterations", C.c_int32)]


EXPORTS = ["feti_create", "feti_create_plan", "feti_solve", "feti_solve_multi", "feti_newton", "feti_newton_steps",
           "feti_checkpoint_write", "feti_checkpoint_read", "feti_elements", "feti_get_sizes", "feti_get_coarse_info",
           "feti_get_factor_info",
           "feti_get_index_maps",
           "feti_get_fixing", "feti_dual_apply", "feti_dual_apply_multi", "feti_dual_apply_noalloc", "feti_prepare", "feti_kernel_stats", "feti_element_stats", "feti_get_schedule",
           "feti_set_spin_timeout", "feti_get_refinement", "feti_last_error",
           "feti_destroy"]

_lib = None


def load(path: str = LIB_PATH):
    """Loads the library once; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfeti.so not found at {path}: run __graft_entry__.build() "
                           "(python -m paper_1508_02599_gb300.build)")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.feti_create.argtypes = [C.POINTER(vp), C.POINTER(FetiMesh), C.POINTER(FetiMaterial), C.POINTER(FetiBC),
                                C.POINTER(FetiOptions), vp]
    lib.feti_create_plan.argtypes = [C.POINTER(vp), C.POINTER(FetiMesh), C.POINTER(FetiMaterial),
                                     C.POINTER(FetiBC), C.POINTER(FetiOptions)]
    lib.feti_solve.argtypes = [vp, vp, C.c_int32, C.POINTER(FetiReport)]
    lib.feti_newton.argtypes = [vp, vp, C.c_int32, C.POINTER(FetiReport)]
    lib.feti_newton_steps.argtypes = [vp, vp, C.c_int32, C.c_int32, vp, C.c_int32, vp, vp, C.POINTER(FetiReport)]
    lib.feti_checkpoint_write.argtypes = [C.c_char_p, vp, C.c_int64, C.c_int32, C.c_int32, C.c_double]
    lib.feti_checkpoint_read.argtypes = [C.c_char_p, vp, C.c_int64, C.POINTER(FetiCheckpointInfo)]
    lib.feti_get_sizes.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.feti_get_coarse_info.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.feti_get_factor_info.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.feti_elements.argtypes = [vp, vp, C.c_int32, vp, vp, C.c_int32]
    lib.feti_get_index_maps.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.feti_get_fixing.argtypes = [vp, vp, vp]
    lib.feti_dual_apply.argtypes = [vp, vp, vp, vp, C.c_int32, C.POINTER(C.c_double)]
    lib.feti_dual_apply_multi.argtypes = [vp, vp, vp, vp, C.c_int32, C.c_int32, C.POINTER(C.c_double)]
    lib.feti_dual_apply_noalloc.argtypes = [vp, vp, vp, vp]
    lib.feti_solve_multi.argtypes = [vp, vp, C.c_int32, vp, C.c_int32, C.POINTER(FetiReport)]
    lib.feti_prepare.argtypes = [vp]
    lib.feti_kernel_stats.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.feti_element_stats.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.feti_get_schedule.argtypes = [vp, vp]
    lib.feti_set_spin_timeout.argtypes = [vp, C.c_uint64]
    lib.feti_get_refinement.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    lib.feti_last_error.argtypes = [vp]
    lib.feti_last_error.restype = C.c_char_p
    lib.feti_destroy.argtypes = [vp]
    lib.feti_destroy.restype = None
    for name in EXPORTS[:-2]:
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib
