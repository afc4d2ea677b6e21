"""ctypes binding of libmfns.so (include/mfns.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  Vectors are passed as
device pointers taken from torch tensors (torch provides device memory and
streams, nothing else).  Importing this module does not need a GPU; loading
the library does need the built ``libmfns.so`` and raises if it is missing.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmfns.so")

# mirror of the #defines in include/mfns.h
OK = 0
ERR_ARG, ERR_OOM, ERR_BUDGET, ERR_UNSUPPORTED, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_CONVERGED = -1, -2, -3, -4, -5, -6, -7
STOKES, STOKES_A, STAB_NS, PMASS = 0, 1, 2, 3
FP64, FP32 = 0, 1
OP_SYSTEM, OP_PMASS = -1, -2
TERM_MASS, TERM_CONV, TERM_NEWTON, TERM_SUPG = 1, 2, 4, 8
TERM_SUPG_NEWTON, TERM_PSPG, TERM_STRONG_VISC, TERMS_ALL = 16, 32, 64, 127
GLOBAL_COARSENING, LOCAL_SMOOTHING = 0, 1   # mfns_problem_desc.hierarchy


class ProblemDesc(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("degree", C.c_int), ("nu", C.c_double), ("dt", C.c_double),
        ("terms", C.c_int), ("div_sign", C.c_double), ("smoother", C.c_int),
        ("smoother_degree", C.c_int), ("mg_order", C.c_int), ("mg_precision", C.c_int),
        ("coarse_stop_n", C.c_int), ("fgmres_restart", C.c_int), ("tol", C.c_double),
        ("maxit", C.c_int), ("cg_iterations", C.c_int), ("lambda_max", C.c_double),
        ("recompute_frozen", C.c_int),
        ("fused_smoother", C.c_int),
        ("hierarchy", C.c_int),
    ]


class Info(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("degree", C.c_int), ("kind", C.c_int), ("n_levels", C.c_int),
        ("n_dofs", C.c_int64), ("n_velocity_dofs", C.c_int64), ("n_cells", C.c_int64),
        ("n_colors", C.c_int), ("level_dofs", C.c_int64 * 32), ("level_degree", C.c_int * 32),
        ("level_cells", C.c_int64 * 32), ("lambda_max", C.c_double * 32), ("device_bytes", C.c_size_t),
        ("cycle_dofs", C.c_int64),
    ]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("seconds", C.c_double),
                ("converged", C.c_int)]


class NewtonDesc(C.Structure):
    _fields_ = [("dt", C.c_double), ("omega", C.c_double), ("rtol", C.c_double), ("atol", C.c_double),
                ("lin_tol", C.c_double), ("max_newton", C.c_int), ("extrapolate", C.c_int)]


class NewtonInfo(C.Structure):
    _fields_ = [("newton_iterations", C.c_int), ("linear_iterations", C.c_int), ("residual0", C.c_double),
                ("residual", C.c_double), ("seconds", C.c_double), ("converged", C.c_int)]


_SIGS = {
    "mfns_ctx_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(C.c_void_p)]),
    "mfns_ctx_destroy": (C.c_int, [C.c_void_p]),
    "mfns_ctx_set_batching": (C.c_int, [C.c_void_p, C.c_int]),
    "mfns_ctx_memory": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "mfns_last_error": (C.c_char_p, []),
    "mfns_mesh_uniform": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "mfns_mesh_refine_ball": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_double, C.c_int]),
    "mfns_mesh_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "mfns_mesh_destroy": (C.c_int, [C.c_void_p]),
    "mfns_problem_create": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(ProblemDesc), C.POINTER(C.c_void_p)]),
    "mfns_problem_create_hp": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(ProblemDesc), C.c_void_p, C.c_int64,
                                         C.POINTER(C.c_void_p)]),
    "mfns_mesh_cells": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "mfns_problem_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "mfns_dof_support_points": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mfns_constrained_dofs": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "mfns_set_lambda_max": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "mfns_problem_destroy": (C.c_int, [C.c_void_p]),
    "mfns_vmult": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "mfns_vmult_host": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                  C.c_int, C.c_int64, C.c_void_p]),
    "mfns_diagonal": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_void_p]),
    "mfns_kernel_timing": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "mfns_apply_constraints": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_void_p]),
    "mfns_smooth": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                              C.c_void_p]),
    "mfns_smooth_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                                      C.c_void_p]),
    "mfns_prolongate_add": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                      C.c_void_p]),
    "mfns_restrict": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                C.c_void_p]),
    "mfns_vcycle": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "mfns_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(SolveInfo), C.c_void_p]),
    "mfns_set_state": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.c_void_p]),
    "mfns_residual": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p]),
    "mfns_bdf_step": (C.c_int, [C.c_void_p, C.POINTER(NewtonDesc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_int64, C.POINTER(NewtonInfo), C.c_void_p]),
    "mfns_max_velocity": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.c_void_p]),
    "mfns_solve_begin": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "mfns_batch_step": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int)]),
    "mfns_solve_status": (C.c_int, [C.c_void_p, C.POINTER(SolveInfo)]),
    "mfns_batch_vcycle": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_void_p),
                                    C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_void_p]),
    "mfns_spacetime_create": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_void_p)]),
    "mfns_spacetime_create_pdisc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_double,
                                              C.POINTER(C.c_void_p)]),
    "mfns_spacetime_support_points": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mfns_spacetime_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.c_void_p,
                                      C.c_void_p]),
    "mfns_spacetime_vmult": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "mfns_spacetime_destroy": (C.c_int, [C.c_void_p]),
    "mfns_spacetime_temporal": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mfns_spacetime_mg_build": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int, C.c_void_p]),
    "mfns_spacetime_mg_level": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                          C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "mfns_spacetime_mg_support_points": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mfns_spacetime_mg_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_void_p,
                                          C.c_int64, C.c_void_p]),
    "mfns_spacetime_vcycle": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "mfns_spacetime_mg_smoother_bytes": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mfns_spacetime_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int,
                                       C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p]),
}

EXPORTED = tuple(_SIGS)
_lib = None


def load(path=LIB_PATH):
    """Load libmfns.so; raises (no fallback) when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmfns.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MfnsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mfns error {code}: {msg}")
        self.code = code


def check(code):
    if code != OK:
        raise MfnsError(code, load().mfns_last_error().decode())
    return code
