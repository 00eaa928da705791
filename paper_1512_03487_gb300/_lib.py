"""ctypes loader for ``liblqcd.so`` and the C structs of ``include/lqcd.h``.

Loading the library performs no CUDA call, so it works on a machine without a
GPU; a missing library raises ImportError (there is no fallback path).
"""
from __future__ import annotations

import ctypes as C
import os

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG_DIR, "liblqcd.so")

# status codes
LQCD_OK = 0
LQCD_ERR_ARG = -1
LQCD_ERR_CUDA = -2
LQCD_ERR_NOT_CONVERGED = -3
LQCD_ERR_NAN = -4
LQCD_ERR_TIMEOUT = -5
LQCD_ERR_UNSUPPORTED = -6
LQCD_ERR_WORKSPACE = -7
# enums
LQCD_F64, LQCD_F32, LQCD_F16, LQCD_F64_DF = 0, 1, 2, 3
LQCD_EVEN, LQCD_ODD, LQCD_FULL = 0, 1, 2
LQCD_WILSON, LQCD_DWF = 0, 1
LQCD_FORCE_TA, LQCD_FORCE_GRAD = 0, 1
LQCD_LEAPFROG, LQCD_MINNORM2 = 0, 1


class lqcd_lattice(C.Structure):
    _fields_ = [("dims", C.c_int * 4), ("n5", C.c_int), ("bc", C.c_double * 4)]


class lqcd_operator(C.Structure):
    _fields_ = [("kind", C.c_int), ("mass", C.c_double), ("M5", C.c_double), ("mf", C.c_double),
                ("prec", C.c_int), ("recon", C.c_int), ("gparity", C.c_int)]


class lqcd_solver_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int), ("sloppy_prec", C.c_int),
                ("sloppy_recon", C.c_int), ("delta", C.c_double), ("check_interval", C.c_int),
                ("use_graph", C.c_int), ("timeout_ms", C.c_double), ("delta_mid", C.c_double),
                ("update_prec", C.c_int), ("reserved", C.c_int)]


class lqcd_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("reliable_updates", C.c_int), ("true_rel_residual", C.c_double),
                ("time_ms", C.c_double), ("status", C.c_int), ("residual_replacements", C.c_int)]


class lqcd_batch_item(C.Structure):
    _fields_ = [("lat", lqcd_lattice), ("mass", C.c_double), ("gauge", C.c_void_p), ("gauge_sloppy", C.c_void_p),
                ("x", C.c_void_p), ("b", C.c_void_p)]


class lqcd_hmc_params(C.Structure):
    _fields_ = [("beta", C.c_double), ("tau", C.c_double), ("nsteps", C.c_int), ("integrator", C.c_int),
                ("fermion", C.c_int)]


class lqcd_hmc_info(C.Structure):
    _fields_ = [("H0", C.c_double), ("H1", C.c_double), ("kinetic0", C.c_double), ("kinetic1", C.c_double),
                ("gauge0", C.c_double), ("gauge1", C.c_double), ("fermion0", C.c_double), ("fermion1", C.c_double),
                ("force_evaluations", C.c_int), ("cg_iterations", C.c_int), ("status", C.c_int)]


class lqcd_mg_params(C.Structure):
    _fields_ = [("block", C.c_int), ("nvec", C.c_int), ("setup_iters", C.c_int), ("pre_smooth", C.c_int),
                ("post_smooth", C.c_int), ("coarse_iters", C.c_int), ("restart", C.c_int)]


_P = C.c_void_p
_LAT = C.POINTER(lqcd_lattice)
_OP = C.POINTER(lqcd_operator)
_PRM = C.POINTER(lqcd_solver_params)
_INFO = C.POINTER(lqcd_solve_info)
_I = C.c_int
_SZ = C.c_size_t

#: name -> (restype, argtypes), one entry per declaration of include/lqcd.h
SIGNATURES = {
    "lqcd_version": (C.c_char_p, []),
    "lqcd_last_error": (C.c_char_p, []),
    "lqcd_launch_count": (C.c_uint64, []),
    "lqcd_release_caches": (None, []),
    "lqcd_spinor_bytes": (_SZ, [_LAT, _I, _I]),
    "lqcd_gauge_bytes": (_SZ, [_LAT, _I, _I]),
    "lqcd_spinor_pack": (_I, [_P, _I, _I, _P, _LAT, _P]),
    "lqcd_spinor_unpack": (_I, [_P, _P, _I, _I, _LAT, _P]),
    "lqcd_gauge_pack": (_I, [_P, _I, _I, _P, _LAT, _P]),
    "lqcd_gauge_unpack": (_I, [_P, _P, _I, _I, _LAT, _P]),
    "lqcd_spinor_upload": (_I, [_P, _I, _I, _P, _P, _LAT, _P]),
    "lqcd_spinor_download": (_I, [_P, _P, _I, _I, _P, _LAT, _P]),
    "lqcd_gauge_upload": (_I, [_P, _I, _I, _P, _P, _LAT, _P]),
    "lqcd_dslash": (_I, [_P, _P, _P, _LAT, _OP, _I, _I, _P]),
    "lqcd_M": (_I, [_P, _P, _P, _LAT, _OP, _I, _I, _P, _P]),
    "lqcd_MdagM": (_I, [_P, _P, _P, _LAT, _OP, _I, _P, _P]),
    "lqcd_operator_workspace_bytes": (_SZ, [_LAT, _OP, _I]),
    "lqcd_eo_prepare": (_I, [_P, _P, _P, _LAT, _OP, _P, _P]),
    "lqcd_eo_reconstruct": (_I, [_P, _P, _P, _LAT, _OP, _P, _P]),
    "lqcd_cg_workspace_bytes": (_SZ, [_LAT, _OP, _PRM, _I]),
    "lqcd_cg_solve": (_I, [_P, _P, _P, _P, _LAT, _OP, _PRM, _I, _INFO, _P, _SZ, _P]),
    "lqcd_cgnr_solve": (_I, [_P, _P, _P, _P, _LAT, _OP, _PRM, _I, _INFO, _P, _SZ, _P]),
    "lqcd_eo_solve_workspace_bytes": (_SZ, [_LAT, _OP, _PRM]),
    "lqcd_eo_solve": (_I, [_P, _P, _P, _P, _LAT, _OP, _PRM, _INFO, _P, _SZ, _P]),
    "lqcd_force": (_I, [_P, _P, _P, _P, _LAT, _OP, _I, _P]),
    "lqcd_colour_matrix_bytes": (_SZ, [_LAT, _I]),
    "lqcd_colour_matrix_pack": (_I, [_P, _I, _P, _LAT, _P]),
    "lqcd_colour_matrix_unpack": (_I, [_P, _P, _I, _LAT, _P]),
    "lqcd_su3_mul": (_I, [_P, _P, _P, _LAT, _I, _P]),
    "lqcd_reduce_workspace_bytes": (_SZ, [_LAT]),
    "lqcd_plaquette": (_I, [C.POINTER(C.c_double), _P, _LAT, _P, _SZ, _P]),
    "lqcd_momentum_kinetic": (_I, [C.POINTER(C.c_double), _P, _LAT, _P, _SZ, _P]),
    "lqcd_gauge_force": (_I, [_P, _P, _LAT, C.c_double, _P]),
    "lqcd_gauge_exp_update": (_I, [_P, _P, C.c_double, _LAT, _P]),
    "lqcd_hmc_workspace_bytes": (_SZ, [_LAT, _OP, _PRM]),
    "lqcd_mg_coarse_bytes": (_SZ, [_LAT, _I, _I, _I]),
    "lqcd_mg_coarse_op_bytes": (_SZ, [_LAT, _I, _I, _I]),
    "lqcd_mg_block_orthonormalize": (_I, [_P, _I, _I, _LAT, _P]),
    "lqcd_mg_restrict": (_I, [_P, _P, _P, _I, _I, _I, _LAT, _P]),
    "lqcd_mg_prolong": (_I, [_P, _P, _P, _I, _I, _I, _LAT, _P]),
    "lqcd_mg_coarse_build": (_I, [_P, _P, _P, _I, _I, _LAT, _OP, _P]),
    "lqcd_mg_coarse_apply": (_I, [_P, _P, _P, _I, _I, _I, _I, _LAT, _P]),
    "lqcd_mg_workspace_bytes": (_SZ, [_LAT, _OP, C.POINTER(lqcd_mg_params)]),
    "lqcd_mg_setup": (_I, [_P, _P, _P, _LAT, _OP, C.POINTER(lqcd_mg_params), _P, _SZ, _P]),
    "lqcd_mg_solve": (_I, [_P, _P, _P, _P, _LAT, _OP, C.POINTER(lqcd_mg_params), _PRM, _INFO, _P, _SZ, _P]),
    "lqcd_hmc_trajectory": (_I, [_P, _P, _P, _LAT, _OP, C.POINTER(lqcd_hmc_params), _PRM,
                                 C.POINTER(lqcd_hmc_info), _P, _SZ, _P]),
    "lqcd_M_noalloc": (_I, [_P, _P, _P, _LAT, _OP, _I, _I, _P]),
    "lqcd_block_cg_workspace_bytes": (_SZ, [_LAT, _OP, _PRM]),
    "lqcd_block_cg_solve": (_I, [_P, _P, _P, _P, _LAT, _OP, _PRM, _INFO, _P, _SZ, _P]),
    "lqcd_batch_cg_workspace_bytes": (_SZ, [_I, C.c_void_p, _I, _PRM]),
    "lqcd_batch_cg_solve": (_I, [_I, C.c_void_p, _I, _PRM, C.c_void_p, _P, _SZ, _P]),
    "lqcd_tune_save": (_I, [C.c_char_p]),
    "lqcd_tune_load": (_I, [C.c_char_p]),
    "lqcd_tune_entries": (_I, []),
    "lqcd_tune_get": (_I, [C.c_char_p]),
    "lqcd_spinor_dot_re": (_I, [C.POINTER(C.c_double), _P, _P, _LAT, _P, _SZ, _P]),
    "lqcd_tune_clear": (None, []),
    "lqcd_tune_set_enabled": (None, [C.c_int]),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib
