"""ctypes declarations of libmc.so (include/mc.h). Argument marshalling only.

Loading fails loudly when the library has not been built: there is no CPU
fallback anywhere in this package.
"""

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmc.so")

MC_MAX_CONTINUA = 4
MC_OK, MC_E_ARG, MC_E_ALLOC, MC_E_CUDA, MC_E_NOCONV, MC_E_TIMEOUT, MC_E_STATE, MC_E_BREAKDOWN = range(8)
MC_PREC_FP64, MC_PREC_FP32_IR, MC_PREC_BF16T_IR = 0, 1, 2
MC_PRECOND_JACOBI, MC_PRECOND_TWO_LEVEL = 0, 1
MC_TWO_LEVEL_MAX_TILES = 2048
MC_TWO_LEVEL_MAX_COUPLED = 4096
MC_INNER_SINGLE_REDUCTION, MC_INNER_TWO_REDUCTIONS = 0, 1
MC_NLMC_CONSERVATIVE = 1
MC_FP64_TWO_PASS, MC_FP64_SINGLE_PASS = 0, 1
MC_SCHEME_COUPLED, MC_SCHEME_D, MC_SCHEME_L, MC_SCHEME_U = -1, 0, 1, 2

dp = C.POINTER(C.c_double)
dpp = C.POINTER(dp)


class mc_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32)]


class mc_opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("precond", C.c_int32), ("max_iter", C.c_int32),
        ("ir_max", C.c_int32), ("rtol", C.c_double), ("inner_rtol", C.c_double),
        ("spin_limit", C.c_int64), ("blocks", C.c_int32), ("threads", C.c_int32),
        ("inner_form", C.c_int32), ("fp64_form", C.c_int32),
    ]


class mc_stats(C.Structure):
    _fields_ = [
        ("steps_done", C.c_int32), ("status", C.c_int32),
        ("iters", C.c_int64 * MC_MAX_CONTINUA), ("max_iters", C.c_int32 * MC_MAX_CONTINUA),
        ("ir_sweeps", C.c_int32), ("reserved", C.c_int32),
        ("rel_residual", C.c_double * MC_MAX_CONTINUA), ("mass_defect", C.c_double),
    ]


# name -> (restype, argtypes); every symbol include/mc.h declares.
SIGNATURES = {
    "mc_default_opts": (C.c_int, [C.POINTER(mc_opts)]),
    "mc_setup": (C.c_int, [C.POINTER(mc_grid), C.c_int32, dpp, dp, dp, dpp, C.c_double,
                           C.POINTER(mc_opts), C.c_void_p, C.POINTER(C.c_void_p)]),
    "mc_set_opts": (C.c_int, [C.c_void_p, C.POINTER(mc_opts)]),
    "mc_set_source": (C.c_int, [C.c_void_p, C.c_int32, dp]),
    "mc_set_well": (C.c_int, [C.c_void_p, C.c_int32, dp, dp]),
    "mc_set_state": (C.c_int, [C.c_void_p, dpp]),
    "mc_get_state": (C.c_int, [C.c_void_p, dpp]),
    "mc_state_device": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "mc_step_decoupled": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(mc_stats)]),
    "mc_step_coupled": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(mc_stats)]),
    "mc_get_coefficients": (C.c_int, [C.c_void_p, C.c_int32, dp, dp, dp]),
    "mc_apply": (C.c_int, [C.c_void_p, C.c_int32, dpp, dpp]),
    "mc_rhs_decoupled": (C.c_int, [C.c_void_p, dpp]),
    "mc_device_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "mc_step_single_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_double,
                                         C.c_double, C.c_void_p, C.c_void_p, C.c_int32,
                                         C.c_double, C.c_int32, C.c_void_p,
                                         C.POINTER(mc_stats)]),
    "mc_nlmc_build": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                C.c_int32, C.POINTER(C.c_void_p)]),
    "mc_nlmc_build_ex": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                   C.c_int32, C.POINTER(C.c_void_p), C.c_int32,
                                   C.POINTER(C.c_void_p)]),
    "mc_nlmc_active": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint8)]),
    "mc_nlmc_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(mc_stats)]),
    "mc_nlmc_set_state": (C.c_int, [C.c_void_p, dp]),
    "mc_nlmc_get_state": (C.c_int, [C.c_void_p, dp]),
    "mc_nlmc_get_operator": (C.c_int, [C.c_void_p, dp, dp, dp]),
    "mc_nlmc_get_basis": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, dp]),
    "mc_nlmc_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "mc_nlmc_destroy": (None, [C.c_void_p]),
    "mc_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(mc_opts),
                                  C.POINTER(C.c_void_p)]),
    "mc_batch_set_team": (C.c_int, [C.c_void_p, C.c_int32]),
    "mc_batch_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(mc_stats)]),
    "mc_batch_instance_stats": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(mc_stats)]),
    "mc_batch_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_int32,
                                    C.c_char_p, C.POINTER(C.c_int32), dp]),
    "mc_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "mc_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "mc_batch_destroy": (None, [C.c_void_p]),
    "mc_fp64_fma_rate": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mc_frac_create": (C.c_int, [C.c_void_p, C.c_int32, dp, C.c_double, C.c_double, dp,
                                 C.POINTER(C.c_void_p)]),
    "mc_frac_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "mc_frac_pieces": (C.c_int, [C.c_void_p, dp, dp, C.POINTER(C.c_int32)]),
    "mc_frac_set_source": (C.c_int, [C.c_void_p, dp]),
    "mc_frac_set_well": (C.c_int, [C.c_void_p, dp, dp]),
    "mc_frac_set_state": (C.c_int, [C.c_void_p, dpp, dp]),
    "mc_frac_get_state": (C.c_int, [C.c_void_p, dpp, dp]),
    "mc_frac_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(mc_stats)]),
    "mc_frac_destroy": (None, [C.c_void_p]),
    "mc_destroy": (None, [C.c_void_p]),
    "mc_last_error": (C.c_char_p, [C.c_void_p]),
    "mc_status_string": (C.c_char_p, [C.c_int]),
}

_lib = None


def load():
    """Load libmc.so once; raises if it is missing or lacks a symbol."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libmc.so is not built (%s); run paper_2209_01158_gb300.build.build()"
                           % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
