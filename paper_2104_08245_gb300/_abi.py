"""ctypes declarations of include/nolsm.h. Argument marshalling only: no arithmetic of the method."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

# nolsm_status
OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_SPD, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_NO_PLATEAU, \
    ERR_UNSUPPORTED, ERR_NO_SOLUTION, ERR_TIMEOUT = range(11)
# nolsm_precision
FP64, FP32, BF16, BF16X3, FP8E4M3, FP16 = range(6)
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "bf16x3": BF16X3, "fp8e4m3": FP8E4M3, "fp16": FP16}
# nolsm_bound_source
BOUND_GERSHGORIN, BOUND_POWER, BOUND_MLP = range(3)
# nolsm_options.inverse
INVERSE_CHOLESKY, INVERSE_NEWTON_SCHULZ = range(2)


class NolsmSystem(ctypes.Structure):
    _fields_ = [("n_mol", c_int32), ("nbf", c_void_p),
                ("s_nnzb", c_int64), ("s_row_ptr", c_void_p), ("s_col_idx", c_void_p), ("s_vals", c_void_p),
                ("h_nnzb", c_int64), ("h_row_ptr", c_void_p), ("h_col_idx", c_void_p), ("h_vals", c_void_p)]


class NolsmOptions(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("refine_steps", c_int32), ("max_iter", c_int32),
                ("tol_ns", c_double), ("tol_accept", c_double), ("tol_n", c_double), ("tol_mu", c_double),
                ("max_bisect", c_int32), ("bound_source", c_int32), ("sub_begin", c_int64), ("sub_end", c_int64),
                ("symmetric_form", c_int32), ("inverse", c_int32), ("wait_ns", c_int64)]


class NolsmBisection(ctypes.Structure):
    _fields_ = [("lo", c_double), ("hi", c_double), ("mu", c_double), ("n_occ", c_double), ("trace_DS", c_double),
                ("steps", c_int32), ("state", c_int32)]


# nolsm_bisection.state
BISECT_ACCEPTED, BISECT_EVALUATE, BISECT_NO_PLATEAU = range(3)


class NolsmElementModel(ctypes.Structure):
    _fields_ = [("pos", c_void_p), ("cell", c_double * 3), ("onsite", c_void_p), ("s_exp", c_double),
                ("hop", c_double), ("hop_len", c_double), ("aniso", c_double), ("dirs", c_void_p)]


class NolsmPlanInfo(ctypes.Structure):
    _fields_ = [("n_mol", c_int32), ("d_nnzb", c_int64), ("d_nvals", c_int64), ("max_n", c_int32),
                ("min_n", c_int32), ("sum_n3", c_double), ("device_bytes", c_int64), ("nb_entries", c_int64),
                ("grouped", c_int32)]


class NolsmStats(ctypes.Structure):
    _fields_ = [("ms_plan", c_double), ("ms_prepare", c_double), ("ms_sign", c_double), ("ms_reduce", c_double),
                ("ms_scatter", c_double), ("solves", c_int64), ("sub_solves", c_int64), ("ns_steps", c_int64),
                ("flops_paper", c_double), ("flops_tensor", c_double), ("flops_tensor_padded", c_double),
                ("flops_fp64", c_double), ("launches", c_int64), ("reruns", c_int64), ("ms_gather", c_double),
                ("ms_factor", c_double), ("flops_fp32", c_double), ("factor_launches", c_int64),
                ("ms_energy_weighted", c_double), ("ms_prep_tensor", c_double), ("flops_prep_tensor", c_double),
                ("flops_prep_tensor_issued", c_double), ("ill_conditioned", c_int64),
                ("ill_conditioned_kept", c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# (name, restype, argtypes) of every entry point of include/nolsm.h
SIGNATURES = [
    ("nolsm_options_default", None, [ctypes.POINTER(NolsmOptions), c_int32]),
    ("nolsm_build_submatrices", c_int32, [ctypes.POINTER(NolsmSystem), c_void_p, ctypes.POINTER(c_void_p)]),
    ("nolsm_plan_query", c_int32, [c_void_p, ctypes.POINTER(NolsmPlanInfo)]),
    ("nolsm_plan_set_elements", c_int32, [c_void_p, ctypes.POINTER(NolsmElementModel)]),
    ("nolsm_build_grouped", c_int32, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_void_p)]),
    ("nolsm_plan_get_maps", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p]),
    ("nolsm_solve_batch", c_int32, [c_void_p, c_double, ctypes.POINTER(NolsmOptions), c_void_p,
                                    ctypes.POINTER(c_double), ctypes.POINTER(c_double), c_void_p, c_void_p,
                                    c_void_p, c_void_p]),
    ("nolsm_scatter_density", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("nolsm_energy_weighted", c_int32, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double)]),
    ("nolsm_combine_submatrices", c_int32, [c_int32, c_void_p, c_void_p, c_void_p, c_int32, c_void_p,
                                            ctypes.POINTER(c_int32), c_void_p, ctypes.POINTER(c_int32)]),
    ("nolsm_find_mu", c_int32, [c_void_p, c_double, c_double, c_double, ctypes.POINTER(NolsmOptions), c_void_p,
                                ctypes.POINTER(c_double), ctypes.POINTER(c_double), ctypes.POINTER(c_int32),
                                ctypes.POINTER(c_double)]),
    ("nolsm_plan_get_prepared", c_int32, [c_void_p, ctypes.POINTER(NolsmOptions), c_void_p, c_void_p, c_void_p,
                                          c_void_p, c_void_p]),
    ("nolsm_spectral_bracket", c_int32, [c_void_p, ctypes.POINTER(NolsmOptions), c_void_p,
                                         ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    ("nolsm_bisect_begin", c_int32, [c_void_p, ctypes.POINTER(NolsmOptions), c_void_p, c_int32]),
    ("nolsm_bisect_point", c_int32, [c_void_p, c_double, ctypes.POINTER(NolsmOptions), c_void_p,
                                     ctypes.POINTER(c_double), ctypes.POINTER(c_int32)]),
    ("nolsm_bisect_side", c_int32, [c_void_p, ctypes.POINTER(NolsmOptions), c_void_p, c_int32]),
    ("nolsm_bisection_start", c_int32, [ctypes.POINTER(NolsmBisection), c_double, c_double, c_double]),
    ("nolsm_bisection_update", c_int32, [ctypes.POINTER(NolsmBisection), c_double, ctypes.POINTER(NolsmOptions),
                                         ctypes.POINTER(c_int32)]),
    ("nolsm_plan_stats", c_int32, [c_void_p, ctypes.POINTER(NolsmStats)]),
    ("nolsm_plan_stats_reset", c_int32, [c_void_p]),
    ("nolsm_plan_destroy", None, [c_void_p]),
    ("nolsm_sign_noalloc", c_int32, [c_int32] + [c_void_p] * 9 + [c_double, ctypes.POINTER(NolsmOptions), c_void_p]
     + [c_void_p] * 5),
    ("nolsm_mlp_param_count", c_int32, []),
    ("nolsm_mlp_create", c_int32, [ctypes.c_uint64, c_void_p, ctypes.POINTER(c_void_p)]),
    ("nolsm_mlp_destroy", None, [c_void_p]),
    ("nolsm_mlp_get_params", c_int32, [c_void_p, c_void_p]),
    ("nolsm_mlp_set_params", c_int32, [c_void_p, c_void_p]),
    ("nolsm_mlp_forward", c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    ("nolsm_mlp_gradient", c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                     ctypes.POINTER(c_double)]),
    ("nolsm_mlp_adam_step", c_int32, [c_void_p, ctypes.c_float, c_void_p]),
    ("nolsm_mlp_train", c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_int32, ctypes.c_float,
                                  c_void_p, c_void_p]),
    ("nolsm_plan_set_mlp", c_int32, [c_void_p, c_void_p]),
    ("nolsm_features", c_int32, [c_void_p, c_double, ctypes.POINTER(NolsmOptions), c_void_p, c_void_p]),
    ("nolsm_power_bounds", c_int32, [c_void_p, ctypes.POINTER(NolsmOptions), c_void_p, c_void_p]),
    ("nolsm_training_data", c_int32, [c_void_p, c_double, ctypes.POINTER(NolsmOptions), c_void_p, c_void_p,
                                      c_void_p]),
    ("nolsm_status_str", ctypes.c_char_p, [c_int32]),
    ("nolsm_tc_shape", c_int32, [c_int32, c_int32, c_int32]),
    ("nolsm_last_error", ctypes.c_char_p, []),
]

_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """The CUDA library. There is no fallback: a missing library is an error."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"NOLSM CUDA library not built ({path}); run __graft_entry__.build() or "
                               "python -m paper_2104_08245_gb300.build")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib
