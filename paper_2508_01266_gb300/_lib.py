"""ctypes binding of liblrcc.so (argument marshalling only).

Every numerical step runs inside the library's CUDA kernels; this module only
converts tensors to pointers.  It raises at import time if the library has not
been built, so no code path can silently run without the native extension.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrcc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")

lib = C.CDLL(LIB_PATH)


class lrcc_dims(C.Structure):
    _fields_ = [("nk", C.c_int32), ("nocc", C.c_int32), ("nvir", C.c_int32), ("naux", C.c_int32),
                ("kmesh", C.c_int32)]


class lrcc_options(C.Structure):
    _fields_ = [("conv_tol", C.c_double), ("refine_tol", C.c_double), ("max_iter", C.c_int32),
                ("diis_depth", C.c_int32), ("diis_period", C.c_int32), ("precision", C.c_int32),
                ("autotune", C.c_int32), ("use_graphs", C.c_int32), ("spin_timeout_cycles", C.c_uint64),
                ("response_form", C.c_int32), ("log_path", C.c_char_p), ("max_batch", C.c_int32),
                ("host_history", C.c_int32)]


VP = C.c_void_p
_SIGS = {
    "lrcc_create": (C.c_int, [C.POINTER(lrcc_dims), C.POINTER(VP)]),
    "lrcc_set_integrals": (C.c_int, [VP, VP, VP, VP, C.c_int32]),
    "lrcc_set_ground_state": (C.c_int, [VP, VP, VP, VP, VP, C.c_int32]),
    "lrcc_jacobian_apply": (C.c_int, [VP, C.c_int32, C.c_int32, VP, VP, VP, VP, C.POINTER(lrcc_options), VP]),
    "lrcc_jacobian_apply_noalloc": (C.c_int, [VP, C.c_int32, VP, VP, VP, VP, VP]),
    "lrcc_polarizability": (C.c_int, [VP, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_double), C.c_int32,
                                      C.POINTER(lrcc_options), VP, C.POINTER(C.c_int32)]),
    "lrcc_polarizability_forms": (C.c_int, [VP, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_double),
                                            C.c_int32, C.POINTER(lrcc_options), VP, VP, C.POINTER(C.c_int32)]),
    "lrcc_response_function": (C.c_int, [VP, C.c_int32, VP, C.POINTER(C.c_double), C.c_int32,
                                         C.POINTER(lrcc_options), VP, C.POINTER(C.c_int32)]),
    "lrcc_last_error": (C.c_char_p, [VP]),
    "lrcc_destroy": (None, [VP]),
    "lrcc_default_options": (None, [C.POINTER(lrcc_options)]),
    "lrcc_kernel_launches": (C.c_int64, [VP]),
    "lrcc_profile": (C.c_int, [VP, C.c_int32]),
    "lrcc_profile_query": (C.c_int, [VP, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_double)]),
    "lrcc_profile_report": (C.c_int, [VP, C.c_char_p, C.c_int64]),
    "lrcc_residual": (C.c_int, [VP, VP, VP, VP, VP]),
    "lrcc_solve_ground_state": (C.c_int, [VP, C.POINTER(lrcc_options), VP, VP, VP, VP, C.c_int32,
                                          C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "lrcc_excitation_energies": (C.c_int, [VP, C.c_int32, C.POINTER(lrcc_options), VP, VP, VP,
                                           C.POINTER(C.c_int32)]),
    "lrcc_batch_polarizability": (C.c_int, [C.POINTER(VP), C.c_int32, C.POINTER(C.c_int32), C.c_int32,
                                            C.POINTER(C.c_double), C.c_int32, C.POINTER(lrcc_options),
                                            C.POINTER(VP), C.POINTER(VP)]),
    "lrcc_plan_create": (C.c_int, [C.POINTER(lrcc_dims), C.c_int64, C.POINTER(VP)]),
    "lrcc_plan_destroy": (None, [VP]),
    "lrcc_plan_info": (C.c_int, [VP, VP, VP, VP]),
    "lrcc_plan_num_ops": (C.c_int32, [VP, C.c_int32]),
    "lrcc_plan_validate": (C.c_int, [VP, C.c_char_p, C.c_int32]),
    "lrcc_plan_op": (C.c_int, [VP, C.c_int32, C.c_int32, VP]),
    "lrcc_plan_gemm": (C.c_int, [VP, C.c_int32, VP, VP, VP, VP, VP, VP, VP]),
    "lrcc_plan_perm": (C.c_int, [VP, C.c_int32, VP, VP, VP]),
    "lrcc_plan_btrans": (C.c_int, [VP, C.c_int32, VP, VP, VP]),
    "lrcc_plan_zero": (C.c_int, [VP, C.c_int32, VP, VP]),
    "lrcc_plan_choice": (C.c_int, [VP, C.c_int32, C.c_int32, VP]),
    "lrcc_small_eig": (C.c_int, [C.c_int32, VP, VP, VP]),
    "lrcc_wait_selftest": (C.c_int, [VP, C.c_int64]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

STATUS = {0: "LRCC_OK", 1: "LRCC_EINVAL", 2: "LRCC_ENOMEM", 3: "LRCC_ECUDA", 4: "LRCC_ENOCONV",
          5: "LRCC_ETIMEOUT", 6: "LRCC_EUNSUPPORTED"}
