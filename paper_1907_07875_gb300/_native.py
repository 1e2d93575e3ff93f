"""ctypes declarations for libgft.so (include/gft.h).  Argument marshalling
only: every computation happens in the library."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgft.so")

c_plan = C.c_void_p
c_status = C.c_int


class PlanInfo(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_stages", C.c_int32), ("n_leaves", C.c_int32),
                ("n_pairs", C.c_int32), ("max_leaf", C.c_int32), ("has_device", C.c_int32),
                ("jacobi_sweeps", C.c_int32), ("flags", C.c_uint32),
                ("fast_mults", C.c_int64), ("fast_adds", C.c_int64), ("jit", C.c_int32),
                ("tile_signals", C.c_int32), ("threads", C.c_int32), ("wide", C.c_int32),
                ("right_pairs", C.c_int32)]


class ApproxInfo(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_haar_layers", C.c_int32), ("n_layers", C.c_int32),
                ("n_units", C.c_int32), ("has_device", C.c_int32), ("tile_signals", C.c_int32),
                ("mults", C.c_int64), ("adds", C.c_int64)]


P = C.c_void_p
I32P = C.POINTER(C.c_int32)
I64P = C.POINTER(C.c_int64)
F64P = C.POINTER(C.c_double)

# name -> (restype, argtypes); the complete exported surface of gft.h
SIGNATURES = {
    "gft_status_string": (C.c_char_p, [C.c_int]),
    "gft_last_error": (C.c_char_p, []),
    "gft_version": (C.c_int32, []),
    "gft_laplacian_from_weights": (c_status, [C.c_int32, P, P, P]),
    "gft_normalized_laplacian_from_weights": (c_status, [C.c_int32, P, P, P]),
    "gft_plan_create_bipartite": (c_status, [C.c_int32, P, P, C.c_uint32, C.POINTER(c_plan)]),
    "gft_plan_create": (c_status, [C.c_int32, P, C.c_int32, P, C.c_uint32, C.POINTER(c_plan)]),
    "gft_plan_create_many": (c_status, [C.c_int32, P, P, P, P, C.c_uint32, P]),
    "gft_find_involution": (c_status, [C.c_int32, P, P, C.c_int64, P, I32P]),
    "gft_search_stages": (c_status, [C.c_int32, P, C.c_int32, C.c_int64, P, I32P]),
    "gft_plan_destroy": (c_status, [c_plan]),
    "gft_plan_get_info": (c_status, [c_plan, C.POINTER(PlanInfo)]),
    "gft_plan_get_stage_pairs": (c_status, [c_plan, C.c_int32, P, I32P]),
    "gft_plan_get_leaves": (c_status, [c_plan, P, P]),
    "gft_plan_get_leaf_laplacian": (c_status, [c_plan, C.c_int32, P]),
    "gft_plan_get_output_map": (c_status, [c_plan, P]),
    "gft_plan_eigenvalues": (c_status, [c_plan, P]),
    "gft_plan_basis": (c_status, [c_plan, P]),
    "gft_plan_forward": (c_status, [c_plan, P, P, C.c_int64, P, C.c_uint32]),
    "gft_plan_inverse": (c_status, [c_plan, P, P, C.c_int64, P, C.c_uint32]),
    "gft_plan_forward_f64": (c_status, [c_plan, P, P, C.c_int64, P]),
    "gft_plan_inverse_f64": (c_status, [c_plan, P, P, C.c_int64, P]),
    "gft_plan_forward_host": (c_status, [c_plan, P, P, C.c_int64, C.c_uint32]),
    "gft_device_error": (c_status, [c_plan, I32P]),
    "gft_plan_kernel_source": (c_status, [c_plan, C.c_int32, P, I64P]),
    "gft_batch_create": (c_status, [C.c_int32, P, P, C.c_uint32, C.POINTER(C.c_void_p)]),
    "gft_batch_forward": (c_status, [C.c_void_p, P, P, P]),
    "gft_batch_get_tile": (c_status, [C.c_void_p, C.c_int32, I32P, I32P]),
    "gft_batch_get_launches": (c_status, [C.c_void_p, I32P]),
    "gft_batch_destroy": (c_status, [C.c_void_p]),
    "gft_approx_create": (c_status, [C.c_int32, P, C.c_int32, P, C.c_int32, C.c_uint32, C.POINTER(C.c_void_p)]),
    "gft_approx_destroy": (c_status, [C.c_void_p]),
    "gft_approx_get_info": (c_status, [C.c_void_p, C.POINTER(ApproxInfo)]),
    "gft_approx_get_units": (c_status, [C.c_void_p, P, P, P, P]),
    "gft_approx_eigenvalues": (c_status, [C.c_void_p, P]),
    "gft_approx_basis": (c_status, [C.c_void_p, P]),
    "gft_approx_forward": (c_status, [C.c_void_p, P, P, C.c_int64, P]),
    "gft_givens_create": (c_status, [C.c_int32, C.c_int32, P, C.POINTER(C.c_void_p)]),
    "gft_givens_destroy": (c_status, [C.c_void_p]),
    "gft_givens_forward": (c_status, [C.c_void_p, P, P, P, C.c_int64, P]),
    "gft_givens_backward": (c_status, [C.c_void_p, P, P, P, P, P, C.c_int64, P]),
    "gft_givens_backward_noalloc": (c_status, [C.c_int32, C.c_int32, P, P, P, P, P, P, C.c_int64, P]),
}

_lib = None


def load():
    """Load libgft.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with `python -c \"import __graft_entry__ as g; "
                           "g.build()\"` (the transform has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
