"""ctypes loader and signatures for libngfreg.so (the C ABI in include/ngfreg.h).

Argument marshalling only.  There is no fallback: if the shared library is
missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libngfreg.so")

RG_OK, RG_EFOLD, RG_EINVAL, RG_ECUDA, RG_ENOMEM, RG_ENONFINITE, RG_ETIMEOUT = 0, 1, -1, -2, -3, -4, -5
RG_ESCRATCH = -6
RG_NOALLOC_MAX_CTAS = 65536
RG_CURV, RG_VCC, RG_KP = 1, 2, 4
RG_PCG_MAX = 63
RG_F32, RG_F16 = 0, 1
RG_HOOK_NO_TMA, RG_HOOK_POLL_LIMIT, RG_HOOK_PASS = 1, 2, 3
RG_SCHED_PERSISTENT, RG_SCHED_HOOK_BARRIER = 8, 16
RG_REPORT_COLS = 11     # {it, J, g.p, t, J new, evaluations, pcg steps, status, min d, max d, in bounds}


class ImageGeom(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("h", C.c_double * 3)]


class GridGeom(C.Structure):
    _fields_ = [("m", C.c_int32 * 3)]


class Params(C.Structure):
    _fields_ = [("eta", C.c_double), ("alpha", C.c_double), ("gamma", C.c_double), ("delta", C.c_double),
                ("delta_adaptive", C.c_int32), ("tau", C.c_double), ("det_lo", C.c_double), ("det_hi", C.c_double)]


class Schedule(C.Structure):
    _fields_ = [("levels", C.c_int32), ("gn_iters", C.c_int32), ("pcg_iters", C.c_int32), ("ls_max", C.c_int32),
                ("armijo_c", C.c_double), ("flags", C.c_int32)]


EXPORTS = [
    "rg_workspace_size", "rg_ctx_create", "rg_ctx_destroy", "rg_set_params", "rg_get_params", "rg_set_stream",
    "rg_set_images", "rg_set_keypoints", "ngf_objective", "ngf_gradient", "gn_linearize", "gn_matvec",
    "regularizer_apply", "gn_pcg_solve", "gn_solve", "rg_pyramid_workspace_size", "register_pyramid",
    "rg_restrict_image", "rg_prolong_grid", "rg_last_error", "rg_version", "rg_profile", "rg_profile_read",
    "rg_launch_count", "ngf_distance_noalloc", "rg_set_tile", "rg_autotune", "kp_workspace_size", "kp_scratch_size",
    "kp_ngf_features", "kp_cost_volume", "kp_mst", "kp_bp_marginals", "kp_match", "kp_launch_count",
    "kp_forstner_workspace_size", "kp_forstner", "register_pyramid_batch", "rg_sync", "rg_debug_hook",
]

_lib = None


class NgfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ngfreg error {code}: {msg}")
        self.code = code


def load():
    """Load libngfreg.so (built by paper_1807_00467_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1807_00467_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, sz, dp, fp = C.c_void_p, C.c_int32, C.c_size_t, C.c_void_p, C.c_void_p
    IG, GG, PP, SP = C.POINTER(ImageGeom), C.POINTER(GridGeom), C.POINTER(Params), C.POINTER(Schedule)
    sig = {
        "rg_workspace_size": ([IG, GG, C.c_int, i32, i32, C.POINTER(sz)], C.c_int),
        "rg_ctx_create": ([C.POINTER(vp), IG, GG, C.c_int, PP, i32, i32, vp, sz, vp], C.c_int),
        "rg_ctx_destroy": ([vp], C.c_int),
        "rg_set_params": ([vp, PP], C.c_int),
        "rg_get_params": ([vp, PP], C.c_int),
        "rg_set_stream": ([vp, vp], C.c_int),
        "rg_set_tile": ([vp, i32], C.c_int),
        "rg_autotune": ([vp, vp, C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "kp_workspace_size": ([C.POINTER(i32), i32, C.POINTER(sz)], C.c_int),
        "kp_scratch_size": ([i32, C.POINTER(sz)], C.c_int),
        "kp_ngf_features": ([C.POINTER(i32), vp, C.c_double, vp, vp], C.c_int),
        "kp_cost_volume": ([C.POINTER(i32), vp, vp, i32, vp, vp, vp], C.c_int),
        "kp_mst": ([i32, vp, vp, C.c_double, vp, vp, sz, vp], C.c_int),
        "kp_bp_marginals": ([i32, vp, vp, vp, vp, C.c_double, C.c_double, vp, vp, sz, vp], C.c_int),
        "kp_match": ([C.POINTER(i32), vp, vp, i32, vp, vp, i32, vp, vp, vp, sz, vp], C.c_int),
        "kp_launch_count": ([], C.c_int64),
        "kp_forstner_workspace_size": ([C.POINTER(i32), C.POINTER(sz)], C.c_int),
        "register_pyramid_batch": ([i32, IG, vp, vp, C.c_int, GG, PP, SP, vp, fp, vp, C.POINTER(sz), vp], C.c_int),
        "kp_forstner": ([C.POINTER(i32), vp, vp, C.c_double, i32, vp, C.POINTER(i32), vp, vp, sz, vp], C.c_int),
        "rg_set_images": ([vp, vp, vp], C.c_int),
        "rg_set_keypoints": ([vp, i32, fp, fp], C.c_int),
        "ngf_objective": ([vp, fp, dp], C.c_int),
        "ngf_gradient": ([vp, fp, dp, fp], C.c_int),
        "gn_linearize": ([vp, fp, dp, fp], C.c_int),
        "gn_matvec": ([vp, fp, fp], C.c_int),
        "regularizer_apply": ([vp, i32, fp, fp, dp, fp], C.c_int),
        "gn_pcg_solve": ([vp, fp, fp, i32, dp], C.c_int),
        "gn_solve": ([vp, fp, SP, C.POINTER(C.c_double)], C.c_int),
        "rg_pyramid_workspace_size": ([IG, GG, C.c_int, i32, i32, i32, C.POINTER(sz)], C.c_int),
        "register_pyramid": ([IG, vp, vp, C.c_int, GG, PP, SP, i32, fp, fp, fp, C.POINTER(C.c_double), vp, sz, vp],
                             C.c_int),
        "rg_restrict_image": ([C.POINTER(i32), C.c_int, vp, vp, vp], C.c_int),
        "rg_prolong_grid": ([C.POINTER(i32), fp, fp, vp], C.c_int),
        "rg_profile": ([vp, i32], C.c_int),
        "rg_profile_read": ([vp, i32, C.POINTER(C.c_double), C.POINTER(C.c_int64)], C.c_int),
        "rg_launch_count": ([], C.c_int64),
        "ngf_distance_noalloc": ([IG, GG, vp, vp, vp, C.c_double, vp, vp], C.c_int),
        "rg_sync": ([vp], C.c_int),
        "rg_debug_hook": ([vp, i32, i32], C.c_int),
        "rg_last_error": ([vp], C.c_char_p),
        "rg_version": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L
