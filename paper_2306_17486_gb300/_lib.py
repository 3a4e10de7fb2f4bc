"""ctypes declarations of the C ABI in include/helm.h (argument marshalling only).

The library is the in-tree build `_build/libhelm.so`.  There is no fallback: if it
is missing, `lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhelm.so")
HEADER = os.path.join(HERE, "..", "include", "helm.h")

vp = C.c_void_p
i32 = C.c_int
f64 = C.c_double
sz = C.c_size_t


class MgOpts(C.Structure):
    _fields_ = [("levels", i32), ("beta", f64), ("omega_jacobi", f64), ("coarse_iters", i32),
                ("sl_includes_gamma", i32), ("boundary_fix", i32), ("bc", i32)]


class FgmresOpts(C.Structure):
    _fields_ = [("restart", i32), ("rtol", f64), ("maxit", i32), ("warmup_iters", i32), ("reorth", i32),
                ("cnn_every", i32), ("fallback", i32)]


class FgmresStats(C.Structure):
    _fields_ = [("iters", i32), ("status", i32), ("rel_res_est", f64), ("rel_res_true", f64)]


class CnnDesc(C.Structure):
    _fields_ = [("c0", i32), ("expansion", i32), ("skip_threshold", i32), ("literal_green", i32),
                ("explicit_unet", i32)]


# name -> (restype, argtypes)
PROTOS = {
    "helm_mg_opts_default": (None, [C.POINTER(MgOpts)]),
    "helm_problem_create": (i32, [vp, i32, i32, i32, f64, f64, C.POINTER(MgOpts), vp, C.POINTER(vp)]),
    "helm_problem_destroy": (i32, [vp]),
    "helm_problem_level_shape": (i32, [vp, i32, C.POINTER(i32), C.POINTER(i32)]),
    "helm_problem_get_field": (i32, [vp, i32, i32, vp, vp]),
    "helm_workspace_size": (i32, [vp, vp, i32, i32, C.POINTER(sz)]),
    "helm_helmholtz_apply": (i32, [vp, vp, vp, i32, vp]),
    "helm_helmholtz_residual_fp64": (i32, [vp, vp, vp, vp, vp, i32, vp, sz, vp]),
    "helm_slmg_vcycle": (i32, [vp, vp, vp, i32, vp, sz, vp]),
    "helm_slmg_vcycle_static": (i32, [vp, vp, vp, i32, vp]),
    "helm_fgmres_opts_default": (None, [C.POINTER(FgmresOpts)]),
    "helm_fgmres_solve": (i32, [vp, vp, vp, vp, i32, C.POINTER(FgmresOpts), vp, vp, vp, sz, vp]),
    "helm_problem_update": (i32, [vp, vp, f64, vp]),
    "helm_tune_set": (i32, [i32, i32, i32, i32]),
    "helm_tune_get": (i32, [i32, i32, i32, C.POINTER(i32)]),
    "helm_tune_clear": (i32, []),
    "helm_solver_plan_create": (i32, [vp, vp, vp, vp, i32, C.POINTER(FgmresOpts), vp, sz, vp, C.POINTER(vp)]),
    "helm_solver_plan_solve": (i32, [vp, vp, vp, vp]),
    "helm_solver_plan_destroy": (i32, [vp]),
    "helm_datagen_pairs": (i32, [vp, vp, vp, vp, vp, i32, i32, i32, vp, sz, vp]),
    "helm_training_field": (i32, [vp, i32, i32, C.c_float, C.c_float, vp, vp]),
    "helm_datagen_workspace_size": (i32, [vp, i32, i32, C.POINTER(sz)]),
    "helm_device_errors": (i32, [C.POINTER(C.c_uint)]),
    "helm_last_error_string": (C.c_char_p, []),
    "helm_version": (C.c_char_p, []),
    "helm_launch_count": (C.c_ulonglong, []),
    "helm_profile_begin": (i32, []),
    "helm_profile_end": (i32, [C.POINTER(i32)]),
    "helm_profile_read": (i32, [i32, C.POINTER(C.c_char_p), C.POINTER(C.c_long), C.POINTER(f64)]),
    "helm_conv_bf16": (i32, [vp, i32, i32, i32, i32, vp, i32, i32, i32, vp, vp, i32, vp, vp, i32, vp, vp, vp, sz,
                              vp]),
    "helm_ib_bf16": (i32, [vp, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
    "helm_implicit_bf16": (i32, [vp, i32, i32, i32, vp, vp, vp]),
    "helm_implicit_rect_bf16": (i32, [vp, i32, i32, i32, i32, vp, vp, vp]),
    "helm_implicit_3pass_bf16": (i32, [vp, i32, i32, i32, i32, vp, vp, vp, sz, vp]),
    "helm_implicit_3pass_workspace_size": (i32, [i32, i32, i32, i32, C.POINTER(sz)]),
    "helm_cnn_create": (i32, [C.POINTER(CnnDesc), C.POINTER(vp)]),
    "helm_cnn_destroy": (i32, [vp]),
    "helm_cnn_num_params": (i32, [vp, C.POINTER(sz)]),
    "helm_cnn_param_info": (i32, [vp, i32, C.POINTER(C.c_char_p), C.POINTER(i32), C.POINTER(i32), C.POINTER(sz)]),
    "helm_cnn_num_bn": (i32, [vp, C.POINTER(i32)]),
    "helm_cnn_bn_info": (i32, [vp, i32, C.POINTER(C.c_char_p), C.POINTER(i32), C.POINTER(sz)]),
    "helm_cnn_set_params": (i32, [vp, vp, vp]),
    "helm_cnn_set_running": (i32, [vp, vp, vp]),
    "helm_cnn_get_running": (i32, [vp, vp, vp]),
    "helm_cnn_set_problem": (i32, [vp, vp, vp, sz, vp]),
    "helm_cnn_get_ghat": (i32, [vp, i32, vp, vp]),
    "helm_cnn_get_ghat_rect": (i32, [vp, i32, i32, vp, vp]),
    "helm_cnn_apply": (i32, [vp, vp, vp, vp, i32, i32, vp, sz, vp]),
    "helm_cnn_precond_apply": (i32, [vp, vp, vp, vp, i32, vp, sz, vp]),
    "helm_cnn_precond_backward": (i32, [vp, vp, vp, vp, vp, vp, i32, vp, sz, vp]),
    "helm_cnn_save": (i32, [vp, C.c_char_p, vp]),
    "helm_cnn_load": (i32, [vp, C.c_char_p, vp, vp]),
    "helm_cnn_train_workspace_size": (i32, [vp, vp, i32, i32, C.POINTER(sz)]),
    "helm_cnn_train_forward": (i32, [C.POINTER(vp), i32, vp, vp, vp, i32, vp, sz, vp]),
    "helm_mse_loss": (i32, [vp, vp, C.c_long, i32, vp, vp, vp, vp]),
    "helm_adam_step": (i32, [vp, vp, vp, vp, C.c_long, f64, f64, f64, f64, i32, vp]),
}

_LIB = None


def header_functions() -> list[str]:
    """Every function name declared in include/helm.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(helm_[a-z0-9_]+)\s*\(", txt)))


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"native library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOS.items():
            if hasattr(L, name):
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
        _LIB = L
    return _LIB


class HelmError(RuntimeError):
    pass


def check(rc: int, what: str = ""):
    if rc != 0:
        msg = lib().helm_last_error_string().decode()
        raise HelmError(f"{what} failed with code {rc}: {msg}")
