"""The C-ABI library builds, loads and exports every symbol include/helm.h declares
(no GPU: nothing here calls a compute entry point)."""
import ctypes
import os

import pytest

import __graft_entry__
from paper_2306_17486_gb300 import _lib


@pytest.fixture(scope="module")
def L():
    __graft_entry__.build()
    return _lib.lib()


def test_header_symbols_exported(L):
    names = _lib.header_functions()
    assert "helm_fgmres_solve" in names and "helm_slmg_vcycle" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # every exported declaration has a ctypes prototype in the binding
    assert not [n for n in names if n not in _lib.PROTOS]


def test_host_side_validation_without_gpu(L):
    # argument checks run on the host before any CUDA call
    assert L.helm_problem_create(None, 64, 64, 8, 0.6, 0.0, None, None, ctypes.byref(ctypes.c_void_p())) == -1
    assert b"invalid" in L.helm_last_error_string()
    o = _lib.MgOpts()
    L.helm_mg_opts_default(ctypes.byref(o))
    assert (o.levels, o.beta, o.omega_jacobi, o.coarse_iters, o.boundary_fix, o.bc) == (3, 0.5, 0.8, 10, 1, 0)
    assert ctypes.sizeof(_lib.MgOpts) == 40
    o.levels = 4
    # 100 is not divisible by 2^4: shape error, before touching the device
    fake = ctypes.c_void_p(0x1000)
    assert L.helm_problem_create(fake, 100, 100, 8, 0.6, 0.0, ctypes.byref(o), None,
                                 ctypes.byref(ctypes.c_void_p())) == -2
    o.bc = 3                                       # no such boundary condition
    assert L.helm_problem_create(fake, 96, 96, 8, 0.6, 0.0, ctypes.byref(o), None,
                                 ctypes.byref(ctypes.c_void_p())) == -1
    assert b"bc must be" in L.helm_last_error_string()
    o.bc = 0
    f = _lib.FgmresOpts()
    L.helm_fgmres_opts_default(ctypes.byref(f))
    assert (f.restart, f.rtol, f.maxit, f.warmup_iters, f.reorth, f.cnn_every) == (10, 1e-6, 2000, 3, 1, 1)
    assert L.helm_version().startswith(b"helm-gb300")
    # network descriptor checks also precede any device allocation
    d = _lib.CnnDesc(16, 6, 512, 0, 2)                # explicit_unet must be 0 or 1
    assert L.helm_cnn_create(ctypes.byref(d), ctypes.byref(ctypes.c_void_p())) == -1
    assert b"explicit_unet" in L.helm_last_error_string()
    d = _lib.CnnDesc(8, 6, 512, 0, 0)                 # kernels exist for c0 = 16 only
    assert L.helm_cnn_create(ctypes.byref(d), ctypes.byref(ctypes.c_void_p())) == -1
    assert ctypes.sizeof(_lib.FgmresStats) == 24


def test_library_is_in_tree_and_built_for_sm103a(L):
    assert os.path.dirname(_lib.LIB_PATH).startswith(os.path.dirname(os.path.abspath(_lib.__file__)))
    from paper_2306_17486_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_tuning_table_lookup_order(L):
    v = ctypes.c_int()
    assert L.helm_tune_clear() == 0
    assert L.helm_tune_get(0, 576, 64, ctypes.byref(v)) == 0 and v.value == 0       # heuristic
    assert L.helm_tune_set(0, 0, 0, 16) == 0                                           # any layer
    assert L.helm_tune_set(0, 576, 0, 8) == 0                                          # height 576, any batch
    assert L.helm_tune_set(0, 576, 64, 4) == 0                                         # height 576, batch 64
    for (h, b), want in {(576, 64): 4, (576, 8): 8, (288, 64): 16}.items():
        assert L.helm_tune_get(0, h, b, ctypes.byref(v)) == 0 and v.value == want, (h, b, v.value)
    assert L.helm_tune_get(1, 576, 64, ctypes.byref(v)) == 0 and v.value == 0         # other knob untouched
    assert L.helm_tune_set(0, 576, 64, 0) == 0                                         # removed: next entry
    assert L.helm_tune_get(0, 576, 64, ctypes.byref(v)) == 0 and v.value == 8
    assert L.helm_tune_set(3, 576, 64, 4) == -1                                        # no such knob
    assert L.helm_tune_set(0, 0, 64, 4) == -1                                          # batch without height
    assert L.helm_tune_set(0, -1, 0, 4) == -1
    assert L.helm_tune_clear() == 0
    assert L.helm_tune_get(0, 576, 8, ctypes.byref(v)) == 0 and v.value == 0
