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


def test_implicit_layer_host_checks_without_gpu(L):
    """The three-pass implicit layer's workspace query (batch x c/2 x m_y x 2m_x complex64)
    and the argument checks of the implicit-layer entry points, all on the host."""
    n = ctypes.c_size_t()
    assert L.helm_implicit_3pass_workspace_size(8, 136, 136, 64, ctypes.byref(n)) == 0
    assert n.value == 8 * 32 * 136 * 272 * 8
    assert L.helm_implicit_3pass_workspace_size(2, 36, 68, 64, ctypes.byref(n)) == 0
    assert n.value == 2 * 32 * 36 * 136 * 8
    assert L.helm_implicit_3pass_workspace_size(0, 36, 68, 64, ctypes.byref(n)) == -1
    fake = ctypes.c_void_p(0x1000)
    other = ctypes.c_void_p(0x2000)
    # odd or non-multiple-of-8 channel counts, aliasing, a missing workspace: EINVAL
    assert L.helm_implicit_rect_bf16(fake, 1, 8, 12, 12, fake, other, None) == -1
    assert L.helm_implicit_rect_bf16(fake, 1, 8, 12, 16, fake, fake, None) == -1
    assert L.helm_implicit_3pass_bf16(fake, 1, 8, 12, 16, fake, other, None, 1 << 20, None) == -1
    # a workspace one byte short: EWORKSPACE before any launch
    assert L.helm_implicit_3pass_bf16(fake, 1, 8, 12, 16, fake, other, fake, 8 * 8 * 24 * 8 - 1, None) == -6
    assert b"workspace" in L.helm_last_error_string()


def test_implicit_three_pass_tuning_knob(L):
    """Knob 2 (HELM_TUNE_IMPLICIT_3PASS) is accepted and looked up like the others."""
    v = ctypes.c_int()
    assert L.helm_tune_clear() == 0
    assert L.helm_tune_set(2, 8, 0, 1) == 0
    assert L.helm_tune_get(2, 8, 64, ctypes.byref(v)) == 0 and v.value == 1
    assert L.helm_tune_get(2, 16, 64, ctypes.byref(v)) == 0 and v.value == 0
    assert L.helm_tune_clear() == 0
