"""GB300 (sm_103a) library for learned multigrid-augmented Helmholtz preconditioning
(arXiv 2306.17486): Python binding of the C ABI in include/helm.h.

This module only marshals arguments: every step of the solver runs in the CUDA
kernels of libhelm.so.  Torch supplies device memory and streams.  There is no CPU
fallback; without the built library every call raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import FgmresOpts, FgmresStats, HelmError, MgOpts, check, lib

STATUS = {0: "active", 1: "converged", 2: "maxit", 3: "nonfinite"}

STATS_DTYPE = np.dtype([("iters", "<i4"), ("status", "<i4"), ("rel_res_est", "<f8"), ("rel_res_true", "<f8")])


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _need(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise HelmError(f"{name} must be a contiguous CUDA tensor of dtype {dtype}")


def _grid(p, t, dtype, name) -> int:
    """Check that t is a contiguous CUDA tensor of `dtype` on the problem's device with
    shape [ny, nx] or [B, ny, nx] of problem p; returns the batch B.  The library
    builds its tensor maps and writes its outputs from p's grid and B, so a tensor of
    any other shape would be read or written out of bounds."""
    _need(t, dtype, name)
    if t.device != p.device:
        raise HelmError(f"{name} is on {t.device}, the problem on {p.device}")
    if t.dim() not in (2, 3) or tuple(t.shape[-2:]) != (p.ny, p.nx) or (t.dim() == 3 and t.shape[0] < 1):
        raise HelmError(f"{name} has shape {tuple(t.shape)}; expected [B, {p.ny}, {p.nx}] or [{p.ny}, {p.nx}]")
    return t.shape[0] if t.dim() == 3 else 1


def _out(p, ref, out, dtype, name):
    """The output buffer: a new tensor shaped like `ref`, or the caller's `out`, which must
    have ref's shape, `dtype` and device and must not alias ref."""
    if out is None:
        return torch.empty(ref.shape, dtype=dtype, device=ref.device)
    _grid(p, out, dtype, name)
    if tuple(out.shape) != tuple(ref.shape):
        raise HelmError(f"{name} has shape {tuple(out.shape)}, expected {tuple(ref.shape)}")
    if out.data_ptr() == ref.data_ptr():
        raise HelmError(f"{name} must not alias the input")
    return out


def _batch_vec(t, B, dtype, name, device):
    _need(t, dtype, name)
    if t.device != device or t.numel() != B:
        raise HelmError(f"{name} must hold {B} entries on {device}")


BOUNDARY_CONDITIONS = {"dirichlet": 0, "neumann": 1, "sommerfeld": 2}   # HELM_BC_*


def mg_opts(levels=3, beta=0.5, omega_jacobi=0.8, coarse_iters=10, sl_includes_gamma=False, boundary_fix=True,
            bc="dirichlet"):
    o = MgOpts()
    lib().helm_mg_opts_default(C.byref(o))
    o.levels, o.beta, o.omega_jacobi = levels, beta, omega_jacobi
    o.coarse_iters, o.sl_includes_gamma, o.boundary_fix = coarse_iters, int(sl_includes_gamma), int(boundary_fix)
    o.bc = BOUNDARY_CONDITIONS[bc]
    return o


def fgmres_opts(restart=10, rtol=1e-6, maxit=2000, warmup_iters=3, reorth=1, cnn_every=1, fallback=True):
    o = FgmresOpts()
    lib().helm_fgmres_opts_default(C.byref(o))
    o.restart, o.rtol, o.maxit, o.warmup_iters, o.reorth = restart, rtol, maxit, warmup_iters, reorth
    o.cnn_every, o.fallback = cnn_every, int(fallback)
    return o


class Problem:
    """One slowness model kappa (CUDA float32 [ny, nx], absorbing layer included).
    Keyword options are those of `mg_opts`, among them bc = 'dirichlet' (the paper's
    zero padding), 'neumann' or 'sommerfeld'."""

    def __init__(self, kappa: torch.Tensor, abl: int, omega_h: float, gamma0: float = 0.0, levels: int = 3,
                 **mg):
        _need(kappa, torch.float32, "kappa")
        self.ny, self.nx = kappa.shape
        self.abl, self.omega_h, self.gamma0, self.levels = abl, omega_h, gamma0, levels
        self.device = kappa.device
        self._opts = mg_opts(levels=levels, **mg)
        h = C.c_void_p()
        check(lib().helm_problem_create(_ptr(kappa), self.nx, self.ny, abl, omega_h, gamma0, C.byref(self._opts),
                                        _stream(), C.byref(h)), "helm_problem_create")
        self.handle = h
        self._ws = None

    def close(self):
        if getattr(self, "handle", None):
            lib().helm_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_shape(self, level):
        nx, ny = C.c_int(), C.c_int()
        check(lib().helm_problem_level_shape(self.handle, level, C.byref(nx), C.byref(ny)), "level_shape")
        return ny.value, nx.value

    def field(self, which: str, level: int = 0) -> torch.Tensor:
        code = {"mass_A": 0, "mass_SL": 1, "dinv_SL": 2, "gamma": 3, "kappa": 4}[which]
        ny, nx = self.level_shape(level)
        dt = torch.float32 if code >= 3 else torch.complex64
        out = torch.empty((ny, nx), dtype=dt, device=self.device)
        check(lib().helm_problem_get_field(self.handle, code, level, _ptr(out), _stream()), "get_field")
        return out

    def workspace(self, batch: int, restart: int = 10, cnn=None) -> torch.Tensor:
        n = C.c_size_t()
        check(lib().helm_workspace_size(self.handle, cnn.handle if cnn is not None else None, batch, restart,
                                        C.byref(n)), "workspace_size")
        if self._ws is None or self._ws.numel() < n.value:
            self._ws = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        return self._ws


def helmholtz_apply(p: Problem, x: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
    """y = h^2 A x for complex64 x [B, ny, nx]."""
    B = _grid(p, x, torch.complex64, "x")
    y = _out(p, x, y, torch.complex64, "y")
    check(lib().helm_helmholtz_apply(p.handle, _ptr(x), _ptr(y), B, _stream()), "helm_helmholtz_apply")
    return y


def helmholtz_residual_fp64(p: Problem, b: torch.Tensor, x: torch.Tensor):
    """(r, ||r||^2) with r = b - h^2 A x evaluated in FP64 (x complex128)."""
    B = _grid(p, b, torch.complex64, "b")
    _grid(p, x, torch.complex128, "x")
    if tuple(x.shape) != tuple(b.shape):
        raise HelmError(f"x has shape {tuple(x.shape)}, b {tuple(b.shape)}")
    r = torch.empty_like(b)
    nr = torch.empty(B, dtype=torch.float64, device=b.device)
    ws = p.workspace(B)
    check(lib().helm_helmholtz_residual_fp64(p.handle, _ptr(b), _ptr(x), _ptr(r), _ptr(nr), B, _ptr(ws),
                                             ws.numel(), _stream()), "helm_helmholtz_residual_fp64")
    return r, nr


def slmg_vcycle(p: Problem, r: torch.Tensor, z: torch.Tensor | None = None) -> torch.Tensor:
    """z = V(r), one shifted-Laplacian V(1,1) cycle."""
    B = _grid(p, r, torch.complex64, "r")
    z = _out(p, r, z, torch.complex64, "z")
    ws = p.workspace(B)
    check(lib().helm_slmg_vcycle(p.handle, _ptr(r), _ptr(z), B, _ptr(ws), ws.numel(), _stream()),
          "helm_slmg_vcycle")
    return z


def slmg_vcycle_static(p: Problem, r: torch.Tensor, z: torch.Tensor | None = None) -> torch.Tensor:
    """z = V(r) like slmg_vcycle, using the library's fixed device scratch instead of a
    workspace (for callers that cannot allocate); raises if the batch needs more scratch
    than the library holds."""
    B = _grid(p, r, torch.complex64, "r")
    z = _out(p, r, z, torch.complex64, "z")
    check(lib().helm_slmg_vcycle_static(p.handle, _ptr(r), _ptr(z), B, _stream()), "helm_slmg_vcycle_static")
    return z


def fgmres_solve(p: Problem, b: torch.Tensor, x: torch.Tensor | None = None, cnn=None, restart=10, rtol=1e-6,
                 maxit=2000, warmup_iters=3, reorth=1, maxit_per_rhs: torch.Tensor | None = None, cnn_every=1,
                 fallback=True):
    """Solve h^2 A x = b (b complex64 [B, ny, nx]); x complex128 (in: x0, out: solution).
    Returns (x, stats) with stats a numpy structured array (iters, status, rel_res_est,
    rel_res_true) per right-hand side."""
    B = _grid(p, b, torch.complex64, "b")
    if x is None:
        x = torch.zeros(b.shape, dtype=torch.complex128, device=b.device)
    _grid(p, x, torch.complex128, "x")
    if tuple(x.shape) != tuple(b.shape):
        raise HelmError(f"x has shape {tuple(x.shape)}, b {tuple(b.shape)}")
    stats = torch.zeros(B * STATS_DTYPE.itemsize, dtype=torch.uint8, device=b.device)
    ws = p.workspace(B, restart, cnn)
    o = fgmres_opts(restart, rtol, maxit, warmup_iters, reorth, cnn_every, fallback)
    caps = None
    if maxit_per_rhs is not None:
        _batch_vec(maxit_per_rhs, B, torch.int32, "maxit_per_rhs", b.device)
        caps = maxit_per_rhs
    check(lib().helm_fgmres_solve(p.handle, cnn.handle if cnn is not None else None, _ptr(b), _ptr(x), B,
                                  C.byref(o), _ptr(caps), _ptr(stats), _ptr(ws), ws.numel(), _stream()),
          "helm_fgmres_solve")
    st = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=STATS_DTYPE)
    return x, st


def problem_update(p: Problem, kappa: torch.Tensor, omega_h: float):
    """Recompute p's setup in place for a new slowness model of the same grid
    (helm_problem_update); a network's encodings of p must be recomputed afterwards."""
    _need(kappa, torch.float32, "kappa")
    if tuple(kappa.shape) != (p.ny, p.nx) or kappa.device != p.device:
        raise HelmError(f"kappa must be [{p.ny}, {p.nx}] on {p.device}")
    check(lib().helm_problem_update(p.handle, _ptr(kappa), omega_h, _stream()), "helm_problem_update")
    p.omega_h = omega_h


class SolverPlan:
    """A captured FGMRES solver for one problem handle, batch size and options
    (helm_solver_plan_*): the right-hand sides go into `self.b`, the solution comes out
    in `self.x`; every restart cycle is one CUDA graph launch on the plan's stream."""

    def __init__(self, p: Problem, batch: int, cnn=None, restart=10, rtol=1e-6, maxit=2000, warmup_iters=3,
                 reorth=1, cnn_every=1, fallback=True, stream: torch.cuda.Stream | None = None):
        self.p, self.cnn, self.batch = p, cnn, batch
        self.stream = stream if stream is not None else torch.cuda.Stream(device=p.device)
        self.b = torch.zeros((batch, p.ny, p.nx), dtype=torch.complex64, device=p.device)
        self.x = torch.zeros((batch, p.ny, p.nx), dtype=torch.complex128, device=p.device)
        self.stats = torch.zeros(batch * STATS_DTYPE.itemsize, dtype=torch.uint8, device=p.device)
        n = C.c_size_t()
        check(lib().helm_workspace_size(p.handle, cnn.handle if cnn is not None else None, batch, restart,
                                        C.byref(n)), "workspace_size")
        self.ws = torch.empty(n.value, dtype=torch.uint8, device=p.device)
        self.opts = fgmres_opts(restart, rtol, maxit, warmup_iters, reorth, cnn_every, fallback)
        h = C.c_void_p()
        torch.cuda.current_stream(p.device).synchronize()
        check(lib().helm_solver_plan_create(p.handle, cnn.handle if cnn is not None else None, _ptr(self.b),
                                            _ptr(self.x), batch, C.byref(self.opts), _ptr(self.ws), self.ws.numel(),
                                            _stream(self.stream), C.byref(h)), "helm_solver_plan_create")
        self.handle = h

    def solve(self, maxit_per_rhs: torch.Tensor | None = None):
        """Solve for the current contents of self.b; returns the per-RHS statistics."""
        caps = None
        if maxit_per_rhs is not None:
            _batch_vec(maxit_per_rhs, self.batch, torch.int32, "maxit_per_rhs", self.b.device)
            caps = maxit_per_rhs
        check(lib().helm_solver_plan_solve(self.handle, _ptr(caps), _ptr(self.stats), _stream(self.stream)),
              "helm_solver_plan_solve")
        self.stream.synchronize()
        return np.frombuffer(self.stats.cpu().numpy().tobytes(), dtype=STATS_DTYPE)

    def close(self):
        if getattr(self, "handle", None):
            lib().helm_solver_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TUNE_KNOBS = {"conv_rows": 0, "ib_sh": 1, "implicit_3pass": 2}


def tune_set(knob: str, height: int, batch: int, value: int):
    """Override a launch heuristic for layers of height `height` run on `batch` images
    (batch 0: any batch; height 0 with batch 0: every layer); value 0 removes the entry."""
    check(lib().helm_tune_set(TUNE_KNOBS[knob], int(height), int(batch), int(value)), "helm_tune_set")


def tune_get(knob: str, height: int, batch: int) -> int:
    """The value a launch of that height and batch takes (0: the heuristic)."""
    v = C.c_int()
    check(lib().helm_tune_get(TUNE_KNOBS[knob], int(height), int(batch), C.byref(v)), "helm_tune_get")
    return v.value


def tune_clear():
    check(lib().helm_tune_clear(), "helm_tune_clear")


def profile(fn) -> list:
    """Run fn() under the library's profiler (helm_profile_*: CUDA events around every
    launch on its own stream) and return [(kernel name, launches, total ms)], largest
    total first."""
    check(lib().helm_profile_begin(), "helm_profile_begin")
    nk = C.c_int()
    try:
        fn()
        torch.cuda.synchronize()
    finally:
        check(lib().helm_profile_end(C.byref(nk)), "helm_profile_end")
    rows = []
    for i in range(nk.value):
        nm, cnt, tot = C.c_char_p(), C.c_long(), C.c_double()
        check(lib().helm_profile_read(i, C.byref(nm), C.byref(cnt), C.byref(tot)), "helm_profile_read")
        rows.append((nm.value.decode(), cnt.value, tot.value))
    rows.sort(key=lambda t: -t[2])
    return rows


def device_errors() -> int:
    f = C.c_uint()
    check(lib().helm_device_errors(C.byref(f)), "helm_device_errors")
    return f.value


def version() -> str:
    return lib().helm_version().decode()


CONV_MODES = {"s1": 0, "s2": 1, "t2": 2, "t1": 3}


def conv_bf16(x: torch.Tensor, w: torch.Tensor, mode: str = "s1", scale=None, shift=None, act=False, add1=None,
              add2=None, raw=False):
    """One tensor-core convolution (see helm_conv_bf16): x BF16 NHWC [B, H, W, Cin],
    w FP32 in PyTorch module layout.  Returns (y BF16 NHWC, yraw FP32 NHWC or None)."""
    _need(x, torch.bfloat16, "x")
    _need(w, torch.float32, "w")
    if x.dim() != 4 or w.device != x.device:
        raise HelmError("x must be BF16 NHWC [B, H, W, Cin]; w on the same device")
    B, H, W, Ci = x.shape
    if w.dim() == 2:
        taps = 1
    elif w.dim() == 4 and tuple(w.shape[2:]) == (3, 3):
        taps = 9
    else:
        raise HelmError(f"w has shape {tuple(w.shape)}; expected [Co, Ci] or a 3x3 kernel")
    m = CONV_MODES[mode]
    transposed = taps == 9 and m in (2, 3)
    Co = w.shape[1] if transposed else w.shape[0]
    if (w.shape[0] if transposed else w.shape[1]) != Ci:
        raise HelmError(f"w has shape {tuple(w.shape)} for {Ci} input channels")
    if taps == 1:
        Ho, Wo = H, W
    elif m == 1:
        Ho, Wo = H // 2, W // 2
    elif m == 2:
        Ho, Wo = 2 * H, 2 * W
    else:
        Ho, Wo = H, W
    for v, nm in ((scale, "scale"), (shift, "shift")):
        if v is not None:
            _batch_vec(v, Co, torch.float32, nm, x.device)
    if add1 is not None:
        _need(add1, torch.bfloat16, "add1")
        if tuple(add1.shape) != (B, Ho, Wo, Co) or add1.device != x.device:
            raise HelmError(f"add1 must be [{B}, {Ho}, {Wo}, {Co}] on {x.device}")
    if add2 is not None:
        _need(add2, torch.bfloat16, "add2")
        if add2.dim() != 4 or add2.shape[0] not in (1, B) or tuple(add2.shape[1:]) != (Ho, Wo, Co) \
                or add2.device != x.device:
            raise HelmError(f"add2 must be [{B} or 1, {Ho}, {Wo}, {Co}] on {x.device}")
    y = torch.empty((B, Ho, Wo, Co), dtype=torch.bfloat16, device=x.device)
    yr = torch.empty((B, Ho, Wo, Co), dtype=torch.float32, device=x.device) if raw else None
    ws = torch.empty(taps * max(16, (Ci + 15) // 16 * 16) * Co * 2 + 4096, dtype=torch.uint8, device=x.device)
    bc = int(add2 is not None and add2.shape[0] == 1 and B > 1)
    check(lib().helm_conv_bf16(_ptr(x), B, H, W, Ci, _ptr(w), Co, taps, m, _ptr(scale), _ptr(shift), int(act),
                               _ptr(add1), _ptr(add2), bc, _ptr(y), _ptr(yr), _ptr(ws), ws.numel(), _stream()),
          "helm_conv_bf16")
    return y, yr


class Cnn:
    """The encoder-solver network: FP32 parameters (`params`, a flat CUDA tensor in the
    library's parameter order) and BN running statistics live on the device.
    explicit_unet=True gives the explicit U-Net of Section 6: the same network without
    the implicit step at the coarsest level."""

    def __init__(self, c0=16, expansion=6, skip_threshold=512, literal_green=False, explicit_unet=False,
                 device="cuda"):
        d = _lib.CnnDesc()
        d.c0, d.expansion, d.skip_threshold, d.literal_green = c0, expansion, skip_threshold, int(literal_green)
        d.explicit_unet = int(explicit_unet)
        self.explicit_unet = bool(explicit_unet)
        h = C.c_void_p()
        check(lib().helm_cnn_create(C.byref(d), C.byref(h)), "helm_cnn_create")
        self.handle = h
        self.device = torch.device(device)
        n = C.c_size_t()
        check(lib().helm_cnn_num_params(h, C.byref(n)), "num_params")
        self.nparams = n.value
        self.spec = []          # (name, shape, offset)
        i = 0
        while True:
            nm, nd, off = C.c_char_p(), C.c_int(), C.c_size_t()
            shp = (C.c_int * 4)()
            if lib().helm_cnn_param_info(h, i, C.byref(nm), C.byref(nd), shp, C.byref(off)) != 0:
                break
            self.spec.append((nm.value.decode(), tuple(shp[:nd.value]), off.value))
            i += 1
        nb = C.c_int()
        check(lib().helm_cnn_num_bn(h, C.byref(nb)), "num_bn")
        self.bn = []            # (name, C, roff)
        for j in range(nb.value):
            nm, cc, ro = C.c_char_p(), C.c_int(), C.c_size_t()
            check(lib().helm_cnn_bn_info(h, j, C.byref(nm), C.byref(cc), C.byref(ro)), "bn_info")
            self.bn.append((nm.value.decode(), cc.value, ro.value))
        self.nrunning = sum(2 * c for _, c, _ in self.bn)
        self.params = torch.zeros(self.nparams, dtype=torch.float32, device=self.device)
        self.running = torch.zeros(self.nrunning, dtype=torch.float32, device=self.device)
        check(lib().helm_cnn_get_running(h, _ptr(self.running), _stream()), "get_running")
        self.set_params()

    def close(self):
        if getattr(self, "handle", None):
            lib().helm_cnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- parameters -------------------------------------------------------------
    def set_params(self, flat: torch.Tensor | None = None):
        if flat is not None:
            self.params.copy_(flat)
        check(lib().helm_cnn_set_params(self.handle, _ptr(self.params), _stream()), "set_params")

    def load_dict(self, pdict: dict):
        """Fill the parameter vector from a name -> array dict (shapes must match)."""
        flat = np.zeros(self.nparams, dtype=np.float32)
        for name, shape, off in self.spec:
            a = np.asarray(pdict[name], dtype=np.float32)
            assert a.shape == shape, (name, a.shape, shape)
            flat[off:off + a.size] = a.ravel()
        self.params.copy_(torch.from_numpy(flat))
        self.set_params()

    def to_dict(self, flat: torch.Tensor | None = None) -> dict:
        v = (self.params if flat is None else flat).detach().cpu().numpy().astype(np.float64)
        return {name: v[off:off + int(np.prod(shape))].reshape(shape) for name, shape, off in self.spec}

    def load_running(self, rdict: dict):
        """rdict: bn name -> (mean, var)."""
        flat = np.zeros(self.nrunning, dtype=np.float32)
        for name, c, ro in self.bn:
            mu, var = rdict[name]
            flat[ro:ro + c] = mu
            flat[ro + c:ro + 2 * c] = var
        self.running.copy_(torch.from_numpy(flat))
        check(lib().helm_cnn_set_running(self.handle, _ptr(self.running), _stream()), "set_running")

    def running_dict(self) -> dict:
        check(lib().helm_cnn_get_running(self.handle, _ptr(self.running), _stream()), "get_running")
        v = self.running.cpu().numpy().astype(np.float64)
        return {name: (v[ro:ro + c].copy(), v[ro + c:ro + 2 * c].copy()) for name, c, ro in self.bn}

    def running_dict_flat(self) -> np.ndarray:
        check(lib().helm_cnn_get_running(self.handle, _ptr(self.running), _stream()), "get_running")
        return self.running.cpu().numpy().copy()

    def load_running_flat(self, flat):
        self.running.copy_(torch.as_tensor(np.asarray(flat, dtype=np.float32)))
        check(lib().helm_cnn_set_running(self.handle, _ptr(self.running), _stream()), "set_running")

    def ghat(self, m) -> torch.Tensor:
        """G_hat (Eq. 15 after crop and DFT) of a coarsest map of side m, or of an
        m_y x m_x map given as a pair: complex64 [nk, 2 m_y, 2 m_x]."""
        my, mx = (m, m) if np.ndim(m) == 0 else (int(m[0]), int(m[1]))
        shapes = dict((n, s) for n, s, _ in self.spec)
        nk = shapes["s.imp.K"][1] if "s.imp.K" in shapes else 1   # explicit U-Net: the call fails
        out = torch.empty((nk, 2 * my, 2 * mx), dtype=torch.complex64, device=self.device)
        if my == mx:
            check(lib().helm_cnn_get_ghat(self.handle, my, _ptr(out), _stream()), "get_ghat")
        else:
            check(lib().helm_cnn_get_ghat_rect(self.handle, my, mx, _ptr(out), _stream()), "get_ghat_rect")
        return out

    # ---- application ------------------------------------------------------------
    def set_problem(self, p: Problem):
        check(lib().helm_cnn_set_problem(self.handle, p.handle, None, 0, _stream()), "helm_cnn_set_problem")

    def apply(self, p: Problem, r: torch.Tensor, train: bool = False, ws: torch.Tensor | None = None):
        """e = s Net(r / s), s = RMS of r over the grid."""
        B = _grid(p, r, torch.complex64, "r")
        e = torch.empty_like(r)
        ws = p.workspace(B, 10, self) if ws is None else ws
        check(lib().helm_cnn_apply(p.handle, self.handle, _ptr(r), _ptr(e), B, int(train), _ptr(ws), ws.numel(),
                                   _stream()), "helm_cnn_apply")
        return e

    def precond(self, p: Problem, r: torch.Tensor):
        """z = e + V(r - A e)."""
        B = _grid(p, r, torch.complex64, "r")
        z = torch.empty_like(r)
        ws = p.workspace(B, 10, self)
        check(lib().helm_cnn_precond_apply(p.handle, self.handle, _ptr(r), _ptr(z), B, _ptr(ws), ws.numel(),
                                           _stream()), "helm_cnn_precond_apply")
        return z

    # ---- training ---------------------------------------------------------------
    def train_workspace(self, p: Problem, batch: int, nprob: int = 1) -> torch.Tensor:
        n = C.c_size_t()
        check(lib().helm_cnn_train_workspace_size(p.handle, self.handle, batch, nprob, C.byref(n)),
              "train_workspace_size")
        ws = getattr(self, "_tws", None)
        if ws is None or ws.numel() < n.value:
            self._tws = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        return self._tws

    def forward_train(self, p, r: torch.Tensor) -> torch.Tensor:
        """Training-mode forward (batch-statistics BN; saves activations for backward).
        `p` is one Problem or a list of Problems: sample b then belongs to
        p[b // (B // len(p))]."""
        probs = list(p) if isinstance(p, (list, tuple)) else [p]
        B = _grid(probs[0], r, torch.complex64, "r")
        if B % len(probs):
            raise HelmError(f"batch {B} is not divisible by the {len(probs)} slowness models")
        ws = self.train_workspace(probs[0], B, len(probs))
        e = torch.empty_like(r)
        arr = (C.c_void_p * len(probs))(*[q.handle.value for q in probs])
        check(lib().helm_cnn_train_forward(arr, len(probs), self.handle, _ptr(r), _ptr(e), B, _ptr(ws), ws.numel(),
                                           _stream()), "helm_cnn_train_forward")
        self._train_nprob = len(probs)
        self._train_p0 = probs[0]
        return e

    def backward(self, p, grad_e: torch.Tensor, grad_params: torch.Tensor | None = None,
                 r: torch.Tensor | None = None):
        """Parameter gradient of the last training forward; with `r` (that forward's
        input) also the input gradient: returns grad_params, or (grad_params, grad_r)."""
        p = p[0] if isinstance(p, (list, tuple)) else p
        B = _grid(p, grad_e, torch.complex64, "grad_e")
        g = torch.empty_like(self.params) if grad_params is None else grad_params
        _batch_vec(g, self.nparams, torch.float32, "grad_params", self.params.device)
        gr = None
        if r is not None:
            if _grid(p, r, torch.complex64, "r") != B or r.shape != grad_e.shape:
                raise HelmError("r must have grad_e's shape")
            gr = torch.empty_like(r)
        ws = self.train_workspace(p, B, getattr(self, "_train_nprob", 1))
        check(lib().helm_cnn_precond_backward(p.handle, self.handle, _ptr(r), _ptr(grad_e), _ptr(gr), _ptr(g), B,
                                              _ptr(ws), ws.numel(), _stream()), "helm_cnn_precond_backward")
        return g if r is None else (g, gr)

    # ---- persistence ------------------------------------------------------------
    def save(self, path: str):
        """helm_cnn_save: parameters, BN statistics and the G_hat the handle holds."""
        check(lib().helm_cnn_save(self.handle, str(path).encode(), _stream()), "helm_cnn_save")

    def load(self, path: str):
        """helm_cnn_load into this handle's parameter vector (same descriptor)."""
        check(lib().helm_cnn_load(self.handle, str(path).encode(), _ptr(self.params), _stream()), "helm_cnn_load")
        check(lib().helm_cnn_get_running(self.handle, _ptr(self.running), _stream()), "get_running")


def mse_loss(e_pred: torch.Tensor, e_true: torch.Tensor, grad: bool = True):
    """Eq. (16) on the device: (loss tensor (float64, shape [1]), gradient or None)."""
    _need(e_pred, torch.complex64, "e_pred")
    _need(e_true, torch.complex64, "e_true")
    if e_true.shape != e_pred.shape or e_true.device != e_pred.device or e_pred.dim() < 2:
        raise HelmError(f"e_pred {tuple(e_pred.shape)} and e_true {tuple(e_true.shape)} must match, batch first")
    B = e_pred.shape[0]
    loss = torch.empty(1, dtype=torch.float64, device=e_pred.device)
    g = torch.empty_like(e_pred) if grad else None
    ws = torch.empty(8192, dtype=torch.uint8, device=e_pred.device)
    check(lib().helm_mse_loss(_ptr(e_pred), _ptr(e_true), e_pred.numel(), B, _ptr(loss), _ptr(g), _ptr(ws),
                              _stream()), "helm_mse_loss")
    return loss, g


class Adam:
    """Adam on the device (helm_adam_step), FP32 moments."""

    def __init__(self, params: torch.Tensor, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        self.p = params
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.lr, self.b1, self.b2, self.eps = lr, betas[0], betas[1], eps
        self.t = 0

    def step(self, grads: torch.Tensor):
        self.t += 1
        check(lib().helm_adam_step(_ptr(self.p), _ptr(grads), _ptr(self.m), _ptr(self.v), self.p.numel(), self.lr,
                                   self.b1, self.b2, self.eps, self.t, _stream()), "helm_adam_step")


class CnnFunction(torch.autograd.Function):
    """torch.autograd wrapper around the training forward / backward kernels:
    e = CnnFunction.apply(params, r, net, problem), with `params` the network's own
    parameter vector (net.params).  Gradients flow to `params` and, when r requires
    one, to r (the library's input gradient, the RMS scale's dependence included)."""

    @staticmethod
    def forward(ctx, params, r, net, problem):
        if params.data_ptr() != net.params.data_ptr():
            raise HelmError("CnnFunction: params must be the network's parameter vector (net.params)")
        ctx.net, ctx.problem = net, problem
        ctx.need_r = ctx.needs_input_grad[1]
        if ctx.need_r:
            ctx.save_for_backward(r)
        return net.forward_train(problem, r)

    @staticmethod
    def backward(ctx, grad_e):
        if ctx.need_r:
            (r,) = ctx.saved_tensors
            g, gr = ctx.net.backward(ctx.problem, grad_e.contiguous(), r=r.contiguous())
            return g, gr, None, None
        g = ctx.net.backward(ctx.problem, grad_e.contiguous())
        return g, None, None, None


def training_field(white: torch.Tensor, sigma: float, noise: float) -> torch.Tensor:
    """Random training vectors (Section 4.3): white is a float32 CUDA tensor [B, 4, n, n]
    of standard normal numbers (planes w0, w1, n0, n1); returns complex64 [B, n, n]
    x = f / RMS(f) + noise (n0 + i n1) with f the periodic Gaussian filter (std sigma
    cells) of w0 + i w1."""
    _need(white, torch.float32, "white")
    if white.dim() != 4 or white.shape[1] != 4 or white.shape[2] != white.shape[3]:
        raise ValueError("white must be [B, 4, n, n]")
    B, n = white.shape[0], white.shape[2]
    x = torch.empty((B, n, n), dtype=torch.complex64, device=white.device)
    check(lib().helm_training_field(_ptr(white), B, n, float(sigma), float(noise), _ptr(x), _stream()),
          "helm_training_field")
    return x


def datagen_pairs(p: Problem, x: torch.Tensor, iters: torch.Tensor, max_iters: int = 20, normalise: bool = True):
    """Eq. (17) on the device: (e, r) complex64 for random x [B, N, N] (complex64) and
    per-sample FGMRES iteration counts `iters` (int32 CUDA tensor)."""
    B = _grid(p, x, torch.complex64, "x")
    _batch_vec(iters, B, torch.int32, "iters", x.device)
    n = C.c_size_t()
    check(lib().helm_datagen_workspace_size(p.handle, B, max_iters, C.byref(n)), "datagen_workspace_size")
    ws = getattr(p, "_dws", None)
    if ws is None or ws.numel() < n.value:
        p._dws = ws = torch.empty(n.value, dtype=torch.uint8, device=x.device)
    e = torch.empty_like(x)
    r = torch.empty_like(x)
    check(lib().helm_datagen_pairs(p.handle, _ptr(x), _ptr(iters), _ptr(e), _ptr(r), B, max_iters, int(normalise),
                                   _ptr(ws), ws.numel(), _stream()), "helm_datagen_pairs")
    return e, r
