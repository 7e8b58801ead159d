"""ctypes binding of libnlem.so.  Argument marshalling only; names follow include/nlem.h."""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(PKG, "lib", "libnlem.so")

PREC_FP32 = 0
PREC_BF16 = 1
INIT_WEIGHTED_MEAN = 0
INIT_NOISY_PATCH = 1
SOLVER_ADMM = 0
SOLVER_IRLS = 1
SOLVER_FAST = 2
LAYOUT_AUTO = 0
LAYOUT_PIXEL = 1
LAYOUT_PAIR = 2
PENALTY_UNIFORM = 0
PENALTY_WEIGHTED = 1

_ERRNAMES = {-1: "NLEM_ERR_INVALID", -2: "NLEM_ERR_CUDA", -3: "NLEM_ERR_OOM", -4: "NLEM_ERR_TIMEOUT",
             -5: "NLEM_ERR_UNSUPPORTED"}


class NlemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class _Box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float), ("hi", ctypes.c_float)]


class _ImageDesc(ctypes.Structure):
    _fields_ = [("image", ctypes.c_void_p), ("out", ctypes.c_void_p), ("iters_used", ctypes.c_void_p),
                ("residual", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("pitch", ctypes.c_int),
                ("patch", ctypes.c_int), ("window", ctypes.c_int), ("h", ctypes.c_float)]


class _Set(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p),
                ("center", ctypes.c_void_p), ("radius", ctypes.c_float)]


class _Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_float), ("check_every", ctypes.c_int), ("precision", ctypes.c_int),
                ("init", ctypes.c_int), ("fp64_check", ctypes.c_int), ("layout", ctypes.c_int),
                ("solver", ctypes.c_int), ("irls_eps", ctypes.c_float), ("penalty", ctypes.c_int),
                ("restart_every", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libnlem.so (built in-tree by __graft_entry__.build()); raises if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libnlem.so not found at {_LIB_PATH}; build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i, ll, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_float
        lib.nlem_last_error.restype = ctypes.c_char_p
        lib.nlem_version.restype = ctypes.c_char_p
        lib.nlem_options_default.argtypes = [ctypes.POINTER(_Options)]
        lib.nlem_ctx_create.argtypes = [ctypes.POINTER(vp), i]
        lib.nlem_ctx_destroy.argtypes = [vp]
        lib.em_solve.argtypes = [vp, vp, vp, i, i, _Box, f, i, vp, vp]
        lib.em_solve_batch.argtypes = [vp, vp, vp, ll, i, i, _Box, f, i, vp, ctypes.POINTER(_Options), vp, vp, vp,
                                       vp, vp, vp]
        lib.nlem_denoise.argtypes = [vp, vp, i, i, i, i, i, f, f, i, _Box, ctypes.POINTER(_Options), vp, vp, vp, vp,
                                     vp, vp]
        lib.nlem_denoise_host.argtypes = [vp, vp, i, i, i, i, f, f, i, _Box, ctypes.POINTER(_Options), vp, vp, vp]
        lib.em_solve_batch_set.argtypes = [vp, vp, vp, ll, i, i, ctypes.POINTER(_Set), f, i, vp,
                                           ctypes.POINTER(_Options), vp, vp, vp, vp]
        lib.nlem_denoise_color.argtypes = [vp, vp, i, i, i, i, i, i, f, f, i, _Box, ctypes.POINTER(_Options), vp, vp,
                                           vp, vp, vp, vp]
        lib.em_solve_batch_host.argtypes = [vp, vp, vp, ll, i, i, _Box, f, i, vp, ctypes.POINTER(_Options), ll, vp,
                                            vp, vp, vp]
        lib.nlem_fp32_peak.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        lib.nlem_denoise_batch.argtypes = [vp, ctypes.POINTER(_ImageDesc), i, f, i, _Box, ctypes.POINTER(_Options), vp]
        lib.nlem_batch_config.argtypes = [vp, ctypes.c_char_p, i]
        lib.nlem_batch_force_config.argtypes = [vp, i, i, i]
        lib.nlem_debug_status.argtypes = [i, ctypes.POINTER(i), ctypes.POINTER(ll), ctypes.POINTER(ll),
                                          ctypes.POINTER(ll)]
        lib.nlem_device_status.argtypes = [vp]
        lib.nlem_selftest_timeout.argtypes = [vp]
        lib.nlem_bf16_weights.argtypes = [vp, vp, i, i, i, i, i, f, vp, vp]
        lib.nlem_ws_num_params.argtypes = [i]
        lib.nlem_ws_num_params.restype = ll
        lib.nlem_ws_create.argtypes = [vp, i, f, ctypes.c_ulonglong, ctypes.POINTER(vp)]
        lib.nlem_ws_destroy.argtypes = [vp]
        lib.nlem_ws_get_params.argtypes = [vp, vp]
        lib.nlem_ws_set_params.argtypes = [vp, vp]
        lib.nlem_ws_save.argtypes = [vp, ctypes.c_char_p]
        lib.nlem_ws_load.argtypes = [vp, ctypes.c_char_p]
        lib.nlem_ws_forward.argtypes = [vp, vp, vp, ll, vp, vp]
        lib.nlem_ws_loss_grad.argtypes = [vp, vp, vp, vp, ll, vp, vp, vp]
        lib.nlem_ws_train_step.argtypes = [vp, vp, vp, vp, ll, f, vp, vp]
        lib.nlem_ws_train.argtypes = [vp, vp, vp, vp, ll, i, i, f, ctypes.c_ulonglong, vp, vp]
        lib.nlem_ws_predict.argtypes = [vp, vp, vp, ll, _Box, vp, vp, vp, vp]
        lib.nlem_features.argtypes = [vp, vp, i, i, i, i, i, f, vp, ll, vp, vp]
        lib.nlem_denoise_ex.argtypes = [vp, vp, i, i, i, i, i, f, f, i, _Box, ctypes.POINTER(_Options), vp, ll, vp, vp,
                                        vp, vp, vp, vp, vp]
        lib.nlem_ws_labels.argtypes = [vp, vp, i, i, i, i, i, f, _Box, vp, ll, ctypes.POINTER(f), i, f, i, i, f, i,
                                       vp, vp, ctypes.POINTER(ll), vp]
        lib.nlem_denoise_warm.argtypes = [vp, vp, vp, i, i, i, i, i, f, f, i, _Box, ctypes.POINTER(_Options), vp, vp,
                                          ctypes.POINTER(ll), vp]
        lib.nlem_denoise_batch_noalloc.argtypes = [ctypes.POINTER(_ImageDesc), i, f, i, _Box,
                                                   ctypes.POINTER(_Options), vp]
        for name in ("nlem_ctx_create", "nlem_ctx_destroy", "em_solve", "em_solve_batch", "em_solve_batch_host",
                     "nlem_denoise",
                     "nlem_denoise_host", "nlem_fp32_peak", "nlem_denoise_batch", "nlem_batch_config", "nlem_batch_force_config", "nlem_debug_status", "nlem_denoise_batch_noalloc",
                     "nlem_device_status", "nlem_bf16_weights", "nlem_ws_create", "nlem_ws_destroy",
                     "nlem_ws_get_params", "nlem_ws_set_params", "nlem_ws_save", "nlem_ws_load", "nlem_ws_forward",
                     "nlem_ws_loss_grad", "nlem_ws_train_step", "nlem_ws_predict", "nlem_features", "nlem_denoise_ex",
                     "nlem_denoise_warm", "nlem_ws_labels"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int):
    if rc < 0:
        raise NlemError(rc, load_library().nlem_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("device tensor required (use nlem_denoise_host for host buffers)")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _image(t):
    """Device pointer and row pitch (elements) of a float32 image [H, W] whose rows are
    contiguous; row-pitched views (for example a column slice of a wider array) are passed as
    they are."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("device tensor required (use nlem_denoise_host for host buffers)")
    if t.dim() != 2 or (t.shape[1] > 1 and t.stride(1) != 1) or t.stride(0) < t.shape[1]:
        raise ValueError("image must be [H, W] with contiguous rows")
    return ctypes.c_void_p(t.data_ptr()), int(t.stride(0)) if t.shape[0] > 1 else int(t.shape[1])


def _need(t, dtype, shape, name):
    import torch
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def _stream(device):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _options(tol=0.0, check_every=1, precision=PREC_FP32, init=INIT_WEIGHTED_MEAN, fp64_check=False,
             layout=0, solver=None, irls_eps=None, penalty=PENALTY_UNIFORM, restart_every=0):
    o = _Options()
    load_library().nlem_options_default(ctypes.byref(o))
    o.tol = float(tol)
    o.check_every = int(check_every)
    o.precision = int(precision)
    o.init = int(init)
    o.fp64_check = 1 if fp64_check else 0
    o.layout = int(layout)
    if solver is not None:
        o.solver = int(solver)
    if irls_eps is not None:
        o.irls_eps = float(irls_eps)
    o.penalty = int(penalty)
    o.restart_every = int(restart_every)
    return o


class Context:
    """Owns an nlem_ctx (workspace, tuning cache) on one CUDA device."""

    def __init__(self, device: int = 0):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.nlem_ctx_create(ctypes.byref(h), int(device)))
        self.handle = h
        self.device = int(device)

    def close(self):
        if self.handle:
            load_library().nlem_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_ctxs: dict[int, Context] = {}


def _ctx(device) -> Context:
    import torch
    dev = torch.device(device).index if device is not None else torch.cuda.current_device()
    if dev is None:
        dev = torch.cuda.current_device()
    c = _ctxs.get(dev)
    if c is None:
        c = _ctxs[dev] = Context(dev)
    return c


def em_solve(points, weights, box=(0.0, 255.0), rho=1.0, iters=100, out=None, ctx: Context | None = None):
    """Problem (1) for one point set: points [n, d] float32 CUDA, weights [n]; returns x [d]."""
    import torch
    n, d = points.shape
    _need(points, torch.float32, (n, d), "points")
    _need(weights, torch.float32, (n,), "weights")
    c = ctx or _ctx(points.device)
    if out is None:
        out = torch.empty(d, dtype=torch.float32, device=points.device)
    _check(load_library().em_solve(c.handle, _ptr(points), _ptr(weights), n, d, _Box(*box), float(rho), int(iters),
                                   _ptr(out), _stream(points.device)))
    return out


def em_solve_batch(points, weights, box=(0.0, 255.0), rho=1.0, iters=100, x0=None, tol=0.0, check_every=1,
                   fp64_check=False, ctx: Context | None = None, out=None, penalty=PENALTY_UNIFORM,
                   solver=SOLVER_ADMM, restart_every=0):
    """Algorithm 1 on B problems: points [B, n, d], weights [B, n] (float32 CUDA).  penalty:
    PENALTY_UNIFORM (Algorithm 1) or PENALTY_WEIGHTED (mu_k = rho w_k; d = 49).  solver SOLVER_FAST:
    accelerated EM-ADMM (d = 49, n <= 448; restart_every 0 = the combined-residual restart test,
    k >= 1 = restart after every k-th step).
    Returns dict(x [B,d], iters_used [B] int32, residual [B], obj64/kkt64 [B] float64 if fp64_check)."""
    import torch
    B, n, d = points.shape
    _need(points, torch.float32, (B, n, d), "points")
    _need(weights, torch.float32, (B, n), "weights")
    if x0 is not None:
        _need(x0, torch.float32, (B, d), "x0")
    c = ctx or _ctx(points.device)
    dev = points.device
    res = out or {}
    x = res.get("x")
    if x is None:
        x = torch.empty((B, d), dtype=torch.float32, device=dev)
    used = res.get("iters_used")
    if used is None:
        used = torch.empty(B, dtype=torch.int32, device=dev)
    resid = res.get("residual")
    if resid is None:
        resid = torch.empty(B, dtype=torch.float32, device=dev)
    obj = kkt = None
    if fp64_check:
        obj = torch.empty(B, dtype=torch.float64, device=dev)
        kkt = torch.empty(B, dtype=torch.float64, device=dev)
    o = _options(tol, check_every, fp64_check=fp64_check, penalty=penalty, solver=solver,
                 restart_every=restart_every)
    _check(load_library().em_solve_batch(c.handle, _ptr(points), _ptr(weights), B, n, d, _Box(*box), float(rho),
                                         int(iters), _ptr(x0), ctypes.byref(o), _ptr(x), _ptr(used), _ptr(resid),
                                         _ptr(obj), _ptr(kkt), _stream(dev)))
    r = dict(x=x, iters_used=used, residual=resid)
    if fp64_check:
        r.update(obj64=obj, kkt64=kkt)
    return r


SET_COORD_BOXES = 1
SET_BALL = 2


def em_solve_batch_set(points, weights, lo=None, hi=None, center=None, radius=None, rho=1.0, iters=100, x0=None,
                       tol=0.0, check_every=1, ctx: Context | None = None, out=None):
    """Algorithm 1 on B problems over a constraint set other than the box: per-coordinate boxes
    (lo, hi: float32 CUDA [d]) or the ball ||x - center|| <= radius (center: float32 CUDA [d]).
    Returns dict(x [B,d], iters_used [B] int32, residual [B])."""
    import torch
    B, n, d = points.shape
    _need(points, torch.float32, (B, n, d), "points")
    _need(weights, torch.float32, (B, n), "weights")
    if x0 is not None:
        _need(x0, torch.float32, (B, d), "x0")
    s = _Set()
    if center is not None:
        _need(center, torch.float32, (d,), "center")
        s.kind, s.center, s.radius = SET_BALL, _ptr(center), float(radius)
    else:
        _need(lo, torch.float32, (d,), "lo")
        _need(hi, torch.float32, (d,), "hi")
        s.kind, s.lo, s.hi = SET_COORD_BOXES, _ptr(lo), _ptr(hi)
    c = ctx or _ctx(points.device)
    dev = points.device
    res = out or {}
    x = res.get("x")
    if x is None:
        x = torch.empty((B, d), dtype=torch.float32, device=dev)
    used = res.get("iters_used")
    if used is None:
        used = torch.empty(B, dtype=torch.int32, device=dev)
    resid = res.get("residual")
    if resid is None:
        resid = torch.empty(B, dtype=torch.float32, device=dev)
    o = _options(tol, check_every)
    _check(load_library().em_solve_batch_set(c.handle, _ptr(points), _ptr(weights), B, n, d, ctypes.byref(s),
                                             float(rho), int(iters), _ptr(x0), ctypes.byref(o), _ptr(x), _ptr(used),
                                             _ptr(resid), _stream(dev)))
    return dict(x=x, iters_used=used, residual=resid)


def _host_ptr(t, dtype, shape, name):
    """Pointer of a contiguous CPU tensor (pinned memory lets the library overlap its copies)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a CPU torch.Tensor")
    _need(t, dtype, shape, name)
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def em_solve_batch_host(points, weights, box=(0.0, 255.0), rho=1.0, iters=100, x0=None, tol=0.0, check_every=1,
                        chunk=0, ctx: Context | None = None, out=None, device=0, penalty=PENALTY_UNIFORM,
                        solver=SOLVER_ADMM, restart_every=0):
    """Algorithm 1 on B problems held in HOST memory: points [B, n, d] and weights [B, n] (CPU float32
    tensors, ideally pinned).  The library copies them in chunks of `chunk` problems (0 = about 1 GiB),
    overlapping the copy of each chunk with the solve of the previous one, and copies the results
    back.  Returns dict(x [B,d], iters_used [B] int32, residual [B]) as CPU tensors."""
    import torch
    B, n, d = points.shape
    pp = _host_ptr(points, torch.float32, (B, n, d), "points")
    wp = _host_ptr(weights, torch.float32, (B, n), "weights")
    x0p = _host_ptr(x0, torch.float32, (B, d), "x0") if x0 is not None else None
    c = ctx or _ctx(torch.device("cuda", device))
    pin = points.is_pinned()
    res = out or {}
    x = res.get("x")
    if x is None:
        x = torch.empty((B, d), dtype=torch.float32, pin_memory=pin)
    used = res.get("iters_used")
    if used is None:
        used = torch.empty(B, dtype=torch.int32, pin_memory=pin)
    resid = res.get("residual")
    if resid is None:
        resid = torch.empty(B, dtype=torch.float32, pin_memory=pin)
    o = _options(tol, check_every, penalty=penalty, solver=solver, restart_every=restart_every)
    _check(load_library().em_solve_batch_host(c.handle, pp, wp, B, n, d, _Box(*box), float(rho), int(iters), x0p,
                                              ctypes.byref(o), int(chunk),
                                              _host_ptr(x, torch.float32, (B, d), "x"),
                                              _host_ptr(used, torch.int32, (B,), "iters_used"),
                                              _host_ptr(resid, torch.float32, (B,), "residual"),
                                              _stream(torch.device("cuda", c.device))))
    return dict(x=x, iters_used=used, residual=resid)


def nlem_denoise(image, patch=7, window=21, h=200.0, rho=1.0, iters=100, box=(0.0, 255.0), tol=0.0, check_every=1,
                 precision=PREC_FP32, init=INIT_WEIGHTED_MEAN, fp64_check=False, ctx: Context | None = None,
                 out=None, layout=LAYOUT_AUTO, solver=SOLVER_ADMM, irls_eps=1e-6, penalty=PENALTY_UNIFORM,
                 restart_every=0):
    """NLEM (Sec. 3) of a float32 CUDA image [H, W].  Returns dict(out [H,W], iters_used,
    residual[, obj64, kkt64]).  layout: LAYOUT_AUTO, LAYOUT_PIXEL (one pixel per CTA) or
    LAYOUT_PAIR (two adjacent pixels per CTA; patch 7, window <= 21, FP32).  solver: SOLVER_ADMM
    (Algorithm 1), SOLVER_IRLS (the surrogate of Eq. 2 with irls_eps, exactly `iters` steps) or
    SOLVER_FAST (accelerated EM-ADMM, 7x7 patches, one pixel per CTA; restart_every as for
    em_solve_batch)."""
    import torch
    H, W = image.shape
    _need(image, torch.float32, (H, W), "image")
    c = ctx or _ctx(image.device)
    dev = image.device
    res = out or {}
    o_img = res.get("out")
    if o_img is None:
        o_img = torch.empty((H, W), dtype=torch.float32, device=dev)
    used = res.get("iters_used")
    if used is None:
        used = torch.empty((H, W), dtype=torch.int32, device=dev)
    resid = res.get("residual")
    if resid is None:
        resid = torch.empty((H, W), dtype=torch.float32, device=dev)
    obj = kkt = None
    if fp64_check:
        obj = torch.empty((H, W), dtype=torch.float64, device=dev)
        kkt = torch.empty((H, W), dtype=torch.float64, device=dev)
    o = _options(tol, check_every, precision, init, fp64_check, layout, solver, irls_eps, penalty, restart_every)
    ip, pitch = _image(image)
    _check(load_library().nlem_denoise(c.handle, ip, H, W, pitch, int(patch), int(window), float(h), float(rho),
                                       int(iters), _Box(*box), ctypes.byref(o), _ptr(o_img), _ptr(used), _ptr(resid),
                                       _ptr(obj), _ptr(kkt), _stream(dev)))
    r = dict(out=o_img, iters_used=used, residual=resid)
    if fp64_check:
        r.update(obj64=obj, kkt64=kkt)
    return r


def nlem_denoise_color(image, patch=5, window=21, h=200.0, rho=1.0, iters=100, box=(0.0, 255.0), tol=0.0,
                       check_every=1, init=INIT_WEIGHTED_MEAN, fp64_check=False, ctx: Context | None = None, out=None):
    """NLEM (Sec. 3) of a planar multichannel float32 CUDA image [C, H, W] (contiguous): the patches stack
    the channels.  Returns dict(out [C, H, W], iters_used [H, W], residual [H, W][, obj64, kkt64])."""
    import torch
    if not isinstance(image, torch.Tensor) or not image.is_cuda or image.dim() != 3:
        raise ValueError("device tensor [C, H, W] required")
    C, H, W = image.shape
    _need(image, torch.float32, (C, H, W), "image")
    if not image.is_contiguous():
        raise ValueError("image must be contiguous [C, H, W]")
    c = ctx or _ctx(image.device)
    dev = image.device
    res = out or {}
    o_img = res.get("out")
    if o_img is None:
        o_img = torch.empty((C, H, W), dtype=torch.float32, device=dev)
    used = res.get("iters_used")
    if used is None:
        used = torch.empty((H, W), dtype=torch.int32, device=dev)
    resid = res.get("residual")
    if resid is None:
        resid = torch.empty((H, W), dtype=torch.float32, device=dev)
    obj = kkt = None
    if fp64_check:
        obj = torch.empty((H, W), dtype=torch.float64, device=dev)
        kkt = torch.empty((H, W), dtype=torch.float64, device=dev)
    o = _options(tol, check_every, PREC_FP32, init, fp64_check)
    _check(load_library().nlem_denoise_color(c.handle, _ptr(image), H, W, W, C, int(patch), int(window), float(h),
                                             float(rho), int(iters), _Box(*box), ctypes.byref(o), _ptr(o_img),
                                             _ptr(used), _ptr(resid), _ptr(obj), _ptr(kkt), _stream(dev)))
    r = dict(out=o_img, iters_used=used, residual=resid)
    if fp64_check:
        r.update(obj64=obj, kkt64=kkt)
    return r


def nlem_denoise_host(image, patch=7, window=21, h=200.0, rho=1.0, iters=100, box=(0.0, 255.0), tol=0.0,
                      check_every=1, precision=PREC_FP32, init=INIT_WEIGHTED_MEAN, ctx: Context | None = None,
                      out=None, iters_used=None, device=0, solver=SOLVER_ADMM, irls_eps=1e-6, penalty=PENALTY_UNIFORM,
                      restart_every=0):
    """NLEM on HOST buffers (numpy float32 [H, W] or CPU torch tensor, ideally pinned):
    copies in, denoises and copies out inside the library.  Returns the host output."""
    import numpy as np
    import torch
    if isinstance(image, np.ndarray):
        img_t = torch.from_numpy(np.ascontiguousarray(image, dtype=np.float32))
    else:
        img_t = image.contiguous()
    if img_t.is_cuda or img_t.dtype != torch.float32:
        raise ValueError("host float32 image required")
    H, W = img_t.shape
    c = ctx or _ctx(torch.device("cuda", device))
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, pin_memory=img_t.is_pinned())
    o = _options(tol, check_every, precision, init, solver=solver, irls_eps=irls_eps, penalty=penalty,
                 restart_every=restart_every)
    ip = ctypes.c_void_p(iters_used.data_ptr()) if iters_used is not None else None
    _check(load_library().nlem_denoise_host(c.handle, ctypes.c_void_p(img_t.data_ptr()), H, W, int(patch),
                                            int(window), float(h), float(rho), int(iters), _Box(*box),
                                            ctypes.byref(o), ctypes.c_void_p(out.data_ptr()), ip,
                                            _stream(torch.device("cuda", c.device))))
    return out


def nlem_fp32_peak(ctx: Context | None = None):
    """Measured FP32 FMA throughput (TFLOP/s) and SM count of the context's device."""
    import torch
    c = ctx or _ctx(torch.device("cuda", torch.cuda.current_device()))
    tf = ctypes.c_double()
    sms = ctypes.c_int()
    _check(load_library().nlem_fp32_peak(c.handle, ctypes.byref(tf), ctypes.byref(sms)))
    return tf.value, sms.value


def nlem_denoise_batch(images, patches, windows, hs, rho=1.0, iters=100, box=(0.0, 255.0), tol=0.0, check_every=1,
                       init=INIT_WEIGHTED_MEAN, ctx: Context | None = None, outs=None, solver=SOLVER_ADMM,
                       restart_every=0):
    """NLEM on a list of float32 CUDA images of uneven sizes in one persistent launch
    (CUDA-graph replayed).  patches, windows, hs: per-image patch size, window size and h.
    solver: SOLVER_ADMM (Algorithm 1) or SOLVER_FAST (accelerated EM-ADMM; restart_every as for
    em_solve_batch).  Returns a list of dicts (out, iters_used, residual), one per image."""
    import torch
    n = len(images)
    if not (len(patches) == len(windows) == len(hs) == n):
        raise ValueError("one patch, window and h per image")
    c = ctx or _ctx(images[0].device)
    dev = images[0].device
    if outs is None:
        outs = [dict(out=torch.empty(im.shape, dtype=torch.float32, device=dev),
                     iters_used=torch.empty(im.shape, dtype=torch.int32, device=dev),
                     residual=torch.empty(im.shape, dtype=torch.float32, device=dev)) for im in images]
    descs = (_ImageDesc * n)()
    for k, im in enumerate(images):
        _need(im, torch.float32, tuple(im.shape), f"images[{k}]")
        H, W = im.shape
        d = descs[k]
        ip, pitch = _image(im)
        d.image = ip.value
        d.out = _ptr(outs[k]["out"]).value
        d.iters_used = _ptr(outs[k]["iters_used"]).value if outs[k].get("iters_used") is not None else None
        d.residual = _ptr(outs[k]["residual"]).value if outs[k].get("residual") is not None else None
        d.H, d.W, d.pitch = H, W, pitch
        d.patch, d.window, d.h = int(patches[k]), int(windows[k]), float(hs[k])
    o = _options(tol, check_every, PREC_FP32, init, solver=solver, restart_every=restart_every)
    _check(load_library().nlem_denoise_batch(c.handle, descs, n, float(rho), int(iters), _Box(*box), ctypes.byref(o),
                                             _stream(dev)))
    return outs


def nlem_batch_config(ctx: Context | None = None) -> str:
    """Launch shape the autotuner chose for the last batch on this context."""
    import torch
    c = ctx or _ctx(torch.device("cuda", torch.cuda.current_device()))
    buf = ctypes.create_string_buffer(512)
    _check(load_library().nlem_batch_config(c.handle, buf, 512))
    return buf.value.decode()


def nlem_denoise_batch_noalloc(images, patches, windows, hs, outs, rho=1.0, iters=100, box=(0.0, 255.0), tol=0.0,
                               check_every=1, init=INIT_WEIGHTED_MEAN, solver=SOLVER_ADMM, restart_every=0):
    """nlem_denoise_batch without any device allocation: the caller supplies every output
    buffer (`outs`: one dict per image with out [H,W] and optionally iters_used, residual);
    the library uses its own fixed scratch array.  At most 256 images per call; calls whose GPU
    work overlaps must not run concurrently (they share that array).  solver and restart_every
    as for nlem_denoise_batch."""
    import torch
    n = len(images)
    if not (len(patches) == len(windows) == len(hs) == len(outs) == n):
        raise ValueError("one patch, window, h and output dict per image")
    dev = images[0].device if n else torch.device("cuda", torch.cuda.current_device())
    for k in range(n):
        for t in (images[k], outs[k]["out"], outs[k].get("iters_used"), outs[k].get("residual")):
            if t is not None and t.device != dev:
                raise ValueError(f"image {k}: every image and output must be on {dev}")
    descs = (_ImageDesc * n)()
    for k, im in enumerate(images):
        _need(im, torch.float32, tuple(im.shape), f"images[{k}]")
        H, W = im.shape
        d = descs[k]
        ip, pitch = _image(im)
        d.image = ip.value
        d.out = _ptr(outs[k]["out"]).value
        d.iters_used = _ptr(outs[k]["iters_used"]).value if outs[k].get("iters_used") is not None else None
        d.residual = _ptr(outs[k]["residual"]).value if outs[k].get("residual") is not None else None
        d.H, d.W, d.pitch = H, W, pitch
        d.patch, d.window, d.h = int(patches[k]), int(windows[k]), float(hs[k])
    o = _options(tol, check_every, PREC_FP32, init, solver=solver, restart_every=restart_every)
    with torch.cuda.device(dev):   # the library runs on the current device: make it the images'
        _check(load_library().nlem_denoise_batch_noalloc(descs, n, float(rho), int(iters), _Box(*box),
                                                         ctypes.byref(o), _stream(dev)))
    return outs


def nlem_batch_force_config(variant, fetch=1, ctas_per_sm=2, ctx: Context | None = None):
    """Pin the batched launch's shape (variant 0 or 1, see include/nlem.h); variant -1 restores
    the autotuner."""
    import torch
    c = ctx or _ctx(torch.device("cuda", torch.cuda.current_device()))
    _check(load_library().nlem_batch_force_config(c.handle, int(variant), int(fetch), int(ctas_per_sm)))


def nlem_debug_status(reset=True):
    """The debug build's bounds-check record (include/nlem.h): dict(count, site, index, limit);
    raises NlemError (-5) in the release build."""
    site, idx, lim, cnt = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(load_library().nlem_debug_status(1 if reset else 0, ctypes.byref(site), ctypes.byref(idx), ctypes.byref(lim),
                                            ctypes.byref(cnt)))
    return dict(count=cnt.value, site=site.value, index=idx.value, limit=lim.value)


def nlem_device_status(ctx: Context | None = None) -> int:
    """Synchronize and raise NlemError if a kernel reported a bounded-wait timeout."""
    import torch
    c = ctx or _ctx(torch.device("cuda", torch.cuda.current_device()))
    return _check(load_library().nlem_device_status(c.handle))


def nlem_selftest_timeout(ctx: Context | None = None) -> int:
    """Run the bounded-wait self-test (include/nlem.h) and return its status code: NLEM_ERR_TIMEOUT
    (-4) when the timeout path works."""
    import torch
    c = ctx or _ctx(torch.device("cuda", torch.cuda.current_device()))
    return int(load_library().nlem_selftest_timeout(c.handle))


def nlem_bf16_weights(image, patch=9, window=21, h=300.0, ctx: Context | None = None, out=None):
    """Mixed-precision weight table [H*W, window^2] of a float32 CUDA image (tensor-core cross
    terms); entries past a pixel's clipped window size are left as they were in `out`."""
    import torch
    H, W = image.shape
    _need(image, torch.float32, (H, W), "image")
    c = ctx or _ctx(image.device)
    if out is None:
        out = torch.full((H * W, window * window), float("nan"), dtype=torch.float32, device=image.device)
    ip, pitch = _image(image)
    _check(load_library().nlem_bf16_weights(c.handle, ip, H, W, pitch, int(patch), int(window), float(h),
                                            _ptr(out), _stream(image.device)))
    return out


class WarmStart:
    """Learned warm-start model (include/nlem.h: nlem_ws_*) on the context's device."""

    def __init__(self, d, nref=441.0, seed=1, ctx: Context | None = None):
        import torch
        self.ctx = ctx or _ctx(torch.device("cuda", torch.cuda.current_device()))
        self.d = int(d)
        h = ctypes.c_void_p()
        _check(load_library().nlem_ws_create(self.ctx.handle, self.d, float(nref), int(seed), ctypes.byref(h)))
        self.handle = h
        self.num_params = int(load_library().nlem_ws_num_params(self.d))

    def close(self):
        if getattr(self, "handle", None):
            load_library().nlem_ws_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        import numpy as np
        out = np.empty(self.num_params, dtype=np.float32)
        _check(load_library().nlem_ws_get_params(self.handle, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters")
        _check(load_library().nlem_ws_set_params(self.handle, p.ctypes.data_as(ctypes.c_void_p)))

    def save(self, path):
        _check(load_library().nlem_ws_save(self.handle, str(path).encode()))

    def load(self, path):
        _check(load_library().nlem_ws_load(self.handle, str(path).encode()))

    def forward(self, feats):
        import torch
        B = feats.shape[0]
        y = torch.empty((B, self.d + 1), dtype=torch.float32, device=feats.device)
        _check(load_library().nlem_ws_forward(self.ctx.handle, self.handle, _ptr(feats), B, _ptr(y),
                                              _stream(feats.device)))
        return y

    def loss_grad(self, feats, targets):
        import torch
        B = feats.shape[0]
        loss = torch.zeros(1, dtype=torch.float32, device=feats.device)
        grad = torch.empty(self.num_params, dtype=torch.float32, device=feats.device)
        _check(load_library().nlem_ws_loss_grad(self.ctx.handle, self.handle, _ptr(feats), _ptr(targets), B,
                                                _ptr(loss), _ptr(grad), _stream(feats.device)))
        return loss, grad

    def train_step(self, feats, targets, lr, loss=None):
        B = feats.shape[0]
        _check(load_library().nlem_ws_train_step(self.ctx.handle, self.handle, _ptr(feats), _ptr(targets), B,
                                                 float(lr), _ptr(loss), _stream(feats.device)))

    def train(self, feats, targets, epochs, batch, lr, seed=0):
        """`epochs` shuffled passes of minibatch Adam over the whole set (nlem_ws_train);
        returns the mean minibatch loss of each epoch."""
        import numpy as np
        N = feats.shape[0]
        hist = np.zeros(max(int(epochs), 1), dtype=np.float32)
        _check(load_library().nlem_ws_train(self.ctx.handle, self.handle, _ptr(feats), _ptr(targets), N, int(epochs),
                                            int(batch), float(lr), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                            hist.ctypes.data_as(ctypes.c_void_p), _stream(feats.device)))
        return [float(x) for x in hist[:int(epochs)]]

    def predict(self, feats, box=(0.0, 255.0)):
        import torch
        B = feats.shape[0]
        dev = feats.device
        y = torch.empty((B, self.d + 1), dtype=torch.float32, device=dev)
        x0 = torch.empty((B, self.d), dtype=torch.float32, device=dev)
        rho = torch.empty(B, dtype=torch.float32, device=dev)
        _check(load_library().nlem_ws_predict(self.ctx.handle, self.handle, _ptr(feats), B, _Box(*box), _ptr(y),
                                              _ptr(x0), _ptr(rho), _stream(dev)))
        return y, x0, rho


def nlem_features(image, patch=7, window=21, h=200.0, pixels=None, ctx: Context | None = None):
    """Warm-start features [npix, 2d+2] of the listed pixels' NLEM problems (all if None)."""
    import torch
    H, W = image.shape
    c = ctx or _ctx(image.device)
    n = pixels.numel() if pixels is not None else H * W
    d = patch * patch
    feats = torch.empty((n, 2 * d + 2), dtype=torch.float32, device=image.device)
    if pixels is not None:
        _need(pixels, torch.int32, (n,), "pixels")
    ip, pitch = _image(image)
    _check(load_library().nlem_features(c.handle, ip, H, W, pitch, int(patch), int(window), float(h),
                                        _ptr(pixels), n, _ptr(feats), _stream(image.device)))
    return feats


def nlem_ws_labels(image, pixels, feats, rho_grid, patch=7, window=21, h=200.0, box=(0.0, 255.0), tol=1e-4,
                   check_every=5, cap=300, tight_tol=1e-6, tight_cap=2000, ctx: Context | None = None, targets=None):
    """Warm-start training labels of the listed pixels (int32 CUDA [n]) of a float32 CUDA image,
    computed in the library (include/nlem.h).  Returns (targets [n, d+1] CUDA, counts per grid
    penalty as a list)."""
    import torch
    H, W = image.shape
    c = ctx or _ctx(image.device)
    n = pixels.numel()
    d = patch * patch
    _need(pixels, torch.int32, (n,), "pixels")
    _need(feats, torch.float32, (n, 2 * d + 2), "feats")
    if targets is None:
        targets = torch.empty((n, d + 1), dtype=torch.float32, device=image.device)
    grid = (ctypes.c_float * len(rho_grid))(*[float(r) for r in rho_grid])
    counts = (ctypes.c_longlong * len(rho_grid))()
    ip, pitch = _image(image)
    _check(load_library().nlem_ws_labels(c.handle, ip, H, W, pitch, int(patch), int(window), float(h), _Box(*box),
                                         _ptr(pixels), n, grid, len(rho_grid), float(tol), int(check_every), int(cap),
                                         float(tight_tol), int(tight_cap), _ptr(feats), _ptr(targets), counts,
                                         _stream(image.device)))
    return targets, list(counts)


def nlem_denoise_ex(image, patch=7, window=21, h=200.0, rho=1.0, iters=100, box=(0.0, 255.0), tol=0.0, check_every=1,
                    init=INIT_WEIGHTED_MEAN, pixels=None, x0=None, rho_pix=None, z_out=False, ctx: Context | None = None,
                    out=None, penalty=PENALTY_UNIFORM, solver=SOLVER_ADMM, restart_every=0):
    """NLEM on a pixel list with optional per-pixel start points / penalties (indexed by
    linear pixel) and the full solution patches; solver SOLVER_ADMM or SOLVER_FAST.  Returns
    dict(out, iters_used, residual[, z])."""
    import torch
    H, W = image.shape
    c = ctx or _ctx(image.device)
    dev = image.device
    d = patch * patch
    res = out or {}
    o = res.get("out")
    if o is None:
        o = torch.zeros((H, W), dtype=torch.float32, device=dev)
    used = res.get("iters_used")
    if used is None:
        used = torch.zeros((H, W), dtype=torch.int32, device=dev)
    resid = res.get("residual")
    if resid is None:
        resid = torch.zeros((H, W), dtype=torch.float32, device=dev)
    z = None
    if z_out:
        z = res.get("z")
        if z is None:
            z = torch.zeros((H * W, d), dtype=torch.float32, device=dev)
    n = pixels.numel() if pixels is not None else 0
    opts = _options(tol, check_every, PREC_FP32, init, penalty=penalty, solver=solver, restart_every=restart_every)
    ip, pitch = _image(image)
    _check(load_library().nlem_denoise_ex(c.handle, ip, H, W, pitch, int(patch), int(window), float(h), float(rho),
                                          int(iters), _Box(*box), ctypes.byref(opts), _ptr(pixels), n, _ptr(x0),
                                          _ptr(rho_pix), _ptr(o), _ptr(used), _ptr(resid), _ptr(z), _stream(dev)))
    r = dict(out=o, iters_used=used, residual=resid)
    if z_out:
        r["z"] = z
    return r


def nlem_denoise_warm(ws: WarmStart, image, patch=7, window=21, h=200.0, rho_fallback=1.0, iters=300,
                      box=(0.0, 255.0), tol=1e-4, check_every=10, count_fallback=True, ctx: Context | None = None,
                      out=None):
    """NLEM with the learned warm start and plain-ADMM fallback.  Returns dict(out,
    iters_used, fallback) (fallback = pixels solved again, or None if not counted)."""
    import torch
    H, W = image.shape
    c = ctx or ws.ctx
    dev = image.device
    res = out or {}
    o = res.get("out")
    if o is None:
        o = torch.empty((H, W), dtype=torch.float32, device=dev)
    used = res.get("iters_used")
    if used is None:
        used = torch.empty((H, W), dtype=torch.int32, device=dev)
    opts = _options(tol, check_every, PREC_FP32, INIT_WEIGHTED_MEAN)
    fb = ctypes.c_longlong(-1)
    ip, pitch = _image(image)
    _check(load_library().nlem_denoise_warm(c.handle, ws.handle, ip, H, W, pitch, int(patch), int(window), float(h),
                                            float(rho_fallback), int(iters), _Box(*box), ctypes.byref(opts), _ptr(o),
                                            _ptr(used), ctypes.byref(fb) if count_fallback else None, _stream(dev)))
    return dict(out=o, iters_used=used, fallback=int(fb.value) if count_fallback else None)
