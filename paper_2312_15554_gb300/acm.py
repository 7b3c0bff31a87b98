"""Thin Python binding of the ACM C ABI (include/acm.h).

Argument marshalling only: every step of the method runs inside libacm.so. The
names mirror the C entry points. Array arguments may be torch tensors (CUDA or
CPU, contiguous) or numpy arrays (host memory); scalars and reports are Python
values. The library is loaded lazily and a missing or unloadable build raises
immediately: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB = None
_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libacm.so")

ACM_OK = 0
ACM_ERR_MAXITER = -4
DERIV_EXACT, DERIV_CENTRAL = 0, 1
FP32, FP64, FP32_THEN_FP64 = 0, 1, 2

EXPORTED = (
    "acm_stokes_default_params", "acm_advdiff_default_params", "acm_create", "acm_destroy",
    "acm_stokes", "acm_stokes_tensor", "acm_advdiff", "acm_advdiff_tensor",
    "acm_fft_r2c", "acm_fft_c2r", "acm_fft_r2c_static", "acm_history",
    "acm_batch_create", "acm_batch_destroy", "acm_batch_stokes", "acm_batch_profile_enable",
    "acm_batch_profile_read", "acm_autotune", "acm_set_tiles", "acm_get_tiles", "acm_batch_autotune", "acm_batch_tiles",
    "acm_batch_history_enable", "acm_batch_history", "acm_fno_create", "acm_fno_destroy", "acm_fno_num_params", "acm_fno_set_params",
    "acm_fno_get_params", "acm_fno_forward", "acm_fno_warm_start", "acm_fno_backward", "acm_fno_adamw", "acm_profile_enable", "acm_profile_read", "acm_last_error", "acm_status_str",
)

KERNEL_KINDS = ("x_stokes_local", "x_stokes_rhs", "y_fwd_stokes", "z_stokes", "y_inv_stokes", "x_solute",
                "y_fwd_solute", "z_solute", "y_inv_solute", "finalize", "other")


class acm_stokes_params(C.Structure):
    _fields_ = [("nu", C.c_double), ("eps", C.c_double), ("alpha0", C.c_double), ("beta0", C.c_double),
                ("b0", C.c_double), ("phi", C.c_double * 3), ("tau", C.c_double * 3),
                ("psi_min_frac", C.c_double), ("eps32", C.c_double), ("max_iter", C.c_int),
                ("adaptive", C.c_int), ("deriv", C.c_int), ("precision", C.c_int), ("check_every", C.c_int),
                ("device_loop", C.c_int), ("pore_scale", C.c_double)]


class acm_advdiff_params(C.Structure):
    _fields_ = [("eta", C.c_double), ("A0", C.c_double), ("B0", C.c_double * 3), ("B0_explicit", C.c_int),
                ("eps", C.c_double), ("max_iter", C.c_int), ("deriv", C.c_int), ("precision", C.c_int),
                ("check_every", C.c_int), ("device_loop", C.c_int)]


class acm_report(C.Structure):
    _fields_ = [("iters", C.c_int), ("iters_fp64", C.c_int), ("converged", C.c_int), ("status", C.c_int),
                ("res", C.c_double * 6), ("tol", C.c_double * 6), ("psi", C.c_double * 3),
                ("time_ms", C.c_double)]

    def as_dict(self):
        return {"iters": self.iters, "iters_fp64": self.iters_fp64, "converged": bool(self.converged),
                "status": self.status, "res": list(self.res), "tol": list(self.tol), "psi": list(self.psi),
                "time_ms": self.time_ms}


class AcmError(RuntimeError):
    def __init__(self, status: int, where: str):
        detail = ""
        if status == -3:
            detail = " [" + load().acm_last_error().decode(errors="replace") + "]"
        super().__init__(f"{where}: {status_str(status)} ({status}){detail}")
        self.status = status


def load(path: str = None):
    """Load libacm.so; raises if it has not been built or cannot be loaded."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libacm.so not built at {path}: run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, cp, dp, ip = C.c_void_p, C.c_char_p, C.POINTER(C.c_double), C.c_int
    lib.acm_stokes_default_params.argtypes = [C.POINTER(acm_stokes_params)]
    lib.acm_advdiff_default_params.argtypes = [C.POINTER(acm_advdiff_params)]
    lib.acm_create.argtypes = [C.POINTER(vp), ip, ip, ip, vp]
    lib.acm_destroy.argtypes = [vp]
    lib.acm_stokes.argtypes = [vp, vp, dp, C.POINTER(acm_stokes_params), vp, vp, vp, vp, vp, dp,
                               C.POINTER(acm_report)]
    lib.acm_stokes_tensor.argtypes = [vp, vp, C.POINTER(acm_stokes_params), vp, dp, dp, C.POINTER(acm_report)]
    lib.acm_advdiff.argtypes = [vp, vp, vp, C.c_double, dp, C.POINTER(acm_advdiff_params), vp, vp, dp, dp,
                                C.POINTER(acm_report)]
    lib.acm_advdiff_tensor.argtypes = [vp, vp, vp, C.c_double, C.POINTER(acm_advdiff_params), vp, dp, dp,
                                       C.POINTER(acm_report)]
    lib.acm_fft_r2c.argtypes = [vp, ip, ip, vp, vp]
    lib.acm_fft_c2r.argtypes = [vp, ip, ip, vp, vp]
    lib.acm_fft_r2c_static.argtypes = [ip, ip, ip, ip, vp, vp, vp]
    lib.acm_batch_create.argtypes = [C.POINTER(vp), ip, C.POINTER(C.c_int), vp]
    lib.acm_batch_destroy.argtypes = [vp]
    lib.acm_batch_stokes.argtypes = [vp, C.POINTER(vp), C.POINTER(acm_stokes_params), C.POINTER(vp),
                                     C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), dp, C.POINTER(acm_report)]
    i5 = C.POINTER(C.c_int)
    lib.acm_autotune.argtypes = [vp, ip, ip, i5]
    lib.acm_set_tiles.argtypes = [vp, ip, i5]
    lib.acm_get_tiles.argtypes = [vp, ip, i5]
    lib.acm_batch_autotune.argtypes = [vp, ip, ip]
    lib.acm_batch_tiles.argtypes = [vp, ip, ip, i5]
    lib.acm_batch_history_enable.argtypes = [vp, ip]
    lib.acm_batch_history.argtypes = [vp, ip, ip, dp, ip, C.POINTER(C.c_int)]
    lib.acm_batch_profile_enable.argtypes = [vp, ip]
    lib.acm_batch_profile_read.argtypes = [vp, dp, C.POINTER(C.c_longlong)]
    fp = C.POINTER(C.c_float)
    lib.acm_fno_create.argtypes = [C.POINTER(vp), ip, ip, ip, ip, ip, ip, ip, vp]
    lib.acm_fno_destroy.argtypes = [vp]
    lib.acm_fno_num_params.argtypes = [vp, C.POINTER(C.c_longlong)]
    lib.acm_fno_set_params.argtypes = [vp, vp]
    lib.acm_fno_get_params.argtypes = [vp, vp]
    lib.acm_fno_forward.argtypes = [vp, ip, vp, vp]
    lib.acm_fno_warm_start.argtypes = [vp, ip, vp, vp, vp]
    lib.acm_fno_backward.argtypes = [vp, ip, vp, vp, dp, vp]
    lib.acm_fno_adamw.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]
    lib.acm_history.argtypes = [vp, ip, dp, ip, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.acm_profile_enable.argtypes = [vp, ip]
    lib.acm_profile_read.argtypes = [vp, dp, C.POINTER(C.c_longlong)]
    lib.acm_last_error.argtypes = []
    lib.acm_last_error.restype = cp
    lib.acm_status_str.argtypes = [ip]
    lib.acm_status_str.restype = cp
    for name in EXPORTED:
        if name not in ("acm_status_str", "acm_last_error"):
            getattr(lib, name).restype = C.c_int
    _LIB = lib
    return lib


def status_str(s: int) -> str:
    return load().acm_status_str(int(s)).decode()


def _check(s: int, where: str, allow_maxiter: bool = False):
    if s == ACM_OK or (allow_maxiter and s == ACM_ERR_MAXITER):
        return s
    raise AcmError(s, where)


def _ptr(x):
    """Raw address of a contiguous torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _dvec(v, n=3):
    return (C.c_double * n)(*[float(a) for a in v])


def stokes_params(**kw) -> acm_stokes_params:
    p = acm_stokes_params()
    load().acm_stokes_default_params(C.byref(p))
    for k, v in kw.items():
        if k in ("phi", "tau"):
            setattr(p, k, (C.c_double * 3)(*v))
        else:
            setattr(p, k, v)
    return p


def advdiff_params(**kw) -> acm_advdiff_params:
    p = acm_advdiff_params()
    load().acm_advdiff_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "B0":
            p.B0 = (C.c_double * 3)(*v)
            p.B0_explicit = 1
        else:
            setattr(p, k, v)
    return p


class acm_ctx:
    """Owns an acm_ctx* for grids of shape (n0, n1, n2) on a CUDA stream (handle or 0)."""

    def __init__(self, shape, stream: int = 0):
        lib = load()
        self.shape = tuple(int(s) for s in shape)
        h = C.c_void_p()
        _check(lib.acm_create(C.byref(h), *self.shape, C.c_void_p(stream)), "acm_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().acm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def acm_create(shape, stream: int = 0) -> acm_ctx:
    return acm_ctx(shape, stream)


def acm_destroy(ctx: acm_ctx):
    ctx.close()


def acm_stokes(ctx, H, g, params=None, init_u=None, init_lambda=None, u=None, p=None, lam=None):
    """acm_stokes: returns (status, K_col, report); fields are written into u, p, lam."""
    K = (C.c_double * 3)()
    rep = acm_report()
    s = load().acm_stokes(ctx.h, _ptr(H), _dvec(g), C.byref(params or stokes_params()), _ptr(init_u),
                          _ptr(init_lambda), _ptr(u), _ptr(p), _ptr(lam), K, C.byref(rep))
    _check(s, "acm_stokes", allow_maxiter=True)
    return s, np.array(K[:]), rep


def acm_stokes_tensor(ctx, H, params=None, u3=None, grad_form=False):
    K = (C.c_double * 9)()
    Kg = (C.c_double * 9)() if grad_form else None
    reps = (acm_report * 3)()
    s = load().acm_stokes_tensor(ctx.h, _ptr(H), C.byref(params or stokes_params()), _ptr(u3), K,
                                 Kg, reps)
    _check(s, "acm_stokes_tensor", allow_maxiter=True)
    return s, np.array(K[:]).reshape(3, 3), (np.array(Kg[:]).reshape(3, 3) if grad_form else None), list(reps)


def acm_advdiff(ctx, H, u, Pe, g_chi, params=None, chi=None, grad_chi=None):
    Dg = (C.c_double * 3)()
    Dx = (C.c_double * 3)()
    rep = acm_report()
    s = load().acm_advdiff(ctx.h, _ptr(H), _ptr(u), float(Pe), _dvec(g_chi), C.byref(params or advdiff_params()),
                           _ptr(chi), _ptr(grad_chi), Dg, Dx, C.byref(rep))
    _check(s, "acm_advdiff", allow_maxiter=True)
    return s, np.array(Dg[:]), np.array(Dx[:]), rep


def acm_advdiff_tensor(ctx, H, u, Pe, params=None, chi3=None):
    D = (C.c_double * 9)()
    Dx = (C.c_double * 9)()
    reps = (acm_report * 3)()
    s = load().acm_advdiff_tensor(ctx.h, _ptr(H), _ptr(u), float(Pe), C.byref(params or advdiff_params()),
                                  _ptr(chi3), D, Dx, reps)
    _check(s, "acm_advdiff_tensor", allow_maxiter=True)
    return s, np.array(D[:]).reshape(3, 3), np.array(Dx[:]).reshape(3, 3), list(reps)


def acm_fft_r2c(ctx, x, out, fp64: bool, nbatch: int = 1):
    _check(load().acm_fft_r2c(ctx.h, int(fp64), nbatch, _ptr(x), _ptr(out)), "acm_fft_r2c")


def acm_fft_c2r(ctx, x, out, fp64: bool, nbatch: int = 1):
    _check(load().acm_fft_c2r(ctx.h, int(fp64), nbatch, _ptr(x), _ptr(out)), "acm_fft_c2r")


def acm_profile_enable(ctx, on: bool = True):
    _check(load().acm_profile_enable(ctx.h, int(bool(on))), "acm_profile_enable")


def acm_profile_read(ctx):
    """Per kernel kind: (device ms, launches) since the previous read."""
    n = len(KERNEL_KINDS)
    ms = (C.c_double * n)()
    cnt = (C.c_longlong * n)()
    _check(load().acm_profile_read(ctx.h, ms, cnt), "acm_profile_read")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


def acm_history(ctx, index: int = 0, cap: int = 20000):
    """Per-iteration records of the last solve: numpy array (iterations, record length)."""
    n = C.c_int()
    ln = C.c_int()
    _check(load().acm_history(ctx.h, int(index), None, 0, C.byref(n), C.byref(ln)), "acm_history")
    k = min(cap, n.value)
    if k == 0 or ln.value == 0:
        return np.zeros((0, max(ln.value, 1)))
    buf = (C.c_double * (k * ln.value))()
    _check(load().acm_history(ctx.h, int(index), buf, k, C.byref(n), C.byref(ln)), "acm_history")
    return np.array(buf[:]).reshape(k, ln.value)


def acm_fft_r2c_static(x, out, fp64: bool, stream: int = None):
    """The allocation-free transform (no context; device buffers only).

    x: real [n0][n1][n2] (float64 when fp64, else float32); out: [n0][n1][n2/2 + 1][2]
    of the same dtype. The C side cannot see buffer sizes or dtypes, so they are
    checked here; stream defaults to torch's current stream of x's device.
    """
    fp64 = bool(fp64)
    want = "float64" if fp64 else "float32"
    for name, t in (("x", x), ("out", out)):
        if not hasattr(t, "data_ptr") or not hasattr(t, "is_cuda"):
            raise ValueError(f"{name} must be a torch tensor")
        if str(t.dtype).replace("torch.", "") != want:
            raise ValueError(f"{name} must be {want} for fp64={fp64}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if x.dim() != 3:
        raise ValueError("x must be a 3-D real field [n0][n1][n2]")
    n0, n1, n2 = (int(s) for s in x.shape)
    if tuple(out.shape) != (n0, n1, n2 // 2 + 1, 2):
        raise ValueError(f"out must have shape {(n0, n1, n2 // 2 + 1, 2)}, got {tuple(out.shape)}")
    if x.is_cuda:
        import torch
        cur = torch.cuda.current_device()
        if x.device.index != cur or not out.is_cuda or out.device.index != cur:
            raise ValueError("x and out must be on the current CUDA device")
        if stream is None:
            stream = torch.cuda.current_stream(x.device).cuda_stream
    _check(load().acm_fft_r2c_static(n0, n1, n2, int(fp64), _ptr(x), _ptr(out), C.c_void_p(stream or 0)),
           "acm_fft_r2c_static")


class acm_batch:
    """Owns an acm_batch* for cells of the given shapes (list of (n0, n1, n2))."""

    def __init__(self, shapes, stream: int = 0):
        lib = load()
        self.shapes = [tuple(int(a) for a in sh) for sh in shapes]
        dims = (C.c_int * (3 * len(self.shapes)))(*[a for sh in self.shapes for a in sh])
        h = C.c_void_p()
        _check(lib.acm_batch_create(C.byref(h), len(self.shapes), dims, C.c_void_p(stream)), "acm_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().acm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def acm_batch_stokes(batch, Hs, params=None, u_out=None, init_u=None, init_lambda=None, lambda_out=None):
    """Returns (status, K [ncells, 3, 3], reports [ncells][3]). The optional
    per-cell buffers are [3 loads][3][V] of the solve's real type."""
    n = len(batch.shapes)

    def arr(xs):
        return None if xs is None else (C.c_void_p * n)(*[_ptr(x) for x in xs])
    hp = arr(Hs)
    K = (C.c_double * (9 * n))()
    reps = (acm_report * (3 * n))()
    s = load().acm_batch_stokes(batch.h, hp, C.byref(params or stokes_params()), arr(init_u), arr(init_lambda),
                                arr(u_out), arr(lambda_out), K, reps)
    _check(s, "acm_batch_stokes", allow_maxiter=True)
    return s, np.array(K[:]).reshape(n, 3, 3), [list(reps[3 * i:3 * i + 3]) for i in range(n)]


TILE_PASSES = ("y_fwd_stokes", "z_stokes", "y_inv_stokes", "y_fwd_solute", "z_solute", "y_inv_solute")


def acm_autotune(ctx, fp64: bool = False, deriv: int = DERIV_EXACT):
    """Times the tile widths of the strided passes; returns {pass: width}."""
    t = (C.c_int * 6)()
    _check(load().acm_autotune(ctx.h, int(fp64), int(deriv), t), "acm_autotune")
    return dict(zip(TILE_PASSES, list(t)))


def acm_set_tiles(ctx, tiles, fp64: bool = False):
    """tiles: {pass: width} or six widths in TILE_PASSES order."""
    if isinstance(tiles, dict):
        tiles = [tiles[k] for k in TILE_PASSES]
    t = (C.c_int * 6)(*[int(x) for x in tiles])
    _check(load().acm_set_tiles(ctx.h, int(fp64), t), "acm_set_tiles")


def acm_get_tiles(ctx, fp64: bool = False):
    t = (C.c_int * 6)()
    _check(load().acm_get_tiles(ctx.h, int(fp64), t), "acm_get_tiles")
    return dict(zip(TILE_PASSES, list(t)))


def acm_batch_autotune(batch, fp64: bool = False, deriv: int = DERIV_EXACT):
    _check(load().acm_batch_autotune(batch.h, int(fp64), int(deriv)), "acm_batch_autotune")


def acm_batch_tiles(batch, cell: int, fp64: bool = False):
    t = (C.c_int * 6)()
    _check(load().acm_batch_tiles(batch.h, cell, int(fp64), t), "acm_batch_tiles")
    return dict(zip(TILE_PASSES, list(t)))


def acm_batch_history_enable(batch, cap: int):
    _check(load().acm_batch_history_enable(batch.h, int(cap)), "acm_batch_history_enable")


def acm_batch_history(batch, cell: int, load_index: int):
    """Records (count, 20) of one problem of the last batched solve (see acm_history)."""
    lib = load()
    cnt = C.c_int()
    _check(lib.acm_batch_history(batch.h, cell, load_index, None, 0, C.byref(cnt)), "acm_batch_history")
    out = np.zeros((cnt.value, 20))
    if cnt.value:
        _check(lib.acm_batch_history(batch.h, cell, load_index, out.ctypes.data_as(C.POINTER(C.c_double)),
                                     cnt.value, C.byref(cnt)), "acm_batch_history")
    return out


def acm_batch_profile_enable(batch, on: bool = True):
    _check(load().acm_batch_profile_enable(batch.h, int(bool(on))), "acm_batch_profile_enable")


def acm_batch_profile_read(batch):
    k = len(KERNEL_KINDS)
    ms = (C.c_double * k)()
    cnt = (C.c_longlong * k)()
    _check(load().acm_batch_profile_read(batch.h, ms, cnt), "acm_batch_profile_read")
    return {name: (ms[i], cnt[i]) for i, name in enumerate(KERNEL_KINDS)}


class acm_fno:
    """Owns an acm_fno* (the learned warm start) for grids of one shape."""

    def __init__(self, shape, width=32, modes=12, layers=4, max_batch=4, stream: int = 0):
        lib = load()
        self.shape = tuple(int(a) for a in shape)
        self.width, self.modes, self.layers, self.max_batch = width, modes, layers, max_batch
        h = C.c_void_p()
        _check(lib.acm_fno_create(C.byref(h), *self.shape, width, modes, layers, max_batch, C.c_void_p(stream)),
               "acm_fno_create")
        self.h = h
        n = C.c_longlong()
        _check(lib.acm_fno_num_params(self.h, C.byref(n)), "acm_fno_num_params")
        self.num_params = n.value

    def close(self):
        if getattr(self, "h", None):
            load().acm_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        _check(load().acm_fno_set_params(self.h, _ptr(theta)), "acm_fno_set_params")

    def get_params(self):
        out = np.zeros(self.num_params, np.float32)
        _check(load().acm_fno_get_params(self.h, _ptr(out)), "acm_fno_get_params")
        return out

    def forward(self, H, out, batch=None):
        b = int(batch if batch is not None else H.shape[0])
        _check(load().acm_fno_forward(self.h, b, _ptr(H), _ptr(out)), "acm_fno_forward")

    def warm_start(self, H, init_u, init_lambda, batch=None):
        """Warm starts of the three unit loads, [batch][3][3][V] FP32 on the device."""
        b = int(batch if batch is not None else H.shape[0])
        _check(load().acm_fno_warm_start(self.h, b, _ptr(H), _ptr(init_u), _ptr(init_lambda)),
               "acm_fno_warm_start")

    def backward(self, H, target, grad=None, batch=None):
        b = int(batch if batch is not None else H.shape[0])
        loss = C.c_double()
        _check(load().acm_fno_backward(self.h, b, _ptr(H), _ptr(target), C.byref(loss), _ptr(grad)),
               "acm_fno_backward")
        return loss.value

    def adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4):
        _check(load().acm_fno_adamw(self.h, lr, beta1, beta2, eps, weight_decay), "acm_fno_adamw")
