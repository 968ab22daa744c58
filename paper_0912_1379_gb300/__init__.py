"""Python binding of the GB300 discrete LCT library (include/lct.h).

Argument marshalling only: every function forwards to the native entry point
of the same name in liblct.so (built in-tree by ``_build.build()``); every
step of the transform runs in the library's CUDA kernels.  PyTorch is used
only for device memory and streams.  If liblct.so is missing the import of
any entry point raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import _build

LCT_C64, LCT_C128 = 0, 1
(LCT_PREC_NATIVE, LCT_PREC_SPLIT_BF16, LCT_PREC_SPLIT_FP16, LCT_PREC_FP16, LCT_PREC_PLAIN64,
 LCT_PREC_PLAIN32) = range(6)
STATUS = ["LCT_OK", "LCT_ERR_ARG", "LCT_ERR_N", "LCT_ERR_NOT_SYMPLECTIC", "LCT_ERR_DTYPE",
          "LCT_ERR_ALIGN", "LCT_ERR_OOM", "LCT_ERR_CUDA", "LCT_ERR_DEVICE", "LCT_ERR_TIMEOUT",
          "LCT_ERR_UNSUPPORTED"]

_lib = None
_lock = threading.Lock()


class LctError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__("%s: %s (%s)" % (where, name, _status_string(status)))


def build(force: bool = False) -> str:
    """Compile liblct.so for sm_103a (in-tree)."""
    return _build.build(force=force)


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            raise RuntimeError("liblct.so is not built (call paper_0912_1379_gb300.build()); "
                               "there is no fallback path")
        lib = ctypes.CDLL(_build.LIB)
        i64, f64, vp, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_int64)
        up = ctypes.POINTER(ctypes.c_uint64)
        plan_p = ctypes.POINTER(vp)
        sig = {
            "lct_plan_create": [plan_p, i64, f64, f64, f64, f64, i32],
            "lct_plan_create_complex": [plan_p, i64, dp, i32],
            "lct_plan_create_batch": [plan_p, i64, lp, dp, lp, i32],
            "lct_plan_set_precision": [vp, i32],
            "lct_execute": [vp, vp, vp, i64, vp],
            "lct_execute_host": [vp, vp, vp, i64, vp],
            "lct_partition": [i64, vp, vp, i32, vp, vp],
            "lct_selftest_timeout": [i32, ctypes.c_double, vp],
            "lct_set_debug": [i32],
            "frft_execute": [i64, f64, f64, vp, vp, i64, i32, vp],
            "frft_hermite_execute": [i64, f64, f64, vp, vp, i64, i32, vp],
            "frft_mehler_execute": [i64, f64, f64, vp, vp, i64, i32, vp],
            "frft_hermite_basis": [i64, dp, dp],
            "frft_hermite_status": [vp],
            "lct_transpose": [i32, vp, vp, i64, i64, i64, i64, vp],
            "lct_output_grid": [vp, i64, dp, dp],
            "lct_input_grid": [i64, dp],
            "lct_plan_phase_turns": [vp, i64, up],
            "lct_device_status": [vp, vp],
            "lct_plan_destroy": [vp],
            "lct_execute_noalloc": [i64, f64, f64, f64, f64, i32, vp, vp, i64, vp],
            "lct_plan_set_variant": [vp, i32],
            "lct_plan_get_variant": [vp, ctypes.POINTER(i32)],
            "lct_plan_autotune": [vp, vp, vp, i64, vp],
            "lct_backward": [vp, vp, vp, vp, vp, vp, i64, vp],
            "lct2d_plan_create": [plan_p, i64, i64, dp, dp, i32],
            "lct2d_execute": [vp, vp, vp, vp, i64, vp],
            "lct2d_backward": [vp, vp, vp, vp, vp, vp, vp, vp, i64, vp],
            "lct2d_plan_destroy": [vp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = i32
        lib.lct_status_string.argtypes = [i32]
        lib.lct_status_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _status_string(status: int) -> str:
    try:
        return _load().lct_status_string(status).decode()
    except Exception:  # library not loadable while formatting an error
        return "?"


def _check(status: int, where: str):
    if status != 0:
        raise LctError(status, where)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    return t.data_ptr()


def dtype_code(torch_dtype) -> int:
    import torch
    if torch_dtype == torch.complex64:
        return LCT_C64
    if torch_dtype == torch.complex128:
        return LCT_C128
    raise TypeError("samples must be complex64 or complex128, got %s" % (torch_dtype,))


# ---------------------------------------------------------------------------
# entry points (same names as include/lct.h)
# ---------------------------------------------------------------------------
def lct_plan_create(N: int, a: float, b: float, c: float, d: float, dtype: int = LCT_C64) -> int:
    h = ctypes.c_void_p()
    _check(_load().lct_plan_create(ctypes.byref(h), N, a, b, c, d, dtype), "lct_plan_create")
    return h.value


def lct_plan_create_complex(N: int, abcd, dtype: int = LCT_C64) -> int:
    p = np.ascontiguousarray(np.asarray(abcd, dtype=np.complex128).view(np.float64))
    if p.shape != (8,):
        raise ValueError("abcd must hold 4 complex values")
    h = ctypes.c_void_p()
    _check(_load().lct_plan_create_complex(ctypes.byref(h), N,
                                           p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           dtype), "lct_plan_create_complex")
    return h.value


def lct_plan_create_batch(N, abcd, offsets, dtype: int = LCT_C64) -> int:
    Ns = np.ascontiguousarray(np.asarray(N, dtype=np.int64))
    p = np.ascontiguousarray(np.asarray(abcd, dtype=np.complex128).reshape(len(Ns), 4)
                             .view(np.float64).reshape(-1))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    if off.shape != Ns.shape:
        raise ValueError("offsets must have one entry per signal")
    h = ctypes.c_void_p()
    lp = ctypes.POINTER(ctypes.c_int64)
    _check(_load().lct_plan_create_batch(ctypes.byref(h), len(Ns), Ns.ctypes.data_as(lp),
                                         p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         off.ctypes.data_as(lp), dtype), "lct_plan_create_batch")
    return h.value


def lct_plan_set_precision(plan: int, precision: int) -> None:
    _check(_load().lct_plan_set_precision(plan, precision), "lct_plan_set_precision")


def lct_plan_set_variant(plan: int, variant: int) -> None:
    _check(_load().lct_plan_set_variant(plan, variant), "lct_plan_set_variant")


def lct_plan_get_variant(plan: int) -> int:
    v = ctypes.c_int()
    _check(_load().lct_plan_get_variant(plan, ctypes.byref(v)), "lct_plan_get_variant")
    return v.value


def lct_plan_autotune(plan: int, inp, out, batch: int, stream=None) -> int:
    """Time the kernel variants on these buffers; returns the chosen one."""
    _check(_load().lct_plan_autotune(plan, _ptr(inp), _ptr(out), batch, _stream_handle(stream)),
           "lct_plan_autotune")
    return lct_plan_get_variant(plan)


def lct_execute(plan: int, inp, out, batch: int, stream=None) -> None:
    _check(_load().lct_execute(plan, _ptr(inp), _ptr(out), batch, _stream_handle(stream)),
           "lct_execute")


def lct_set_debug(on: bool) -> None:
    """Debug mode: synchronous output scan and status check after each
    lct_execute (see include/lct.h)."""
    _check(_load().lct_set_debug(1 if on else 0), "lct_set_debug")


def lct_selftest_timeout(which: int, limit_ms: float, stream=None) -> int:
    """Status of one on-purpose bounded device wait (LCT_ERR_TIMEOUT = 9 when
    it gave up as designed); see include/lct.h."""
    return int(_load().lct_selftest_timeout(which, limit_ms, _stream_handle(stream)))


def lct_partition(N, world: int, abcd=None):
    """Owner rank of every signal (cost-balanced, largest first) and the
    per-rank loads; see lct_partition in include/lct.h."""
    n = np.ascontiguousarray(np.asarray(N, dtype=np.int64))
    owner = np.empty(len(n), dtype=np.int32)
    load = np.empty(world, dtype=np.float64)
    p = None
    if abcd is not None:       # [count, 4] real or complex (a, b, c, d)
        p = np.ascontiguousarray(np.asarray(abcd, dtype=np.complex128).reshape(len(n), 4)
                                 .view(np.float64).reshape(-1))
    _check(_load().lct_partition(len(n), n.ctypes.data, 0 if p is None else p.ctypes.data, world,
                                 owner.ctypes.data, load.ctypes.data), "lct_partition")
    return owner, load


def lct_execute_host(plan: int, h_in, h_out, batch: int, stream=None) -> None:
    """lct_execute on host buffers (page-locked tensors for overlap): the
    library pipelines copy-in, transform and copy-out over chunks."""
    _check(_load().lct_execute_host(plan, _ptr(h_in), _ptr(h_out), batch, _stream_handle(stream)),
           "lct_execute_host")


def lct_backward(plan: int, grad_out, inp, out, grad_in, grad_abd, batch: int, stream=None) -> None:
    """grad_in = L^H grad_out; grad_abd (float64 device tensor or None)
    receives (dl/da, dl/db, dl/dd) per signal (batch plans) or summed."""
    _check(_load().lct_backward(plan, _ptr(grad_out), _ptr(inp), _ptr(out), _ptr(grad_in),
                                _ptr(grad_abd), batch, _stream_handle(stream)), "lct_backward")


def lct2d_plan_create(ny: int, nx: int, abcd_y, abcd_x, dtype: int = LCT_C64) -> int:
    py = np.ascontiguousarray(np.asarray(abcd_y, dtype=np.float64))
    px = np.ascontiguousarray(np.asarray(abcd_x, dtype=np.float64))
    if py.shape != (4,) or px.shape != (4,):
        raise ValueError("abcd_x and abcd_y must hold 4 real values")
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    _check(_load().lct2d_plan_create(ctypes.byref(h), ny, nx, py.ctypes.data_as(dp),
                                     px.ctypes.data_as(dp), dtype), "lct2d_plan_create")
    return h.value


def lct2d_execute(plan: int, inp, mid, out, batch: int, stream=None) -> None:
    _check(_load().lct2d_execute(plan, _ptr(inp), _ptr(mid), _ptr(out), batch,
                                 _stream_handle(stream)), "lct2d_execute")


def lct2d_backward(plan: int, grad_out, inp, mid, out, grad_mid, grad_in, grad_abd, batch: int,
                   stream=None) -> None:
    _check(_load().lct2d_backward(plan, _ptr(grad_out), _ptr(inp), _ptr(mid), _ptr(out),
                                  _ptr(grad_mid), _ptr(grad_in), _ptr(grad_abd), batch,
                                  _stream_handle(stream)), "lct2d_backward")


def lct2d_plan_destroy(plan: int) -> None:
    _check(_load().lct2d_plan_destroy(plan), "lct2d_plan_destroy")


def frft_execute(N: int, z: complex, inp, out, batch: int, dtype: int = LCT_C64, stream=None) -> None:
    z = complex(z)
    _check(_load().frft_execute(N, z.real, z.imag, _ptr(inp), _ptr(out), batch, dtype,
                                _stream_handle(stream)), "frft_execute")


def frft_hermite_execute(N: int, z: complex, inp, out, batch: int, dtype: int = LCT_C64,
                         stream=None) -> None:
    """Hermite-zero discrete fractional transform F_z = sqrt(2 pi) U^T D(z) U
    of signals sampled at the zeros of H_N (see include/lct.h)."""
    z = complex(z)
    _check(_load().frft_hermite_execute(N, z.real, z.imag, _ptr(inp), _ptr(out), batch, dtype,
                                        _stream_handle(stream)), "frft_hermite_execute")


def frft_mehler_execute(N: int, z: complex, inp, out, batch: int, dtype: int = LCT_C64,
                        stream=None) -> None:
    """F_z for complex z on the real nodes y_j = x_j: the matrix of eq. (fasy)
    times the samples (eq. (primcuad)), as one weighted convolution (see
    include/lct.h)."""
    z = complex(z)
    _check(_load().frft_mehler_execute(N, z.real, z.imag, _ptr(inp), _ptr(out), batch, dtype,
                                       _stream_handle(stream)), "frft_mehler_execute")


def lct_transpose(inp, out, rows: int, cols: int, vec: int = 1, batch: int = 1, dtype: int = LCT_C64,
                  stream=None) -> None:
    """[batch][rows][cols][vec] -> [batch][cols][rows][vec] on the device."""
    _check(_load().lct_transpose(dtype, _ptr(inp), _ptr(out), rows, cols, vec, batch,
                                 _stream_handle(stream)), "lct_transpose")


def frft_hermite_status(stream=None) -> int:
    """Synchronise and return the Hermite tensor-core kernels' status (0 = ok,
    9 = a bounded wait gave up); does not raise."""
    return int(_load().frft_hermite_status(_stream_handle(stream)))


def frft_hermite_basis(N: int, with_matrix: bool = True):
    """(nodes x [N], U [N, N] or None) of the Hermite-zero transform,
    computed on the current GPU."""
    x = np.empty(N, dtype=np.float64)
    U = np.empty((N, N), dtype=np.float64) if with_matrix else None
    dp = ctypes.POINTER(ctypes.c_double)
    _check(_load().frft_hermite_basis(N, x.ctypes.data_as(dp),
                                      U.ctypes.data_as(dp) if U is not None else None),
           "frft_hermite_basis")
    return x, U


def lct_output_grid(plan: int, index: int = 0, N: Optional[int] = None):
    """(y complex128 [N], rho float64 [N]) of signal `index`."""
    if N is None:
        raise ValueError("pass N (the signal length of that index)")
    y = np.empty(2 * N, dtype=np.float64)
    rho = np.empty(N, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(_load().lct_output_grid(plan, index, y.ctypes.data_as(dp), rho.ctypes.data_as(dp)),
           "lct_output_grid")
    return y.view(np.complex128), rho


def lct_input_grid(N: int) -> np.ndarray:
    x = np.empty(N, dtype=np.float64)
    _check(_load().lct_input_grid(N, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "lct_input_grid")
    return x


def lct_plan_phase_turns(plan: int, index: int = 0):
    out = (ctypes.c_uint64 * 5)()
    _check(_load().lct_plan_phase_turns(plan, index, out), "lct_plan_phase_turns")
    return tuple(int(v) for v in out)


def lct_device_status(plan: int, stream=None) -> int:
    """Synchronise and return the device status (0 = ok); does not raise."""
    return int(_load().lct_device_status(plan, _stream_handle(stream)))


def lct_plan_destroy(plan: int) -> None:
    _check(_load().lct_plan_destroy(plan), "lct_plan_destroy")


def lct_status_string(status: int) -> str:
    return _status_string(status)


LCT_NOALLOC_MAX_N = 4096
LCT_NOALLOC_MAX_POINTS = 1 << 21


def lct_execute_noalloc(N: int, a: float, b: float, c: float, d: float, inp, out, batch: int,
                        dtype: int = LCT_C64, stream=None) -> None:
    """FP64 transform that allocates no device memory (static 32 MiB work
    array; batch * N <= LCT_NOALLOC_MAX_POINTS, N <= LCT_NOALLOC_MAX_N).
    Calls that overlap on the GPU race on the shared array."""
    _check(_load().lct_execute_noalloc(N, a, b, c, d, dtype, _ptr(inp), _ptr(out), batch,
                                       _stream_handle(stream)), "lct_execute_noalloc")


# ---------------------------------------------------------------------------
# convenience: an owning plan object
# ---------------------------------------------------------------------------
class Plan:
    """Owning wrapper of an lct_plan handle."""

    def __init__(self, handle: int, N, dtype: int):
        self.handle = handle
        self.N = N
        self.dtype = dtype

    @classmethod
    def create(cls, N: int, a, b, c, d, dtype: int = LCT_C64) -> "Plan":
        if any(isinstance(v, complex) for v in (a, b, c, d)):
            return cls(lct_plan_create_complex(N, [a, b, c, d], dtype), N, dtype)
        return cls(lct_plan_create(N, a, b, c, d, dtype), N, dtype)

    @classmethod
    def batch(cls, N, abcd, offsets, dtype: int = LCT_C64) -> "Plan":
        return cls(lct_plan_create_batch(N, abcd, offsets, dtype), N, dtype)

    def set_precision(self, precision: int) -> "Plan":
        lct_plan_set_precision(self.handle, precision)
        return self

    def execute(self, inp, out, batch: int, stream=None) -> None:
        lct_execute(self.handle, inp, out, batch, stream)

    def execute_host(self, h_in, h_out, batch: int, stream=None) -> None:
        lct_execute_host(self.handle, h_in, h_out, batch, stream)

    def set_variant(self, variant: int) -> "Plan":
        lct_plan_set_variant(self.handle, variant)
        return self

    def autotune(self, inp, out, batch: int, stream=None) -> int:
        return lct_plan_autotune(self.handle, inp, out, batch, stream)

    def destroy(self) -> None:
        if self.handle:
            lct_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Plan2D:
    """Owning wrapper of an lct2d_plan handle."""

    def __init__(self, handle: int):
        self.handle = handle

    def destroy(self) -> None:
        if self.handle:
            lct2d_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# autograd: the library's forward and backward kernels as torch Functions
# ---------------------------------------------------------------------------
def _torch_fns():
    import torch

    class LCTFunction(torch.autograd.Function):
        """G = LCT(x) for x [batch, N] complex (cuda); abcd float64 [4]
        (shared) or [batch, 4] (per signal).  Backward: lct_backward."""

        @staticmethod
        def forward(ctx, x, abcd):
            x = x.contiguous()
            code = dtype_code(x.dtype)
            xb = x.reshape(-1, x.shape[-1])
            batch, N = xb.shape
            p = abcd.detach().to("cpu", torch.float64).numpy()
            if p.ndim == 1:
                plan = Plan(lct_plan_create(N, *[float(v) for v in p], code), N, code)
            else:
                plan = Plan(lct_plan_create_batch([N] * batch, p, np.arange(batch) * N, code), N, code)
            out = torch.empty_like(xb)
            plan.execute(xb, out, batch)
            ctx.plan, ctx.batch, ctx.shape, ctx.pshape = plan, batch, x.shape, p.shape
            ctx.pdev = abcd.device
            ctx.save_for_backward(xb, out)
            return out.reshape(x.shape)

        @staticmethod
        def backward(ctx, g):
            xb, out = ctx.saved_tensors
            g = g.contiguous().reshape(xb.shape)
            grad_in = torch.empty_like(xb)
            want_p = ctx.needs_input_grad[1]
            gp = None
            if want_p:
                gp = torch.zeros((ctx.batch, 3) if len(ctx.pshape) == 2 else (3,),
                                 dtype=torch.float64, device=xb.device)
            lct_backward(ctx.plan.handle, g, xb, out, grad_in, gp, ctx.batch)
            grad_abcd = None
            if want_p:
                z = torch.zeros_like(gp[..., :1])
                grad_abcd = torch.cat([gp[..., 0:2], z, gp[..., 2:3]], dim=-1)   # c: no effect for b != 0
                grad_abcd = grad_abcd.to(ctx.pdev)
            # the plan lives as long as ctx: backward may run more than once
            # (retain_graph), and Plan.__del__ frees it afterwards
            return grad_in.reshape(ctx.shape), grad_abcd

    class LCT2DFunction(torch.autograd.Function):
        """Separable 2-D LCT of x [batch, ny, nx]: rows with abcd_x, then
        columns with abcd_y (float64 [4] each).  Backward: lct2d_backward."""

        @staticmethod
        def forward(ctx, x, abcd_x, abcd_y):
            x = x.contiguous()
            code = dtype_code(x.dtype)
            xb = x.reshape(-1, x.shape[-2], x.shape[-1])
            batch, ny, nx = xb.shape
            px = abcd_x.detach().to("cpu", torch.float64).numpy()
            py = abcd_y.detach().to("cpu", torch.float64).numpy()
            plan = Plan2D(lct2d_plan_create(ny, nx, py, px, code))
            mid = torch.empty_like(xb)
            out = torch.empty_like(xb)
            lct2d_execute(plan.handle, xb, mid, out, batch)
            ctx.plan, ctx.batch, ctx.shape = plan, batch, x.shape
            ctx.pdev = (abcd_x.device, abcd_y.device)
            ctx.save_for_backward(xb, mid, out)
            return out.reshape(x.shape)

        @staticmethod
        def backward(ctx, g):
            xb, mid, out = ctx.saved_tensors
            g = g.contiguous().reshape(xb.shape)
            grad_mid = torch.empty_like(xb)
            grad_in = torch.empty_like(xb)
            want_p = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
            gp = torch.zeros(6, dtype=torch.float64, device=xb.device) if want_p else None
            lct2d_backward(ctx.plan.handle, g, xb, mid, out, grad_mid, grad_in, gp, ctx.batch)
            gx = gy = None
            if want_p:
                z = torch.zeros(1, dtype=torch.float64, device=xb.device)
                gx = torch.cat([gp[0:2], z, gp[2:3]]).to(ctx.pdev[0])
                gy = torch.cat([gp[3:5], z, gp[5:6]]).to(ctx.pdev[1])
            return grad_in.reshape(ctx.shape), gx, gy

    return LCTFunction, LCT2DFunction


_FNS = None


def _fns():
    global _FNS
    if _FNS is None:
        _FNS = _torch_fns()
    return _FNS


def lct(x, abcd):
    """Differentiable LCT of the last axis of x (complex64/128 cuda tensor).
    abcd: float64 tensor [4] or [batch, 4] with ad - bc = 1 (b != 0 for
    gradients); gradients flow to x and to (a, b, d)."""
    return _fns()[0].apply(x, abcd)


def lct2d(x, abcd_x, abcd_y):
    """Differentiable separable 2-D LCT of x [..., ny, nx]."""
    return _fns()[1].apply(x, abcd_x, abcd_y)


from .sharded import lct2d_sharded  # noqa: E402,F401
