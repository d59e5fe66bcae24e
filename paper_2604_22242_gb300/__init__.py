"""Python binding of libfx.so, the fused-expression library (include/fx.h).

Argument marshalling only: every step of an evaluation runs in the
library's CUDA kernels. The functions keep the C names; a non-zero status
raises ``FxError`` carrying the library's message. The library must be built
(``python -m paper_2604_22242_gb300.build``); without it every call raises.

PyTorch is used for device memory and streams only: ``colmajor`` makes a
column-major device matrix (a 2-D tensor with strides ``(1, ld)``) and
``bind_tensor`` binds one to a slot.
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "FxError", "FX_F32", "FX_F64", "FX_BF16", "FX_F16", "FX_MAX_SLOTS", "lib", "lib_path",
    "fx_list", "fx_expr_create", "fx_expr_destroy", "fx_expr_info", "fx_expr_slot_name",
    "fx_expr_bind", "fx_expr_set_scalar", "fx_expr_get_scalar", "fx_eval", "fx_eval_unfused",
    "fx_eval_host", "fx_eval_batch", "fx_eval_backward", "fx_tune", "fx_expr_launch_shape",
    "fx_expr_set_launch_shape", "fx_fp64_fma_rate", "fx_expr_slot_dtype",
    "fx_selftest_wait_timeout", "fx_tune_batch",
    "fx_expr_last_launches", "fx_expr_sync_status", "fx_last_error_string", "fx_status_string", "BatchItem",
    "colmajor", "bind_tensor", "Expr", "FusedLoss", "DTYPE_OF",
]

FX_F32, FX_F64, FX_BF16, FX_F16 = 0, 1, 2, 3
FX_MAX_SLOTS = 24
FX_MAX_SCALARS = 8
KINDS = {0: "elementwise", 1: "full_reduce", 2: "dim_reduce", 3: "multi"}
TUNE = {"off": 0, "cache": 1, "search": 2}

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "libfx.so")


class FxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fx status {status}: {msg}")
        self.status = status


class BatchItem(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p * FX_MAX_SLOTS), ("ld", ctypes.c_int64 * FX_MAX_SLOTS),
                ("rows", ctypes.c_int64), ("cols", ctypes.c_int64)]


_lib = None


def lib():
    """The loaded library (loaded on first use; raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(lib_path):
        raise FxError(-100, f"{lib_path} is missing: build it with "
                            "`python -m paper_2604_22242_gb300.build`")
    L = ctypes.CDLL(lib_path)
    vp, i64, i32, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "fx_list_count": (i32, []),
        "fx_list_get": (st, [i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(i32),
                             ctypes.POINTER(ctypes.c_char_p)]),
        "fx_expr_create": (st, [ctypes.c_char_p, i32, pp]),
        "fx_expr_destroy": (st, [vp]),
        "fx_expr_info": (st, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                              ctypes.POINTER(i32)]),
        "fx_expr_slot_name": (st, [vp, i32, ctypes.POINTER(ctypes.c_char_p)]),
        "fx_expr_bind": (st, [vp, i32, vp, i64, i64, i64]),
        "fx_expr_set_scalar": (st, [vp, i32, ctypes.c_double]),
        "fx_expr_get_scalar": (st, [vp, i32, ctypes.POINTER(ctypes.c_double)]),
        "fx_eval": (st, [vp, vp]),
        "fx_eval_unfused": (st, [vp, vp]),
        "fx_eval_host": (st, [vp, pp, pp, vp]),
        "fx_eval_batch": (st, [vp, i64, ctypes.POINTER(BatchItem), vp, i32]),
        "fx_eval_backward": (st, [vp, vp, pp, vp]),
        "fx_tune": (st, [vp, i32, vp]),
        "fx_expr_launch_shape": (st, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                      ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "fx_expr_set_launch_shape": (st, [vp, i32, i32, i32, i32]),
        "fx_fp64_fma_rate": (st, [vp, ctypes.POINTER(ctypes.c_double)]),
        "fx_expr_slot_dtype": (st, [vp, i32, ctypes.POINTER(i32)]),
        "fx_selftest_wait_timeout": (st, [vp, ctypes.POINTER(ctypes.c_uint)]),
        "fx_tune_batch": (st, [vp, i64, ctypes.POINTER(BatchItem), i32, vp]),
        "fx_expr_last_launches": (i32, [vp]),
        "fx_expr_sync_status": (st, [vp, vp]),
        "fx_last_error_string": (ctypes.c_char_p, []),
        "fx_status_string": (ctypes.c_char_p, [i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise FxError(status, lib().fx_last_error_string().decode())


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * max(1, len(ptrs)))()
    for i, p in enumerate(ptrs):
        arr[i] = p if p else None
    return arr


# ---------------------------------------------------------------- C functions

def fx_list():
    """[(name, storage dtype, formula), ...] of every compiled instantiation."""
    L = lib()
    out = []
    for i in range(L.fx_list_count()):
        n, f = ctypes.c_char_p(), ctypes.c_char_p()
        d = ctypes.c_int()
        _check(L.fx_list_get(i, ctypes.byref(n), ctypes.byref(d), ctypes.byref(f)))
        out.append((n.value.decode(), d.value, f.value.decode()))
    return out


def fx_expr_create(name: str, storage: int):
    h = ctypes.c_void_p()
    _check(lib().fx_expr_create(name.encode(), storage, ctypes.byref(h)))
    return h


def fx_expr_destroy(h):
    _check(lib().fx_expr_destroy(h))


def fx_expr_info(h):
    a, b, c, k = (ctypes.c_int() for _ in range(4))
    _check(lib().fx_expr_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(k)))
    return a.value, b.value, c.value, KINDS[k.value]


def fx_expr_slot_name(h, slot: int) -> str:
    n = ctypes.c_char_p()
    _check(lib().fx_expr_slot_name(h, slot, ctypes.byref(n)))
    return n.value.decode()


def fx_expr_bind(h, slot: int, ptr: int, rows: int, cols: int, ld: int):
    _check(lib().fx_expr_bind(h, slot, ptr or None, rows, cols, ld))


def fx_expr_set_scalar(h, idx: int, v: float):
    _check(lib().fx_expr_set_scalar(h, idx, float(v)))


def fx_expr_get_scalar(h, idx: int) -> float:
    v = ctypes.c_double()
    _check(lib().fx_expr_get_scalar(h, idx, ctypes.byref(v)))
    return v.value


def fx_eval(h, stream: int = 0):
    _check(lib().fx_eval(h, stream or None))


def fx_eval_unfused(h, stream: int = 0):
    _check(lib().fx_eval_unfused(h, stream or None))


def fx_eval_host(h, host_in, host_out, stream: int = 0):
    """host_in / host_out: lists of host addresses (pinned memory)."""
    _check(lib().fx_eval_host(h, _ptr_array(host_in), _ptr_array(host_out), stream or None))


def fx_eval_batch(h, items, stream: int = 0, use_graph: bool = True):
    """items: a ctypes array of BatchItem."""
    _check(lib().fx_eval_batch(h, len(items), items, stream or None, 1 if use_graph else 0))


def fx_eval_backward(h, grad_out_ptr, grad_ptrs, stream: int = 0):
    _check(lib().fx_eval_backward(h, grad_out_ptr or None, _ptr_array(grad_ptrs), stream or None))


def fx_tune(h, mode: str = "search", stream: int = 0):
    _check(lib().fx_tune(h, TUNE[mode], stream or None))


def fx_tune_batch(h, items, mode: str = "search", stream: int = 0):
    """items: a ctypes array of BatchItem (as for fx_eval_batch)."""
    _check(lib().fx_tune_batch(h, len(items), items, TUNE[mode], stream or None))


def fx_expr_launch_shape(h):
    """(block, unroll, blocks_per_sm, pipeline) currently in force."""
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().fx_expr_launch_shape(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                      ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def fx_expr_slot_dtype(h, slot: int) -> int:
    """Storage type code (FX_F32, FX_F64, FX_BF16, FX_F16) of a slot's buffer."""
    v = ctypes.c_int()
    _check(lib().fx_expr_slot_dtype(h, slot, ctypes.byref(v)))
    return v.value


def fx_selftest_wait_timeout(stream: int = 0) -> int:
    """Error word after a bounded wait that nothing releases (1 expected)."""
    v = ctypes.c_uint()
    _check(lib().fx_selftest_wait_timeout(stream or None, ctypes.byref(v)))
    return v.value


def fx_fp64_fma_rate(stream: int = 0) -> float:
    """Measured FP64 FMA throughput of the current device, flop/s."""
    v = ctypes.c_double()
    _check(lib().fx_fp64_fma_rate(stream or None, ctypes.byref(v)))
    return v.value


def fx_expr_set_launch_shape(h, block: int, unroll: int, blocks_per_sm: int = 0,
                             pipeline: int = 0):
    _check(lib().fx_expr_set_launch_shape(h, block, unroll, blocks_per_sm, pipeline))


def fx_expr_last_launches(h) -> int:
    return lib().fx_expr_last_launches(h)


def fx_expr_sync_status(h, stream: int = 0):
    _check(lib().fx_expr_sync_status(h, stream or None))


def fx_last_error_string() -> str:
    return lib().fx_last_error_string().decode()


def fx_status_string(s: int) -> str:
    return lib().fx_status_string(s).decode()


# ---------------------------------------------------------------- torch helpers

def _torch():
    import torch
    return torch


def DTYPE_OF(storage: int):
    torch = _torch()
    return {FX_F32: torch.float32, FX_F64: torch.float64, FX_BF16: torch.bfloat16,
            FX_F16: torch.float16}[storage]


def colmajor(rows: int, cols: int, dtype, device="cuda", ld: int | None = None):
    """An uninitialised column-major rows x cols device matrix (strides (1, ld))."""
    torch = _torch()
    ld = max(rows, 1) if ld is None else ld
    base = torch.empty(max(cols, 1) * ld, dtype=dtype, device=device)
    return base.as_strided((rows, cols), (1, ld))


def bind_tensor(h, slot: int, t):
    """Binds a 2-D tensor with unit row stride (column-major) or a 1-D
    tensor (a column vector) to ``slot``."""
    if t.dim() == 1:
        rows, cols, ld = t.shape[0], 1, max(t.shape[0], 1)
        if t.numel() > 1 and t.stride(0) != 1:
            raise ValueError("a vector must be contiguous")
    elif t.dim() == 2:
        rows, cols = t.shape
        if rows > 1 and t.stride(0) != 1:
            raise ValueError("matrices are column-major: stride(0) must be 1")
        ld = t.stride(1) if cols > 1 else max(rows, 1)
        ld = max(ld, rows, 1)
    else:
        raise ValueError("bind a 1-D or 2-D tensor")
    fx_expr_bind(h, slot, t.data_ptr(), rows, cols, ld)


class Expr:
    """An expression object with its slots bound to torch tensors."""

    def __init__(self, name: str, storage: int):
        self.h = fx_expr_create(name, storage)
        self.name, self.storage = name, storage
        self.n_in, self.n_out, self.n_scal, self.kind = fx_expr_info(self.h)
        self.slots = [fx_expr_slot_name(self.h, k) for k in range(self.n_in + self.n_out)]
        self._keep = {}

    def bind(self, slot, t):
        k = self.slots.index(slot) if isinstance(slot, str) else slot
        bind_tensor(self.h, k, t)
        self._keep[k] = t
        return self

    def set_scalar(self, idx, v):
        fx_expr_set_scalar(self.h, idx, v)
        return self

    def eval(self, stream=None):
        fx_eval(self.h, _stream_ptr(stream))

    def eval_unfused(self, stream=None):
        fx_eval_unfused(self.h, _stream_ptr(stream))

    def close(self):
        if self.h:
            fx_expr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    if stream is None:
        torch = _torch()
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def FusedLoss():
    """A torch.autograd.Function over an accu(...) tree: forward is the fused
    reduction, backward the fused reverse pass (fx_eval_backward)."""
    torch = _torch()

    class _F(torch.autograd.Function):
        @staticmethod
        def forward(ctx, name, storage, *inputs):
            ex = Expr(name, storage)
            for k, t in enumerate(inputs):
                ex.bind(k, t)
            rdt = torch.float64 if storage == FX_F64 else torch.float32
            out = torch.empty((1, 1), dtype=rdt, device=inputs[0].device)
            ex.bind(ex.n_in, out)
            ex.eval()
            ctx.ex = ex
            ctx.save_for_backward(*inputs)
            return out.reshape(())

        @staticmethod
        def backward(ctx, gL):
            ex = ctx.ex
            inputs = ctx.saved_tensors
            grads = []
            for t in inputs:
                if t.dim() == 1:
                    grads.append(torch.empty_like(t))
                else:
                    grads.append(colmajor(t.shape[0], t.shape[1], t.dtype, t.device))
            gl = gL.to(torch.float64 if ex.storage == FX_F64 else torch.float32).reshape(1).contiguous()
            fx_eval_backward(ex.h, gl.data_ptr(), [g.data_ptr() for g in grads],
                             _stream_ptr(None))
            ctx.keep = gl
            return (None, None, *grads)

    return _F
