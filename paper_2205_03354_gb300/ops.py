"""Device entry points taking torch tensors (marshalling only)."""
from __future__ import annotations

import ctypes

import torch

from ._lib_loader import check, lib
from .stencil import Stencil

F64, F32 = 0, 1
BC_PERIODIC, BC_GHOSTED, BC_ZERO = 0, 1, 2
_BC = {"periodic": BC_PERIODIC, "ghosted": BC_GHOSTED, "zero": BC_ZERO}
_P = ctypes.POINTER(Stencil)
_I64P = ctypes.POINTER(ctypes.c_int64)

lib.sc_apply_composed.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _I64P, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
lib.sc_apply_composed.restype = ctypes.c_int
lib.sc_apply_host_work_bytes.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _I64P]
lib.sc_apply_host_work_bytes.restype = ctypes.c_size_t
lib.sc_apply_composed_host.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _I64P, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
lib.sc_apply_composed_host.restype = ctypes.c_int


def dtype_code(t) -> int:
    if t == torch.float64:
        return F64
    if t == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t}")


def bc_code(bc) -> int:
    return _BC[bc] if isinstance(bc, str) else int(bc)


def dims_arg(dims):
    arr = (ctypes.c_int64 * 3)(*(list(dims) + [1] * (3 - len(dims))))
    return arr


def stream_arg(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def require_device(name: str, t, dtype=None) -> None:
    """Every device entry point takes contiguous CUDA tensors; anything else is
    refused here, before the library could be handed a host address."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}")


def apply_composed(s: Stencil, x: torch.Tensor, y: torch.Tensor, bc="periodic", h=(1, 1),
                   dims=None, stream=None) -> torch.Tensor:
    """y = A x with the composed stencil s (flat evaluation) on the device.
    ``dims`` = interior (nx, ny[, nz]); defaults to y's shape reversed."""
    if not (x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous CUDA tensors")
    if x.dtype != y.dtype:
        raise TypeError("x and y dtypes differ")
    if dims is None:
        dims = tuple(reversed(y.shape))
    check(lib.sc_apply_composed(ctypes.byref(s), dtype_code(y.dtype), bc_code(bc), dims_arg(dims),
                                int(h[0]), int(h[1]), ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(y.data_ptr()), stream_arg(stream)))
    return y


def apply_host_work_bytes(s: Stencil, dtype, bc, dims) -> int:
    return int(lib.sc_apply_host_work_bytes(ctypes.byref(s), dtype_code(dtype), bc_code(bc), dims_arg(dims)))


def apply_composed_host(s: Stencil, x: torch.Tensor, y: torch.Tensor, work: torch.Tensor,
                        bc="periodic", h=(1, 1), dims=None, stream=None) -> torch.Tensor:
    """Same operator with x, y in host memory (pinned for speed); copies in
    and out through the device work buffer ``work`` inside the call."""
    if x.is_cuda or y.is_cuda or not work.is_cuda:
        raise ValueError("x, y must be host tensors and work a device tensor")
    if dims is None:
        dims = tuple(reversed(y.shape))
    check(lib.sc_apply_composed_host(ctypes.byref(s), dtype_code(y.dtype), bc_code(bc), dims_arg(dims),
                                     int(h[0]), int(h[1]), ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                                     work.numel() * work.element_size(), stream_arg(stream)))
    return y


lib.sc_apply_composition_work_bytes.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, _I64P]
lib.sc_apply_composition_work_bytes.restype = ctypes.c_size_t
lib.sc_apply_composition.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, _I64P, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.c_int32, ctypes.c_void_p]
lib.sc_apply_composition.restype = ctypes.c_int
ARITH_NATIVE, ARITH_PAIR = 0, 1


def apply_composition_work_bytes(outer: Stencil, inner: Stencil, dtype, bc, dims) -> int:
    return int(lib.sc_apply_composition_work_bytes(ctypes.byref(outer), ctypes.byref(inner), dtype_code(dtype),
                                                   bc_code(bc), dims_arg(dims)))


def apply_composition(outer: Stencil, inner: Stencil, x: torch.Tensor, y: torch.Tensor, work=None,
                      bc="periodic", h=(1, 1), dims=None, stream=None, arith="native") -> torch.Tensor:
    """y = outer(inner(x)): the composed operator in nested form (two passes
    through a device temporary); arith="pair" evaluates FP64 Laplacian
    factors in pairs of FP32 numbers."""
    require_device("x", x)
    require_device("y", y, x.dtype)
    if dims is None:
        dims = tuple(reversed(y.shape))
    nb = apply_composition_work_bytes(outer, inner, y.dtype, bc, dims)
    if work is None:
        work = torch.empty(max(nb, 1), dtype=torch.uint8, device=y.device)
    require_device("work", work)
    check(lib.sc_apply_composition(ctypes.byref(outer), ctypes.byref(inner), dtype_code(y.dtype), bc_code(bc),
                                   dims_arg(dims), int(h[0]), int(h[1]), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                                   work.numel() * work.element_size(), ARITH_PAIR if arith == "pair" else ARITH_NATIVE,
                                   stream_arg(stream)))
    return y


lib.sc_apply_varcoef.argtypes = [_P, _P, ctypes.c_int32, _I64P, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
lib.sc_apply_varcoef.restype = ctypes.c_int


def apply_varcoef(outer: Stencil, inner: Stencil, m, x, y, work, h=(1, 1), dims=None, stream=None):
    """y = outer(m * inner(x)), periodic (the variable-mobility composition)."""
    require_device("x", x)
    require_device("y", y, x.dtype)
    require_device("m", m, x.dtype)
    require_device("work", work)
    if dims is None:
        dims = tuple(reversed(y.shape))
    check(lib.sc_apply_varcoef(ctypes.byref(outer), ctypes.byref(inner), dtype_code(y.dtype), dims_arg(dims),
                               int(h[0]), int(h[1]), ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                               work.numel() * work.element_size(), stream_arg(stream)))
    return y


EVAL_NAMES = {0: "flat", 1: "nested", 2: "pair", 3: "fused"}


class TuneChoice(ctypes.Structure):
    _fields_ = [("eval", ctypes.c_int32), ("planes", ctypes.c_int32), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {"eval": EVAL_NAMES[self.eval], "planes": int(self.planes), "ms": float(self.ms)}


_TUNE_ARGS = [_P, _P, ctypes.c_int32, ctypes.c_int32, _I64P, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
lib.sc_autotune_apply.argtypes = _TUNE_ARGS + [ctypes.POINTER(TuneChoice), ctypes.c_void_p]
lib.sc_autotune_apply.restype = ctypes.c_int
lib.sc_apply_tuned.argtypes = _TUNE_ARGS + [ctypes.c_void_p]
lib.sc_apply_tuned.restype = ctypes.c_int
lib.sc_tuned_choice.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, _I64P, ctypes.POINTER(TuneChoice)]
lib.sc_tuned_choice.restype = ctypes.c_int
lib.sc_tune_set.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, _I64P, ctypes.POINTER(TuneChoice)]
lib.sc_tune_set.restype = ctypes.c_int


def _tune_args(outer, inner, x, y, work, bc, h, dims):
    require_device("x", x)
    require_device("y", y, x.dtype)
    require_device("work", work)
    if dims is None:
        dims = tuple(reversed(y.shape))
    return (ctypes.byref(outer), ctypes.byref(inner), dtype_code(y.dtype), bc_code(bc), dims_arg(dims),
            int(h[0]), int(h[1]), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
            ctypes.c_void_p(work.data_ptr()), work.numel() * work.element_size())


def autotune_apply(outer: Stencil, inner: Stencil, x, y, work, bc="periodic", h=(1, 1), dims=None,
                   stream=None) -> dict:
    """Times the evaluation schedules x halo-blocking depths and caches the
    fastest for this shape (y is overwritten)."""
    c = TuneChoice()
    check(lib.sc_autotune_apply(*_tune_args(outer, inner, x, y, work, bc, h, dims), ctypes.byref(c),
                                stream_arg(stream)))
    return c.as_dict()


def apply_tuned(outer: Stencil, inner: Stencil, x, y, work, bc="periodic", h=(1, 1), dims=None, stream=None):
    """y = compose(outer, inner) x with the tuned schedule for this shape."""
    check(lib.sc_apply_tuned(*_tune_args(outer, inner, x, y, work, bc, h, dims), stream_arg(stream)))
    return y


lib.sc_apply_tuned_host_work_bytes.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, _I64P]
lib.sc_apply_tuned_host_work_bytes.restype = ctypes.c_size_t
lib.sc_apply_tuned_host.argtypes = _TUNE_ARGS + [ctypes.c_void_p]
lib.sc_apply_tuned_host.restype = ctypes.c_int


def apply_tuned_host_work_bytes(outer: Stencil, inner: Stencil, dtype, bc, dims) -> int:
    return int(lib.sc_apply_tuned_host_work_bytes(ctypes.byref(outer), ctypes.byref(inner), dtype_code(dtype),
                                                  bc_code(bc), dims_arg(dims)))


def apply_tuned_host(outer: Stencil, inner: Stencil, x, y, work, bc="periodic", h=(1, 1), dims=None, stream=None):
    """The tuned apply with x and y in host memory (pinned for link-speed
    copies), pipelined over slabs of the slowest axis: one slab's copy-in,
    the previous slab's apply and the one before's copy-out run at once.
    x and y must not overlap.  Asynchronous: synchronise the stream before
    reading y."""
    for name, t in (("x", x), ("y", y)):
        if not (isinstance(t, torch.Tensor) and not t.is_cuda and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous host tensor")
    if y.dtype != x.dtype:
        raise TypeError("x and y must have the same dtype")
    require_device("work", work)
    if dims is None:
        dims = tuple(reversed(y.shape))
    check(lib.sc_apply_tuned_host(ctypes.byref(outer), ctypes.byref(inner), dtype_code(y.dtype), bc_code(bc),
                                  dims_arg(dims), int(h[0]), int(h[1]), ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                                  work.numel() * work.element_size(), stream_arg(stream)))
    return y


def tune_set(outer: Stencil, inner: Stencil, dtype, bc, dims, choice: dict) -> None:
    """Records a saved tuning choice ({"eval", "planes", "ms"}) for a shape so
    that apply_tuned reuses it without timing."""
    names = {v: k for k, v in EVAL_NAMES.items()}
    c = TuneChoice(names[choice["eval"]], int(choice["planes"]), float(choice.get("ms", 0.0)))
    check(lib.sc_tune_set(ctypes.byref(outer), ctypes.byref(inner), dtype_code(dtype), bc_code(bc),
                          dims_arg(dims), ctypes.byref(c)))
