"""Serving loop binding (marshalling only): sc_server_create / sc_submit /
sc_poll / sc_server_drain / sc_server_destroy."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib_loader import check, lib
from .solvers import _PREC

EPENDING = 9


class ServerCfg(ctypes.Structure):
    _fields_ = [("arena_dev", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t),
                ("max_active", ctypes.c_int32), ("slice_ms", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("order", ctypes.c_int32), ("n", ctypes.c_int64 * 3),
                ("prec", ctypes.c_int32), ("rtol", ctypes.c_double), ("maxit", ctypes.c_int64),
                ("f_host", ctypes.c_void_p), ("ghost_host", ctypes.c_void_p), ("x_host", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("prec", ctypes.c_int32), ("iters", ctypes.c_int64),
                ("rel_res", ctypes.c_double), ("queue_s", ctypes.c_double), ("latency_s", ctypes.c_double)]

    def as_dict(self):
        return {"status": int(self.status), "prec": "mixed" if self.prec == 1 else "f64",
                "iters": int(self.iters), "rel_res": float(self.rel_res), "queue_s": float(self.queue_s),
                "latency_s": float(self.latency_s)}


lib.sc_request_bytes.argtypes = [ctypes.POINTER(Request)]
lib.sc_request_bytes.restype = ctypes.c_size_t
lib.sc_server_create.argtypes = [ctypes.POINTER(ServerCfg), ctypes.POINTER(ctypes.c_void_p)]
lib.sc_server_create.restype = ctypes.c_int
lib.sc_server_destroy.argtypes = [ctypes.c_void_p]
lib.sc_server_destroy.restype = ctypes.c_int
lib.sc_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
lib.sc_submit.restype = ctypes.c_int
lib.sc_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Result)]
lib.sc_poll.restype = ctypes.c_int
lib.sc_server_drain.argtypes = [ctypes.c_void_p, ctypes.c_double]
lib.sc_server_drain.restype = ctypes.c_int


def make_request(f: np.ndarray, ghost: np.ndarray, x: np.ndarray, order=2, prec="auto", rtol=1e-10,
                 maxit=10_000_000) -> Request:
    for a in (f, ghost, x):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be C-contiguous float64 arrays")
    r = Request()
    r.ndim, r.order = x.ndim, order
    for a, s in enumerate(reversed(x.shape)):
        r.n[a] = s
    r.prec = _PREC[prec] if isinstance(prec, str) else int(prec)
    r.rtol, r.maxit = rtol, maxit
    r.f_host, r.ghost_host, r.x_host = f.ctypes.data, ghost.ctypes.data, x.ctypes.data
    return r


def request_bytes(r: Request) -> int:
    return int(lib.sc_request_bytes(ctypes.byref(r)))


class Server:
    """Continuous-batching plate-problem server on the current device."""

    def __init__(self, arena: torch.Tensor, max_active: int = 256, slice_ms: float = 2.0):
        if not arena.is_cuda:
            raise ValueError("arena must be a CUDA tensor")
        self._arena = arena
        cfg = ServerCfg(arena.data_ptr(), arena.numel() * arena.element_size(), max_active, slice_ms)
        h = ctypes.c_void_p()
        check(lib.sc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, f, ghost, x, **kw) -> int:
        r = make_request(f, ghost, x, **kw)
        t = ctypes.c_uint64()
        check(lib.sc_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = (f, ghost, x)
        return t.value

    def poll(self, ticket: int):
        res = Result()
        rc = lib.sc_poll(self._h, ticket, ctypes.byref(res))
        if rc == EPENDING:
            return None
        check(rc)
        self._keep.pop(ticket, None)
        return res.as_dict()

    def drain(self, timeout_s: float = 600.0):
        check(lib.sc_server_drain(self._h, timeout_s))

    def close(self):
        if self._h:
            check(lib.sc_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
