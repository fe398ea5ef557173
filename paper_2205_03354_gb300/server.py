"""Serving loop binding (marshalling only): sc_server_create / sc_submit /
sc_poll / sc_server_drain / sc_server_status / sc_server_destroy."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib_loader import check, lib
from .solvers import _PREC

EPENDING = 9


REQ_PLATE, REQ_CH = 0, 1


class ServerCfg(ctypes.Structure):
    _fields_ = [("arena_dev", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t),
                ("max_active", ctypes.c_int32), ("slice_ms", ctypes.c_double), ("pcg_min_points", ctypes.c_int64),
                ("fail_slice", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("solver", ctypes.c_int32), ("ndim", ctypes.c_int32),
                ("order", ctypes.c_int32),
                ("n", ctypes.c_int64 * 3), ("prec", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("maxit", ctypes.c_int64), ("f_host", ctypes.c_void_p), ("ghost_host", ctypes.c_void_p),
                ("u_host", ctypes.c_void_p), ("h_num", ctypes.c_int64), ("h_den", ctypes.c_int64),
                ("dt", ctypes.c_double), ("M", ctypes.c_double), ("kappa", ctypes.c_double),
                ("chem", ctypes.c_int32), ("rho", ctypes.c_double), ("ca", ctypes.c_double),
                ("cb", ctypes.c_double), ("x_host", ctypes.c_void_p)]


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
lib.sc_server_status.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_size_t),
                                 ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(ctypes.c_int32)]
lib.sc_server_status.restype = ctypes.c_int


def _host_f64(*arrays):
    for a in arrays:
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be C-contiguous float64 arrays")


_RSOLVER = {"auto": -1, "persistent": 0, "pcg": 2}


def make_request(f: np.ndarray, ghost: np.ndarray, x: np.ndarray, order=2, prec="auto", rtol=1e-10,
                 maxit=10_000_000, solver="auto") -> Request:
    """A plate problem (Sec. 3.3): f and the ghosted exact field in, x out.
    solver: "persistent" (batched), "pcg" (preconditioned) or "auto" (by size)."""
    _host_f64(f, ghost, x)
    r = Request()
    r.kind = REQ_PLATE
    r.solver = _RSOLVER[solver] if isinstance(solver, str) else int(solver)
    r.ndim, r.order = x.ndim, order
    for a, s in enumerate(reversed(x.shape)):
        r.n[a] = s
    r.prec = _PREC[prec] if isinstance(prec, str) else int(prec)
    r.rtol, r.maxit = rtol, maxit
    r.f_host, r.ghost_host, r.x_host = f.ctypes.data, ghost.ctypes.data, x.ctypes.data
    return r


def make_ch_request(u: np.ndarray, x: np.ndarray, h, dt, M=1.0, kappa=1e-4, chem="cubic", rho=0.0, ca=0.0,
                    cb=0.0, order=2, prec="auto", rtol=1e-10, maxit=1_000_000) -> Request:
    """One semi-implicit Cahn-Hilliard step (Sec. 4.1) of the field u into x."""
    _host_f64(u, x)
    if u.shape != x.shape:
        raise ValueError("u and x must have the same shape")
    r = Request()
    r.kind = REQ_CH
    r.solver = 0
    r.ndim, r.order = x.ndim, order
    for a, s in enumerate(reversed(x.shape)):
        r.n[a] = s
    r.prec = _PREC[prec] if isinstance(prec, str) else int(prec)
    r.rtol, r.maxit = rtol, maxit
    r.u_host, r.x_host = u.ctypes.data, x.ctypes.data
    r.h_num, r.h_den = int(h[0]), int(h[1])
    r.dt, r.M, r.kappa = dt, M, kappa
    r.chem = 0 if chem == "cubic" else 1
    r.rho, r.ca, r.cb = rho, ca, cb
    return r


def request_bytes(r: Request) -> int:
    return int(lib.sc_request_bytes(ctypes.byref(r)))


class Server:
    """Continuous-batching server of plate problems and Cahn-Hilliard steps on
    the current device."""

    def __init__(self, arena: torch.Tensor, max_active: int = 256, slice_ms: float = 2.0, fail_slice: int = 0,
                 pcg_min_points: int = 0):
        if not arena.is_cuda:
            raise ValueError("arena must be a CUDA tensor")
        self._arena = arena
        cfg = ServerCfg(arena.data_ptr(), arena.numel() * arena.element_size(), max_active, slice_ms,
                        pcg_min_points, fail_slice)
        h = ctypes.c_void_p()
        check(lib.sc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, f, ghost, x, **kw) -> int:
        """Queues a plate problem; returns its ticket."""
        r = make_request(f, ghost, x, **kw)
        t = ctypes.c_uint64()
        check(lib.sc_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = (f, ghost, x)
        return t.value

    def submit_ch(self, u, x, h, dt, **kw) -> int:
        """Queues one Cahn-Hilliard step of u (result into x); returns its ticket."""
        r = make_ch_request(u, x, h, dt, **kw)
        t = ctypes.c_uint64()
        check(lib.sc_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = (u, x)
        return t.value

    def status(self) -> dict:
        err, act, pend = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        free, tot = ctypes.c_size_t(), ctypes.c_size_t()
        check(lib.sc_server_status(self._h, ctypes.byref(err), ctypes.byref(free), ctypes.byref(tot),
                                   ctypes.byref(act), ctypes.byref(pend)))
        return {"worker_error": int(err.value), "free_bytes": int(free.value), "arena_bytes": int(tot.value),
                "active": int(act.value), "pending": int(pend.value)}

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
