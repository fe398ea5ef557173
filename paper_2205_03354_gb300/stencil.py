"""Exact stencils: a ctypes mirror of ``sc_stencil`` and the host-only
algebra entry points (composition, Laplacians, weights)."""
from __future__ import annotations

import ctypes
from fractions import Fraction

import numpy as np

from ._lib_loader import check, lib

MAX_PTS = 2197
D1_C2, D2_C2, D1_C4, D2_C4, D1_FWD, D2_FWD = range(6)
_F64, _F32 = 0, 1


class Stencil(ctypes.Structure):
    """Mirror of sc_stencil: weight at off[i] is num[i]/den * h^-hpow."""

    _fields_ = [("ndim", ctypes.c_int32), ("npts", ctypes.c_int32), ("hpow", ctypes.c_int32),
                ("radius", ctypes.c_int32), ("den", ctypes.c_int64),
                ("off", (ctypes.c_int32 * 3) * MAX_PTS), ("num", ctypes.c_int64 * MAX_PTS)]

    def points(self) -> dict:
        """{(dx[, dy[, dz]]): Fraction} of the exact coefficients."""
        out = {}
        for i in range(self.npts):
            k = tuple(int(self.off[i][a]) for a in range(self.ndim))
            out[k] = Fraction(int(self.num[i]), int(self.den))
        return out

    def __repr__(self):
        return f"Stencil(ndim={self.ndim}, npts={self.npts}, hpow={self.hpow}, radius={self.radius})"


_P = ctypes.POINTER(Stencil)
for name, args in [("sc_stencil_1d", [ctypes.c_int32, _P]),
                   ("sc_stencil_embed", [_P, ctypes.c_int32, ctypes.c_int32, _P]),
                   ("sc_stencil_add", [_P, _P, _P]),
                   ("sc_laplacian", [ctypes.c_int32, ctypes.c_int32, _P]),
                   ("sc_compose_stencil", [_P, _P, _P]),
                   ("sc_stencil_weights", [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p])]:
    getattr(lib, name).argtypes = args
    getattr(lib, name).restype = ctypes.c_int


def stencil_1d(kind: int) -> Stencil:
    out = Stencil()
    check(lib.sc_stencil_1d(kind, ctypes.byref(out)))
    return out


def stencil_embed(s1d: Stencil, ndim: int, axis: int) -> Stencil:
    out = Stencil()
    check(lib.sc_stencil_embed(ctypes.byref(s1d), ndim, axis, ctypes.byref(out)))
    return out


def stencil_add(a: Stencil, b: Stencil) -> Stencil:
    out = Stencil()
    check(lib.sc_stencil_add(ctypes.byref(a), ctypes.byref(b), ctypes.byref(out)))
    return out


def laplacian(ndim: int, order: int) -> Stencil:
    out = Stencil()
    check(lib.sc_laplacian(ndim, order, ctypes.byref(out)))
    return out


def compose_stencil(outer: Stencil, inner: Stencil) -> Stencil:
    out = Stencil()
    check(lib.sc_compose_stencil(ctypes.byref(outer), ctypes.byref(inner), ctypes.byref(out)))
    return out


def stencil_weights(s: Stencil, h_num: int, h_den: int, dtype=np.float64) -> np.ndarray:
    """Correctly rounded weights for h = h_num/h_den, in the order of s.off."""
    dt = np.dtype(dtype)
    out = np.zeros(s.npts, dtype=dt)
    code = _F64 if dt == np.float64 else _F32
    check(lib.sc_stencil_weights(ctypes.byref(s), h_num, h_den, code,
                                 out.ctypes.data_as(ctypes.c_void_p)))
    return out
