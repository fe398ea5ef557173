"""Matrix-free FP64 apply of a stencil on a structured grid, and a dense
matrix builder for tiny grids.

Oracle (test infrastructure only; see ``oracle/__init__.py``).

y_i = sum_k w_k x_{i+k}: the stencil's definition (Def. 2.1, the weighted
sum of source values around each target point), evaluated at every grid
point with numpy shifted slices, in a fixed order of the offsets.  Arrays are
indexed [z][y][x] (or [y][x]); an offset vector is (dx, dy[, dz]) in the order
of the paper's (x, y, z) and is mapped onto the reversed array axes.

Boundary handling (the paper is silent on discrete boundaries for the apply):
  "periodic" : indices wrap around (the Cahn-Hilliard domain of Sec. 4.1);
  "ghosted"  : x carries an R-wide ghost ring, y covers the interior only;
  "zero"     : values outside the grid are zero (the homogeneous operator the
               Krylov solve uses after the ghost data moved to the RHS).
"""
from __future__ import annotations

import numpy as np


def _axis_shift(off: tuple) -> tuple:
    """offset (dx, dy, dz...) -> per-array-axis shift (..., dy, dx)."""
    return tuple(reversed(off))


def apply(weights: dict, x: np.ndarray, bc: str, radius: int | None = None) -> np.ndarray:
    """FP64 matrix-free apply.  ``weights``: {offset -> float}."""
    x = np.asarray(x, dtype=np.float64)
    offs = sorted(weights)
    if radius is None:
        radius = max(max(abs(v) for v in k) for k in offs)
    R = radius
    if bc == "periodic":
        y = np.zeros_like(x)
        for k in offs:
            sh = _axis_shift(k)
            # np.roll(x, -s)[i] == x[i + s]
            y += weights[k] * np.roll(x, tuple(-s for s in sh), axis=tuple(range(x.ndim)))
        return y
    if bc == "zero":
        xp = np.pad(x, R)
        return apply(weights, xp, "ghosted", R)
    if bc == "ghosted":
        n = tuple(s - 2 * R for s in x.shape)
        if min(n) < 0:
            raise ValueError("ghosted input smaller than its ghost ring")
        y = np.zeros(n, dtype=np.float64)
        for k in offs:
            sh = _axis_shift(k)
            sl = tuple(slice(R + s, R + s + m) for s, m in zip(sh, n))
            y += weights[k] * x[sl]
        return y
    raise ValueError(f"unknown bc {bc!r}")


def dense_matrix(coeffs: dict, shape: tuple, bc: str) -> np.ndarray:
    """Dense matrix M with (M x)_i = sum_k c_k x_{i+k} on a tiny grid, built
    entry by entry with Python loops (object dtype keeps Fractions exact).

    bc = "periodic": rows and columns both index the N^d grid (wrapping);
    bc = "zero":     rows and columns index the grid, out-of-grid sources drop.
    """
    ndim = len(shape)
    npts = int(np.prod(shape))
    M = np.zeros((npts, npts), dtype=object)
    M[:] = 0
    idx = np.arange(npts).reshape(shape)
    for flat in range(npts):
        pos = np.unravel_index(flat, shape)  # array order (.., y, x)
        for k, c in coeffs.items():
            sh = _axis_shift(k)
            tgt = []
            ok = True
            for p, s, n in zip(pos, sh, shape):
                q = p + s
                if bc == "periodic":
                    q %= n
                elif not (0 <= q < n):
                    ok = False
                    break
                tgt.append(q)
            if ok:
                M[flat, idx[tuple(tgt)]] += c
    if ndim == 0:
        raise ValueError("empty shape")
    return M


def apply_at(weights: dict, x: np.ndarray, bc: str, points: np.ndarray, radius: int | None = None) -> np.ndarray:
    """The same sum evaluated only at the listed output points (rows of array
    indices in array-axis order), one point at a time: lets a full-size
    device result be checked on a sample."""
    x = np.asarray(x)
    offs = sorted(weights)
    if radius is None:
        radius = max(max(abs(v) for v in k) for k in offs)
    R = radius
    out = np.zeros(len(points), dtype=np.float64)
    shape_out = tuple(s - 2 * R for s in x.shape) if bc == "ghosted" else x.shape
    for n, p in enumerate(points):
        acc = 0.0
        for k in offs:
            sh = _axis_shift(k)
            idx = []
            ok = True
            for pi, s, m in zip(p, sh, shape_out):
                q = int(pi) + s
                if bc == "periodic":
                    q %= m
                elif bc == "ghosted":
                    q += R
                elif not (0 <= q < m):
                    ok = False
                    break
                idx.append(q)
            if ok:
                acc += float(weights[k]) * float(x[tuple(idx)])
        out[n] = acc
    return out


def apply_varcoef(outer: dict, inner: dict, m: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = outer(m * inner(x)) on a periodic grid: the composition of Sec.
    2.2.3 with a pointwise coefficient between the factors (the variable
    mobility of d/dx(M d/dx(d2/dx2 f)): compose d/dx with d2/dx2, scale by M
    at each grid point, compose the result with d/dx)."""
    t = apply(inner, x, "periodic")
    return apply(outer, np.asarray(m, dtype=np.float64) * t, "periodic")
