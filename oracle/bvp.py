"""The biharmonic boundary-value problem of Sec. 3.3.

Oracle (test infrastructure only; see ``oracle/__init__.py``).

Lap(Lap f) = g on the unit square (or cube) with the simply supported plate
data of Sec. 3.3, Eq. bc: f = 0 and the normal second derivative = 0 on the
boundary, for the manufactured f = prod_a sin(k_a pi x_a), giving
g = pi^4 (sum_a k_a^2)^2 f (the paper's case is k = (1, 1), g = 4 pi^4 f).

Readings of what the paper leaves open:
  * grid: N interior nodes per axis, h = 1/(N+1), x_i = i h, i = 1..N;
  * "exact" boundary data: the R-wide ghost ring around the interior
    (R = stencil radius: boundary node plus outer nodes) holds the exact f;
    the composed stencil is applied at interior nodes only and the ghost
    contribution moves to the right-hand side, b = g - A_ghost(ring);
  * "odd_reflect" boundary data: f_0 = 0 and f_{-m} = -f_m about each
    boundary node (the central-difference form of f = 0, f_xx = 0), which
    turns Lap o Lap into the square of the Dirichlet Laplacian.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import apply as ap
from .cg import cg


def interior_shape(n: int, ndim: int) -> tuple:
    return (n,) * ndim


def rhs_exact_ghost(weights: dict, g_int: np.ndarray, ring: np.ndarray, R: int) -> np.ndarray:
    """b = g - A(ring with zero interior) on the interior (Sec. 3.3 with the
    ghost ring known)."""
    z = np.array(ring, dtype=np.float64, copy=True)
    inner = tuple(slice(R, s - R) for s in z.shape)
    z[inner] = 0.0
    return np.asarray(g_int, dtype=np.float64) - ap.apply(weights, z, "ghosted", R)


def apply_interior(weights: dict, x: np.ndarray, R: int) -> np.ndarray:
    """The homogeneous interior operator (zero ghost ring)."""
    return ap.apply(weights, x, "zero", R)


def pad_odd(x: np.ndarray, R: int) -> np.ndarray:
    """Ghost ring by odd reflection about the boundary nodes 0 and N+1:
    value 0 on the boundary node, -x_m at distance m beyond it."""
    out = np.asarray(x, dtype=np.float64)
    for ax in range(out.ndim):
        n = out.shape[ax]
        parts = []
        # low side: array positions for nodes (1-R) .. 0
        for node in range(1 - R, 1):
            if node == 0:
                parts.append(np.zeros_like(np.take(out, [0], axis=ax)))
            else:
                parts.append(-np.take(out, [-node - 1], axis=ax))
        parts.append(out)
        for node in range(n + 1, n + R + 1):
            if node == n + 1:
                parts.append(np.zeros_like(np.take(out, [0], axis=ax)))
            else:
                m = node - (n + 1)  # distance beyond the boundary node
                parts.append(-np.take(out, [n - m], axis=ax))
        out = np.concatenate(parts, axis=ax)
    return out


def apply_odd(weights: dict, x: np.ndarray, R: int) -> np.ndarray:
    return ap.apply(weights, pad_odd(x, R), "ghosted", R)


def solve_exact_ghost(weights: dict, g_int, ring, R: int, rtol=1e-10, maxit=1_000_000):
    """CG from x0 = 0 on the interior system.  Returns (x, iters, relres, ok)."""
    b = rhs_exact_ghost(weights, g_int, ring, R)
    return cg(lambda v: apply_interior(weights, v, R), b, None, rtol, maxit)


def assemble_interior(weights: dict, shape: tuple) -> sp.csr_matrix:
    """Sparse matrix of the interior operator (zero ghosts), for the
    independent direct solve."""
    ndim = len(shape)
    npts = int(np.prod(shape))
    idx = np.arange(npts).reshape(shape)
    rows, cols, vals = [], [], []
    for k, w in weights.items():
        sh = tuple(reversed(k))
        # row i couples to column i + s wherever both lie inside the grid
        src = [slice(max(0, -s), n - max(0, s)) for s, n in zip(sh, shape)]
        dst = [slice(a.start + s, a.stop + s) for a, s in zip(src, sh)]
        r = idx[tuple(src)].ravel()
        c = idx[tuple(dst)].ravel()
        rows.append(r)
        cols.append(c)
        vals.append(np.full(r.shape, w, dtype=np.float64))
    if ndim == 0:
        raise ValueError("empty shape")
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(npts, npts))


def solve_direct(weights: dict, g_int, ring, R: int) -> np.ndarray:
    """Sparse direct solve of the same interior system (library oracle)."""
    b = rhs_exact_ghost(weights, g_int, ring, R)
    A = assemble_interior(weights, b.shape)
    return spla.spsolve(A.tocsc(), b.ravel()).reshape(b.shape)
