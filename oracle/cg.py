"""Textbook conjugate gradients (Hestenes-Stiefel) in FP64.

Oracle (test infrastructure only; see ``oracle/__init__.py``).

The paper solves its linear systems through PETSc without naming the Krylov
method or a preconditioner (Sec. 4); the reading taken here is unpreconditioned
CG, which applies because the composed operators used (the biharmonic on the
interior with the ghost data moved to the right-hand side, and
I + dt eps^2 Lap o Lap on a periodic grid) are symmetric positive definite.
"""
from __future__ import annotations

import numpy as np


def cg(matvec, b: np.ndarray, x0: np.ndarray | None = None, rtol: float = 1e-10,
       maxit: int = 1_000_000):
    """Solve A x = b.  Stops when ||b - A x_k||_2 <= rtol ||b||_2 measured on the
    recurrence residual, then reports the true residual too.

    Returns (x, iterations, true relative residual, converged flag)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - matvec(x)
    bnorm = float(np.sqrt(np.vdot(b, b)))
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, True
    p = r.copy()
    rr = float(np.vdot(r, r))
    it = 0
    converged = np.sqrt(rr) <= rtol * bnorm
    while not converged and it < maxit:
        q = matvec(p)
        pq = float(np.vdot(p, q))
        if not pq > 0.0:
            break
        alpha = rr / pq
        x += alpha * p
        r -= alpha * q
        rr_new = float(np.vdot(r, r))
        it += 1
        converged = np.sqrt(rr_new) <= rtol * bnorm
        beta = rr_new / rr
        rr = rr_new
        p = r + beta * p
    true_res = float(np.linalg.norm(b - matvec(x)) / bnorm)
    return x, it, true_res, bool(converged)
