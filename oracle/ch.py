"""One semi-implicit Cahn-Hilliard step on a periodic grid (Sec. 4).

Oracle (test infrastructure only; see ``oracle/__init__.py``).

Sec. 4.1, Eq. cahn:  dc/dt = div( M grad( f'(c) - kappa Lap c ) ).
The linear fourth-order part is implicit and the nonlinear part explicit
(Sec. 4.1, last paragraph), with Lap o Lap built by composing the Laplacian
with itself.  One first-order IMEX step therefore solves

    (I + dt M kappa Lap_h o Lap_h) c^{n+1} = c^n + dt M Lap_h f'(c^n).

Free energies:
  "cubic":       f(c) = (c^2 - 1)^2 / 4,  f'(c) = c^3 - c;
  "double_well": f(c) = rho (c - ca)^2 (c - cb)^2   (Sec. 4.1),
                 f'(c) = 2 rho (c - ca)(c - cb)(2c - ca - cb).
Grid reading: N points per axis, spacing h, x_i = i h, periodic.
"""
from __future__ import annotations

import numpy as np

from . import apply as ap
from . import stencil as st
from .cg import cg


def fprime(c: np.ndarray, chem: tuple) -> np.ndarray:
    if chem[0] == "cubic":
        return c ** 3 - c
    if chem[0] == "linear":  # f(c) = a c^2 / 2: a linear model used to pin the time steppers
        return chem[1] * c
    if chem[0] == "double_well":
        _, rho, ca, cb = chem
        return 2.0 * rho * (c - ca) * (c - cb) * (2.0 * c - ca - cb)
    raise ValueError(chem)


def fchem(c: np.ndarray, chem: tuple) -> np.ndarray:
    if chem[0] == "cubic":
        return (c * c - 1.0) ** 2 / 4.0
    if chem[0] == "double_well":
        _, rho, ca, cb = chem
        return rho * (c - ca) ** 2 * (c - cb) ** 2
    raise ValueError(chem)


def operators(ndim: int, h, order: int = 2):
    """FP64 weights of Lap_h and of the composed Lap_h o Lap_h."""
    lap = st.laplacian(ndim, order)
    bil = st.compose(lap, lap)
    return st.fp_weights(lap, h, np.float64), st.fp_weights(bil, h, np.float64)


def rhs(c: np.ndarray, lap_w: dict, dt: float, M: float, chem: tuple) -> np.ndarray:
    """c^n + dt M Lap_h f'(c^n)."""
    return c + dt * M * ap.apply(lap_w, fprime(c, chem), "periodic")


def step(c: np.ndarray, h, dt: float, M: float, kappa: float, chem: tuple,
         rtol: float = 1e-10, order: int = 2, maxit: int = 100000):
    """One IMEX step solved by CG from x0 = c^n.  Returns
    (c_new, iterations, true relative residual, converged)."""
    lap_w, bil_w = operators(c.ndim, h, order)
    b = rhs(c, lap_w, dt, M, chem)
    s = dt * M * kappa

    def matvec(v):
        return v + s * ap.apply(bil_w, v, "periodic")

    return cg(matvec, b, c, rtol, maxit)


def lap_symbol(shape: tuple, h: float, order: int = 2) -> np.ndarray:
    """Eigenvalues of the periodic Lap_h on the DFT modes theta_a = 2 pi k/N:
    sum over axes of the 1D symbol (2 cos t - 2)/h^2 (2nd order) or
    (-2 cos 2t + 32 cos t - 30)/(12 h^2) (4th order)."""
    sym = np.zeros(shape)
    for ax, n in enumerate(shape):
        t = 2.0 * np.pi * np.fft.fftfreq(n)
        if order == 2:
            s1 = (2.0 * np.cos(t) - 2.0) / h ** 2
        else:
            s1 = (-2.0 * np.cos(2 * t) + 32.0 * np.cos(t) - 30.0) / (12.0 * h ** 2)
        bshape = [1] * len(shape)
        bshape[ax] = n
        sym = sym + s1.reshape(bshape)
    return sym


def step_fft(c: np.ndarray, h: float, dt: float, M: float, kappa: float, chem: tuple,
             order: int = 2) -> np.ndarray:
    """The same step solved exactly in the DFT basis, where the periodic
    operators are diagonal (a special case that reduces to numpy.fft)."""
    lam = lap_symbol(c.shape, h, order)
    chat = np.fft.fftn(c)
    fhat = np.fft.fftn(fprime(c, chem))
    new = (chat + dt * M * lam * fhat) / (1.0 + dt * M * kappa * lam * lam)
    return np.real(np.fft.ifftn(new))


def mass(c: np.ndarray) -> float:
    return float(np.sum(c, dtype=np.float64))


def free_energy(c: np.ndarray, h: float, kappa: float, chem: tuple) -> float:
    """F(c) = int f_chem(c) + kappa/2 |grad c|^2 (Sec. 4.1), discretised with
    forward differences on the periodic grid and the midpoint rule."""
    grad2 = np.zeros_like(c)
    for ax in range(c.ndim):
        d = (np.roll(c, -1, axis=ax) - c) / h
        grad2 += d * d
    return float(h ** c.ndim * np.sum(fchem(c, chem) + 0.5 * kappa * grad2))


# Semi-implicit backward differentiation (SBDF) schemes of orders 1-3 for the
# same splitting (the paper uses IMEX schemes of orders one to three in Sec.
# 4.3 without naming them; these are the standard SBDF family).  With
# history u^n, u^(n-1), ... and N(u) = M Lap f'(u):
#   sum_j a_j u^(n+1-j) / dt = -M kappa Lap Lap u^(n+1) + sum_j b_j N(u^(n-j)),
# the BDF coefficients a for the implicit part and the extrapolation b for
# the explicit part.  Divided by a_0:
#   (I + g dt M kappa Lap Lap) u^(n+1) = sum_j al_j u^(n-j) + g dt M Lap sum_j b_j f'(u^(n-j))
# with g = 1 / a_0 and al_j = -a_(j+1) / a_0.
SBDF = {
    1: {"a": (1.0, -1.0), "b": (1.0,)},
    2: {"a": (1.5, -2.0, 0.5), "b": (2.0, -1.0)},
    3: {"a": (11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0), "b": (3.0, -3.0, 1.0)},
}


def sbdf_coefficients(order: int):
    """(al, b, g) of the divided form above."""
    a, b = SBDF[order]["a"], SBDF[order]["b"]
    g = 1.0 / a[0]
    al = tuple(-a[j + 1] / a[0] for j in range(order))
    return al, b, g


def step_sbdf_fft(hist: list, h: float, dt: float, M: float, kappa: float, chem: tuple, order: int,
                  lap_order: int = 2) -> np.ndarray:
    """One SBDF step from hist = [u^n, u^(n-1), ...] (order fields), solved
    exactly in the DFT basis where the periodic operators are diagonal."""
    al, b, g = sbdf_coefficients(order)
    lam = lap_symbol(hist[0].shape, h, lap_order)
    rhs = sum(al[j] * np.fft.fftn(hist[j]) for j in range(order))
    nl = sum(b[j] * np.fft.fftn(fprime(hist[j], chem)) for j in range(order))
    new = (rhs + g * dt * M * lam * nl) / (1.0 + g * dt * M * kappa * lam * lam)
    return np.real(np.fft.ifftn(new))
