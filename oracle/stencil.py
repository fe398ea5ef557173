"""Exact-rational finite-difference stencils and stencil composition.

Oracle (test infrastructure only; see ``oracle/__init__.py``).

A stencil is a finite map from integer offset vectors u_i in Z^d to rational
coefficients c_i, together with an integer h-power p: the weight applied at
offset u_i is a_i = c_i * h**(-p)  (Def. 2.1: weights proportional to h^-p,
and x_i - x_0 = h u_i, Sec. 2.1).

Composition C = B(A) (Sec. 2.2, Eq. C=B(A)): offsets add, weights multiply,
  c_k = sum_{u_i + v_j = k} a_i b_j,  p_C = p_A + p_B.
Taylor vector (Eq. CompactNotation): t_alpha = sum_i c_i u_i^alpha / alpha!.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass
from fractions import Fraction

import numpy as np


@dataclass(frozen=True)
class Stencil:
    """coeffs: {offset tuple -> Fraction}; hpow: weights scale as h**-hpow."""

    coeffs: tuple  # tuple of (offset tuple, Fraction), sorted by offset
    hpow: int

    @staticmethod
    def make(coeffs: dict, hpow: int) -> "Stencil":
        items = [(tuple(int(v) for v in k), Fraction(c)) for k, c in coeffs.items()]
        items = [(k, c) for k, c in items if c != 0]
        dims = {len(k) for k, _ in items}
        if len(dims) > 1:
            raise ValueError("mixed dimensions in one stencil")
        return Stencil(tuple(sorted(items)), int(hpow))

    @property
    def ndim(self) -> int:
        return len(self.coeffs[0][0]) if self.coeffs else 0

    def as_dict(self) -> dict:
        return dict(self.coeffs)

    @property
    def npts(self) -> int:
        return len(self.coeffs)

    @property
    def radius(self) -> int:
        return max((max(abs(v) for v in k) for k, _ in self.coeffs), default=0)


# ---------------------------------------------------------------------------
# 1D building blocks printed in the paper (weights a_i = c_i / h^p)
# ---------------------------------------------------------------------------

def d1_central2() -> Stencil:
    """(f(x_1) - f(x_-1)) / (2h): Sec. 2.1.1, Eq. f'stencil.

    Some passages (Sec. 3.1 and the order-of-accuracy example) print the
    weights as {1/h, -1/h}; the Taylor vectors the paper derives need 1/(2h),
    which is the reading used here.
    """
    return Stencil.make({(1,): Fraction(1, 2), (-1,): Fraction(-1, 2)}, 1)


def d2_central2() -> Stencil:
    """[1, -2, 1] / h^2: Sec. 2.1.2, Eq. CenterSecondDerivative."""
    return Stencil.make({(-1,): 1, (0,): -2, (1,): 1}, 2)


def d1_central4() -> Stencil:
    """(8 f_1 - f_2 + f_-2 - 8 f_-1) / (12h): Sec. 2.2.2, Eq. 4orderf'."""
    return Stencil.make({(1,): Fraction(8, 12), (2,): Fraction(-1, 12),
                         (-2,): Fraction(1, 12), (-1,): Fraction(-8, 12)}, 1)


def d2_central4() -> Stencil:
    """[-1, 16, -30, 16, -1] / (12 h^2): the fourth-order second derivative the
    paper composes with itself in Sec. 3.2 (the integer weights are those of
    the apply-sweep workload; the paper does not print them)."""
    return Stencil.make({(-2,): Fraction(-1, 12), (-1,): Fraction(16, 12),
                         (0,): Fraction(-30, 12), (1,): Fraction(16, 12),
                         (2,): Fraction(-1, 12)}, 2)


def d1_forward() -> Stencil:
    """(f(x_1) - f(x_0)) / h: Sec. 2.2.1 and Appendix A."""
    return Stencil.make({(1,): 1, (0,): -1}, 1)


def d2_forward() -> Stencil:
    """(f(x_2) - 2 f(x_1) + f(x_0)) / h^2: Sec. 2.2.1 and Appendix A."""
    return Stencil.make({(2,): 1, (1,): -2, (0,): 1}, 2)


STENCIL_1D = {
    "d1_c2": d1_central2, "d2_c2": d2_central2, "d1_c4": d1_central4,
    "d2_c4": d2_central4, "d1_fwd": d1_forward, "d2_fwd": d2_forward,
}


# ---------------------------------------------------------------------------
# Algebra
# ---------------------------------------------------------------------------

def compose(outer: Stencil, inner: Stencil) -> Stencil:
    """C = B(A) with B = outer, A = inner (Sec. 2.2, Eq. C=B(A)).

    Every source point x_i of A is shifted by every point x_j of B and weighted
    by a_i b_j; the h-powers add (derivative order abar + bbar)."""
    if outer.ndim != inner.ndim:
        raise ValueError("composition needs stencils of equal dimension")
    acc: dict = {}
    for vj, bj in outer.coeffs:
        for ui, ai in inner.coeffs:
            k = tuple(a + b for a, b in zip(ui, vj))
            acc[k] = acc.get(k, Fraction(0)) + ai * bj
    return Stencil.make(acc, outer.hpow + inner.hpow)


def add(a: Stencil, b: Stencil) -> Stencil:
    """Linear combination of two stencils with the same h-power (Sec. 2.1: the
    Taylor series of source points form a vector space)."""
    if a.hpow != b.hpow or a.ndim != b.ndim:
        raise ValueError("can only add stencils with equal h-power and dimension")
    acc = a.as_dict()
    for k, c in b.coeffs:
        acc[k] = acc.get(k, Fraction(0)) + c
    return Stencil.make(acc, a.hpow)


def embed(s1d: Stencil, ndim: int, axis: int) -> Stencil:
    """A 1D stencil acting along ``axis`` of a ``ndim``-dimensional lattice
    (the identity on the other axes), Sec. 2.3."""
    if s1d.ndim != 1:
        raise ValueError("embed takes a 1D stencil")
    out = {}
    for (k,), c in s1d.coeffs:
        off = [0] * ndim
        off[axis] = k
        out[tuple(off)] = c
    return Stencil.make(out, s1d.hpow)


def outer_product(sx: Stencil, sy: Stencil) -> Stencil:
    """Composition of stencils acting on different axes = outer (tensor)
    product, Sec. 2.3.  Offsets are concatenated, h-powers add."""
    out = {}
    for kx, cx in sx.coeffs:
        for ky, cy in sy.coeffs:
            out[kx + ky] = cx * cy
    return Stencil.make(out, sx.hpow + sy.hpow)


def laplacian(ndim: int, order: int) -> Stencil:
    """Sum over axes of the 1D second-derivative stencil of the given order
    (2 -> [1,-2,1]/h^2, 4 -> [-1,16,-30,16,-1]/(12h^2)); Sec. 3.3 builds the
    Laplacian once and composes it with itself."""
    base = {2: d2_central2, 4: d2_central4}[order]()
    s = embed(base, ndim, 0)
    for ax in range(1, ndim):
        s = add(s, embed(base, ndim, ax))
    return s


def bilaplacian(ndim: int, order: int) -> Stencil:
    """Lap o Lap by composition (Sec. 3.3)."""
    lap = laplacian(ndim, order)
    return compose(lap, lap)


# ---------------------------------------------------------------------------
# Taylor vectors (Eq. CompactNotation) and validity rules (Def. 2.2)
# ---------------------------------------------------------------------------

def taylor_coeff(s: Stencil, alpha: tuple) -> Fraction:
    """t_alpha = sum_i c_i u_i^alpha / alpha!  (multi-index, exact)."""
    tot = Fraction(0)
    denom = 1
    for a in alpha:
        denom *= math.factorial(a)
    for u, c in s.coeffs:
        term = 1
        for ui, a in zip(u, alpha):
            term *= ui ** a
        tot += c * term
    return tot / denom


def taylor_vector_1d(s: Stencil, nterms: int) -> tuple[int, list]:
    """For a 1D stencil return (beta, T) in the paper's notation: beta is the
    derivative order (first alpha with t_alpha != 0), and T lists the
    coefficients of h^j f^(beta+j), j = 0..nterms-1 (Sec. 2.1).  Dividing by
    h^p shifts the series p slots left, so T_j = t_{beta + j}."""
    if s.ndim != 1:
        raise ValueError("1D only")
    beta = None
    for a in range(0, 64):
        if taylor_coeff(s, (a,)) != 0:
            beta = a
            break
    if beta is None:
        raise ValueError("zero stencil")
    return beta, [taylor_coeff(s, (beta + j,)) for j in range(nterms)]


def derivative_and_accuracy_1d(s: Stencil) -> tuple[int, int]:
    """(derivative order, order of accuracy q) per Def. 2.2: the leading
    coefficient must be 1, its index is the derivative order, the next nonzero
    entry sits at index q."""
    beta, T = taylor_vector_1d(s, 24)
    if T[0] != 1:
        raise ValueError("leading Taylor coefficient is not one (Def. 2.2)")
    if beta != s.hpow:
        raise ValueError("derivative order differs from the h-power")
    for j in range(1, len(T)):
        if T[j] != 0:
            return beta, j
    raise ValueError("no error term found within 24 terms")


def taylor_matrix(s: Stencil, beta: tuple, nterms: int) -> list:
    """2D analogue of the paper's outer-product Taylor matrices (Sec. 2.3):
    entry [i][j] is the coefficient of h^(i+j) f^(beta_x+i, beta_y+j)."""
    if s.ndim != 2:
        raise ValueError("2D only")
    return [[taylor_coeff(s, (beta[0] + i, beta[1] + j)) for j in range(nterms)]
            for i in range(nterms)]


def moment(s: Stencil, powers: tuple) -> Fraction:
    """sum_i c_i prod_a u_{i,a}^{powers_a}  (no factorials)."""
    tot = Fraction(0)
    for u, c in s.coeffs:
        term = 1
        for ui, a in zip(u, powers):
            term *= ui ** a
        tot += c * term
    return tot


# ---------------------------------------------------------------------------
# Floating-point weights: exactly the rational c_i * h^-p, rounded once
# ---------------------------------------------------------------------------

def exact_weights(s: Stencil, h: Fraction) -> dict:
    """{offset -> Fraction} of the scaled weights c_i * h^-p for rational h."""
    h = Fraction(h)
    scale = h ** (-s.hpow)
    return {k: c * scale for k, c in s.coeffs}


def round_f64(q: Fraction) -> float:
    """Nearest double to the rational q (Python's int/int true division is
    correctly rounded, ties to even)."""
    return q.numerator / q.denominator


def round_f32(q: Fraction) -> np.float32:
    """Nearest float32 to the rational q, ties to even, decided by exact
    comparison of the candidates around the double nearest to q."""
    guess = np.float32(round_f64(q))
    cands = {guess, np.nextafter(guess, np.float32(np.inf)),
             np.nextafter(guess, np.float32(-np.inf))}
    best = None
    for c in cands:
        if not np.isfinite(c):
            continue
        err = abs(Fraction(float(c)) - q)
        if best is None or err < best[0]:
            best = (err, c)
        elif err == best[0]:
            # tie: keep the candidate with an even significand
            bits_c = int(np.array(c, dtype=np.float32).view(np.uint32))
            if bits_c % 2 == 0:
                best = (err, c)
    return np.float32(best[1])


def fp_weights(s: Stencil, h: Fraction, dtype) -> dict:
    """Correctly rounded floating-point weights {offset -> value}."""
    ex = exact_weights(s, h)
    if np.dtype(dtype) == np.float64:
        return {k: round_f64(v) for k, v in ex.items()}
    if np.dtype(dtype) == np.float32:
        return {k: round_f32(v) for k, v in ex.items()}
    raise ValueError("dtype must be float64 or float32")


def all_offsets_box(ndim: int, r: int):
    """Every offset of the (2r+1)^ndim box, lexicographic."""
    return list(itertools.product(range(-r, r + 1), repeat=ndim))
