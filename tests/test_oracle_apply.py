"""Pins of the oracle's matrix-free apply and CG."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import apply as ap
from oracle import stencil as st
from oracle.cg import cg


def _asym2d():
    return st.outer_product(st.d1_forward(), st.d2_forward())


def test_apply_equals_dense_matrix_periodic_and_zero():
    """Brute force with one-sided stencils, so a sign or axis mix-up fails."""
    rng = np.random.default_rng(1)
    for s, shape in [(_asym2d(), (6, 7)),
                     (st.outer_product(st.outer_product(st.d1_forward(), st.d1_central2()), st.d2_forward()), (5, 4, 6)),
                     (st.bilaplacian(2, 4), (9, 11))]:
        w = {k: float(v) for k, v in s.coeffs}
        x = rng.uniform(-1, 1, shape)
        for bc in ["periodic", "zero"]:
            M = ap.dense_matrix(w, shape, bc).astype(np.float64)
            y = ap.apply(w, x, bc)
            assert np.allclose(y.ravel(), M @ x.ravel(), rtol=1e-13, atol=1e-13)


def test_ghosted_matches_periodic_padding():
    rng = np.random.default_rng(2)
    s = st.bilaplacian(3, 4)
    w = {k: float(v) for k, v in s.coeffs}
    x = rng.uniform(-1, 1, (12, 10, 9))
    R = 4
    xp = np.pad(x, R, mode="wrap")
    assert np.array_equal(ap.apply(w, xp, "ghosted", R), ap.apply(w, x, "periodic"))


@pytest.mark.parametrize("ndim,order,n", [(2, 2, 32), (2, 4, 24), (3, 2, 12), (3, 4, 16)])
def test_fourier_modes_are_eigenvectors(ndim, order, n):
    """On a periodic grid every DFT mode is an eigenvector of Lap o Lap with
    eigenvalue (sum_a lambda(theta_a))^2, lambda the 1D symbol
    (2 - 2cos t)/h^2 or (30 - 32 cos t + 2 cos 2t)/(12 h^2)."""
    h = 1.0 / n
    B = st.bilaplacian(ndim, order)
    w = st.fp_weights(B, Fraction(1, n), np.float64)
    rng = np.random.default_rng(3)
    for _ in range(4):
        ks = rng.integers(0, n, ndim)
        grids = np.meshgrid(*[np.arange(n)] * ndim, indexing="ij")  # array axes (z,)y,x
        phase = sum(2 * np.pi * k * g / n for k, g in zip(ks, grids))
        v = np.cos(phase)
        lam = 0.0
        for k in ks:
            t = 2 * np.pi * k / n
            lam += (2 - 2 * np.cos(t)) / h**2 if order == 2 else (30 - 32 * np.cos(t) + 2 * np.cos(2 * t)) / (12 * h**2)
        sigma = lam * lam
        y = ap.apply(w, v, "periodic")
        scale = sum(abs(x) for x in w.values())
        assert np.max(np.abs(y - sigma * v)) <= 64 * np.finfo(float).eps * scale


def test_checkerboard_is_the_largest_mode():
    """Checkerboard on an even grid: eigenvalue sum|w| h^-4 (64/h^4 for the
    13-point operator)."""
    n = 16
    B = st.bilaplacian(2, 2)
    w = st.fp_weights(B, Fraction(1, n), np.float64)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    v = (-1.0) ** (x + y)
    assert np.array_equal(ap.apply(w, v, "periodic"), 64.0 * n**4 * v)


def test_cg_matches_direct_solve():
    rng = np.random.default_rng(4)
    A = rng.normal(size=(40, 40))
    A = A @ A.T + 40 * np.eye(40)
    b = rng.normal(size=40)
    x, it, res, ok = cg(lambda v: A @ v, b, None, 1e-12)
    assert ok and res <= 1e-11
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-11)
    # exact arithmetic would finish in at most n steps; a well-conditioned
    # 40x40 system stays close to that
    assert it <= 80


def test_cg_zero_rhs_and_x0():
    x, it, res, ok = cg(lambda v: 2 * v, np.zeros(5))
    assert ok and it == 0 and np.all(x == 0)
    b = np.arange(1.0, 6.0)
    x, it, res, ok = cg(lambda v: 2 * v, b, b / 2)
    assert ok and it == 0 and np.allclose(x, b / 2)


def _random_one_sided(ndim, seed):
    """A stencil with random weights on an asymmetric set of offsets (radius
    2, some axes reaching further one way than the other), so that a swapped
    axis, a flipped sign or a ghost ring offset by one shows up."""
    rng = np.random.default_rng(seed)
    coeffs = {}
    for _ in range(9):
        off = tuple(int(v) for v in rng.integers(-1, 3, ndim))
        coeffs[off] = Fraction(int(rng.integers(1, 50)) * (1 if rng.random() < 0.5 else -1), 7)
    coeffs[(2,) + (0,) * (ndim - 1)] = Fraction(3)  # reach radius 2 along x only
    return st.Stencil.make(coeffs, 0)


def _edge_points(shape, rng, nrand):
    """Every corner of the grid, points on every face and edge, and random
    interior points (array-axis order)."""
    pts = set()
    lo_hi = [(0, 1, n - 2, n - 1) for n in shape]
    for p in np.ndindex(*(4,) * len(shape)):
        pts.add(tuple(lo_hi[a][p[a]] for a in range(len(shape))))
    for _ in range(nrand):
        pts.add(tuple(int(rng.integers(0, n)) for n in shape))
    return np.array(sorted(pts))


@pytest.mark.parametrize("ndim,shape", [(2, (9, 13)), (3, (6, 7, 9))])
def test_apply_at_matches_apply_every_boundary(ndim, shape):
    """apply_at (one point at a time) against the whole-grid apply for every
    boundary treatment, on one-sided stencils (forward-difference outer
    products and random asymmetric ones), at every corner, face and edge and
    at random points: the same sum, so agreement to 1e-15 of sum |w x|."""
    rng = np.random.default_rng(31 + ndim)
    stencils = [_random_one_sided(ndim, 5 + ndim)]
    if ndim == 2:
        stencils.append(st.outer_product(st.d1_forward(), st.d2_forward()))
    else:
        stencils.append(st.outer_product(st.outer_product(st.d1_forward(), st.d2_forward()), st.d1_forward()))
    for s in stencils:
        w = {k: float(v) for k, v in s.coeffs}
        R = s.radius
        absw = {k: abs(v) for k, v in w.items()}
        for bc in ("periodic", "zero", "ghosted"):
            xshape = tuple(n + 2 * R for n in shape) if bc == "ghosted" else shape
            x = rng.uniform(-1, 1, xshape)
            full = ap.apply(w, x, bc, R)
            assert full.shape == shape
            pts = _edge_points(shape, rng, 40)
            got = ap.apply_at(w, x, bc, pts, R)
            ref = full[tuple(pts.T)]
            scale = ap.apply(absw, np.abs(x), bc, R)[tuple(pts.T)]
            assert np.all(np.abs(got - ref) <= 1e-15 * scale), (bc, s)


def test_apply_at_hand_computed_values():
    """Values worked out by hand: a forward difference in x at the last
    column reads the wrapped first column (periodic), nothing (zero), or the
    ghost ring (ghosted)."""
    w = {(1, 0): 1.0, (0, 0): -1.0}  # (x_{i+1} - x_i), offsets in (dx, dy) order
    x = np.arange(12.0).reshape(3, 4)  # rows y, columns x
    pt = np.array([[1, 3]])  # y = 1, x = 3 (last column)
    assert ap.apply_at(w, x, "periodic", pt)[0] == x[1, 0] - x[1, 3]
    assert ap.apply_at(w, x, "zero", pt)[0] == -x[1, 3]
    xg = np.arange(30.0).reshape(5, 6)  # 3 x 4 interior with a ring of width 1
    assert ap.apply_at(w, xg, "ghosted", pt, 1)[0] == xg[2, 5] - xg[2, 4]


def test_varcoef_with_constant_coefficient_is_the_composed_stencil():
    """A constant coefficient m0 between the factors gives m0 times the
    composed stencil (Eq. C=B(A))."""
    rng = np.random.default_rng(12)
    outer = st.embed(st.d1_central2(), 2, 0)
    inner = st.compose(st.embed(st.d1_central2(), 2, 0), st.embed(st.d2_central2(), 2, 0))
    wo = {k: float(v) for k, v in outer.coeffs}
    wi = {k: float(v) for k, v in inner.coeffs}
    wc = {k: float(v) for k, v in st.compose(outer, inner).coeffs}
    x = rng.uniform(-1, 1, (12, 17))
    y = ap.apply_varcoef(wo, wi, np.full(x.shape, 2.5), x)
    assert np.allclose(y, 2.5 * ap.apply(wc, x, "periodic"), rtol=0, atol=1e-12)


def test_varcoef_is_exact_for_quartic_data_and_linear_mobility():
    """d/dx(M d/dx(d2/dx2 x^4)) with M = a + b x is 24 a + 48 b x, and the
    central stencils reproduce it exactly (d2c2 x^4 = 12 x^2 + 2 h^2, whose
    central derivative is 24 x; M times that is quadratic, whose central
    derivative is exact).  Checked in exact rationals on points away from the
    periodic seam."""
    h = Fraction(1, 4)
    n = 40
    xs = [h * i for i in range(n)]
    a, b = Fraction(3, 2), Fraction(-2, 5)
    d1 = {k[0]: v / h for k, v in st.d1_central2().coeffs}
    d2 = {k[0]: v / (h * h) for k, v in st.d2_central2().coeffs}
    f = [xv ** 4 for xv in xs]
    t1 = {i: sum(w * f[i + o] for o, w in d2.items()) for i in range(2, n - 2)}
    t2 = {i: sum(w * t1[i + o] for o, w in d1.items()) for i in range(3, n - 3)}
    mt = {i: (a + b * xs[i]) * t2[i] for i in t2}
    y = {i: sum(w * mt[i + o] for o, w in d1.items()) for i in range(4, n - 4)}
    assert all(y[i] == 24 * a + 48 * b * xs[i] for i in y)
    # the oracle's floating-point evaluation agrees on the same interior points
    wo = {(k,): float(v) for k, v in d1.items()}
    wi = {(k,): float(v) for k, v in d2.items()}
    wi3 = {}
    for (k1,), v1 in wo.items():
        for (k2,), v2 in wi.items():
            wi3[(k1 + k2,)] = wi3.get((k1 + k2,), 0.0) + v1 * v2
    yo = ap.apply_varcoef(wo, wi3, np.array([float(a + b * xv) for xv in xs]), np.array([float(v) for v in f]))
    for i in range(6, n - 6):
        assert abs(yo[i] - float(y[i])) <= 1e-9 * max(1.0, abs(float(y[i])))
