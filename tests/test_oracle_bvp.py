"""Pins of the oracle's biharmonic BVP (Sec. 3.3)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import apply as ap
from oracle import bvp
from oracle import stencil as st
from synth_inputs import manufactured


def _setup(n, ndim=2, order=2, ks=None):
    B = st.bilaplacian(ndim, order)
    R = B.radius
    w = st.fp_weights(B, Fraction(1, n + 1), np.float64)
    m = manufactured.bvp_case(n, ndim, R, ks or (1,) * ndim)
    return w, R, m


def test_polynomial_solution_is_reproduced_exactly():
    """Lap o Lap is exact on polynomials of degree <= 5 (moment conditions),
    so with the ghost ring holding a quintic the discrete solution IS the
    quintic at the nodes.  Catches a wrong ghost ring, RHS sign or index."""
    n, R = 12, 2
    h = 1.0 / (n + 1)
    B = st.bilaplacian(2, 2)
    w = st.fp_weights(B, Fraction(1, n + 1), np.float64)
    idx = np.arange(1 - R, n + R + 1) * h
    Y, X = np.meshgrid(idx, idx, indexing="ij")

    def u(x, y):
        return x**4 / 24 + x**2 * y**2 / 4 - 0.3 * x**3 * y + y**5 - 2 * x * y + 0.7

    def g(x, y):  # Delta^2 u
        return 1.0 + 2.0 + 120.0 * y

    ring = u(X, Y)
    gi = g(X[R:-R, R:-R], Y[R:-R, R:-R])
    x, it, res, ok = bvp.solve_exact_ghost(w, gi, ring, R, rtol=1e-13)
    assert ok
    assert np.max(np.abs(x - ring[R:-R, R:-R])) < 1e-9


def test_cg_matches_sparse_direct_solve():
    for n in (16, 24):
        w, R, m = _setup(n)
        x, it, res, ok = bvp.solve_exact_ghost(w, m["g"], m["u_padded"], R, rtol=1e-12)
        xd = bvp.solve_direct(w, m["g"], m["u_padded"], R)
        assert ok
        assert np.max(np.abs(x - xd)) <= 1e-9 * np.max(np.abs(xd))


def test_second_order_convergence():
    """Sec. 3.3: composing second-order Laplacians gives a second-order
    biharmonic solve (l_inf error vs the exact solution)."""
    errs = []
    for n in (16, 32, 64):
        w, R, m = _setup(n)
        x, it, res, ok = bvp.solve_exact_ghost(w, m["g"], m["u_padded"], R, rtol=1e-10)
        assert ok and res <= 1e-10
        errs.append(np.max(np.abs(x - m["u_exact"])))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < r < 2.3 for r in rates), (errs, rates)


def test_odd_reflection_is_dirichlet_laplacian_squared():
    """With the odd-reflection ghost reading, the interior operator equals
    L_D^2 (L_D the Dirichlet Laplacian), entry for entry."""
    n, R = 6, 2
    B = st.bilaplacian(2, 2)
    L = st.laplacian(2, 2)
    wB = {k: float(v) for k, v in B.coeffs}
    wL = {k: float(v) for k, v in L.coeffs}
    LD = ap.dense_matrix(wL, (n, n), "zero").astype(np.float64)
    cols = []
    for j in range(n * n):
        e = np.zeros(n * n)
        e[j] = 1.0
        cols.append(bvp.apply_odd(wB, e.reshape(n, n), R).ravel())
    A = np.array(cols).T
    assert np.array_equal(A, LD @ LD)


def test_odd_reflection_closed_form():
    """The discrete solution for g = 4 pi^4 sin(pi x) sin(pi y) is
    (4 pi^4 / mu) sin(pi x) sin(pi y), mu = 64 sin^4(pi h / 2)/h^4."""
    n, R = 20, 2
    h = 1.0 / (n + 1)
    B = st.bilaplacian(2, 2)
    w = st.fp_weights(B, Fraction(1, n + 1), np.float64)
    xs = np.arange(1, n + 1) * h
    Y, X = np.meshgrid(xs, xs, indexing="ij")
    u = np.sin(np.pi * X) * np.sin(np.pi * Y)
    g = 4 * np.pi**4 * u
    from oracle.cg import cg
    x, it, res, ok = cg(lambda v: bvp.apply_odd(w, v, R), g, None, 1e-13)
    mu = 64 * np.sin(np.pi * h / 2) ** 4 / h**4
    assert ok
    assert np.max(np.abs(x - 4 * np.pi**4 / mu * u)) < 1e-9


@pytest.mark.parametrize("ndim,order", [(3, 2), (2, 4)])
def test_other_operators_converge(ndim, order):
    """The 25-point 3D and 33-point 4th-order 2D biharmonic solves converge at
    their order with exact ghosts (errors shrink by ~2^order)."""
    errs = []
    ns = (8, 16) if ndim == 3 else (16, 32)
    for n in ns:
        w, R, m = _setup(n, ndim, order)
        x, it, res, ok = bvp.solve_exact_ghost(w, m["g"], m["u_padded"], R, rtol=1e-12)
        assert ok
        errs.append(np.max(np.abs(x - m["u_exact"])))
    rate = np.log2(errs[0] / errs[1])
    assert rate > order - 0.4, (errs, rate)
