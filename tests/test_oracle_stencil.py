"""Pins of the oracle's exact stencil algebra against the paper and against
mathematics that does not depend on the oracle's own composition code."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import apply as ap
from oracle import stencil as st
from tests.conftest import frac


def build(name: str) -> st.Stencil:
    """'a o b o c' -> compose(a, compose(b, c))."""
    parts = [p.strip() for p in name.split(" o ")]
    s = st.STENCIL_1D[parts[-1]]()
    for p in reversed(parts[:-1]):
        s = st.compose(st.STENCIL_1D[p](), s)
    return s


def test_taylor_vectors_match_paper(golden):
    for e in golden["taylor_1d"]:
        s = build(e["name"])
        beta, T = st.taylor_vector_1d(s, len(e["T"]))
        assert beta == e["beta"], e["name"]
        assert T == [frac(t) for t in e["T"]], (e["name"], T)


def test_composed_1d_stencils_match_paper(golden):
    for e in golden["stencils_1d"]:
        s = build(e["name"])
        want = {(int(k),): Fraction(v, e["den"]) for k, v in e["num"].items() if v != 0}
        assert s.as_dict() == want, e["name"]
        assert s.hpow == e["hpow"]


def test_bilaplacian_13pt_matches_paper(golden):
    g = golden["bilaplacian_2d_13pt"]
    want = {tuple(int(v) for v in k.split(",")): Fraction(n, g["den"]) for k, n in g["num"].items()}
    b = st.bilaplacian(2, 2)
    assert b.as_dict() == want
    assert b.hpow == g["hpow"]
    lap = golden["laplacian_2d_5pt"]
    want_l = {tuple(int(v) for v in k.split(",")): Fraction(n) for k, n in lap["num"].items()}
    assert st.laplacian(2, 2).as_dict() == want_l
    # the 5:13 point ratio of the sparsity discussion
    assert (st.laplacian(2, 2).npts, b.npts) == (5, 13)


def test_taylor_matrices_2d_match_paper(golden):
    for e in golden["taylor_2d"]:
        s = st.outer_product(build(e["x"]), build(e["y"]))
        n = len(e["M"])
        M = st.taylor_matrix(s, tuple(e["beta"]), n)
        assert M == [[frac(v) for v in row] for row in e["M"]], (e["x"], e["y"])


def test_composition_is_commutative_and_associative():
    names = list(st.STENCIL_1D)
    for a, b in itertools.product(names, repeat=2):
        A, B = st.STENCIL_1D[a](), st.STENCIL_1D[b]()
        assert st.compose(A, B) == st.compose(B, A)
    A, B, C = st.d1_forward(), st.d2_central4(), st.d1_central2()
    assert st.compose(st.compose(A, B), C) == st.compose(A, st.compose(B, C))
    L = st.laplacian(3, 4)
    D = st.embed(st.d1_forward(), 3, 1)
    assert st.compose(L, D) == st.compose(D, L)


def test_order_of_accuracy_lemma_and_proposition():
    """q_C = min(q_A, q_B) with leading coefficient t_qA, t_qB or their sum
    (Lemma Accuracy, Proposition CoeffAccuracy), over every pair of central
    1D stencils."""
    cen = ["d1_c2", "d2_c2", "d1_c4", "d2_c4"]
    for a, b in itertools.product(cen, repeat=2):
        A, B = st.STENCIL_1D[a](), st.STENCIL_1D[b]()
        pa, qa = st.derivative_and_accuracy_1d(A)
        pb, qb = st.derivative_and_accuracy_1d(B)
        C = st.compose(B, A)
        pc, qc = st.derivative_and_accuracy_1d(C)
        assert pc == pa + pb
        assert qc == min(qa, qb)
        ta = st.taylor_vector_1d(A, qa + 1)[1][qa]
        tb = st.taylor_vector_1d(B, qb + 1)[1][qb]
        tc = st.taylor_vector_1d(C, qc + 1)[1][qc]
        want = (ta + tb) if qa == qb else (ta if qa < qb else tb)
        assert tc == want, (a, b)


@pytest.mark.parametrize("ndim,order", [(2, 2), (3, 2), (2, 4), (3, 4)])
def test_bilaplacian_moment_conditions(ndim, order):
    """Lap o Lap reproduces Delta^2 exactly on polynomials up to degree 5:
    sum w = 0, odd moments vanish, second moments vanish, and
    Delta^2 (x^4/24) = 1, Delta^2 (x^2 y^2 / 4) = 2 (written as moments)."""
    B = st.bilaplacian(ndim, order)
    for powers in itertools.product(range(6), repeat=ndim):
        deg = sum(powers)
        if deg > 5:
            continue
        m = st.moment(B, powers)
        fact = math.prod(math.factorial(p) for p in powers)
        t = m / fact
        if deg == 4:
            if max(powers) == 4:
                assert t == 1, powers
            elif sorted(powers)[-2:] == [2, 2]:
                assert t == 2, powers
            else:
                assert t == 0, powers
        else:
            assert t == 0, powers
    # derivative order 4 = 2 + 2
    assert B.hpow == 4
    # leading error term: 2nd order -> coefficient of h^2 d^6/dx^6 is 1/12+1/12
    six = [0] * ndim
    six[0] = 6
    t6 = st.moment(B, tuple(six)) / math.factorial(6)
    if order == 2:
        assert t6 == Fraction(1, 6)
    else:  # fourth order: the h^2 term vanishes, the h^4 term is -1/90-1/90
        assert t6 == 0
        eight = [0] * ndim
        eight[0] = 8
        assert st.moment(B, tuple(eight)) / math.factorial(8) == Fraction(-1, 45)


def test_derived_bilaplacian_weights():
    """Point counts and weight classes of the composed operators the hot path
    applies (13, 25, 33 and 73 points), pinned independently by the dense
    matrix product below."""
    assert [st.bilaplacian(d, o).npts for d, o in [(2, 2), (3, 2), (2, 4), (3, 4)]] == [13, 25, 33, 73]
    b33 = {k: v * 144 for k, v in st.bilaplacian(2, 4).coeffs}
    assert b33[(0, 0)] == 4628 and b33[(1, 0)] == -1952 and b33[(2, 0)] == 376
    assert b33[(3, 0)] == -32 and b33[(4, 0)] == 1 and b33[(1, 1)] == 512
    assert b33[(2, 1)] == -32 and b33[(2, 2)] == 2
    b73 = {k: v * 144 for k, v in st.bilaplacian(3, 4).coeffs}
    assert b73[(0, 0, 0)] == 9642 and b73[(1, 0, 0)] == -2912 and b73[(2, 0, 0)] == 436
    b25 = st.bilaplacian(3, 2).as_dict()
    assert b25[(0, 0, 0)] == 42 and b25[(1, 0, 0)] == -12 and b25[(1, 1, 0)] == 2 and b25[(2, 0, 0)] == 1
    for d, o in [(2, 2), (3, 2), (2, 4), (3, 4)]:
        assert sum(st.bilaplacian(d, o).as_dict().values()) == 0


@pytest.mark.parametrize("ndim,order,n", [(2, 2, 5), (2, 2, 6), (2, 4, 9), (3, 2, 5)])
def test_composed_matrix_equals_matrix_product(ndim, order, n):
    """Brute force: on a periodic grid the matrix of Lap o Lap equals the
    product of two Laplacian matrices, entry for entry in exact arithmetic."""
    L = st.laplacian(ndim, order)
    B = st.compose(L, L)
    shape = (n,) * ndim
    ML = ap.dense_matrix(L.as_dict(), shape, "periodic")
    MB = ap.dense_matrix(B.as_dict(), shape, "periodic")
    assert (ML.dot(ML) == MB).all()


def test_asymmetric_composition_matrix_product():
    """Composition order and offset signs, caught with one-sided stencils:
    the matrix of B(A) equals M_B M_A on a periodic grid."""
    A = st.outer_product(st.d1_forward(), st.d2_forward())
    Bs = st.outer_product(st.d2_forward(), st.d1_central4())
    C = st.compose(Bs, A)
    shape = (7, 6)
    MA = ap.dense_matrix(A.as_dict(), shape, "periodic")
    MB = ap.dense_matrix(Bs.as_dict(), shape, "periodic")
    MC = ap.dense_matrix(C.as_dict(), shape, "periodic")
    assert (MB.dot(MA) == MC).all()


def test_table3_nonzero_counts(golden):
    rows = golden["table3"]["rows"][:2]
    for r in rows:
        n = int(200 / r["h"])
        assert n * n == r["size"]
        for s, key in [(st.laplacian(2, 2), "nnz_lap"), (st.bilaplacian(2, 2), "nnz_bilap")]:
            M = ap.dense_matrix({k: float(v) for k, v in s.coeffs}, (n, n), "periodic").astype(np.float64)
            assert int(np.count_nonzero(M)) == r[key]
    # the remaining rows follow from 5 and 13 entries per row on larger grids
    for r in golden["table3"]["rows"]:
        assert r["nnz_lap"] == 5 * r["size"] and r["nnz_bilap"] == 13 * r["size"]


def test_table2_spectral_radius(golden):
    """Spectral radius of B = Lap o Lap on the periodic [0,200]^2 grid (h = 8
    gives an odd grid, N = 25, where the checkerboard mode is absent and the
    radius is 0.0155, not 64/h^4) and of A = I + dt B, dt = h/4."""
    B = st.bilaplacian(2, 2)
    for r in golden["table2"]["rows"][:2]:
        h = r["h"]
        n = int(round(200 / h))
        w = st.fp_weights(B, Fraction(h), np.float64)
        M = ap.dense_matrix(w, (n, n), "periodic").astype(np.float64)
        ev = np.linalg.eigvalsh(0.5 * (M + M.T))
        rho_b = float(np.max(np.abs(ev)))
        # printed to the digits shown: agree to half a unit of the last digit
        assert abs(rho_b - r["rho_B"]) <= (5e-5 if h == 8 else 1e-12), (h, rho_b)
        dt = r["dt"]
        ea = 1.0 + dt * ev
        assert abs(np.max(ea) - r["rho_A"]) < 1e-3 * r["rho_A"]
        assert abs(np.max(ea) / np.min(ea) - r["cond_A"]) < 1e-3 * r["cond_A"]
    # even grids: the checkerboard is an eigenvector with eigenvalue 64/h^4
    for r in golden["table2"]["rows"][2:]:
        h = r["h"]
        n = int(round(200 / h))
        y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        v = (-1.0) ** (x + y)
        w = st.fp_weights(B, Fraction(h).limit_denominator(), np.float64)
        Bv = ap.apply(w, v, "periodic")
        lam = float(np.vdot(v, Bv) / np.vdot(v, v))
        assert np.allclose(Bv, lam * v, rtol=0, atol=1e-9 * abs(lam))
        assert lam == pytest.approx(r["rho_B"], rel=1e-12)
        assert 1 + r["dt"] * lam == pytest.approx(r["rho_A"], rel=1e-12)


def test_weight_rounding_is_correct():
    """fp_weights: a single correct rounding of the exact rational weight."""
    B = st.bilaplacian(2, 4)
    for n in [16, 100, 8192, 1000003]:
        h = Fraction(1, n)
        ex = st.exact_weights(B, h)
        w64 = st.fp_weights(B, h, np.float64)
        w32 = st.fp_weights(B, h, np.float32)
        for k, q in ex.items():
            v = w64[k]
            # the neighbours of the chosen double are no closer
            for nb in (np.nextafter(v, np.inf), np.nextafter(v, -np.inf)):
                assert abs(Fraction(v) - q) <= abs(Fraction(float(nb)) - q)
            f = w32[k]
            for nb in (np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf))):
                assert abs(Fraction(float(f)) - q) <= abs(Fraction(float(nb)) - q)
    # ties go to the even significand
    a = np.float32(1.0)
    b = np.nextafter(a, np.float32(2.0))
    mid = (Fraction(float(a)) + Fraction(float(b))) / 2
    assert st.round_f32(mid) == a  # 1.0 has an even significand
    c = np.nextafter(b, np.float32(2.0))
    mid2 = (Fraction(float(b)) + Fraction(float(c))) / 2
    assert st.round_f32(mid2) == c
    assert st.round_f64(Fraction(1, 3)) == 1.0 / 3.0


def _random_stencil(rng, ndim, radius, npts):
    coeffs = {}
    while len(coeffs) < npts:
        off = tuple(int(v) for v in rng.integers(-radius, radius + 1, size=ndim))
        coeffs[off] = Fraction(int(rng.integers(-9, 10)) or 1, int(rng.integers(1, 7)))
    return st.Stencil.make(coeffs, int(rng.integers(0, 3)))


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_taylor_coefficients_of_a_composition_are_the_cauchy_product(ndim):
    """For C = A o B (Eq. C=B(A): offsets add, weights multiply) the binomial
    theorem gives t^C_alpha = sum_{beta <= alpha} t^A_beta t^B_(alpha - beta):
    the Taylor coefficients of a composition are the Cauchy product of the
    factors'.  Random rational stencils with arbitrary offsets; exact
    arithmetic.  A slip in the composition (an offset or weight mix-up) or
    in the Taylor coefficients (a factorial or power) breaks the identity."""
    rng = np.random.default_rng(20 + ndim)
    for _ in range(6):
        A = _random_stencil(rng, ndim, 3, 5)
        B = _random_stencil(rng, ndim, 2, 4)
        C = st.compose(A, B)
        assert C.hpow == A.hpow + B.hpow
        for alpha in itertools.product(range(4), repeat=ndim):
            want = Fraction(0)
            for beta in itertools.product(*(range(a + 1) for a in alpha)):
                gamma = tuple(a - b for a, b in zip(alpha, beta))
                want += st.taylor_coeff(A, beta) * st.taylor_coeff(B, gamma)
            assert st.taylor_coeff(C, alpha) == want, (alpha, A, B)
