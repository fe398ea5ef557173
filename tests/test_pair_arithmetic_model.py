"""The FP64-in-FP32-pairs evaluation of a Laplacian composition, modelled on
the CPU: numpy float32 arithmetic (IEEE round-to-nearest per operation)
following the device passes' sequence of error-free transformations -- the
exact integer split of each double into (hi, lo), pair sums as a tree of
TwoSums, exact scaling by power-of-two weights, a TwoProduct for the centre
weight, Fast2Sum normalisation, the final scale as a pair and the exact
rebuild of the double.  Checked against the oracle's FP64 apply of the
composed stencil (Eq. C=B(A)), this pins the error model behind the GPU
tolerance: a few units of 2^-48 of sum_k |w_k x_k| per pass, well inside the
2^-42 elementwise bound the GPU parity tests use.  Test infrastructure only:
nothing here runs on the device or is imported by the library.
"""
from fractions import Fraction

import numpy as np

from oracle import apply as oap
from oracle import stencil as ost
from synth_inputs import fields

F32 = np.float32


def split(x):
    """hi: the leading 24 significand bits of x (truncated), lo: the next 29
    bits rounded to float32; x = hi + lo + rest, |rest| <= 2^-48 |x|."""
    b = x.view(np.uint64)
    hi = (b & np.uint64(0xFFFFFFFFE0000000)).view(np.float64)
    return hi.astype(F32), (x - hi).astype(F32)


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def fma(a, b, c):
    """a b + c rounded once to float32 (the product is exact in float64)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def pair_sum(a, b):
    s, e = two_sum(a[0], b[0])
    return [s, e + (a[1] + b[1])]


def acc_add(acc, v):
    s, e = two_sum(acc[0], v[0])
    return [s, acc[1] + (e + v[1])]


def scale_exact(acc, k):  # k a power of two: both parts scale exactly
    return [acc[0] * F32(k), acc[1] * F32(k)]


def two_product(h, l, k):
    p = h * F32(k)
    e = fma(h, np.full_like(h, k), -p)  # exact error of the rounded product
    return [p, fma(l, np.full_like(l, k), e)]


def lap_pass(H, L, c0, c1, c2):
    """One pass t = L_int(x) on pairs (periodic), in the device pass's order."""
    ndim = H.ndim

    def nb(d, ax):
        return [np.roll(H, -d, axis=ax), np.roll(L, -d, axis=ax)]

    x_ax = ndim - 1  # the fastest axis
    A = pair_sum(nb(-1, x_ax), nb(1, x_ax))
    Az = pair_sum(nb(-1, 0), nb(1, 0))
    if ndim == 3:
        Az = acc_add(Az, pair_sum(nb(-1, 1), nb(1, 1)))
    A = acc_add(A, Az)
    A = scale_exact(A, c1)
    A = acc_add(A, two_product(H, L, c0))
    B = pair_sum(nb(-2, x_ax), nb(2, x_ax))
    Bz = pair_sum(nb(-2, 0), nb(2, 0))
    if ndim == 3:
        Bz = acc_add(Bz, pair_sum(nb(-2, 1), nb(2, 1)))
    B = acc_add(B, Bz)
    assert c2 == -1.0
    s, e = two_sum(A[0], -B[0])  # A - B
    A = [s, A[1] + (e - B[1])]
    h = A[0] + A[1]  # Fast2Sum
    return h, A[1] - (h - A[0])


def apply_pair_model(x, n):
    """y = s^2 L_int(L_int x), s = 1/(12 h^2), h = 1/n, FP64 in and out."""
    ndim = x.ndim
    c0, c1, c2 = -30.0 * ndim, 16.0, -1.0
    with np.errstate(over="ignore", invalid="ignore"):
        H, L = split(x)
        T = lap_pass(H, L, c0, c1, c2)
        Zh, Zl = lap_pass(T[0], T[1], c0, c1, c2)
    scale = float(n) ** 4 / 144.0
    m, e = np.frexp(scale)
    m, e = 2.0 * m, int(e) - 1  # scale = m 2^e, m in [1, 2)
    sh = F32(m)
    sl = F32(m - float(sh))
    p = Zh * sh
    err = fma(Zh, np.full_like(Zh, sh), -p)
    err = fma(Zh, np.full_like(Zh, sl), err)
    err = fma(Zl, np.full_like(Zl, sh), err)
    zh = p + err
    zl = err - (zh - p)
    # both parts to double exactly, then one FP64 add (48 bits fit)
    return np.ldexp(zh.astype(np.float64) + zl.astype(np.float64), e)


def _check(shape, seed, bound):
    n = shape[-1]
    x = fields.uniform(shape, seed=seed)
    y = apply_pair_model(x, n)
    oL = ost.laplacian(len(shape), 4)
    oc = ost.compose(oL, oL)
    w = ost.fp_weights(oc, Fraction(1, n), np.float64)
    y_ref = oap.apply(w, x, "periodic", oc.radius)
    absL = ost.Stencil.make({k: abs(v) for k, v in oL.coeffs}, oL.hpow)
    mag = oap.apply(ost.fp_weights(ost.compose(absL, absL), Fraction(1, n), np.float64), np.abs(x), "periodic",
                    oc.radius)
    rel = np.max(np.abs(y - y_ref) / mag)
    assert rel <= bound, rel
    return rel


def test_pair_model_2d_within_error_model():
    rel = _check((24, 32), seed=101, bound=2.0 ** -45)
    print(f"2D pair model: max |y - y_ref| / ((|B| o |A|)|x|) = {rel:.3e} (2^{np.log2(rel):.1f})")


def test_pair_model_3d_within_error_model():
    rel = _check((10, 12, 16), seed=102, bound=2.0 ** -45)
    print(f"3D pair model: max |y - y_ref| / ((|B| o |A|)|x|) = {rel:.3e} (2^{np.log2(rel):.1f})")


def test_pair_model_detects_a_dropped_error_term():
    """The model is sensitive: dropping the TwoSum error terms (plain FP32
    sums of the pairs) breaks the bound by many orders of magnitude."""
    global two_sum
    keep = two_sum
    try:
        two_sum = lambda a, b: (a + b, np.zeros_like(a))  # noqa: E731
        x = fields.uniform((24, 32), seed=103)
        y = apply_pair_model(x, 32)
        oL = ost.laplacian(2, 4)
        oc = ost.compose(oL, oL)
        y_ref = oap.apply(ost.fp_weights(oc, Fraction(1, 32), np.float64), x, "periodic", oc.radius)
        assert np.max(np.abs(y - y_ref)) / np.max(np.abs(y_ref)) > 2.0 ** -30
    finally:
        two_sum = keep
