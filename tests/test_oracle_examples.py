"""Convergence examples of Sec. 3.1 and Sec. 3.2 (oracle pins)."""
import numpy as np

from oracle import stencil as st


def _eval_1d(s, f, x0, h):
    return sum(float(c) * f(x0 + k[0] * h) for k, c in s.coeffs) / h ** s.hpow


def _fit(hs, errs):
    p, logc = np.polyfit(np.log(hs), np.log(errs), 1)
    return p, np.exp(logc)


def test_sec31_third_derivative(golden):
    """f = sin x cos x, f''' at pi by composing the central first and second
    derivatives: second order with leading coefficient (1/4) f^(5)(pi) = 4."""
    e = golden["convergence"]["ex1d"]
    s = st.compose(st.d1_central2(), st.d2_central2())
    f = lambda x: np.sin(x) * np.cos(x)
    exact = 4 * np.sin(np.pi) ** 2 - 4 * np.cos(np.pi) ** 2
    hs = np.array([2.0 ** -k for k in range(3, 8)])
    errs = np.array([abs(_eval_1d(s, f, np.pi, h) - exact) for h in hs])
    p, C = _fit(hs, errs)
    assert abs(p - 2) < 0.01 and abs(p - e["rate"]) < 0.01
    assert abs(C - e["C_theory"]) < 0.1 and abs(C - e["C"]) < 0.1


def test_sec32_mixed_derivative(golden):
    """f^(4,3) of sin(x + y) at (2 pi, pi/3): fourth order, coefficient 1/30."""
    e = golden["convergence"]["ex2d"]
    sx = st.compose(st.d2_central4(), st.d2_central4())
    sy = st.compose(st.d1_central4(), st.d2_central4())
    s = st.outer_product(sx, sy)
    x0, y0 = 2 * np.pi, np.pi / 3
    f = lambda x, y: np.sin(x + y)
    exact = np.sin(x0) * np.sin(y0) - np.cos(x0) * np.cos(y0)
    hs = np.array([0.4, 0.3, 0.2, 0.15])
    errs = []
    for h in hs:
        v = sum(float(c) * f(x0 + k[0] * h, y0 + k[1] * h) for k, c in s.coeffs) / h ** s.hpow
        errs.append(abs(v - exact))
    p, C = _fit(hs, np.array(errs))
    assert abs(p - 4) < 0.05 and abs(p - e["rate"]) < 0.05
    assert abs(C - 1 / 30) < 0.003 and abs(C - e["C"]) < 0.003
