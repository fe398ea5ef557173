"""Pins of the von Neumann stability constants (Sec. 2.2.3, Table 1,
Appendix B)."""
import numpy as np

from oracle import stability as sb
from oracle import stencil as st
from tests.conftest import frac


def test_table1_alphas(golden):
    d1, d2 = st.d1_central2(), st.d2_central2()
    schemes = {
        "compact": st.Stencil.make({(-2,): 1, (-1,): -4, (0,): 6, (1,): -4, (2,): 1}, 4),
        "d2_c2 o d2_c2": st.compose(d2, d2),
        "d1_c2 o d1_c2 o d2_c2": st.compose(d1, st.compose(d1, d2)),
    }
    for row in golden["stability"]["table1"]:
        s = schemes[row["scheme"]]
        a = sb.alpha(s.as_dict(), -1)  # df/dt = -D f
        assert abs(a - float(frac(row["alpha"]))) < 1e-10, (row, a)
        assert [-s.radius, s.radius] == row["support"]


def test_appendix_b_bracket_minimum(golden):
    """min over theta of cos t + 2 cos 2t - cos 3t - 2 is -128/27."""
    s = st.compose(st.d1_central2(), st.compose(st.d1_central2(), st.d2_central2()))
    th = np.linspace(0, np.pi, 200001)
    # 2 * (4 * symbol) == -(bracket): the stencil carries 1/4
    bracket = -2.0 * sb.symbol(s.as_dict(), th)
    assert abs(bracket.min() - float(frac(golden["stability"]["appendixB_bracket_min"]))) < 1e-8
    assert np.allclose(bracket, np.cos(th) + 2 * np.cos(2 * th) - np.cos(3 * th) - 2)


def test_heat_equation_alphas(golden):
    d1 = st.d1_central2()
    composed = st.compose(d1, d1)
    assert abs(sb.alpha(composed.as_dict(), +1) - float(frac(golden["stability"]["heat_composed_alpha"]))) < 1e-10
    assert abs(sb.alpha(st.d2_central2().as_dict(), +1) - float(frac(golden["stability"]["heat_compact_alpha"]))) < 1e-10
