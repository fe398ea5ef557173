"""von Neumann stability of explicit steps with composed stencils
(Sec. 2.2.3 and Appendix B).

Oracle (test infrastructure only; see ``oracle/__init__.py``).

For df/dt = sign * D f with D a 1D stencil of h-power p and forward Euler in
time, inserting f_j^n = xi^n e^{i k j h} gives the growth factor
    xi(theta) = 1 + sign * dt/h^p * sum_j c_j e^{i j theta},  theta = k h.
For a symmetric stencil the sum is real; |xi| <= 1 for every theta holds iff
dt <= alpha h^p with alpha = 2 / max_theta(-sign * sum_j c_j cos(j theta)).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize_scalar


def symbol(coeffs: dict, theta: np.ndarray) -> np.ndarray:
    """Real part of sum_j c_j e^{i j theta} (1D stencil {(j,): c_j})."""
    out = np.zeros_like(np.asarray(theta, dtype=np.float64))
    for (j,), c in coeffs.items():
        out = out + float(c) * np.cos(j * theta)
    return out


def alpha(coeffs: dict, sign: int) -> float:
    """Largest alpha with dt <= alpha h^p stable (sign: +1 for df/dt = +D f,
    -1 for df/dt = -D f).  Grid search followed by a bounded refinement."""
    th = np.linspace(0.0, np.pi, 20001)
    g = -sign * symbol(coeffs, th)
    i = int(np.argmax(g))
    lo = th[max(i - 1, 0)]
    hi = th[min(i + 1, len(th) - 1)]
    res = minimize_scalar(lambda t: sign * float(symbol(coeffs, np.array(t))),
                          bounds=(lo, hi), method="bounded",
                          options={"xatol": 1e-14})
    gmax = max(float(g[i]), -float(res.fun))
    return 2.0 / gmax
