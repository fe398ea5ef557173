"""Seeded request trace for the serving workload: Poisson arrivals of
biharmonic plate solves of mixed 2D/3D sizes."""
import numpy as np


def trace(nreq: int, seed: int, rate_per_s: float, n2d=(32, 2048), n3d=(32, 256),
          frac_3d: float = 0.5, kmax: int = 8, ch_frac: float = 0.0) -> list:
    """Each request: arrival time (s), ndim, interior size n (log-uniform in
    the given range, rounded to an integer), wave numbers k in [1, kmax], and
    its kind: a Cahn-Hilliard step with probability ch_frac (drawn from a
    stream of its own, so that ch_frac = 0 leaves the plate trace as it was),
    else a plate problem."""
    kinds = np.random.default_rng(seed + 7919).uniform(size=nreq) < ch_frac
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=nreq)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(nreq):
        ndim = 3 if rng.uniform() < frac_3d else 2
        lo, hi = n3d if ndim == 3 else n2d
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        ks = tuple(int(k) for k in rng.integers(1, kmax + 1, size=ndim))
        out.append({"id": i, "t": float(t[i]), "ndim": ndim, "n": n, "ks": ks,
                    "kind": "ch" if kinds[i] else "plate"})
    return out
