"""Manufactured solutions of the biharmonic plate problem and Cahn-Hilliard
initial data (continuous data only).

Plate: u = prod_a sin(k_a pi x_a) on the unit square/cube, whose biharmonic is
g = pi^4 (sum_a k_a^2)^2 u.  Grid: N interior nodes per axis, h = 1/(N+1),
node i at x = i h; the padded array also covers the R ghost nodes
i = 1-R .. 0 and N+1 .. N+R on each side.  Arrays are indexed [z][y][x].
"""
import numpy as np


def bvp_case(n: int, ndim: int, R: int, ks=None) -> dict:
    ks = tuple(ks) if ks is not None else (1,) * ndim
    h = 1.0 / (n + 1)
    nodes = np.arange(1 - R, n + R + 1) * h
    grids = np.meshgrid(*([nodes] * ndim), indexing="ij")  # array axes (z,)y,x
    # ks are given in (x, y, z) order; array axis a holds coordinate ndim-1-a
    u = np.ones_like(grids[0])
    for a in range(ndim):
        k = ks[ndim - 1 - a]
        u = u * np.sin(k * np.pi * grids[a])
    inner = tuple(slice(R, R + n) for _ in range(ndim))
    lam = np.pi ** 4 * float(sum(k * k for k in ks)) ** 2
    return {"h": h, "R": R, "n": n, "ndim": ndim, "ks": ks,
            "u_padded": u, "u_exact": u[inner].copy(), "g": lam * u[inner]}


def ch_uniform(n: int, ndim: int, seed: int, amp: float = 0.05, batch: int | None = None) -> np.ndarray:
    """Cahn-Hilliard initial field uniform in [-amp, amp] from a seed; with
    ``batch`` the seeds are seed, seed+1, ..."""
    if batch is None:
        return np.random.default_rng(seed).uniform(-amp, amp, size=(n,) * ndim)
    return np.stack([np.random.default_rng(seed + b).uniform(-amp, amp, size=(n,) * ndim)
                     for b in range(batch)])


def ch_spinodal_ic(n: int, ndim: int, length: float, c0: float = 0.5, eps: float = 0.01) -> np.ndarray:
    """The cosine initial condition of the spinodal-decomposition benchmark
    (Sec. 4.1) on an n^ndim periodic grid of side ``length``, x_i = i h."""
    h = length / n
    x1 = np.arange(n) * h
    if ndim == 2:
        y, x = np.meshgrid(x1, x1, indexing="ij")
        return c0 + eps * (np.cos(0.105 * x) * np.cos(0.11 * y)
                           + (np.cos(0.13 * x) * np.cos(0.087 * y)) ** 2
                           + np.cos(0.025 * x - 0.15 * y) * np.cos(0.07 * x - 0.02 * y))
    z, y, x = np.meshgrid(x1, x1, x1, indexing="ij")
    return c0 + eps * (np.cos(0.105 * x) * np.cos(0.11 * y) * np.cos(0.11 * z)
                       + (np.cos(0.13 * x) * np.cos(0.087 * y) * np.cos(0.1 * z)) ** 2
                       + np.cos(0.025 * x - 0.15 * y - 0.1 * z) * np.cos(0.07 * x - 0.02 * y + 0.01 * z))


def bvp_case_separable(n: int, ndim: int, R: int, ks=None) -> dict:
    """The same arrays as bvp_case, built from the 1D factors by broadcasting
    (the same products in the same order, so the same values), without the
    full coordinate grids: fast enough to generate 256^3 requests on the fly."""
    ks = tuple(ks) if ks is not None else (1,) * ndim
    h = 1.0 / (n + 1)
    nodes = np.arange(1 - R, n + R + 1) * h
    u = np.ones((1,) * ndim)
    for a in range(ndim):
        k = ks[ndim - 1 - a]
        shape = [1] * ndim
        shape[a] = nodes.size
        u = u * np.sin(k * np.pi * nodes).reshape(shape)
    inner = tuple(slice(R, R + n) for _ in range(ndim))
    lam = np.pi ** 4 * float(sum(k * k for k in ks)) ** 2
    ue = np.ascontiguousarray(u[inner])
    return {"h": h, "R": R, "n": n, "ndim": ndim, "ks": ks, "u_padded": np.ascontiguousarray(u),
            "u_exact": ue, "g": lam * ue}
