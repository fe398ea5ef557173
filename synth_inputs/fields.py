"""Seeded random fields."""
import numpy as np


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0, dtype=np.float64) -> np.ndarray:
    """Uniform [lo, hi) field from numpy's PCG64 generator seeded with ``seed``;
    drawn in float64 and then cast, so the float32 field is the rounded float64
    field of the same seed."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=tuple(shape)).astype(dtype)


def wide_range(shape, seed: int, lo_exp: int, hi_exp: int, zero_frac: float = 0.0,
               patch: int = 0) -> np.ndarray:
    """FP64 field of random sign whose magnitudes are 2^e * m, e uniform in
    [lo_exp, hi_exp) and m uniform in [1, 2); a fraction ``zero_frac`` of the
    points is set to 0, and, with ``patch`` > 0, a cube of that edge in the
    field's first corner holds one constant value (both make exact
    cancellations in a zero-sum stencil)."""
    rng = np.random.default_rng(seed)
    shape = tuple(shape)
    e = rng.integers(lo_exp, hi_exp, size=shape)
    m = rng.uniform(1.0, 2.0, size=shape)
    s = np.where(rng.random(size=shape) < 0.5, -1.0, 1.0)
    x = s * np.ldexp(m, e)
    if zero_frac > 0:
        x[rng.random(size=shape) < zero_frac] = 0.0
    if patch > 0:
        x[tuple(slice(0, patch) for _ in shape)] = x.flat[0]
    return x
