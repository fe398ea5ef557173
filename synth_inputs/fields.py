"""Seeded random fields."""
import numpy as np


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0, dtype=np.float64) -> np.ndarray:
    """Uniform [lo, hi) field from numpy's PCG64 generator seeded with ``seed``;
    drawn in float64 and then cast, so the float32 field is the rounded float64
    field of the same seed."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=tuple(shape)).astype(dtype)
