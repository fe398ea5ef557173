"""The seeded input generators that the oracle and the GPU path share: each
generator does what its docstring states (no method arithmetic lives here,
so these are properties of the inputs, not of the paper's method)."""
import math

import numpy as np
import pytest

from synth_inputs import fields, manufactured, requests


def test_trace_is_seeded_and_within_its_ranges():
    a = requests.trace(2000, seed=2205, rate_per_s=6.0)
    b = requests.trace(2000, seed=2205, rate_per_s=6.0)
    assert a == b
    assert requests.trace(50, seed=2206, rate_per_s=6.0) != a[:50]
    for r in a:
        lo, hi = (32, 256) if r["ndim"] == 3 else (32, 2048)
        assert lo <= r["n"] <= hi
        assert len(r["ks"]) == r["ndim"] and all(1 <= k <= 8 for k in r["ks"])
        assert r["kind"] == "plate"
    t = np.array([r["t"] for r in a])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0.0)
    # exponential gaps with mean 1/rate: the mean of 1999 gaps within 5 standard errors
    gap = np.diff(t).mean()
    assert abs(gap - 1 / 6.0) <= 5 * (1 / 6.0) / math.sqrt(1999)
    # half 2D, half 3D (binomial, 5 standard deviations)
    n3 = sum(r["ndim"] == 3 for r in a)
    assert abs(n3 - 1000) <= 5 * math.sqrt(2000 * 0.25)


def test_trace_sizes_are_log_uniform():
    """log n is uniform on [log lo, log hi]: each of four equal bins of log n
    holds a quarter of the 2D requests (5 standard deviations)."""
    a = [r for r in requests.trace(4000, seed=7, rate_per_s=1.0) if r["ndim"] == 2]
    x = (np.log([r["n"] for r in a]) - math.log(32)) / (math.log(2048) - math.log(32))
    counts, _ = np.histogram(x, bins=4, range=(0.0, 1.0))
    m = len(a)
    assert np.all(np.abs(counts - m / 4) <= 5 * math.sqrt(m * 0.25 * 0.75) + 2)


def test_trace_cahn_hilliard_kinds_leave_the_plate_trace_unchanged():
    plain = requests.trace(1000, seed=11, rate_per_s=3.0)
    mixed = requests.trace(1000, seed=11, rate_per_s=3.0, ch_frac=0.3)
    for p, m in zip(plain, mixed):
        assert {k: v for k, v in p.items() if k != "kind"} == {k: v for k, v in m.items() if k != "kind"}
    nch = sum(r["kind"] == "ch" for r in mixed)
    assert abs(nch - 300) <= 5 * math.sqrt(1000 * 0.3 * 0.7)
    assert all(r["kind"] == "plate" for r in requests.trace(200, seed=11, rate_per_s=3.0, ch_frac=0.0))


@pytest.mark.parametrize("n,ndim,R,ks", [(9, 2, 2, (1, 3)), (7, 3, 1, (2, 1, 3)), (12, 2, 1, None)])
def test_separable_plate_case_equals_the_grid_built_one(n, ndim, R, ks):
    a = manufactured.bvp_case(n, ndim, R, ks)
    b = manufactured.bvp_case_separable(n, ndim, R, ks)
    for key in ("u_padded", "u_exact", "g"):
        assert np.array_equal(a[key], b[key]), key
    assert a["h"] == b["h"] and a["R"] == b["R"]


def test_plate_case_is_the_stated_manufactured_solution():
    """u = prod sin(k_a pi x_a) sampled at x = i h (i = 1-R .. N+R), g = pi^4
    (sum k^2)^2 u on the interior, and ks given in (x, y, z) order."""
    n, R, ks = 10, 2, (1, 2, 3)
    c = manufactured.bvp_case(n, 3, R, ks)
    h = 1.0 / (n + 1)
    i = np.arange(1 - R, n + R + 1)
    z, y, x = np.meshgrid(i * h, i * h, i * h, indexing="ij")
    u = np.sin(1 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(3 * np.pi * z)
    assert np.allclose(c["u_padded"], u, rtol=0, atol=1e-15)
    assert np.array_equal(c["u_exact"], c["u_padded"][R:R + n, R:R + n, R:R + n])
    assert np.allclose(c["g"], np.pi ** 4 * 14.0 ** 2 * c["u_exact"], rtol=1e-15, atol=0)
    # node 0 and node N+1 lie on the boundary, where u vanishes
    assert np.max(np.abs(c["u_padded"][R - 1])) < 1e-14 and np.max(np.abs(c["u_padded"][R + n])) < 1e-14


def test_field_generators():
    u = fields.uniform((64, 32), seed=3)
    assert np.array_equal(u, fields.uniform((64, 32), seed=3))
    assert u.min() >= -1.0 and u.max() < 1.0 and u.dtype == np.float64
    assert fields.uniform((16,), seed=3, dtype="float32").dtype == np.float32
    c = manufactured.ch_uniform(16, 2, seed=5, amp=0.05, batch=3)
    assert c.shape == (3, 16, 16) and np.array_equal(c[1], manufactured.ch_uniform(16, 2, seed=6))
    assert np.max(np.abs(c)) <= 0.05
    s2 = manufactured.ch_spinodal_ic(50, 2, 200.0)
    s3 = manufactured.ch_spinodal_ic(16, 3, 64.0)
    assert s2.shape == (50, 50) and s3.shape == (16, 16, 16)
    # c0 + eps (three terms of magnitude <= 1): within c0 +- 3 eps
    for s in (s2, s3):
        assert np.all(np.abs(s - 0.5) <= 3 * 0.01 * (1 + 1e-12))
    assert s2[0, 0] == pytest.approx(0.5 + 0.01 * 3.0)
