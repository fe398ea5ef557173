"""The C-ABI library without a GPU: it loads, exports every function the
headers declare, and its exact host algebra matches the oracle bit for bit."""
import ctypes
import math
from fractions import Fraction

import numpy as np
import torch
import pytest

from tests.libutil import ensure_built, header_functions

ensure_built()
import paper_2205_03354_gb300 as sc  # noqa: E402
from oracle import stencil as ost  # noqa: E402

KIND = {"d1_c2": sc.D1_C2, "d2_c2": sc.D2_C2, "d1_c4": sc.D1_C4, "d2_c4": sc.D2_C4,
        "d1_fwd": sc.D1_FWD, "d2_fwd": sc.D2_FWD}


def test_every_declared_symbol_is_exported():
    names = header_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(sc.lib, n)]
    assert not missing, missing


def _same(lib_s, orc_s):
    assert lib_s.hpow == orc_s.hpow
    assert lib_s.points() == {k: v for k, v in orc_s.coeffs}


def test_1d_stencils_and_compositions_match_oracle():
    for a, ka in KIND.items():
        _same(sc.stencil_1d(ka), ost.STENCIL_1D[a]())
        for b, kb in KIND.items():
            _same(sc.compose_stencil(sc.stencil_1d(ka), sc.stencil_1d(kb)),
                  ost.compose(ost.STENCIL_1D[a](), ost.STENCIL_1D[b]()))


@pytest.mark.parametrize("ndim,order", [(2, 2), (3, 2), (2, 4), (3, 4), (1, 2), (1, 4)])
def test_laplacian_and_bilaplacian_match_oracle(ndim, order):
    L = sc.laplacian(ndim, order)
    _same(L, ost.laplacian(ndim, order))
    _same(sc.compose_stencil(L, L), ost.bilaplacian(ndim, order))
    # triple composition (radius 6 in 3D at 2nd order) still exact
    if order == 2:
        _same(sc.compose_stencil(L, sc.compose_stencil(L, L)),
              ost.compose(ost.laplacian(ndim, 2), ost.bilaplacian(ndim, 2)))


def test_mixed_axis_composition_matches_oracle():
    x = sc.stencil_embed(sc.stencil_1d(sc.D1_FWD), 2, 0)
    y = sc.stencil_embed(sc.stencil_1d(sc.D2_C4), 2, 1)
    _same(sc.compose_stencil(x, y), ost.outer_product(ost.d1_forward(), ost.d2_central4()))
    _same(sc.stencil_add(sc.stencil_embed(sc.stencil_1d(sc.D2_C4), 2, 0), y), ost.laplacian(2, 4))


@pytest.mark.parametrize("ndim,order", [(2, 2), (3, 2), (2, 4), (3, 4)])
def test_weights_bit_exact(ndim, order):
    L = sc.laplacian(ndim, order)
    B = sc.compose_stencil(L, L)
    ob = ost.bilaplacian(ndim, order)
    keys = [k for k, _ in ob.coeffs]
    for (hn, hd) in [(1, 64), (1, 65), (1, 8192), (1, 512), (1, 1024), (1, 2049), (8, 1), (1, 2), (3, 7)]:
        h = Fraction(hn, hd)
        for dt in (np.float64, np.float32):
            w = sc.stencil_weights(B, hn, hd, dt)
            ow = ost.fp_weights(ob, h, dt)
            want = np.array([ow[k] for k in keys], dtype=dt)
            assert np.array_equal(w.view(np.uint64 if dt == np.float64 else np.uint32),
                                  want.view(np.uint64 if dt == np.float64 else np.uint32)), (hn, hd, dt)


def test_errors_are_reported():
    a = sc.laplacian(2, 2)
    b = sc.laplacian(3, 2)
    with pytest.raises(sc.ScError) as e:
        sc.compose_stencil(a, b)
    assert e.value.status == 1
    big = sc.Stencil()
    big.ndim, big.npts, big.hpow, big.radius, big.den = 1, 1, 0, 0, 1
    big.off[0][0] = 0
    big.num[0] = 2 ** 62
    with pytest.raises(sc.ScError) as e:
        sc.compose_stencil(big, big)
    assert e.value.status == 8  # SC_EOVERFLOW
    with pytest.raises(sc.ScError):
        sc.laplacian(4, 2)
    with pytest.raises(sc.ScError):
        sc.stencil_weights(a, 0, 1)


def test_saved_tuning_round_trips_without_a_gpu():
    """A saved tuning choice is recorded and read back by the host cache; bad
    choices are rejected before any device work."""
    import torch
    from paper_2205_03354_gb300.ops import TuneChoice, dims_arg, lib
    L = sc.laplacian(3, 2)
    sc.tune_set(L, L, torch.float64, "periodic", (40, 36, 20), {"eval": "pair", "planes": 32, "ms": 1.5})
    out = TuneChoice()
    assert lib.sc_tuned_choice(ctypes.byref(L), ctypes.byref(L), sc.F64, sc.BC_PERIODIC,
                               dims_arg((40, 36, 20)), ctypes.byref(out)) == 0
    assert out.as_dict() == {"eval": "pair", "planes": 32, "ms": 1.5}
    # another shape stays untuned
    assert lib.sc_tuned_choice(ctypes.byref(L), ctypes.byref(L), sc.F64, sc.BC_PERIODIC,
                               dims_arg((40, 36, 21)), ctypes.byref(out)) == 1
    # the fused schedule is a valid choice (it runs the nested one where it does not apply)
    ok = TuneChoice(3, 0, 0.0)
    assert lib.sc_tune_set(ctypes.byref(L), ctypes.byref(L), sc.F64, sc.BC_PERIODIC,
                           dims_arg((40, 36, 20)), ctypes.byref(ok)) == 0
    for bad in (TuneChoice(4, 0, 0.0), TuneChoice(-1, 0, 0.0), TuneChoice(0, -1, 0.0), TuneChoice(1, 5000, 0.0)):
        assert lib.sc_tune_set(ctypes.byref(L), ctypes.byref(L), sc.F64, sc.BC_PERIODIC,
                               dims_arg((40, 36, 20)), ctypes.byref(bad)) == 1


def _lib_stencil(coeffs: dict, hpow: int) -> "sc.Stencil":
    """A library stencil in canonical form (sorted offsets, no zero weights,
    reduced common denominator) from {offset: Fraction}."""
    items = sorted((k, v) for k, v in coeffs.items() if v != 0)
    den = 1
    for _, v in items:
        den = den * v.denominator // math.gcd(den, v.denominator)
    s = sc.Stencil()
    s.ndim = len(items[0][0])
    s.npts = len(items)
    s.hpow = hpow
    s.radius = max(max(abs(c) for c in k) for k, _ in items)
    nums = [int(v * den) for _, v in items]
    g = den
    for n_ in nums:
        g = math.gcd(g, n_)
    s.den = den // g
    for i, ((k, _), n_) in enumerate(zip(items, nums)):
        for a, c in enumerate(k):
            s.off[i][a] = c
        s.num[i] = n_ // g
    return s


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_random_compositions_match_oracle(ndim):
    """The library's exact composition on arbitrary rational stencils (not
    only the paper's) equals the oracle's, point for point."""
    rng = np.random.default_rng(40 + ndim)
    for _ in range(8):
        st_ = []
        for radius, npts in ((3, 6), (2, 5)):
            coeffs = {}
            while len(coeffs) < npts:
                off = tuple(int(v) for v in rng.integers(-radius, radius + 1, size=ndim))
                coeffs[off] = Fraction(int(rng.integers(1, 10)) * (-1) ** int(rng.integers(0, 2)),
                                       int(rng.integers(1, 13)))
            st_.append((coeffs, int(rng.integers(0, 3))))
        (ca, pa), (cb, pb) = st_
        got = sc.compose_stencil(_lib_stencil(ca, pa), _lib_stencil(cb, pb))
        want = ost.compose(ost.Stencil.make(ca, pa), ost.Stencil.make(cb, pb))
        _same(got, want)


def test_random_weights_correctly_rounded():
    """Weights of arbitrary rational stencils (numerators up to 10^6,
    denominators up to 12) at arbitrary rational h (numerator and
    denominator up to 10^4, h^-p with p up to 4, so every exact value fits
    the documented 127 bits): FP64 and FP32 values bit-identical to the
    oracle's correctly rounded exact rationals."""
    rng = np.random.default_rng(77)
    for _ in range(60):
        ndim = int(rng.integers(1, 4))
        coeffs = {}
        while len(coeffs) < 5:
            off = tuple(int(v) for v in rng.integers(-2, 3, size=ndim))
            coeffs[off] = Fraction(int(rng.integers(-10 ** 6, 10 ** 6)) or 1, int(rng.integers(1, 13)))
        hpow = int(rng.integers(0, 5))
        s = _lib_stencil(coeffs, hpow)
        os_ = ost.Stencil.make(coeffs, hpow)
        hn, hd = int(rng.integers(1, 10 ** 4)), int(rng.integers(1, 10 ** 4))
        keys = [k for k, _ in os_.coeffs]
        for dt in (np.float64, np.float32):
            w = sc.stencil_weights(s, hn, hd, dt)
            ow = ost.fp_weights(os_, Fraction(hn, hd), dt)
            want = np.array([ow[k] for k in keys], dtype=dt)
            assert np.array_equal(w.view(np.uint64 if dt == np.float64 else np.uint32),
                                  want.view(np.uint64 if dt == np.float64 else np.uint32)), (coeffs, hpow, hn, hd, dt)



def test_weights_beyond_127_bits_report_overflow():
    """An exact weight that needs more than 127 bits is refused with
    SC_EOVERFLOW, not rounded from a wrapped value."""
    s = _lib_stencil({(0,): Fraction(10 ** 15), (1,): Fraction(-1)}, 4)
    with pytest.raises(sc.ScError) as e:
        sc.stencil_weights(s, 1, 10 ** 6, np.float64)  # 10^15 * 10^24 > 2^127
    assert e.value.status == 8  # SC_EOVERFLOW


def test_random_add_and_embed_match_oracle():
    """Sums of random rational stencils (with cancelling points) and 1D
    stencils embedded along every axis: the library equals the oracle."""
    rng = np.random.default_rng(91)
    for _ in range(20):
        ndim = int(rng.integers(1, 4))
        hp = int(rng.integers(0, 3))
        mk = []
        for _s in range(2):
            coeffs = {}
            while len(coeffs) < (4 if ndim == 1 else 6):  # 5 offsets exist in 1D
                off = tuple(int(v) for v in rng.integers(-2, 3, size=ndim))
                coeffs[off] = Fraction(int(rng.integers(-9, 10)) or 2, int(rng.integers(1, 9)))
            mk.append(coeffs)
        k0 = next(iter(mk[0]))
        mk[1][k0] = -mk[0][k0]  # one point cancels exactly
        got = sc.stencil_add(_lib_stencil(mk[0], hp), _lib_stencil(mk[1], hp))
        _same(got, ost.add(ost.Stencil.make(mk[0], hp), ost.Stencil.make(mk[1], hp)))
        one_d = {(int(i),): Fraction(int(rng.integers(-9, 10)) or 1, int(rng.integers(1, 9)))
                 for i in rng.choice(np.arange(-3, 4), size=4, replace=False)}
        for axis in range(ndim):
            got = sc.stencil_embed(_lib_stencil(one_d, hp), ndim, axis)
            _same(got, ost.embed(ost.Stencil.make(one_d, hp), ndim, axis))


def test_composition_overflow_is_refused():
    """Products or sums beyond int64 are refused with SC_EOVERFLOW."""
    big = _lib_stencil({(0,): Fraction(2 ** 40), (1,): Fraction(3)}, 0)
    with pytest.raises(sc.ScError) as e:
        sc.compose_stencil(big, big)  # 2^80
    assert e.value.status == 8


def test_host_pipeline_work_space_is_two_slabs():
    """The host-buffer apply stages about two slabs (an eighth of the grid
    each, plus the composed halo) instead of the whole grid once the slowest
    axis holds two slabs of 4 Rc planes; shorter grids take the whole-grid
    space (input with its ring, output, schedule work)."""
    L = sc.laplacian(3, 4)
    es = 8
    big = (512, 512, 512)
    whole = 2 * 512 ** 3 * es
    wb = sc.apply_tuned_host_work_bytes(L, L, torch.float64, "periodic", big)
    assert 0 < wb < 0.9 * whole
    # two staging + two ring-filled + two output slabs of 64 planes (+ 8 halo)
    assert wb >= (2 * 72 * 512 * 512 + 2 * 72 * 520 * 520 + 2 * 64 * 512 * 512) * es
    short = (64, 64, 31)  # 31 < 2 x 16 planes: whole grid
    wb = sc.apply_tuned_host_work_bytes(L, L, torch.float64, "ghosted", short)
    assert wb >= (72 * 72 * 39 + 64 * 64 * 31) * es
