"""GPU parity of the composed-stencil apply against the FP64 oracle.

Tolerances (derived from the arithmetic of each schedule):
  * FP64: normwise ||y - y_ref||_2 <= 1e-12 ||y_ref||_2 on random fields, and
    elementwise |y - y_ref| <= npts * eps64 * sum_k |w_k x_{i+k}|;
  * FP32 (inputs and weights rounded to float32, accumulation in float32):
    elementwise |y - y_ref| <= npts * eps32 * sum_k |w_k x_{i+k}|, where
    y_ref is the exact-input FP64 oracle sum of the same float32 data.
"""
from fractions import Fraction

import zlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.libutil import ensure_built  # noqa: E402

ensure_built()
import paper_2205_03354_gb300 as sc  # noqa: E402
from oracle import apply as oap  # noqa: E402
from oracle import stencil as ost  # noqa: E402
from synth_inputs import fields  # noqa: E402

DEV = "cuda:0"


def lib_bilap(ndim, order):
    L = sc.laplacian(ndim, order)
    return sc.compose_stencil(L, L)


def oracle_weights(s, h, dt):
    """Oracle's own correctly rounded weights of the oracle's own composition."""
    return ost.fp_weights(s, h, dt)


def check(y_gpu, x_host, w, bc, R, dt, npts):
    y_ref = oap.apply(w, x_host.astype(np.float64), bc, R)
    absw = {k: abs(float(v)) for k, v in w.items()}
    mag = oap.apply(absw, np.abs(x_host.astype(np.float64)), bc, R)
    eps = np.finfo(dt).eps
    err = np.abs(y_gpu.astype(np.float64) - y_ref)
    assert np.all(err <= npts * eps * mag + 1e-300), float(np.max(err / (mag + 1e-300)))
    if dt == np.float64:
        assert np.linalg.norm(err) <= 1e-12 * np.linalg.norm(y_ref)


CASES = [
    # ndim, order, interior dims (x, y[, z]) spanning several tiles + ragged tails
    (2, 2, (1100, 301)), (2, 4, (1100, 301)), (2, 4, (1101, 97)), (2, 2, (16, 9)),
    (3, 2, (150, 40, 37)), (3, 4, (150, 40, 37)), (3, 4, (67, 19, 23)), (3, 2, (8, 8, 8)),
]


@pytest.mark.parametrize("ndim,order,dims", CASES)
@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("bc", ["periodic", "zero", "ghosted"])
def test_apply_matches_oracle(ndim, order, dims, dt, bc):
    os_ = ost.bilaplacian(ndim, order)
    R = os_.radius
    n = dims[0]
    h = Fraction(1, n)
    w = oracle_weights(os_, h, dt)
    shape = tuple(reversed(dims))
    xshape = tuple(s + 2 * R for s in shape) if bc == "ghosted" else shape
    x = fields.uniform(xshape, seed=zlib.crc32(repr((ndim, order, dims, bc)).encode()), dtype=dt)
    s = lib_bilap(ndim, order)
    xt = torch.from_numpy(x).to(DEV)
    yt = torch.full(shape, float("nan"), dtype=xt.dtype, device=DEV)
    sc.apply_composed(s, xt, yt, bc=bc, h=(1, n), dims=dims)
    torch.cuda.synchronize()
    check(yt.cpu().numpy(), x, w, bc, R, dt, os_.npts)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_other_supports(dt):
    """Stencils outside the Lap o Lap class go through the box kernels:
    a one-sided mixed derivative (2D, radius 2) and a 3D box of radius 1."""
    rng = np.random.default_rng(5)
    cases = [
        (sc.compose_stencil(sc.stencil_embed(sc.stencil_1d(sc.D2_FWD), 2, 0),
                            sc.stencil_embed(sc.stencil_1d(sc.D1_C2), 2, 1)),
         ost.outer_product(ost.d2_forward(), ost.d1_central2()), (300, 50)),
        (sc.compose_stencil(sc.compose_stencil(sc.stencil_embed(sc.stencil_1d(sc.D1_C2), 3, 0),
                                               sc.stencil_embed(sc.stencil_1d(sc.D1_FWD), 3, 1)),
                            sc.stencil_embed(sc.stencil_1d(sc.D1_C2), 3, 2)),
         ost.outer_product(ost.outer_product(ost.d1_central2(), ost.d1_forward()), ost.d1_central2()),
         (70, 20, 11)),
    ]
    for s, os_, dims in cases:
        assert s.points() == {k: v for k, v in os_.coeffs}
        w = oracle_weights(os_, Fraction(1, 8), dt)
        shape = tuple(reversed(dims))
        x = rng.uniform(-1, 1, shape).astype(dt)
        for bc in ["periodic", "zero"]:
            yt = torch.empty(shape, dtype=torch.float64 if dt == np.float64 else torch.float32, device=DEV)
            sc.apply_composed(s, torch.from_numpy(x).to(DEV), yt, bc=bc, h=(1, 8), dims=dims)
            torch.cuda.synchronize()
            check(yt.cpu().numpy(), x, w, bc, os_.radius, dt, os_.npts)


@pytest.mark.parametrize("ndim,dims,dt,bc", [(2, (520, 257), np.float64, "periodic"),   # 8 slabs, ragged
                                          (3, (96, 80, 72), np.float32, "periodic"),   # 5 slabs
                                          (3, (40, 30, 20), np.float64, "ghosted"),    # whole grid
                                          (3, (48, 40, 70), np.float64, "ghosted"),    # 5 slabs
                                          (3, (36, 28, 66), np.float32, "zero"),
                                          (2, (300, 77), np.float32, "zero")])
def test_tuned_host_entry_point_matches_device_one(ndim, dims, dt, bc):
    """The asynchronous host-buffer tuned apply (slab pipeline, or the whole
    grid when it is shorter than two slabs), called three times in a row on
    one work space with different inputs: each result equals the
    device-buffer tuned apply bit for bit."""
    L = sc.laplacian(ndim, 4)
    R = 4
    shape = tuple(reversed(dims))
    xshape = tuple(v + 2 * R for v in shape) if bc == "ghosted" else shape
    tdt = torch.float64 if dt == np.float64 else torch.float32
    xs = [torch.from_numpy(fields.uniform(xshape, seed=40 + k, dtype=dt)).pin_memory() for k in range(3)]
    ys = [torch.full(shape, float("nan"), dtype=tdt).pin_memory() for _ in range(3)]
    work = torch.empty(sc.apply_tuned_host_work_bytes(L, L, tdt, bc, dims), dtype=torch.uint8, device=DEV)
    for x, y in zip(xs, ys):
        sc.apply_tuned_host(L, L, x, y, work, bc=bc, h=(1, dims[0]), dims=dims)
    torch.cuda.current_stream().synchronize()
    wd = torch.empty(sc.apply_composition_work_bytes(L, L, tdt, bc, dims), dtype=torch.uint8, device=DEV)
    for x, y in zip(xs, ys):
        yd = torch.empty(shape, dtype=tdt, device=DEV)
        sc.apply_tuned(L, L, x.to(DEV), yd, wd, bc=bc, h=(1, dims[0]), dims=dims)
        torch.cuda.synchronize()
        assert torch.equal(yd.cpu(), y)


def _host_vs_device(L, ndim, dims, dt, bc, seed):
    R = 2 * L.radius
    shape = tuple(reversed(dims))
    xshape = tuple(v + 2 * R for v in shape) if bc == "ghosted" else shape
    x = torch.from_numpy(fields.uniform(xshape, seed=seed, dtype=dt)).pin_memory()
    y = torch.full(shape, float("nan"), dtype=x.dtype).pin_memory()
    work = torch.empty(sc.apply_tuned_host_work_bytes(L, L, x.dtype, bc, dims), dtype=torch.uint8, device=DEV)
    sc.apply_tuned_host(L, L, x, y, work, bc=bc, h=(1, dims[0]), dims=dims)
    torch.cuda.current_stream().synchronize()
    wd = torch.empty(sc.apply_composition_work_bytes(L, L, x.dtype, bc, dims), dtype=torch.uint8, device=DEV)
    yd = torch.empty(shape, dtype=x.dtype, device=DEV)
    sc.apply_tuned(L, L, x.to(DEV), yd, wd, bc=bc, h=(1, dims[0]), dims=dims)
    torch.cuda.synchronize()
    return y, yd.cpu()


@pytest.mark.parametrize("ndim,dims,dt,bc,how,planes", [
    (3, (80, 48, 64), np.float32, "periodic", "fused", 0),
    (2, (256, 200), np.float32, "periodic", "fused", 64),
    (3, (72, 40, 66), np.float32, "zero", "nested", 16),
    (3, (64, 40, 48), np.float64, "periodic", "pair", 0),
    (2, (512, 300), np.float64, "periodic", "pair", 32),
    (3, (48, 36, 40), np.float64, "zero", "pair", 0),
    (3, (40, 36, 50), np.float64, "ghosted", "pair", 16),
])
def test_host_slabs_run_the_whole_grid_schedule(ndim, dims, dt, bc, how, planes):
    """Each slab of the host-buffer pipeline runs the schedule recorded for
    the whole grid (fused, nested or pair arithmetic, with its planes per
    CTA) on a ghosted slab: the result equals the device apply of the whole
    grid bit for bit."""
    L = sc.laplacian(ndim, 4)
    tdt = torch.float64 if dt == np.float64 else torch.float32
    sc.tune_set(L, L, tdt, bc, dims, {"eval": how, "planes": planes})
    y, yd = _host_vs_device(L, ndim, dims, dt, bc, seed=61)
    assert torch.equal(y, yd)


def test_host_slabs_radius_one_pair_runs_native():
    """Pair arithmetic with radius-1 factors has no ghosted form: the slabs of
    a periodic grid run the native FP64 nested passes, within the FP64 apply
    tolerance of the whole-grid pair apply."""
    L = sc.laplacian(3, 2)
    dims = (64, 40, 48)
    sc.tune_set(L, L, torch.float64, "periodic", dims, {"eval": "pair", "planes": 0})
    y, yd = _host_vs_device(L, 3, dims, np.float64, "periodic", seed=62)
    err = (y - yd).abs().max().item()
    assert err <= 1e-11 * yd.abs().max().item()


def test_host_pipeline_alternating_shapes_on_one_work_space():
    """Calls of different shapes back to back on one work space (the second
    call's staging lies where the first call's output buffers were): every
    result equals its device apply bit for bit."""
    L = sc.laplacian(3, 4)
    shapes = [(96, 64, 80), (40, 24, 36), (96, 64, 80), (64, 48, 20)]
    wb = max(sc.apply_tuned_host_work_bytes(L, L, torch.float64, "periodic", d) for d in shapes)
    work = torch.empty(wb, dtype=torch.uint8, device=DEV)
    xs, ys = [], []
    for k, d in enumerate(shapes):
        x = torch.from_numpy(fields.uniform(tuple(reversed(d)), seed=70 + k, dtype=np.float64)).pin_memory()
        y = torch.full(tuple(reversed(d)), float("nan"), dtype=torch.float64).pin_memory()
        sc.apply_tuned_host(L, L, x, y, work, bc="periodic", h=(1, d[0]), dims=d)
        xs.append(x)
        ys.append(y)
    torch.cuda.current_stream().synchronize()
    for d, x, y in zip(shapes, xs, ys):
        wd = torch.empty(sc.apply_composition_work_bytes(L, L, torch.float64, "periodic", d), dtype=torch.uint8,
                         device=DEV)
        yd = torch.empty(tuple(reversed(d)), dtype=torch.float64, device=DEV)
        sc.apply_tuned(L, L, x.to(DEV), yd, wd, bc="periodic", h=(1, d[0]), dims=d)
        torch.cuda.synchronize()
        assert torch.equal(yd.cpu(), y)


def test_host_pipeline_refuses_overlapping_host_buffers():
    L = sc.laplacian(2, 4)
    dims = (256, 128)
    x = torch.zeros(2 * 256 * 128, dtype=torch.float64).pin_memory()
    work = torch.empty(sc.apply_tuned_host_work_bytes(L, L, torch.float64, "periodic", dims), dtype=torch.uint8,
                       device=DEV)
    with pytest.raises(sc.ScError):
        sc.apply_tuned_host(L, L, x[:256 * 128], x[100:100 + 256 * 128], work, bc="periodic", h=(1, 256),
                            dims=dims)


def test_host_buffer_entry_point_matches_device_one():
    s = lib_bilap(2, 4)
    x = torch.from_numpy(fields.uniform((257, 520), seed=9)).pin_memory()
    y = torch.empty_like(x).pin_memory()
    work = torch.empty(sc.apply_host_work_bytes(s, torch.float64, "periodic", (520, 257)),
                       dtype=torch.uint8, device=DEV)
    sc.apply_composed_host(s, x, y, work, bc="periodic", h=(1, 520))
    yd = torch.empty((257, 520), dtype=torch.float64, device=DEV)
    sc.apply_composed(s, x.to(DEV), yd, bc="periodic", h=(1, 520))
    torch.cuda.synchronize()
    assert torch.equal(yd.cpu(), y)


# every evaluation schedule the apply sweep can launch at its full sizes, with
# the planes per CTA (halo-blocking depth) the sweep's tuning chose for it
FULL_SIZE_SCHEDULES = [
    (2, 8192, np.float64, "pair", 32), (2, 8192, np.float64, "flat", 0),
    (2, 8192, np.float32, "flat", 128), (2, 8192, np.float32, "nested", 64),
    (3, 512, np.float64, "pair", 32), (3, 512, np.float64, "nested", 0),
    (3, 512, np.float32, "nested", 64), (3, 512, np.float32, "flat", 0),
    (3, 512, np.float32, "fused", 0), (3, 512, np.float32, "fused", 32),
    (2, 8192, np.float32, "fused", 0), (2, 8192, np.float32, "fused", 256),
]


def sample_points(n, ndim, seed=77, count=400):
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, n, size=(count, ndim))
    corners = [[0] * ndim, [n - 1] * ndim, [0, n - 1] + [0] * (ndim - 2), [n - 1, 0] + [n - 1] * (ndim - 2),
               [1] * ndim, [n - 2] * ndim, [3] * ndim, [n - 4] * ndim, [n // 2] * ndim,
               [n // 2 - 1] + [0] * (ndim - 1), [0] * (ndim - 1) + [n // 2 - 1], [0] * (ndim - 1) + [n // 2]]
    pts[:len(corners)] = corners
    return pts


def sampled_reference(x, n, ndim, pts):
    """Oracle values at the sampled points and the two magnitude sums the
    tolerances use: sum |c_k x| of the composed weights, and (|B| o |A|)|x|
    of the factors."""
    oL = ost.laplacian(ndim, 4)
    oc = ost.compose(oL, oL)
    x64 = x.astype(np.float64)
    w = oracle_weights(oc, Fraction(1, n), np.float64)
    ref = oap.apply_at(w, x64, "periodic", pts, oc.radius)
    absw = {k: abs(float(v)) for k, v in w.items()}
    mag_flat = oap.apply_at(absw, np.abs(x64), "periodic", pts, oc.radius)
    absL = ost.Stencil.make({k: abs(v) for k, v in oL.coeffs}, oL.hpow)
    wabs = ost.fp_weights(ost.compose(absL, absL), Fraction(1, n), np.float64)
    mag_nested = oap.apply_at(wabs, np.abs(x64), "periodic", pts, oc.radius)
    return ref, mag_flat, mag_nested, oc.npts, oL.npts


def schedule_tolerance(how, dt, npts_c, npts_l, mag_flat, mag_nested):
    """Elementwise bound of each schedule (see the module docstring and the
    nested and pair tests): flat npts eps sum|w x|; nested (2 n_A + 2) eps
    (|B| o |A|)|x| (+ npts eps32 for float32 factor weights); pair 2^-42."""
    eps = np.finfo(dt).eps
    if how == "flat":
        return npts_c * eps * mag_flat
    if how == "pair":
        return 2.0 ** -42 * mag_nested
    # nested and fused: the same two FP32 sums per point, in any order
    b = (2 * npts_l + 2) * eps * mag_nested
    if dt == np.float32:
        b = b + npts_c * eps * mag_nested
    return b


@pytest.mark.parametrize("ndim,n,dt,how,planes", FULL_SIZE_SCHEDULES)
def test_full_size_schedules_sampled(ndim, n, dt, how, planes):
    """The apply-sweep sizes (8192^2, 512^3, periodic, 4th-order Lap o Lap) run
    through apply_tuned with each evaluation schedule and depth recorded by
    tune_set -- the path and launch configuration the bench times -- checked on
    400+ sampled points (corners, the folded-row seam n/2, random) against the
    oracle evaluated point by point."""
    shape = (n,) * ndim
    x = fields.uniform(shape, seed=1234 + ndim, dtype=dt)
    L = sc.laplacian(ndim, 4)
    xt = torch.from_numpy(x).to(DEV)
    yt = torch.full_like(xt, float("nan"))
    wb = sc.apply_composition_work_bytes(L, L, xt.dtype, "periodic", shape)
    work = torch.empty(wb, dtype=torch.uint8, device=DEV)
    sc.tune_set(L, L, xt.dtype, "periodic", shape, {"eval": how, "planes": planes, "ms": 0.0})
    sc.apply_tuned(L, L, xt, yt, work, h=(1, n))
    torch.cuda.synchronize()
    del work
    pts = sample_points(n, ndim)
    y = yt.cpu().numpy()
    got = y[tuple(pts.T)].astype(np.float64)
    ref, mag_flat, mag_nested, npts_c, npts_l = sampled_reference(x, n, ndim, pts)
    tol = schedule_tolerance(how, dt, npts_c, npts_l, mag_flat, mag_nested)
    err = np.abs(got - ref)
    assert np.all(err <= tol), float(np.max(err / tol))
    if dt == np.float64:
        assert np.linalg.norm(err) <= 1e-12 * np.linalg.norm(ref)
    assert not np.isnan(y).any()


FUSED_CASES = [
    # ndim, order, dims (x, y[, z]), boundary: several tiles, ragged tails in every axis
    (3, 4, (136, 40, 21), "periodic"), (3, 2, (72, 24, 8), "periodic"), (3, 4, (72, 24, 8), "periodic"),
    (3, 4, (67, 19, 23), "zero"), (3, 2, (50, 33, 9), "zero"), (3, 4, (66, 21, 13), "ghosted"),
    (3, 2, (70, 17, 11), "ghosted"), (3, 4, (9, 5, 4), "zero"),
    (2, 4, (1100, 301), "periodic"), (2, 2, (128, 8), "periodic"), (2, 4, (1101, 97), "zero"),
    (2, 2, (250, 33), "ghosted"), (2, 4, (244, 40), "ghosted"), (2, 4, (7, 5), "zero"),
]


@pytest.mark.parametrize("ndim,order,dims,bc", FUSED_CASES)
def test_fused_nested_matches_oracle(ndim, order, dims, bc):
    """The single-pass fused nested apply (FP32): the composed operator
    within the two-pass nested bound for every boundary, with ragged tiles,
    and not merely the two-pass kernels (its rounding differs from theirs
    somewhere on a random field)."""
    L = sc.laplacian(ndim, order)
    oL = ost.laplacian(ndim, order)
    oc = ost.compose(oL, oL)
    R = oc.radius
    n = dims[0]
    shape = tuple(reversed(dims))
    xshape = tuple(v + 2 * R for v in shape) if bc == "ghosted" else shape
    x = fields.uniform(xshape, seed=zlib.crc32(repr(("fused", ndim, order, dims, bc)).encode()), dtype=np.float32)
    xt = torch.from_numpy(x).to(DEV)
    yf = torch.full(shape, float("nan"), dtype=torch.float32, device=DEV)
    yn = torch.full(shape, float("nan"), dtype=torch.float32, device=DEV)
    work = torch.empty(sc.apply_composition_work_bytes(L, L, torch.float32, bc, dims), dtype=torch.uint8,
                       device=DEV)
    sc.tune_set(L, L, torch.float32, bc, dims, {"eval": "fused", "planes": 0})
    sc.apply_tuned(L, L, xt, yf, work, bc=bc, h=(1, n), dims=dims)
    sc.apply_composition(L, L, xt, yn, work, bc=bc, h=(1, n), dims=dims)
    torch.cuda.synchronize()
    w = oracle_weights(oc, Fraction(1, n), np.float64)
    y_ref = oap.apply(w, x.astype(np.float64), bc, R)
    absL = ost.Stencil.make({k: abs(v) for k, v in oL.coeffs}, oL.hpow)
    wabs = ost.fp_weights(ost.compose(absL, absL), Fraction(1, n), np.float64)
    mag = oap.apply(wabs, np.abs(x.astype(np.float64)), bc, R)
    eps = np.finfo(np.float32).eps
    bound = (2 * oL.npts + 2 + oc.npts) * eps * mag
    err = np.abs(yf.cpu().numpy().astype(np.float64) - y_ref)
    assert np.all(err <= bound), float(np.max(err / (mag + 1e-300)))
    assert not torch.equal(yf, yn)


def test_invalid_arguments_are_rejected():
    s = lib_bilap(2, 2)
    x = torch.zeros((8, 8), dtype=torch.float64, device=DEV)
    with pytest.raises(sc.ScError):
        sc.apply_composed(s, x, x, bc="periodic", h=(1, 8))  # aliasing
    y = torch.zeros((8, 8), dtype=torch.float64, device=DEV)
    with pytest.raises(sc.ScError):
        sc.apply_composed(s, x, y, bc="periodic", h=(1, 8), dims=(0, 8))
    with pytest.raises(sc.ScError):
        sc.apply_composed(s, x, y, bc="periodic", h=(1, 8), dims=(3, 8))
    s1 = sc.stencil_1d(sc.D2_C2)
    with pytest.raises(sc.ScError):
        sc.apply_composed(s1, x, y, bc="periodic", h=(1, 8))


COMP_CASES = [(2, 2, (1100, 301)), (2, 4, (1101, 97)), (3, 2, (150, 40, 37)), (3, 4, (67, 19, 23)),
              (3, 4, (64, 64, 20))]


@pytest.mark.parametrize("ndim,order,dims", COMP_CASES)
@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("bc", ["periodic", "zero", "ghosted"])
def test_composition_nested_matches_oracle(ndim, order, dims, dt, bc):
    """y = B(A x) from the factors (two passes) equals the oracle's apply of
    the composed stencil, within the rounding bound of the nested sums."""
    L = sc.laplacian(ndim, order)
    oL = ost.laplacian(ndim, order)
    oc = ost.compose(oL, oL)
    R = oc.radius
    n = dims[0]
    w = oracle_weights(oc, Fraction(1, n), np.float64)
    shape = tuple(reversed(dims))
    xshape = tuple(s + 2 * R for s in shape) if bc == "ghosted" else shape
    x = fields.uniform(xshape, seed=zlib.crc32(repr(("nested", ndim, order, dims, bc)).encode()), dtype=dt)
    xt = torch.from_numpy(x).to(DEV)
    yt = torch.full(shape, float("nan"), dtype=xt.dtype, device=DEV)
    sc.apply_composition(L, L, xt, yt, bc=bc, h=(1, n), dims=dims)
    torch.cuda.synchronize()
    y_ref = oap.apply(w, x.astype(np.float64), bc, R)
    absL = ost.Stencil.make({k: abs(v) for k, v in oL.coeffs}, oL.hpow)
    wabs = ost.fp_weights(ost.compose(absL, absL), Fraction(1, n), np.float64)
    mag = oap.apply(wabs, np.abs(x.astype(np.float64)), bc, R)
    eps = np.finfo(dt).eps
    bound = (2 * oL.npts + 2) * eps * mag
    if dt == np.float32:
        bound = bound + oc.npts * np.finfo(np.float32).eps * mag  # float32 weights of each factor
    err = np.abs(yt.cpu().numpy().astype(np.float64) - y_ref)
    assert np.all(err <= bound), float(np.max(err / (mag + 1e-300)))
    if dt == np.float64:
        assert np.linalg.norm(err) <= 1e-12 * np.linalg.norm(y_ref)


def test_star_stencils_use_star_class():
    """Laplacians (axis points only) in 2D/3D, orders 2/4, all boundaries."""
    for ndim, order, dims in [(2, 2, (130, 70)), (2, 4, (300, 33)), (3, 2, (40, 30, 20)), (3, 4, (72, 17, 19))]:
        L = sc.laplacian(ndim, order)
        oL = ost.laplacian(ndim, order)
        for dt in (np.float64, np.float32):
            w = oracle_weights(oL, Fraction(1, dims[0]), dt)
            for bc in ("periodic", "zero", "ghosted"):
                shape = tuple(reversed(dims))
                xs = tuple(s + 2 * oL.radius for s in shape) if bc == "ghosted" else shape
                x = fields.uniform(xs, seed=11, dtype=dt)
                yt = torch.empty(shape, dtype=torch.float64 if dt == np.float64 else torch.float32, device=DEV)
                sc.apply_composed(L, torch.from_numpy(x).to(DEV), yt, bc=bc, h=(1, dims[0]), dims=dims)
                torch.cuda.synchronize()
                check(yt.cpu().numpy(), x, w, bc, oL.radius, dt, oL.npts)


PAIR_CASES = [(2, 4, (8192, 40)), (2, 2, (1100, 301)), (2, 4, (1101, 97)), (3, 4, (150, 40, 37)),
              (3, 2, (64, 20, 30)), (3, 4, (68, 33, 17)), (2, 4, (6, 9)), (2, 4, (1102, 17)),
              (3, 4, (12, 10, 9)), (3, 2, (4, 5, 6))]


def _nested_check(L, oL, x, yt, bc, n, elem_tol):
    oc = ost.compose(oL, oL)
    R = oc.radius
    w = oracle_weights(oc, Fraction(1, n), np.float64)
    y_ref = oap.apply(w, x, bc, R)
    absL = ost.Stencil.make({k: abs(v) for k, v in oL.coeffs}, oL.hpow)
    wabs = ost.fp_weights(ost.compose(absL, absL), Fraction(1, n), np.float64)
    mag = oap.apply(wabs, np.abs(x), bc, R)
    err = np.abs(yt.cpu().numpy() - y_ref)
    assert np.all(err <= elem_tol * mag), float(np.max(err / (mag + 1e-300)))
    assert np.linalg.norm(err) <= 1e-12 * np.linalg.norm(y_ref)


@pytest.mark.parametrize("ndim,order,dims", PAIR_CASES)
@pytest.mark.parametrize("bc", ["periodic", "zero", "ghosted"])
def test_pair_arithmetic_fp64_matches_oracle(ndim, order, dims, bc):
    """FP64 composition evaluated in pairs of FP32 numbers: elementwise
    within 2^-42 of (|B| o |A|)|x| (a few units of 2^-48 per pass, with room),
    normwise within the FP64 target 1e-12."""
    L = sc.laplacian(ndim, order)
    oL = ost.laplacian(ndim, order)
    R = 2 * oL.radius
    n = dims[0]
    shape = tuple(reversed(dims))
    xshape = tuple(s + 2 * R for s in shape) if bc == "ghosted" else shape
    x = fields.uniform(xshape, seed=zlib.crc32(repr(("pair", ndim, order, dims, bc)).encode()))
    yt = torch.full(shape, float("nan"), dtype=torch.float64, device=DEV)
    sc.apply_composition(L, L, torch.from_numpy(x).to(DEV), yt, bc=bc, h=(1, n), dims=dims, arith="pair")
    yn = torch.full(shape, float("nan"), dtype=torch.float64, device=DEV)
    sc.apply_composition(L, L, torch.from_numpy(x).to(DEV), yn, bc=bc, h=(1, n), dims=dims, arith="native")
    torch.cuda.synchronize()
    _nested_check(L, oL, x, yt, bc, n, 2.0 ** -42)
    # even rows take the pair passes (their rounding differs from the native
    # nested passes somewhere), as long as the boundary is periodic or the
    # factors have radius 2; otherwise exactly the native passes run
    paired = n % 2 == 0 and (bc == "periodic" or oL.radius == 2)
    assert torch.equal(yt, yn) != paired


def test_pair_arithmetic_out_of_range_inputs_fall_back():
    """Values that cannot be split into normal floats (tiny, huge, zero mixed
    in) raise the device flag; the native FP64 passes then recompute y."""
    dims = (128, 64)
    L = sc.laplacian(2, 4)
    oL = ost.laplacian(2, 4)
    x = fields.uniform((64, 128), seed=3)
    x[5, 7] = 1e-200
    x[40, 100] = 1e200
    x[10, :] = 0.0
    yt = torch.empty((64, 128), dtype=torch.float64, device=DEV)
    sc.apply_composition(L, L, torch.from_numpy(x).to(DEV), yt, bc="periodic", h=(1, 128), dims=dims, arith="pair")
    torch.cuda.synchronize()
    oc = ost.compose(oL, oL)
    w = oracle_weights(oc, Fraction(1, 128), np.float64)
    y_ref = oap.apply(w, x, "periodic", 4)
    absL = ost.Stencil.make({k: abs(v) for k, v in oL.coeffs}, oL.hpow)
    wabs = ost.fp_weights(ost.compose(absL, absL), Fraction(1, 128), np.float64)
    mag = oap.apply(wabs, np.abs(x), "periodic", 4)
    err = np.abs(yt.cpu().numpy() - y_ref)
    assert np.all(err <= (2 * oL.npts + 2) * np.finfo(np.float64).eps * mag)
    # and a field fully in range gives a different (pair) rounding but the same tolerance
    x2 = fields.uniform((64, 128), seed=4)
    sc.apply_composition(L, L, torch.from_numpy(x2).to(DEV), yt, bc="periodic", h=(1, 128), dims=dims, arith="pair")
    torch.cuda.synchronize()
    _nested_check(L, oL, x2, yt, "periodic", 128, 2.0 ** -42)


@pytest.mark.parametrize("ndim,n,dt", [(2, 512, np.float64), (3, 64, np.float32), (3, 48, np.float64)])
def test_autotuned_apply_matches_oracle(ndim, n, dt):
    """The autotuner picks a schedule and depth; the tuned apply must still
    be the composed operator (FP64: within the pair/FP64 bounds, FP32: the
    FP32 nested bound)."""
    L = sc.laplacian(ndim, 4)
    oL = ost.laplacian(ndim, 4)
    shape = (n,) * ndim
    x = fields.uniform(shape, seed=31, dtype=dt)
    xt = torch.from_numpy(x).to(DEV)
    yt = torch.empty_like(xt)
    wb = sc.apply_composition_work_bytes(L, L, xt.dtype, "periodic", shape)
    work = torch.empty(wb, dtype=torch.uint8, device=DEV)
    choice = sc.autotune_apply(L, L, xt, yt, work, h=(1, n))
    assert choice["eval"] in ("flat", "nested", "pair") and choice["ms"] > 0
    yt.fill_(float("nan"))
    sc.apply_tuned(L, L, xt, yt, work, h=(1, n))
    torch.cuda.synchronize()
    tol = 2.0 ** -42 if dt == np.float64 else (2 * oL.npts + 2 + 73) * np.finfo(np.float32).eps
    _nested_check(L, oL, x.astype(np.float64), yt.double(), "periodic", n, tol) if dt == np.float64 else None
    if dt == np.float32:
        oc = ost.compose(oL, oL)
        w = oracle_weights(oc, Fraction(1, n), np.float64)
        y_ref = oap.apply(w, x.astype(np.float64), "periodic", oc.radius)
        absL = ost.Stencil.make({k: abs(v) for k, v in oL.coeffs}, oL.hpow)
        mag = oap.apply(ost.fp_weights(ost.compose(absL, absL), Fraction(1, n), np.float64),
                        np.abs(x.astype(np.float64)), "periodic", oc.radius)
        assert np.all(np.abs(yt.cpu().numpy() - y_ref) <= tol * mag)


@pytest.mark.parametrize("how,planes", [("flat", 16), ("nested", 0), ("pair", 32)])
def test_saved_tuning_runs_the_recorded_schedule(how, planes):
    """A choice recorded with tune_set is what apply_tuned runs: the same bits
    as calling that schedule directly."""
    n = 48
    L = sc.laplacian(3, 4)
    x = torch.from_numpy(fields.uniform((n,) * 3, seed=77, dtype=np.float64)).to(DEV)
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    wb = sc.apply_composition_work_bytes(L, L, x.dtype, "periodic", (n,) * 3)
    work = torch.empty(wb, dtype=torch.uint8, device=DEV)
    sc.tune_set(L, L, x.dtype, "periodic", (n,) * 3, {"eval": how, "planes": planes, "ms": 0.0})
    sc.apply_tuned(L, L, x, y1, work, h=(1, n))
    if how == "flat":
        sc.apply_composed(sc.compose_stencil(L, L), x, y2, h=(1, n))
    else:
        sc.apply_composition(L, L, x, y2, work, h=(1, n), arith="pair" if how == "pair" else "native")
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("ndim,dims,bc", [(2, (256, 96), "periodic"), (3, (48, 40, 36), "periodic"),
                                          (3, (40, 24, 20), "ghosted"), (2, (130, 70), "zero")])
def test_pair_arithmetic_wide_dynamic_range(ndim, dims, bc):
    """Fields whose magnitudes span 2^-60 .. 2^90 (inside the pair path's
    window), with exact zeros and a constant patch: the split into FP32
    pairs, the error-free sums and the exact rebuild keep every output
    within 2^-42 of (|B| o |A|)|x|, and the pair passes (not the native
    fallback) produced it."""
    L = sc.laplacian(ndim, 4)
    oL = ost.laplacian(ndim, 4)
    R = 2 * oL.radius
    n = dims[0]
    shape = tuple(reversed(dims))
    xshape = tuple(s + 2 * R for s in shape) if bc == "ghosted" else shape
    x = fields.wide_range(xshape, seed=zlib.crc32(repr(("wide", ndim, dims, bc)).encode()), lo_exp=-60,
                          hi_exp=90, zero_frac=0.05, patch=8)
    xt = torch.from_numpy(x).to(DEV)
    yt = torch.full(shape, float("nan"), dtype=torch.float64, device=DEV)
    yn = torch.full(shape, float("nan"), dtype=torch.float64, device=DEV)
    sc.apply_composition(L, L, xt, yt, bc=bc, h=(1, n), dims=dims, arith="pair")
    sc.apply_composition(L, L, xt, yn, bc=bc, h=(1, n), dims=dims, arith="native")
    torch.cuda.synchronize()
    _nested_check(L, oL, x, yt, bc, n, 2.0 ** -42)
    assert not torch.equal(yt, yn)


def _mobility_factors(ndim, axis=0):
    """d/dx and d/dx composed with d2/dx2, along one axis (library and oracle)."""
    d1 = sc.stencil_embed(sc.stencil_1d(sc.D1_C2), ndim, axis)
    d2 = sc.stencil_embed(sc.stencil_1d(sc.D2_C2), ndim, axis)
    o1 = ost.embed(ost.d1_central2(), ndim, axis)
    o2 = ost.embed(ost.d2_central2(), ndim, axis)
    return d1, sc.compose_stencil(d1, d2), o1, ost.compose(o1, o2)


@pytest.mark.parametrize("ndim,dims,axis", [(2, (130, 70), 0), (2, (96, 64), 1), (3, (40, 30, 20), 2)])
@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_varcoef_apply_matches_oracle(ndim, dims, axis, dt):
    """d/dx(M d/dx(d2/dx2 x)) with a random positive mobility M (Sec. 2.2.3)
    against the oracle's definition, elementwise within the rounding of two
    short sums and one product."""
    outer, inner, oo, oi = _mobility_factors(ndim, axis)
    n = dims[0]
    shape = tuple(reversed(dims))
    rng = np.random.default_rng(ndim * 10 + axis)
    x = rng.uniform(-1, 1, shape).astype(dt)
    m = rng.uniform(0.5, 2.0, shape).astype(dt)
    xt, mt = torch.from_numpy(x).to(DEV), torch.from_numpy(m).to(DEV)
    yt = torch.full(shape, float("nan"), dtype=xt.dtype, device=DEV)
    work = torch.empty(x.size * x.itemsize, dtype=torch.uint8, device=DEV)
    sc.apply_varcoef(outer, inner, mt, xt, yt, work, h=(1, n), dims=dims)
    torch.cuda.synchronize()
    wo = oracle_weights(oo, Fraction(1, n), dt)
    wi = oracle_weights(oi, Fraction(1, n), dt)
    ref = oap.apply_varcoef(wo, wi, m.astype(np.float64), x.astype(np.float64))
    ao = {k: abs(float(v)) for k, v in wo.items()}
    ai = {k: abs(float(v)) for k, v in wi.items()}
    mag = oap.apply_varcoef(ao, ai, np.abs(m.astype(np.float64)), np.abs(x.astype(np.float64)))
    tol = (oo.npts + oi.npts + 2) * np.finfo(dt).eps * mag
    err = np.abs(yt.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= tol), float(np.max(err / (mag + 1e-300)))


def test_varcoef_explicit_stability_limit():
    """Explicit Euler steps of f_t = -d/dx(M d/dx(d2/dx2 f)) with M = 1 through
    the composed operator (Sec. 2.2.3, Table 1): stable at 0.98 x (27/32) h^4,
    unstable at 1.05 x (27/32) h^4 (the worst mode grows by |1 - 2.1| per step)."""
    n = 256
    outer, inner, _, _ = _mobility_factors(2, 0)
    rng = np.random.default_rng(3)
    u0 = torch.from_numpy(rng.uniform(-1, 1, (4, n))).to(DEV)
    m = torch.ones_like(u0)
    y = torch.empty_like(u0)
    work = torch.empty(u0.numel() * 8, dtype=torch.uint8, device=DEV)
    h4 = (1.0 / n) ** 4
    growth = {}
    for fac in (0.98, 1.05):
        u = u0.clone()
        dt = fac * 27.0 / 32.0 * h4
        for _ in range(300):
            sc.apply_varcoef(outer, inner, m, u, y, work, h=(1, n))
            u -= dt * y
        growth[fac] = float(u.abs().max() / u0.abs().max())
    assert growth[0.98] <= 1.0 + 1e-9, growth
    assert growth[1.05] > 100.0, growth
