"""The product path has no CPU fallback: every entry point that takes device
tensors refuses host tensors (and wrong dtypes) in the binding, before the
library could be handed a host address, and nothing is computed on the CPU.
Runs without a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests.libutil import ensure_built  # noqa: E402

ensure_built()
import paper_2205_03354_gb300 as sc  # noqa: E402
from paper_2205_03354_gb300 import solvers  # noqa: E402


def _host(*shape, dtype=torch.float64):
    return torch.zeros(shape, dtype=dtype)


def test_applies_refuse_host_tensors():
    L = sc.laplacian(2, 2)
    x, y = _host(16, 16), _host(16, 16)
    work = torch.zeros(1 << 16, dtype=torch.uint8)
    with pytest.raises(ValueError):
        sc.apply_composed(sc.compose_stencil(L, L), x, y, h=(1, 16))
    with pytest.raises(ValueError):
        sc.apply_composition(L, L, x, y, h=(1, 16))
    with pytest.raises(ValueError):
        sc.apply_composition(L, L, x, y, work, h=(1, 16), arith="pair")
    with pytest.raises(ValueError):
        sc.autotune_apply(L, L, x, y, work, h=(1, 16))
    with pytest.raises(ValueError):
        sc.apply_tuned(L, L, x, y, work, h=(1, 16))


def test_solvers_refuse_host_tensors():
    f, g, x = _host(16, 16), _host(20, 20), _host(16, 16)
    with pytest.raises(ValueError):
        sc.make_bvp(f, g, x)
    with pytest.raises(ValueError):
        sc.solve_biharmonic(f, g, x)
    c = sc.make_ch((16, 16), 1, (1, 16), 1e-6, 1.0, 1e-4)
    u = _host(1, 16, 16)
    for call in (lambda: sc.ch_step(c, u), lambda: sc.ch_run(c, u, 2), lambda: sc.ch_stats(c, u),
                 lambda: solvers.ch_stats_noalloc(c, u)):
        with pytest.raises(ValueError):
            call()
    # a float32 field is refused as well (the solvers take FP64 fields)
    with pytest.raises(ValueError):
        sc.ch_step(c, _host(1, 16, 16, dtype=torch.float32))


def test_server_refuses_a_host_arena():
    with pytest.raises(ValueError):
        sc.Server(torch.zeros(1 << 20, dtype=torch.uint8))


def test_host_buffer_entry_point_refuses_without_device_work():
    """The host-buffer apply takes host x/y but a device work buffer; a host
    work buffer is refused."""
    L = sc.laplacian(2, 2)
    x = np.zeros((16, 16))
    with pytest.raises(ValueError):
        sc.apply_composed_host(sc.compose_stencil(L, L), torch.from_numpy(x), torch.from_numpy(x.copy()),
                               torch.zeros(1 << 16, dtype=torch.uint8), h=(1, 16))


def test_overlapping_device_ranges_are_refused_before_any_launch():
    """x and y (and a work space) must be disjoint byte ranges, not merely
    different pointers: y starting inside x's ghosted extent, or a work space
    overlapping either, is refused with SC_EINVAL.  The addresses are never
    dereferenced (the check runs before anything is enqueued)."""
    import ctypes

    from paper_2205_03354_gb300._lib_loader import lib
    from paper_2205_03354_gb300.ops import dims_arg

    L = sc.laplacian(2, 4)
    B = sc.compose_stencil(L, L)
    dims = dims_arg((64, 64))
    base = 1 << 40
    # ghosted input (64 + 8)^2 doubles; y placed 8 bytes before its end
    x = base
    y = base + (72 * 72 - 1) * 8
    rc = lib.sc_apply_composed(ctypes.byref(B), 0, 1, dims, 1, 64, ctypes.c_void_p(x), ctypes.c_void_p(y), None)
    assert rc == 1  # SC_EINVAL
    # the same y is fine for a periodic input of 64^2 doubles only if it lies beyond it
    y2 = base + 64 * 64 * 8 - 8
    rc = lib.sc_apply_composed(ctypes.byref(B), 0, 0, dims, 1, 64, ctypes.c_void_p(x), ctypes.c_void_p(y2), None)
    assert rc == 1
    y3 = base + 64 * 64 * 8 * 2  # disjoint x and y; the work space starts inside y
    rc = lib.sc_apply_composition(ctypes.byref(L), ctypes.byref(L), 0, 0, dims, ctypes.c_int64(1), ctypes.c_int64(64),
                                  ctypes.c_void_p(x), ctypes.c_void_p(y3), ctypes.c_void_p(y3 + 64),
                                  ctypes.c_size_t(1 << 30), 0, None)
    assert rc == 1
