"""sc_ch_stats_noalloc, the statistics entry point for callers that cannot
allocate device memory (their host program owns all device allocations, or
cudaMalloc's possible device synchronisation is not acceptable to them).

Called straight through the C ABI on two calls in a row of different sizes
(a 3D batch, then a smaller 2D field), it must give the same mass and free
energy as sc_ch_stats (the entry point that takes a caller-provided work
buffer) within the 1e-12 relative tolerance of that function's own oracle
test, and -- because the two share their reduction kernel -- the same values
as the CPU oracle's mass and free energy, computed independently.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.libutil import ensure_built  # noqa: E402

ensure_built()
import paper_2205_03354_gb300 as sc  # noqa: E402
from paper_2205_03354_gb300.solvers import Ch  # noqa: E402
from oracle import ch as och  # noqa: E402
from synth_inputs import manufactured  # noqa: E402

DEV = "cuda:0"


def _call_noalloc(c, u):
    m = (ctypes.c_double * c.batch)()
    e = (ctypes.c_double * c.batch)()
    rc = sc.lib.sc_ch_stats_noalloc(ctypes.byref(c), ctypes.c_void_p(u.data_ptr()), m, e,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, sc.lib.sc_last_error()
    return list(m), list(e)


def test_no_alloc_stats_match_work_buffer_variant():
    cases = [((3, 96), 2, 2), ((2, 40), 1, 3)]  # ((ndim, n), batch, seed): second call is smaller
    for (ndim, n), batch, seed in cases:
        u = torch.from_numpy(manufactured.ch_uniform(n, ndim, seed=seed, amp=0.6, batch=batch)).to(DEV)
        c = sc.make_ch((n,) * ndim, batch, (1, n), 1e-6, 1.0, 0.02 ** 2)
        assert isinstance(c, Ch)
        m_ref, e_ref = sc.ch_stats(c, u)
        m, e = _call_noalloc(c, u)
        un = u.cpu().numpy()
        for b in range(batch):
            scale = float(u[b].abs().sum())
            assert abs(m[b] - m_ref[b]) <= 1e-12 * scale
            assert abs(e[b] - e_ref[b]) <= 1e-12 * abs(e_ref[b])
            assert abs(m[b] - och.mass(un[b])) <= 1e-12 * scale
            e_or = och.free_energy(un[b], 1.0 / n, 0.02 ** 2, ("cubic",))
            assert abs(e[b] - e_or) <= 1e-12 * abs(e_or)


def test_no_alloc_rejects_oversized_fields():
    c = sc.make_ch((4097, 4097), 1, (1, 4097), 1e-6, 1.0, 1e-4)
    u = torch.zeros(1, dtype=torch.float64, device=DEV)  # never read: rejected first
    m = (ctypes.c_double * 1)()
    e = (ctypes.c_double * 1)()
    rc = sc.lib.sc_ch_stats_noalloc(ctypes.byref(c), ctypes.c_void_p(u.data_ptr()), m, e, None)
    assert rc == 1  # SC_EINVAL
    assert b"at most" in sc.lib.sc_last_error()
