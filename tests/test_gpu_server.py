"""The serving loop: continuous batching of plate-problem solves.

Each result obtained through the server, while other requests of other sizes
and dimensions are in flight, must be the same as the result of solving that
request alone (same precision): bit for bit, since the engine's reductions
do not depend on the batch.  A small arena forces queueing and admission as
memory frees up.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.libutil import ensure_built  # noqa: E402

ensure_built()
import paper_2205_03354_gb300 as sc  # noqa: E402
from synth_inputs import manufactured  # noqa: E402

DEV = "cuda:0"


def _case(n, ndim, ks):
    m = manufactured.bvp_case(n, ndim, 2, ks)
    return np.ascontiguousarray(m["g"]), np.ascontiguousarray(m["u_padded"])


def _solo(f, g, prec, solver="persistent"):
    ft, gt = torch.from_numpy(f).to(DEV), torch.from_numpy(g).to(DEV)
    x = torch.empty(f.shape, dtype=torch.float64, device=DEV)
    info = sc.solve_biharmonic(ft, gt, x, prec=prec, solver=solver, rtol=1e-10)
    return x.cpu().numpy(), info


SPECS = [(40, 2, (1, 1)), (24, 2, (3, 2)), (12, 3, (1, 2, 1)), (64, 2, (2, 5)), (17, 2, (1, 1)),
         (10, 3, (2, 1, 3)), (33, 2, (4, 4)), (20, 3, (1, 1, 1))]


def test_results_same_alone_and_in_the_mix():
    arena = torch.empty(512 << 20, dtype=torch.uint8, device=DEV)
    srv = sc.Server(arena, max_active=64, slice_ms=1.0)
    try:
        tickets, bufs = [], []
        for n, nd, ks in SPECS:
            f, g = _case(n, nd, ks)
            x = np.full(f.shape, np.nan)
            tickets.append(srv.submit(f, g, x, prec="auto"))
            bufs.append((f, g, x))
        srv.drain(300.0)
        for t, (f, g, x) in zip(tickets, bufs):
            res = srv.poll(t)
            assert res is not None and res["status"] == 0 and res["rel_res"] <= 1e-10, res
            assert res["latency_s"] >= res["queue_s"] >= 0.0
            solo, info = _solo(f, g, res["prec"])
            assert info["iters"] == res["iters"]
            assert np.array_equal(solo, x)
    finally:
        srv.close()


def test_small_arena_queues_and_admits_as_memory_frees():
    f0, g0 = _case(64, 2, (1, 1))
    need = sc.request_bytes(sc.make_request(f0, g0, np.empty_like(f0)))
    arena = torch.empty(2 * need + (4 << 20), dtype=torch.uint8, device=DEV)  # about two at a time
    srv = sc.Server(arena, max_active=8, slice_ms=0.5)
    try:
        tickets, bufs = [], []
        for k in range(6):
            f, g = _case(64, 2, (1 + k % 3, 1))
            x = np.full(f.shape, np.nan)
            tickets.append(srv.submit(f, g, x, prec="f64"))
            bufs.append(x)
        done = {}
        import time
        t0 = time.time()
        while len(done) < len(tickets) and time.time() - t0 < 300:
            for t in tickets:
                if t not in done:
                    r = srv.poll(t)
                    if r is not None:
                        done[t] = r
            time.sleep(0.002)
        assert len(done) == 6
        assert all(r["status"] == 0 and r["rel_res"] <= 1e-10 for r in done.values())
        assert max(r["queue_s"] for r in done.values()) > 0.0  # some had to wait for memory
        assert all(np.isfinite(x).all() for x in bufs)
        # unknown ticket and oversized request
        with pytest.raises(sc.ScError):
            srv.poll(10 ** 9)
        fb, gb = _case(400, 2, (1, 1))
        with pytest.raises(sc.ScError) as e:
            srv.submit(fb, gb, np.empty_like(fb))
        assert e.value.status == 2  # SC_ENOMEM
    finally:
        srv.close()


def test_burst_of_many_requests_all_converge():
    """Many small requests of both dimensions at once: the persistent launch
    then spans most of the GPU (the CTA map is at its largest); every result
    must converge and match its solo solve."""
    arena = torch.empty(2 << 30, dtype=torch.uint8, device=DEV)
    srv = sc.Server(arena, max_active=512, slice_ms=1.0)
    rng = np.random.default_rng(9)
    try:
        jobs = []
        for k in range(160):
            nd = 2 if k % 3 else 3
            n = int(rng.integers(12, 48)) if nd == 2 else int(rng.integers(8, 16))
            f, g = _case(n, nd, tuple(int(v) for v in rng.integers(1, 4, size=nd)))
            x = np.full(f.shape, np.nan)
            jobs.append((srv.submit(f, g, x, prec="auto"), f, g, x))
        srv.drain(600.0)
        for t, f, g, x in jobs:
            r = srv.poll(t)
            assert r["status"] == 0 and r["rel_res"] <= 1e-10, r
        for t, f, g, x in jobs[:12]:
            solo, info = _solo(f, g, "auto")
            assert np.array_equal(solo, x)
    finally:
        srv.close()


def _ch_solo(u0, n, ndim, h, dt, kappa, prec, chem_kw):
    u = torch.from_numpy(u0.copy()).to(DEV).reshape((1,) + u0.shape)
    c = sc.make_ch((n,) * ndim, 1, h, dt, 1.0, kappa, prec=prec, rtol=1e-10, **chem_kw)
    info = sc.ch_step(c, u)[0]
    return u[0].cpu().numpy(), info


def test_plate_and_cahn_hilliard_requests_same_alone_and_in_the_mix():
    """Plate problems and Cahn-Hilliard steps (2D and 3D, cubic and double
    well, FP64 and mixed precision) of several sizes served together: every
    result is bit-identical to the same request solved alone (sc_ch_step
    with batch 1 / sc_solve_biharmonic), and the Cahn-Hilliard steps match
    the oracle's DFT closed form."""
    from oracle import ch as och
    arena = torch.empty(1 << 30, dtype=torch.uint8, device=DEV)
    srv = sc.Server(arena, max_active=64, slice_ms=1.0)
    ch_specs = [(64, 2, (1, 64), 2e-5, 0.05 ** 2, "auto", {}), (96, 2, (1, 96), 1e-6, 0.01 ** 2, "mixed", {}),
                (24, 3, (1, 24), 1e-5, 0.05 ** 2, "f64", {}),
                (48, 2, (200, 48), 0.05, 2.0, "auto", dict(chem="double_well", rho=5.0, ca=0.3, cb=0.7))]
    try:
        jobs = []
        for k, (n, nd, ks) in enumerate(SPECS[:5]):
            f, g = _case(n, nd, ks)
            x = np.full(f.shape, np.nan)
            jobs.append(("plate", srv.submit(f, g, x, prec="auto"), (f, g), x))
            if k < len(ch_specs):
                cn, cnd, h, dt, kap, prec, kw = ch_specs[k]
                u0 = manufactured.ch_uniform(cn, cnd, seed=50 + k, amp=0.3) + (0.5 if kw else 0.0)
                u0 = np.ascontiguousarray(u0)
                xc = np.full(u0.shape, np.nan)
                jobs.append(("ch", srv.submit_ch(u0, xc, h, dt, kappa=kap, prec=prec, **kw),
                             (u0, cn, cnd, h, dt, kap, prec, kw), xc))
        srv.drain(300.0)
        for kind, t, args, x in jobs:
            res = srv.poll(t)
            assert res is not None and res["status"] == 0 and res["rel_res"] <= 1e-10, (kind, res)
            if kind == "plate":
                solo, info = _solo(*args, res["prec"])
            else:
                u0, cn, cnd, h, dt, kap, prec, kw = args
                solo, info = _ch_solo(u0, cn, cnd, h, dt, kap, res["prec"], kw)
                chem = ("double_well", 5.0, 0.3, 0.7) if kw else ("cubic",)
                ref = och.step_fft(u0, h[0] / h[1], dt, 1.0, kap, chem)
                assert np.max(np.abs(x - ref)) <= 1e-8 * max(1.0, np.max(np.abs(ref)))
            assert info["iters"] == res["iters"], kind
            assert np.array_equal(solo, x), kind
    finally:
        srv.close()


def test_failed_time_slice_frees_the_arena_and_refuses_new_work():
    """Failure detection without a GPU fault: the scheduler's test hook makes
    its second time slice fail as a failed launch would.  The requests then
    resident end with SC_ECUDA, their arena space comes back (free bytes equal
    the arena again), later submissions are refused with the same error, and
    the device keeps working."""
    arena = torch.empty(256 << 20, dtype=torch.uint8, device=DEV)
    srv = sc.Server(arena, max_active=16, slice_ms=0.2, fail_slice=2)
    try:
        jobs = []
        for n, nd, ks in SPECS:
            f, g = _case(n, nd, ks)
            x = np.full(f.shape, np.nan)
            try:
                jobs.append(srv.submit(f, g, x, prec="f64"))
            except sc.ScError as e:  # the failure may already have happened
                assert e.status == 7 and jobs
        srv.drain(120.0)
        res = [srv.poll(t) for t in jobs]
        assert all(r is not None for r in res)
        assert any(r["status"] == 7 for r in res)  # SC_ECUDA for those resident at the failure
        assert all(r["status"] in (0, 7) for r in res)
        st = srv.status()
        assert st["worker_error"] == 7 and st["active"] == 0 and st["pending"] == 0
        assert st["free_bytes"] == st["arena_bytes"]
        f, g = _case(16, 2, (1, 1))
        with pytest.raises(sc.ScError) as e:
            srv.submit(f, g, np.empty_like(f))
        assert e.value.status == 7
    finally:
        srv.close()
    f, g = _case(16, 2, (1, 1))
    solo, info = _solo(f, g, "f64")
    assert info["status"] == 0 and info["rel_res"] <= 1e-10


def test_large_plates_go_to_the_preconditioned_solver_alongside_batched_ones():
    """Plate problems of at least 2^16 points are routed (by the automatic
    rule) to the preconditioned solver on the server's second scheduler
    thread while small ones are batched: every result equals its solo solve
    with the same solver, bit for bit, and the large ones take tens of
    iterations."""
    arena = torch.empty(2 << 30, dtype=torch.uint8, device=DEV)
    srv = sc.Server(arena, max_active=64, slice_ms=1.0)
    try:
        jobs = []
        for n, nd, ks in [(300, 2, (1, 2)), (40, 2, (1, 1)), (41, 3, (1, 1, 2)), (24, 2, (3, 2)), (512, 2, (2, 1)),
                          (12, 3, (1, 2, 1))]:
            f, g = _case(n, nd, ks)
            x = np.full(f.shape, np.nan)
            big = f.size >= (1 << 16)
            jobs.append((big, srv.submit(f, g, x, prec="f64"), f, g, x))
        srv.drain(300.0)
        for big, t, f, g, x in jobs:
            r = srv.poll(t)
            assert r is not None and r["status"] == 0 and r["rel_res"] <= 1e-10, r
            solo, info = _solo(f, g, "f64", "pcg" if big else "persistent")
            assert info["iters"] == r["iters"]
            if big:
                assert r["iters"] <= 80
            assert np.array_equal(solo, x)
        st = srv.status()
        assert st["free_bytes"] == st["arena_bytes"] and st["active"] == 0 and st["pending"] == 0
    finally:
        srv.close()
