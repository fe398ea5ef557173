"""Solver entry points (marshalling only): sc_solve_biharmonic[_batch],
sc_ch_step, sc_ch_stats."""
from __future__ import annotations

import ctypes

import torch

from ._lib_loader import check, lib
from .ops import require_device, stream_arg

PREC_F64, PREC_MIXED, PREC_AUTO = 0, 1, 2
SOLVER_PERSISTENT, SOLVER_PLAIN, SOLVER_PCG = 0, 1, 2
_PREC = {"f64": PREC_F64, "mixed": PREC_MIXED, "auto": PREC_AUTO}
_SOLVER = {"persistent": SOLVER_PERSISTENT, "plain": SOLVER_PLAIN, "pcg": SOLVER_PCG}


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("outer", ctypes.c_int64), ("rel_res", ctypes.c_double),
                ("status", ctypes.c_int32), ("prec", ctypes.c_int32), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {"iters": int(self.iters), "outer": int(self.outer), "rel_res": float(self.rel_res),
                "status": int(self.status), "prec": "mixed" if self.prec == PREC_MIXED else "f64",
                "seconds": float(self.seconds)}


class Bvp(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("order", ctypes.c_int32), ("n", ctypes.c_int64 * 3),
                ("prec", ctypes.c_int32), ("solver", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("maxit", ctypes.c_int64), ("f_dev", ctypes.c_void_p), ("ghost_dev", ctypes.c_void_p),
                ("x_dev", ctypes.c_void_p)]


class Ch(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("order", ctypes.c_int32), ("n", ctypes.c_int64 * 3),
                ("batch", ctypes.c_int32), ("h_num", ctypes.c_int64), ("h_den", ctypes.c_int64),
                ("dt", ctypes.c_double), ("M", ctypes.c_double), ("kappa", ctypes.c_double),
                ("chem", ctypes.c_int32), ("rho", ctypes.c_double), ("ca", ctypes.c_double),
                ("cb", ctypes.c_double), ("prec", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("rtol", ctypes.c_double), ("maxit", ctypes.c_int64)]


_BP = ctypes.POINTER(Bvp)
_CP = ctypes.POINTER(Ch)
_IP = ctypes.POINTER(SolveInfo)
lib.sc_bvp_work_bytes.argtypes = [_BP]
lib.sc_bvp_work_bytes.restype = ctypes.c_size_t
lib.sc_bvp_batch_work_bytes.argtypes = [_BP, ctypes.c_int32]
lib.sc_bvp_batch_work_bytes.restype = ctypes.c_size_t
lib.sc_solve_biharmonic.argtypes = [_BP, ctypes.c_void_p, ctypes.c_size_t, _IP, ctypes.c_void_p]
lib.sc_solve_biharmonic.restype = ctypes.c_int
lib.sc_solve_biharmonic_batch.argtypes = [_BP, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, _IP,
                                          ctypes.c_void_p]
lib.sc_solve_biharmonic_batch.restype = ctypes.c_int
lib.sc_ch_work_bytes.argtypes = [_CP]
lib.sc_ch_work_bytes.restype = ctypes.c_size_t
lib.sc_ch_step.argtypes = [_CP, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, _IP, ctypes.c_void_p]
lib.sc_ch_step.restype = ctypes.c_int
lib.sc_ch_stats.argtypes = [_CP, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
lib.sc_ch_stats.restype = ctypes.c_int


def _work(nbytes: int, device, work):
    if work is not None:
        require_device("work", work)
        if work.numel() * work.element_size() < nbytes:
            raise ValueError("work buffer too small")
        return work
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)


def make_bvp(f: torch.Tensor, ghost: torch.Tensor, x: torch.Tensor, order=2, prec="auto",
             solver="persistent", rtol=1e-10, maxit=10_000_000) -> Bvp:
    for t in (f, ghost, x):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("f, ghost and x must be contiguous float64 CUDA tensors")
    nd = x.dim()
    b = Bvp()
    b.ndim, b.order = nd, order
    for a, s in enumerate(reversed(x.shape)):
        b.n[a] = s
    b.prec = _PREC[prec] if isinstance(prec, str) else int(prec)
    b.solver = _SOLVER[solver] if isinstance(solver, str) else int(solver)
    b.rtol, b.maxit = rtol, maxit
    b.f_dev, b.ghost_dev, b.x_dev = f.data_ptr(), ghost.data_ptr(), x.data_ptr()
    return b


def bvp_work_bytes(b: Bvp) -> int:
    return int(lib.sc_bvp_work_bytes(ctypes.byref(b)))


def solve_biharmonic(f, ghost, x, order=2, prec="auto", solver="persistent", rtol=1e-10,
                     maxit=10_000_000, work=None, stream=None) -> dict:
    """Plate problem of Sec. 3.3 on the device; x (interior) is overwritten."""
    b = make_bvp(f, ghost, x, order, prec, solver, rtol, maxit)
    nb = bvp_work_bytes(b)
    if nb == 0:
        check(lib.sc_solve_biharmonic(ctypes.byref(b), None, 0, ctypes.byref(SolveInfo()), None))
    w = _work(nb, x.device, work)
    info = SolveInfo()
    check(lib.sc_solve_biharmonic(ctypes.byref(b), ctypes.c_void_p(w.data_ptr()), nb, ctypes.byref(info),
                                  stream_arg(stream)))
    return info.as_dict()


def solve_biharmonic_batch(problems: list, work=None, stream=None) -> list:
    """problems: list of Bvp (see make_bvp), solved together."""
    arr = (Bvp * len(problems))(*problems)
    nb = int(lib.sc_bvp_batch_work_bytes(arr, len(problems)))
    if nb == 0:
        check(lib.sc_solve_biharmonic_batch(arr, len(problems), None, 0, (SolveInfo * len(problems))(), None))
    dev = torch.device("cuda", torch.cuda.current_device())
    w = _work(nb, dev, work)
    infos = (SolveInfo * len(problems))()
    check(lib.sc_solve_biharmonic_batch(arr, len(problems), ctypes.c_void_p(w.data_ptr()), nb, infos,
                                        stream_arg(stream)))
    return [i.as_dict() for i in infos]


def make_ch(shape, batch, h, dt, M=1.0, kappa=1e-4, chem="cubic", rho=0.0, ca=0.0, cb=0.0, order=2,
            prec="auto", solver="persistent", rtol=1e-10, maxit=1_000_000) -> Ch:
    c = Ch()
    c.ndim, c.order, c.batch = len(shape), order, batch
    for a, s in enumerate(reversed(shape)):
        c.n[a] = s
    c.h_num, c.h_den = int(h[0]), int(h[1])
    c.dt, c.M, c.kappa = dt, M, kappa
    c.chem = 0 if chem == "cubic" else 1
    c.rho, c.ca, c.cb = rho, ca, cb
    c.prec = _PREC[prec] if isinstance(prec, str) else int(prec)
    c.solver = _SOLVER[solver] if isinstance(solver, str) else int(solver)
    c.rtol, c.maxit = rtol, maxit
    return c


def ch_work_bytes(c: Ch) -> int:
    return int(lib.sc_ch_work_bytes(ctypes.byref(c)))


def ch_step(c: Ch, u: torch.Tensor, work=None, stream=None) -> list:
    """One IMEX step of every field in u (batch x n^d, float64, in place)."""
    if not (u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()):
        raise ValueError("u must be a contiguous float64 CUDA tensor")
    nb = ch_work_bytes(c)
    if nb == 0:
        check(lib.sc_ch_step(ctypes.byref(c), ctypes.c_void_p(u.data_ptr()), None, 0,
                             (SolveInfo * max(1, c.batch))(), None))
    w = _work(nb, u.device, work)
    infos = (SolveInfo * c.batch)()
    check(lib.sc_ch_step(ctypes.byref(c), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(w.data_ptr()), nb,
                         infos, stream_arg(stream)))
    return [i.as_dict() for i in infos]


lib.sc_ch_step_sbdf.argtypes = [_CP, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_size_t, _IP, ctypes.c_void_p]
lib.sc_ch_step_sbdf.restype = ctypes.c_int


def ch_step_sbdf(c: Ch, u: torch.Tensor, hist, order: int, work=None, stream=None) -> list:
    """One SBDF step of the given order (1-3): u (u^n) in place -> u^(n+1);
    hist (order >= 2: (order - 1) x batch x n^d) -> the next step's history."""
    require_device("u", u, torch.float64)
    if order > 1:
        require_device("hist", hist, torch.float64)
    nb = ch_work_bytes(c)
    w = _work(nb, u.device, work)
    infos = (SolveInfo * c.batch)()
    check(lib.sc_ch_step_sbdf(ctypes.byref(c), int(order), ctypes.c_void_p(u.data_ptr()),
                              ctypes.c_void_p(hist.data_ptr() if order > 1 else 0), ctypes.c_void_p(w.data_ptr()),
                              nb, infos, stream_arg(stream)))
    return [i.as_dict() for i in infos]


def ch_stats(c: Ch, u: torch.Tensor, work=None, stream=None):
    """(mass[batch], energy[batch]) as Python lists."""
    require_device("u", u, torch.float64)
    n = 1
    for a in range(c.ndim):
        n *= c.n[a]
    nb = (2 * ((n + 4095) // 4096) + 2) * 8
    w = _work(nb, u.device, work)
    m = (ctypes.c_double * c.batch)()
    e = (ctypes.c_double * c.batch)()
    check(lib.sc_ch_stats(ctypes.byref(c), ctypes.c_void_p(u.data_ptr()), m, e, ctypes.c_void_p(w.data_ptr()),
                          nb, stream_arg(stream)))
    return list(m), list(e)


lib.sc_ch_stats_noalloc.argtypes = [_CP, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
lib.sc_ch_stats_noalloc.restype = ctypes.c_int


def ch_stats_noalloc(c: Ch, u: torch.Tensor, stream=None):
    """sc_ch_stats without a work buffer (fixed library scratch, at most 2^24
    grid points per field; calls sharing a device must not overlap)."""
    require_device("u", u, torch.float64)
    m = (ctypes.c_double * c.batch)()
    e = (ctypes.c_double * c.batch)()
    check(lib.sc_ch_stats_noalloc(ctypes.byref(c), ctypes.c_void_p(u.data_ptr()), m, e, stream_arg(stream)))
    return list(m), list(e)


lib.sc_noalloc_forget.argtypes = []
lib.sc_noalloc_forget.restype = None


def noalloc_forget():
    """Drop the kept scratch addresses (call after cudaDeviceReset)."""
    lib.sc_noalloc_forget()


lib.sc_ch_run_work_bytes.argtypes = [_CP, ctypes.c_int64]
lib.sc_ch_run_work_bytes.restype = ctypes.c_size_t
lib.sc_ch_run.argtypes = [_CP, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                          _IP, ctypes.c_void_p]
lib.sc_ch_run.restype = ctypes.c_int


def ch_run(c: Ch, u: torch.Tensor, nsteps: int, use_graph=True, work=None, stream=None) -> list:
    """nsteps IMEX steps of every field of u in place; returns per-step lists
    of per-field info dicts."""
    require_device("u", u, torch.float64)
    nb = int(lib.sc_ch_run_work_bytes(ctypes.byref(c), nsteps))
    w = _work(nb, u.device, work)
    infos = (SolveInfo * (nsteps * c.batch))()
    check(lib.sc_ch_run(ctypes.byref(c), ctypes.c_void_p(u.data_ptr()), nsteps, 1 if use_graph else 0,
                        ctypes.c_void_p(w.data_ptr()), nb, infos, stream_arg(stream)))
    d = [i.as_dict() for i in infos]
    return [d[k * c.batch:(k + 1) * c.batch] for k in range(nsteps)]


lib.sc_selftest_barrier_timeout.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]
lib.sc_selftest_barrier_timeout.restype = ctypes.c_int


def selftest_barrier_timeout(spin_limit: int = 1 << 14, stream=None) -> int:
    """Runs the solver barrier with a member that never arrives; returns the
    status the bounded wait reports (SC_ETIMEOUT = 5)."""
    w = torch.empty(4096, dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))
    st = ctypes.c_int32(-1)
    check(lib.sc_selftest_barrier_timeout(ctypes.c_void_p(w.data_ptr()), 4096, spin_limit, ctypes.byref(st),
                                          stream_arg(stream)))
    return st.value


class SolverTuning(ctypes.Structure):
    _fields_ = [("log2_scale", ctypes.c_int32), ("ms", ctypes.c_float * 5)]

    def as_dict(self):
        return {"log2_scale": int(self.log2_scale), "ms_by_log2_scale": {k - 2: float(self.ms[k]) for k in range(5)}}


lib.sc_autotune_solver.argtypes = [_BP, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.POINTER(SolverTuning), ctypes.c_void_p]
lib.sc_autotune_solver.restype = ctypes.c_int
lib.sc_autotune_ch.argtypes = [_CP, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                               ctypes.POINTER(SolverTuning), ctypes.c_void_p]
lib.sc_autotune_ch.restype = ctypes.c_int
lib.sc_solver_tile_scale_set.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
lib.sc_solver_tile_scale_set.restype = ctypes.c_int
lib.sc_solver_tile_scale_get.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
lib.sc_solver_tile_scale_get.restype = ctypes.c_int


def autotune_solver(probs: list, iters: int = 200, work=None, stream=None) -> dict:
    """Times the persistent engine's tile scales on a plate batch (x buffers
    are overwritten) and keeps the fastest for the classes present."""
    arr = (Bvp * len(probs))(*probs)
    nb = int(lib.sc_bvp_batch_work_bytes(arr, len(probs)))
    w = _work(nb, torch.device("cuda", torch.cuda.current_device()), work)
    t = SolverTuning()
    check(lib.sc_autotune_solver(arr, len(probs), iters, ctypes.c_void_p(w.data_ptr()), nb, ctypes.byref(t),
                                 stream_arg(stream)))
    return t.as_dict()


def autotune_ch(c: Ch, u: torch.Tensor, iters: int = 100, work=None, stream=None) -> dict:
    require_device("u", u, torch.float64)
    nb = ch_work_bytes(c)
    w = _work(nb, u.device, work)
    t = SolverTuning()
    check(lib.sc_autotune_ch(ctypes.byref(c), ctypes.c_void_p(u.data_ptr()), iters, ctypes.c_void_p(w.data_ptr()),
                             nb, ctypes.byref(t), stream_arg(stream)))
    return t.as_dict()


def solver_tile_scale_set(ndim: int, prec: str, log2_scale: int) -> None:
    check(lib.sc_solver_tile_scale_set(ndim, _PREC[prec], log2_scale))


def solver_tile_scale_get(ndim: int, prec: str) -> int:
    v = ctypes.c_int32()
    check(lib.sc_solver_tile_scale_get(ndim, _PREC[prec], ctypes.byref(v)))
    return int(v.value)
