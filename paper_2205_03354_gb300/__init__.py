"""Python binding of libstencilcomp, the GB300 (sm_103a) stencil-composition
library (Mishra, Salac & Knepley, arXiv 2205.03354).

Argument marshalling only: every function forwards to the C ABI declared in
include/stencilcomp.h under the same name with an ``sc_`` prefix.  Device
arrays are torch CUDA tensors (PyTorch provides device memory and streams);
all computation runs in the library's CUDA kernels.  There is no CPU
fallback: if the compiled library is missing, import fails loudly.
"""
from __future__ import annotations

from ._lib_loader import lib, LIB_PATH, ScError, check  # noqa: F401
from .stencil import (Stencil, stencil_1d, stencil_embed, stencil_add, laplacian,  # noqa: F401
                      compose_stencil, stencil_weights, D1_C2, D2_C2, D1_C4, D2_C4, D1_FWD, D2_FWD)
from .ops import (apply_composed, apply_composed_host, apply_host_work_bytes,  # noqa: F401
                  apply_composition, apply_composition_work_bytes, autotune_apply, apply_tuned, tune_set,
                  apply_tuned_host, apply_tuned_host_work_bytes, apply_varcoef,
                  F64, F32, BC_PERIODIC, BC_GHOSTED, BC_ZERO)
from .solvers import (solve_biharmonic, solve_biharmonic_batch, make_bvp, bvp_work_bytes,  # noqa: F401
                      make_ch, ch_step, ch_step_sbdf, ch_run, ch_stats, ch_work_bytes, SolveInfo, Bvp, Ch,
                      autotune_solver, autotune_ch, solver_tile_scale_set, solver_tile_scale_get)
from .server import Server, make_ch_request, make_request, request_bytes  # noqa: F401
