"""CPU oracle for the stencil-composition hot path (test infrastructure only).

This package is the independent, slow, obviously-correct reference that the
CUDA library is checked against.  It is *test infrastructure*: only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import it.  The product path (the C-ABI
library and its Python binding) never imports, calls or links anything here,
and nothing here imports the product package.

Modules
-------
stencil    exact-rational stencils, composition (Sec. 2.2, Eq. C=B(A)), Taylor
           vectors (Eq. CompactNotation), validity rules (Def. 2.2),
           higher-dimensional embedding (Sec. 2.3), correctly rounded weights.
apply      matrix-free FP64 apply of a stencil on a structured grid, plus a
           dense-matrix builder for tiny grids (brute-force pins).
cg         textbook conjugate gradients in FP64.
bvp        the biharmonic boundary-value problem of Sec. 3.3.
ch         one semi-implicit Cahn-Hilliard step (Sec. 4, Eq. cahn), mass and
           free energy, and the DFT closed form of a periodic step.
stability  von Neumann growth factors of Sec. 2.2.3 and Appendix B.

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against values the paper prints, closed forms,
invariants or brute force.  No function here is "parity unpinned".
"""
