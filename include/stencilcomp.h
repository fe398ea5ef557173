/*
 * stencilcomp.h -- C ABI of the GB300 (sm_103a) stencil-composition library.
 *
 * Method: Mishra, Salac & Knepley, "On the order of accuracy for finite
 * difference approximations of partial differential equations using stencil
 * composition" (arXiv 2205.03354).  Stencils are composed exactly (Sec. 2.2,
 * Eq. C=B(A)); the composed wide stencil is applied matrix-free on 2D/3D
 * structured grids, inside conjugate-gradient solves of the biharmonic plate
 * problem (Sec. 3.3) and of semi-implicit Cahn-Hilliard steps (Sec. 4).
 *
 * Conventions for every entry point:
 *  - All functions return an sc_status (0 = SC_OK).  sc_last_error() gives a
 *    short human-readable reason for the last failure on the calling thread.
 *  - The caller owns every buffer it passes; the library never frees caller
 *    memory.  "_dev" pointers are CUDA device pointers on the current device,
 *    "_host" pointers are host memory (pinned memory gives faster copies).
 *  - Grids are dense row-major arrays with x fastest: a 3D grid of dims
 *    {nx, ny, nz} is indexed [z][y][x], a 2D grid [y][x].  An offset vector is
 *    written (dx, dy, dz).
 *  - "stream" is a cudaStream_t (0 = legacy default stream).  Device work is
 *    enqueued on it; functions that must read results back (solves) block
 *    until their work on that stream has finished.
 *  - The library never calls cudaMalloc on a user path: every device buffer,
 *    including scratch ("work") space, is passed in by the caller, whose size
 *    is given by the matching *_work_bytes query.  The serving loop
 *    sub-allocates from a caller-provided device arena.  One exception: the
 *    preconditioned solver (SC_SOLVER_PCG) runs its dense transform products
 *    through cuBLAS, which allocates its own handle resources and GEMM work
 *    space; the handle (and a non-blocking stream) is created on a thread's
 *    first such solve on a device and kept until that thread exits.
 *  - Invalid arguments return SC_EINVAL before any device work is enqueued.
 *
 * The Python binding (paper_2205_03354_gb300) exposes each function under
 * the same name without the "sc_" prefix.
 */
#ifndef STENCILCOMP_H
#define STENCILCOMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sc_stream_t; /* identical to cudaStream_t */

typedef enum {
  SC_OK = 0,
  SC_EINVAL = 1,      /* bad argument (size, pointer, alignment, mode)       */
  SC_ENOMEM = 2,      /* caller-provided work/arena space too small          */
  SC_ENOTCONV = 3,    /* iteration cap reached before the tolerance          */
  SC_EBREAKDOWN = 4,  /* CG breakdown: p^T A p <= 0 or a non-finite scalar    */
  SC_ETIMEOUT = 5,    /* a bounded device wait gave up (never expected)       */
  SC_EBUSY = 6,       /* server: no admission possible right now              */
  SC_ECUDA = 7,       /* a CUDA runtime call failed                           */
  SC_EOVERFLOW = 8,   /* exact integer arithmetic would overflow              */
  SC_EPENDING = 9     /* server: request still in flight                      */
} sc_status;

typedef enum { SC_F64 = 0, SC_F32 = 1 } sc_dtype;

/* Boundary handling of an apply:
 *  SC_BC_PERIODIC: x and y have dims n; indices wrap around.
 *  SC_BC_GHOSTED:  x has dims n + 2R (an R-wide ghost ring, R = stencil
 *                  radius), y has dims n (the interior).
 *  SC_BC_ZERO:     x and y have dims n; values outside the grid are zero. */
typedef enum { SC_BC_PERIODIC = 0, SC_BC_GHOSTED = 1, SC_BC_ZERO = 2 } sc_bc;

/* 1D stencils printed in the paper (a_i = num_i / den * h^-hpow). */
typedef enum {
  SC_D1_C2 = 0,  /* (f_1 - f_-1)/(2h),           Sec. 2.1.1, Eq. f'stencil      */
  SC_D2_C2 = 1,  /* [1,-2,1]/h^2,                Sec. 2.1.2                    */
  SC_D1_C4 = 2,  /* (8f_1 - f_2 + f_-2 - 8f_-1)/(12h), Sec. 2.2.2, Eq. 4orderf' */
  SC_D2_C4 = 3,  /* [-1,16,-30,16,-1]/(12h^2),   the fourth-order 2nd derivative
                    composed in Sec. 3.2                                       */
  SC_D1_FWD = 4, /* (f_1 - f_0)/h,               Sec. 2.2.1                    */
  SC_D2_FWD = 5  /* (f_2 - 2f_1 + f_0)/h^2,      Sec. 2.2.1                    */
} sc_kind1d;

#define SC_MAX_NDIM 3
#define SC_MAX_PTS 2197 /* 13^3: every 3D stencil of radius <= 6 */
#define SC_MAX_APPLY_RADIUS 4

/* An exact stencil (Def. 2.1): weight at offset off[i] is
 * num[i] / den * h^-hpow.  Offsets unused beyond ndim are 0.  Points are kept
 * sorted lexicographically by (dx, dy, dz) with no zero weights, and den > 0
 * with gcd(den, num...) = 1.  Plain value type: no library-owned memory. */
typedef struct {
  int32_t ndim;
  int32_t npts;
  int32_t hpow;
  int32_t radius; /* max |offset component| */
  int64_t den;
  int32_t off[SC_MAX_PTS][SC_MAX_NDIM];
  int64_t num[SC_MAX_PTS];
} sc_stencil;

/* Library version, e.g. 100 for 1.0.0. */
int32_t sc_version(void);
/* Reason for the last non-OK status returned on this thread ("" if none). */
const char *sc_last_error(void);

/* ---- Exact stencil algebra (host only, no device work) ------------------ */

/* One of the 1D stencils above (ndim = 1). */
int sc_stencil_1d(int32_t kind, sc_stencil *out);

/* A 1D stencil acting along `axis` (0 = x) of an ndim-dimensional lattice,
 * the identity on the other axes (Sec. 2.3). */
int sc_stencil_embed(const sc_stencil *s1d, int32_t ndim, int32_t axis, sc_stencil *out);

/* a + b for stencils of equal ndim and hpow (the Taylor series of source
 * points form a vector space, Sec. 2.1).  SC_EOVERFLOW on int64 overflow. */
int sc_stencil_add(const sc_stencil *a, const sc_stencil *b, sc_stencil *out);

/* Sum over axes of the 1D second-derivative stencil of `order` (2 or 4):
 * the Laplacian the paper composes with itself (Sec. 3.3). */
int sc_laplacian(int32_t ndim, int32_t order, sc_stencil *out);

/* Stencil composition C = B(A), B = outer, A = inner (Sec. 2.2, Eq. C=B(A)):
 * offsets add, weights multiply, c_k = sum_{u_i+v_j=k} a_i b_j, and the
 * h-powers add.  Exact in int64; SC_EOVERFLOW if any intermediate would
 * overflow, SC_EINVAL if the result exceeds SC_MAX_PTS points or the
 * dimensions differ.  Composition is only meaningful when the same inner
 * stencil is used at every outer point (Sec. 5, closing caveat), which holds
 * by construction here.  `out` may alias neither input. */
int sc_compose_stencil(const sc_stencil *outer, const sc_stencil *inner, sc_stencil *out);

/* Floating-point weights of s for lattice spacing h = h_num / h_den
 * (h_num, h_den > 0): each weight is the exact rational num_i/den *
 * (h_den/h_num)^hpow rounded ONCE to the nearest double (dtype SC_F64) or
 * float (SC_F32), ties to even.  host_out receives npts values in the order
 * of s->off.  SC_EOVERFLOW if the exact value needs more than 127 bits. */
int sc_stencil_weights(const sc_stencil *s, int64_t h_num, int64_t h_den, int32_t dtype,
                       void *host_out);

/* ---- Matrix-free apply (device) ------------------------------------------ */

/* y = A x with the composed stencil s (flat evaluation, y_i = sum_k w_k
 * x_{i+k}, weights from sc_stencil_weights with h = h_num/h_den), on a grid
 * of interior dims {nx, ny[, nz]} = dims[0..ndim-1].  s->ndim must be 2 or 3
 * and s->radius <= SC_MAX_APPLY_RADIUS.  x and y are device arrays of `dtype`
 * (layout per `bc` above) and must not overlap.  Asynchronous on `stream`. */
int sc_apply_composed(const sc_stencil *s, int32_t dtype, int32_t bc, const int64_t *dims,
                      int64_t h_num, int64_t h_den, const void *x_dev, void *y_dev,
                      sc_stream_t stream);

/* The composed operator C = B(A) evaluated in nested form, y = B(A x) (the
 * double sum of Eq. C=B(A)), from the two factors outer = B and inner = A
 * instead of the composed weights: A is applied on the grid extended by
 * B's radius into a temporary in work_dev, then B.  Same operator and
 * boundary semantics as sc_apply_composed(compose(B, A)) up to rounding
 * (the two factors' weights are rounded separately); fewer arithmetic
 * operations when both factors are sparse (2 x 13 instead of 73 FMAs per
 * point for the 3D fourth-order Lap o Lap), at the price of the temporary's
 * traffic.  For SC_BC_GHOSTED, x carries a ring of width
 * outer->radius + inner->radius.  work_bytes >=
 * sc_apply_composition_work_bytes(...).
 *
 * arith = SC_ARITH_NATIVE evaluates in dtype.  arith = SC_ARITH_PAIR (dtype
 * SC_F64 only) evaluates Laplacian factors -- symmetric star stencils with
 * one integer numerator per distance, radius 1 or 2 -- in pairs of FP32
 * numbers with error-free transformations (GB300 has 64x more FP32 than
 * FP64 FMA throughput): the doubles are split exactly with integer bit
 * operations and the result is rebuilt exactly; the error is a few units of
 * 2^-48 of sum |w x|, inside the FP64 apply tolerance.  Nonzero inputs with
 * magnitude outside [2^-74, 2^100] set a device flag and the native FP64
 * passes recompute the result (they are always enqueued and return at once
 * when the flag is clear).  Other factor shapes fall back to SC_ARITH_NATIVE. */
typedef enum { SC_ARITH_NATIVE = 0, SC_ARITH_PAIR = 1 } sc_arith;
size_t sc_apply_composition_work_bytes(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype,
                                        int32_t bc, const int64_t *dims);
int sc_apply_composition(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                         const int64_t *dims, int64_t h_num, int64_t h_den, const void *x_dev, void *y_dev,
                         void *work_dev, size_t work_bytes, int32_t arith, sc_stream_t stream);

/* Same as sc_apply_composed, with x and y in HOST memory: copies x to the
 * device work space, applies, copies y back and waits for the stream.
 * work_bytes >= sc_apply_host_work_bytes(...). */
size_t sc_apply_host_work_bytes(const sc_stencil *s, int32_t dtype, int32_t bc,
                                const int64_t *dims);
int sc_apply_composed_host(const sc_stencil *s, int32_t dtype, int32_t bc, const int64_t *dims,
                           int64_t h_num, int64_t h_den, const void *x_host, void *y_host,
                           void *work_dev, size_t work_bytes, sc_stream_t stream);



/* y = outer(m * inner(x)) on a periodic grid: a composition with a pointwise
 * coefficient between its factors -- the variable-mobility operator
 * d/dx(M d/dx(d2/dx2 f)) of Sec. 2.2.3 (inner = d/dx composed with d2/dx2,
 * m = M at the grid points, outer = d/dx), which a fixed composed stencil
 * cannot express.  With constant m it equals m times sc_apply_composed of
 * compose(outer, inner).  x, m, y: n^ndim values of dtype (row-major, x
 * fastest); work_bytes >= n^ndim values (the scaled intermediate).  x, y, m
 * and work must not overlap (x may equal m).  Asynchronous on `stream`. */
int sc_apply_varcoef(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, const int64_t *dims,
                     int64_t h_num, int64_t h_den, const void *m_dev, const void *x_dev, void *y_dev,
                     void *work_dev, size_t work_bytes, sc_stream_t stream);

/* ---- Autotuner -------------------------------------------------------------- */

typedef enum {
  SC_EVAL_FLAT = 0,   /* sc_apply_composed on compose(outer, inner)           */
  SC_EVAL_NESTED = 1, /* sc_apply_composition, native arithmetic               */
  SC_EVAL_PAIR = 2,   /* sc_apply_composition, FP32-pair arithmetic (FP64)     */
  SC_EVAL_FUSED = 3   /* nested B(A x) in one pass, the intermediate kept on
                         chip (FP32; both factors sums of 1D stencils along the
                         axes, equal radius 1 or 2; periodic grids of at least
                         72 x 24 x 8 in 3D and 128 x 8 in 2D); other operators
                         run SC_EVAL_NESTED                                    */
} sc_eval;

typedef struct {
  int32_t eval;    /* sc_eval                                                  */
  int32_t planes;  /* output planes per CTA (halo-blocking depth; 0 = the
                      occupancy model)                                         */
  double ms;       /* measured time of one apply                               */
} sc_tune_choice;

/* Times every evaluation schedule of the operator compose(outer, inner) --
 * flat composed weights, nested native, fused nested (FP32, where it
 * applies), nested FP32-pair (FP64 only) --
 * crossed with several halo-blocking depths (planes per CTA: the occupancy
 * model, 16, 32, 64, 128) on the caller's x/y/work and stream (one warm-up
 * and the median of three runs each; y is overwritten), caches the fastest
 * for this (shape, dtype, boundary, factors) in the process and returns it.
 * Blocks until the timing runs finish.  work_bytes >=
 * sc_apply_composition_work_bytes(outer, inner, ...). */
int sc_autotune_apply(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                      const int64_t *dims, int64_t h_num, int64_t h_den, const void *x_dev, void *y_dev,
                      void *work_dev, size_t work_bytes, sc_tune_choice *out, sc_stream_t stream);
/* y = compose(outer, inner) x with the cached choice for this shape (the flat
 * composed apply with the occupancy model when untuned).  Asynchronous. */
int sc_apply_tuned(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                   const int64_t *dims, int64_t h_num, int64_t h_den, const void *x_dev, void *y_dev,
                   void *work_dev, size_t work_bytes, sc_stream_t stream);
/* The cached choice for a shape (SC_EINVAL if not tuned). */
int sc_tuned_choice(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                    const int64_t *dims, sc_tune_choice *out);
/* The tuned apply (as sc_apply_tuned) with x and y in HOST memory, for data
 * that lives on the host.  The grid is cut along its slowest axis (z in 3D,
 * y in 2D) into about eight slabs of at least 4 (R_outer + R_inner) planes;
 * for each slab the input planes it reads (its planes and that halo) are
 * copied into the device work space on a library copy-in stream (the halo
 * planes shared with the previous slab device to device), the in-plane
 * boundary ring is filled on the device, the tuned schedule of the WHOLE
 * grid's shape runs on the slab (as a ghosted grid) on `stream`, and the
 * slab's output planes are copied back on a library copy-out stream; two
 * buffer sets alternate, so slab k + 1's copy-in, slab k's apply and slab
 * k - 1's copy-out overlap.  Grids shorter than two slabs are copied, applied
 * and copied back whole.  The result equals sc_apply_tuned's on the same
 * grid bit for bit, except for a pair-arithmetic schedule with radius-1
 * factors on a periodic grid, whose slabs run the native FP64 nested passes
 * (within the FP64 apply tolerance).  Asynchronous: `stream` is made to wait
 * for the last copy-out; synchronise it before reading y_host.  Consecutive
 * calls on one device overlap (a call's first copy-in waits only until the
 * previous call's applies have read their inputs).  x_host and y_host must
 * not overlap (SC_EINVAL); pinned host buffers let the copies run at link
 * speed.  work_bytes >= sc_apply_tuned_host_work_bytes(...) (about two slabs
 * of input and output plus the schedule's work space for one slab; the
 * whole-grid size for short grids); one work space may serve consecutive
 * calls.  Calls from several host threads are serialised by the library. */
size_t sc_apply_tuned_host_work_bytes(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype,
                                      int32_t bc, const int64_t *dims);
int sc_apply_tuned_host(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                        const int64_t *dims, int64_t h_num, int64_t h_den, const void *x_host, void *y_host,
                        void *work_dev, size_t work_bytes, sc_stream_t stream);
/* Records a choice for a shape in the process cache without timing, e.g. one
 * saved from an earlier sc_autotune_apply run, so that sc_apply_tuned reuses
 * it (a later sc_autotune_apply for the shape replaces it).  eval is an
 * sc_eval; planes in [0, 4096]; SC_EVAL_PAIR on an operator the pair path
 * does not cover runs nested native arithmetic.  in->ms is stored as given.
 * SC_EINVAL for a bad operator, shape or choice; no device work. */
int sc_tune_set(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                const int64_t *dims, const sc_tune_choice *in);

/* ---- Solvers (device) ------------------------------------------------------ */

typedef enum {
  SC_PREC_F64 = 0,   /* FP64 CG throughout                                     */
  SC_PREC_MIXED = 1, /* FP32 stencil applies and vector updates with FP32
                        accumulation; FP64 solution, right-hand side and true
                        residual refreshed by reliable updates                 */
  SC_PREC_AUTO = 2   /* MIXED when the closed-form condition number estimate
                        kappa satisfies kappa * 2^-24 <= 1e-2, else F64        */
} sc_prec;

typedef enum {
  SC_SOLVER_PERSISTENT = 0, /* one cooperative launch runs the whole CG loop  */
  SC_SOLVER_PLAIN = 1,      /* one kernel per CG operation, host-driven loop  */
  SC_SOLVER_PCG = 2         /* plate problems only: FP64 CG preconditioned by
                               the inverse of L_D^2 (L_D the Dirichlet
                               Laplacian) applied with sine transforms (cuBLAS
                               GEMMs, FP32 accuracy; the lowest 16^d modes in
                               FP64); tens of iterations where plain CG needs
                               O(N^2) (large grids).  The loop's scalars stay on
                               the device; an iteration is replayed from a CUDA
                               graph on the calling thread's own stream        */
} sc_solver_kind;

typedef struct {
  int64_t iters;   /* inner CG iterations                                      */
  int64_t outer;   /* FP64 residual refreshes (mixed precision)                */
  double rel_res;  /* final TRUE relative residual ||b - A x||_2 / ||b||_2,
                      recomputed in FP64 after the solve                       */
  int32_t status;  /* SC_OK, SC_ENOTCONV, SC_EBREAKDOWN or SC_ETIMEOUT          */
  int32_t prec;    /* precision actually used (SC_PREC_F64 / SC_PREC_MIXED)     */
  double seconds;  /* wall time of the call                                    */
} sc_solve_info;

/* The biharmonic plate problem of Sec. 3.3: Lap(Lap u) = g on the unit square
 * (ndim 2) or cube (ndim 3) with N = n[a] interior nodes per axis,
 * h = 1/(N+1) (all n[a] equal), node i at x = i h.  The operator is the
 * composed Lap o Lap of the given Laplacian order (2: 13/25 points; the
 * persistent solver supports order 2).  Boundary data: the R-wide ghost ring
 * (R = 2 for order 2) of ghost_dev, an (N+2R)^ndim array laid out like the
 * interior arrays, holds the exact solution (only the ring is read); its
 * contribution moves to the right-hand side, b = g - A(ring), and the
 * interior system is solved by CG from x = 0 to ||b - A x|| <= rtol ||b||.
 * f_dev: g on the interior (N^ndim doubles); x_dev: solution (N^ndim doubles,
 * overwritten). */
typedef struct {
  int32_t ndim;
  int32_t order;
  int64_t n[3];
  int32_t prec;   /* sc_prec */
  int32_t solver; /* sc_solver_kind */
  double rtol;
  int64_t maxit;  /* cap on inner iterations (SC_ENOTCONV when reached) */
  const double *f_dev;
  const double *ghost_dev;
  double *x_dev;
} sc_bvp;

/* Device work space needed by sc_solve_biharmonic / ..._batch. */
size_t sc_bvp_work_bytes(const sc_bvp *p);
int sc_solve_biharmonic(const sc_bvp *p, void *work_dev, size_t work_bytes, sc_solve_info *info,
                        sc_stream_t stream);

/* `count` independent plate problems of uneven sizes and dimensions solved
 * together: one persistent launch per precision class, each problem on its
 * own group of CTAs (the batched persistent solver).  Results are
 * bit-identical to solving each problem alone with the same solver and
 * precision.  infos[count] receives per-problem results. */
size_t sc_bvp_batch_work_bytes(const sc_bvp *probs, int32_t count);
int sc_solve_biharmonic_batch(const sc_bvp *probs, int32_t count, void *work_dev, size_t work_bytes,
                              sc_solve_info *infos, sc_stream_t stream);

/* One semi-implicit Cahn-Hilliard step (Sec. 4.1, Eq. cahn, linear fourth-
 * order part implicit, nonlinear part explicit) on a periodic n^ndim grid of
 * spacing h = h_num/h_den, for `batch` independent fields stored back to back:
 *   (I + dt M kappa Lap_h o Lap_h) u_new = u + dt M Lap_h f'(u),
 * Lap_h the Laplacian of the given order (2), f'(u) = u^3 - u (chem 0) or
 * 2 rho (u - ca)(u - cb)(2u - ca - cb) (chem 1, the double well of Sec. 4.1).
 * CG starts from u; after it the mean of u_new is set to that of the
 * right-hand side (the periodic operator conserves the mean exactly, so
 * this removes only rounding drift).  u_dev is updated in place;
 * infos[batch] receives per-field results. */
typedef struct {
  int32_t ndim;
  int32_t order;
  int64_t n[3];
  int32_t batch;
  int64_t h_num, h_den;
  double dt, M, kappa;
  int32_t chem;
  double rho, ca, cb;
  int32_t prec;
  int32_t solver;
  double rtol;
  int64_t maxit;
} sc_ch;

size_t sc_ch_work_bytes(const sc_ch *p);
int sc_ch_step(const sc_ch *p, double *u_dev, void *work_dev, size_t work_bytes, sc_solve_info *infos,
               sc_stream_t stream);

/* One step of the semi-implicit backward differentiation scheme of order
 * 1, 2 or 3 (SBDF1-3) for the same splitting: with history u^n, u^(n-1),
 * u^(n-2) and N(u) = M Lap f'(u),
 *   (I + g dt M kappa Lap o Lap) u^(n+1) = sum_j al_j u^(n-j) + g dt M Lap sum_j b_j f'(u^(n-j)),
 * g = 1, 2/3, 6/11; al = (1), (4/3, -1/3), (18/11, -9/11, 2/11); b = (1), (2, -1),
 * (3, -3, 1).  The paper (Sec. 4.3) uses IMEX schemes of orders one to three
 * without naming them; SBDF is the standard family of that kind.  u_dev: u^n
 * in, u^(n+1) out (batch x n^ndim).  hist_dev (order >= 2): order - 1 slices
 * of batch x n^ndim values, slice 0 = u^(n-1), slice 1 = u^(n-2); on return
 * they hold u^n and u^(n-1), the history of the next step.  The caller
 * starts a run with lower orders (or a history of its own).  Same work space
 * and solver options as sc_ch_step; order 1 is sc_ch_step. */
int sc_ch_step_sbdf(const sc_ch *p, int32_t order, double *u_dev, double *hist_dev, void *work_dev,
                    size_t work_bytes, sc_solve_info *info, sc_stream_t stream);

/* nsteps Cahn-Hilliard steps of every field (the same step as sc_ch_step,
 * persistent solver), set up once.  With use_graph != 0 one whole step --
 * right-hand-side kernels, solver-state reset, the cooperative persistent
 * launch that solves all `batch` fields, and a kernel that records the
 * step's per-field results in device memory -- is captured once into a CUDA
 * graph and replayed, with no host synchronisation between steps.
 * infos[nsteps * batch] receives per-step, per-field results (step-major).
 * work_bytes >= sc_ch_run_work_bytes(p, nsteps).  Blocking. */
size_t sc_ch_run_work_bytes(const sc_ch *p, int64_t nsteps);
int sc_ch_run(const sc_ch *p, double *u_dev, int64_t nsteps, int32_t use_graph, void *work_dev,
              size_t work_bytes, sc_solve_info *infos, sc_stream_t stream);

/* Mass sum(u) and free energy F(u) = h^d sum[f(u) + kappa/2 sum_a (D+_a u)^2]
 * (forward differences, periodic) of each field, written to host arrays
 * mass[batch], energy[batch].  Deterministic reduction order. */
int sc_ch_stats(const sc_ch *p, const double *u_dev, double *mass_host, double *energy_host,
                void *work_dev, size_t work_bytes, sc_stream_t stream);


/* Same statistics as sc_ch_stats without any work buffer, for callers that
 * cannot allocate device memory (a host program whose own pool allocator
 * owns all device memory, or a latency-critical loop where cudaMalloc, which
 * may synchronise the device, is not allowed).  The paper has no counterpart:
 * this is a deployment convenience.  The partial sums live in a fixed array
 * of 2 * 4096 + 8 doubles inside the library, resident on each GPU that uses
 * it until the process exits; fields of more than 2^24 grid points are
 * rejected with SC_EINVAL.  The first call on a device looks the array's
 * device address up (cudaGetSymbolAddress) with that device current and
 * should happen outside any stream capture; the address is kept for later
 * calls on that device.  All calls share the array: calls that may overlap
 * on the GPU (other streams or host threads) race and must be serialised by
 * the caller.  Allocates nothing. */
int sc_ch_stats_noalloc(const sc_ch *p, const double *u_dev, double *mass_host, double *energy_host,
                        sc_stream_t stream);

/* Drops the device addresses sc_ch_stats_noalloc kept.  A process that calls
 * cudaDeviceReset on a device must call this afterwards, before the next
 * sc_ch_stats_noalloc on that device: the reset ends the context the kept
 * address belonged to.  Host-only; no device call. */
void sc_noalloc_forget(void);


/* ---- Autotuner of the persistent solver ------------------------------------ */

/* The persistent engine cuts every problem into tiles of about a target
 * number of points (FP32: 1024 in 2D, 2048 in 3D; FP64 4x fewer), which sets
 * both the tile count per problem (the work a CTA group shares) and the
 * planes a tile streams (its halo-blocking depth).  The target is scaled by
 * 2^log2_scale, log2_scale in -2..2, separately for each (dimensionality,
 * precision class); default 0.  sc_autotune_solver times `iters` inner
 * iterations of the caller's batch (plate problems; their x is overwritten)
 * at every scale on `stream`, keeps the fastest for the classes present in
 * the batch (process-wide, later solves and server slices use it) and
 * reports the times.  Synchronous.  A problem's results depend on the scale
 * it was laid out with (the reduction groups follow the tiles) and on nothing
 * else: the same scale gives the same bits.  work_bytes as for
 * sc_solve_biharmonic_batch, which already covers every scale. */
typedef struct {
  int32_t log2_scale;  /* the chosen scale                                 */
  float ms[5];         /* time of the timed iterations at scales -2 .. 2   */
} sc_solver_tuning;
int sc_autotune_solver(const sc_bvp *probs, int32_t count, int32_t iters, void *work_dev, size_t work_bytes,
                       sc_solver_tuning *out, sc_stream_t stream);
/* The same for a batch of Cahn-Hilliard steps (u is advanced partly). */
int sc_autotune_ch(const sc_ch *p, double *u_dev, int32_t iters, void *work_dev, size_t work_bytes,
                   sc_solver_tuning *out, sc_stream_t stream);
/* Set / read the scale of one class (prec: SC_PREC_F64 or SC_PREC_MIXED). */
int sc_solver_tile_scale_set(int32_t ndim, int32_t prec, int32_t log2_scale);
int sc_solver_tile_scale_get(int32_t ndim, int32_t prec, int32_t *log2_scale);

/* Failure-detection self-test of the solver's bounded group barrier: runs
 * the barrier for a group of two CTAs with only one launched, so the release
 * never comes, once with each reduction protocol (every CTA reading the
 * partials; the last arriver publishing the result); each wait gives up after
 * spin_limit polls (1..2^24, ~100 ns each) and *status_out receives
 * SC_ETIMEOUT when both did.  Nothing traps or faults; the context stays
 * usable.  work_bytes >= 4096. */
int sc_selftest_barrier_timeout(void *work_dev, size_t work_bytes, int64_t spin_limit, int32_t *status_out,
                                sc_stream_t stream);

/* ---- Serving loop: continuous batching of plate solves and CH steps -------- */

/* A server owns one scheduler thread on the device that is current when it is
 * created.  Requests -- plate problems (Sec. 3.3) and semi-implicit
 * Cahn-Hilliard steps (Sec. 4.1, Eq. cahn) of any size -- are queued by
 * sc_submit and admitted, in arrival order with skipping of requests that do
 * not fit yet, whenever the caller-provided device arena has room for their
 * fields and Krylov state and fewer than max_active requests are resident.
 * Resident requests advance together in persistent launches of at most
 * slice_ms milliseconds each (every request on its own group of CTAs);
 * between slices finished requests are retired (their result copied to the
 * caller's host buffer, their memory freed) and newly admitted ones join.
 * Plate problems routed to the preconditioned solver (see sc_request.solver)
 * are admitted from a queue of their own, by the same arena, and solved one at
 * a time by a second scheduler thread on its own stream.  A request's result
 * does not depend on what else is in flight: it is bit-identical to
 * sc_solve_biharmonic (with the same solver and precision) / sc_ch_step
 * (batch 1).  The server never allocates device memory: everything lives in
 * the arena. */
typedef struct {
  void *arena_dev;     /* device memory owned by the caller                   */
  size_t arena_bytes;  /* its size: the admission budget                     */
  int32_t max_active;  /* resident requests at most (1..4096)                */
  double slice_ms;     /* length of one persistent launch (> 0)              */
  int64_t pcg_min_points; /* plate requests with solver -1 go to the
                          preconditioned solver from this many grid points
                          on (0: 65536)                                     */
  int32_t fail_slice;  /* failure-detection test hook, normally 0: with k > 0
                          the scheduler treats its k-th time slice as failed
                          (as if the launch had returned an error; nothing is
                          launched wrongly and the GPU is not involved), so
                          that the recovery path can be tested             */
} sc_server_cfg;

typedef enum {
  SC_REQ_PLATE = 0,  /* plate problem: f_host, ghost_host -> x_host          */
  SC_REQ_CH = 1      /* one Cahn-Hilliard step of u_host -> x_host           */
} sc_request_kind;

/* One request with HOST buffers, read at admission (f_host / ghost_host /
 * u_host) and written when it completes (x_host); all must stay valid until
 * sc_poll reports it done.  Plate problems: the fields of sc_bvp.  Cahn-
 * Hilliard steps: the fields of sc_ch with batch 1, u_host the field at step
 * n (n^ndim values) and x_host receiving the field at step n + 1. */
typedef struct {
  int32_t kind;        /* sc_request_kind                                   */
  int32_t solver;      /* plate problems: SC_SOLVER_PERSISTENT (batched with
                          the other resident requests), SC_SOLVER_PCG (the
                          preconditioned solver, one request at a time on a
                          second scheduler thread, concurrently with the
                          batched slices), or -1: SC_SOLVER_PCG for grids of at
                          least sc_server_cfg.pcg_min_points points, else
                          batched.  Cahn-Hilliard steps are always batched.   */
  int32_t ndim;
  int32_t order;
  int64_t n[3];
  int32_t prec;
  double rtol;
  int64_t maxit;
  const double *f_host;      /* plate                                       */
  const double *ghost_host;  /* plate                                       */
  const double *u_host;      /* Cahn-Hilliard                               */
  int64_t h_num, h_den;      /* Cahn-Hilliard: spacing                      */
  double dt, M, kappa;       /* Cahn-Hilliard                               */
  int32_t chem;              /* Cahn-Hilliard: 0 cubic, 1 double well       */
  double rho, ca, cb;        /* Cahn-Hilliard: double well                  */
  double *x_host;            /* result                                      */
} sc_request;

typedef struct {
  int32_t status;    /* solve status (SC_OK, SC_ENOTCONV, ...)              */
  int32_t prec;      /* precision used                                      */
  int64_t iters;
  double rel_res;    /* true relative residual                              */
  double queue_s;    /* submit -> admission                                 */
  double latency_s;  /* submit -> result copied to x_host                   */
} sc_result;

typedef struct sc_server sc_server;

/* Device bytes a request occupies while resident (fields + Krylov state),
 * for the default routing of solver -1 (65536 points). */
size_t sc_request_bytes(const sc_request *req);
int sc_server_create(const sc_server_cfg *cfg, sc_server **out);
/* Stops the scheduler; requests still queued or resident are abandoned. */
int sc_server_destroy(sc_server *srv);
/* Queues a request (never blocks).  SC_EINVAL for a malformed request,
 * SC_ENOMEM if it could never fit in the arena; once a time slice has
 * failed, every later submission returns that slice's error. */
int sc_submit(sc_server *srv, const sc_request *req, uint64_t *ticket);
/* SC_EPENDING while the request is queued or resident; SC_OK once it is
 * done (x_host written, *out filled; the ticket is then released);
 * SC_EINVAL for an unknown ticket.  Requests resident when a slice failed
 * are done with that error as their status (their arena space is freed). */
int sc_poll(sc_server *srv, uint64_t ticket, sc_result *out);
/* Waits until nothing is queued or resident, at most timeout_s seconds
 * (SC_ETIMEOUT otherwise). */
int sc_server_drain(sc_server *srv, double timeout_s);
/* Snapshot of the scheduler: the error of the first failed slice (SC_OK if
 * none), free arena bytes (of sc_server's usable arena), requests resident
 * and queued.  Host-only. */
int sc_server_status(sc_server *srv, int32_t *worker_error, size_t *free_bytes, size_t *arena_bytes,
                     int32_t *active, int32_t *pending);

#ifdef __cplusplus
}
#endif
#endif /* STENCILCOMP_H */
