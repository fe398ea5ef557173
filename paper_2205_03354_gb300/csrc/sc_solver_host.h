// Host-side description of one linear solve, shared by the solver and the
// serving translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/stencilcomp.h"

namespace sc {

struct SolveProb;  // sc_solver.cuh

struct ProbSpec {
  int ndim, order, R;
  int64_t n[3];
  int bc;                 // SC_BC_ZERO (plate interior) or SC_BC_PERIODIC (Cahn-Hilliard)
  int64_t h_num, h_den;   // lattice spacing
  double a, b;            // operator a I + b (Lap o Lap)
  double rtol;
  long long maxit;
  double *x;              // solution / initial guess (device, FP64)
  int mean_fix, mixed, solver;
};

struct ProbAux {
  int nbox;
  double *scratch;  // set-up scratch (padded grid)
  double *ones;     // vector of ones (plain mean fix)
  // preconditioned solver (SC_SOLVER_PCG) only
  double *z = nullptr;             // preconditioned residual (FP64)
  float *u0 = nullptr, *u1 = nullptr;  // FP32 transform buffers
  float *S = nullptr;              // DST-I matrix, N x N
  double *lam1 = nullptr;          // 1D Dirichlet eigenvalues, N
  double *part = nullptr, *out = nullptr;  // dot-product partials; results (8) and loop scalars
  // the lowest K0^ndim modes in FP64: their rows of the transform (K0 x N
  // and its transpose), transform work space and the FP64 result
  double *Sl = nullptr, *SlT = nullptr, *wa = nullptr, *wb = nullptr, *wc = nullptr, *zl = nullptr;
};

// Low-mode block edge of the preconditioner (modes with every index < K0
// are transformed in FP64).
int pcg_low_modes(int ndim, long long N);

// Preconditioned plate solve (sc_pcg.cu): res[0] iterations, res[1] true
// relative residual, res[2] status.  Synchronous.
int run_pcg(const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t st, double *res);
// Dot-product partial slots the preconditioned solver needs for n points.
long long pcg_parts(long long n);

// Sub-allocates 256-byte aligned pieces of a caller buffer (base == nullptr:
// sizing only).
struct Carver {
  char *base;
  size_t off = 0, cap;
  Carver(void *b, size_t c) : base(static_cast<char *>(b)), cap(c) {}
  void *take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    void *p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
};

double kappa_estimate(const ProbSpec &sp, double h);
// Resident persistent-CG CTAs on the device (dims: bit 0 2D, bit 1 3D).
int max_group_ctas(bool mixed, int dims = 3);
int bvp_spec(const sc_bvp *b, ProbSpec &sp);
// Work-space layout of one problem (sizes only when cv.base == nullptr).
void layout(const ProbSpec &sp, Carver &cv, SolveProb &P, ProbAux &aux);
// Weights, initial state and alignment flags of one problem (synchronous).
int upload_prob(const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t st);
// Right-hand side b = g - A(ring) and x = 0 of a plate problem (enqueued).
int setup_bvp(const sc_bvp *bp, const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t st);
// Right-hand side u + dt M Lap f'(u) of a Cahn-Hilliard step; x (= u, the
// initial guess) in place (enqueued).
int setup_ch(const sc_ch *cp, const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t st);
// Validated spec of a one-field Cahn-Hilliard step on the device field u.
int ch_single_spec(const sc_ch *c, double *u, ProbSpec &sp);
struct SolveState;
// Copies the solver states of the n problems described at dprobs to host
// (one gather kernel into dout, one copy; synchronous).
int gather_states(const SolveProb *dprobs, int n, SolveState *dout, SolveState *host, cudaStream_t st);
// Runs the persistent engine over `hp` (both precision classes) for at most
// `budget` iterations or `slice_ms` milliseconds per launch (0: no limit);
// synchronous.  dprobs/dmap/dbars: device descriptor space.
int run_persistent(std::vector<SolveProb> &hp, SolveProb *dprobs, int *dmap, unsigned *dbars,
                   cudaStream_t st, long long budget, double slice_ms);

}  // namespace sc
