// Host-side description of one linear solve, shared by the solver and the
// serving translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

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
};

double kappa_estimate(const ProbSpec &sp, double h);
int max_group_ctas(bool mixed);

}  // namespace sc
