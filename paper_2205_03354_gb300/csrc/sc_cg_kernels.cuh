// The persistent CG kernels: one cooperative launch runs every problem of a
// batch, each on its own CTA group (see cg_run in sc_solver.cuh).
#pragma once
#include "sc_cg_kernels.h"
#include "sc_internal.h"
#include "sc_solver.cuh"

namespace sc {

// DIMS: 1 = 2D problems only, 2 = 3D only, 3 = both (a kernel holding only
// the tile routines it needs uses fewer registers, so more CTAs fit).
// TI = void: both precision classes in one launch, chosen per problem.
template <typename TI, int R, int DIMS>
__global__ void __launch_bounds__(CG_NTHR, DIMS == 3 ? 3 : 4)
    cg_persistent_kernel(const SolveProb *__restrict__ probs, const int *__restrict__ cta_prob,
                         long long budget, unsigned long long slice_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[CG_NTHR / 32];
  __shared__ int flag;
  const int pi = cta_prob[blockIdx.x];
  if (pi < 0) return;
  const SolveProb &P = probs[pi];
  if (P.st->phase == 2) return;
  GroupCtx G{&P, int(blockIdx.x) - P.cta0, 0u, 0u, red, &flag};
  if (DIMS & 1) {
    if (P.ndim == 2) cg_run<TI, 2, R>(G, smem, budget, slice_ns);
  }
  if (DIMS & 2) {
    if (P.ndim == 3) cg_run<TI, 3, R>(G, smem, budget, slice_ns);
  }
}

template <int R, int DIMS>
__global__ void __launch_bounds__(CG_NTHR, 3)
    cg_persistent_both(const SolveProb *__restrict__ probs, const int *__restrict__ cta_prob, long long budget,
                       unsigned long long slice_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[CG_NTHR / 32];
  __shared__ int flag;
  const int pi = cta_prob[blockIdx.x];
  if (pi < 0) return;
  const SolveProb &P = probs[pi];
  if (P.st->phase == 2) return;
  GroupCtx G{&P, int(blockIdx.x) - P.cta0, 0u, 0u, red, &flag};
  if (P.mixed) {
    if ((DIMS & 1) && P.ndim == 2) cg_run<float, 2, R>(G, smem, budget, slice_ns);
    if ((DIMS & 2) && P.ndim == 3) cg_run<float, 3, R>(G, smem, budget, slice_ns);
  } else {
    if ((DIMS & 1) && P.ndim == 2) cg_run<double, 2, R>(G, smem, budget, slice_ns);
    if ((DIMS & 2) && P.ndim == 3) cg_run<double, 3, R>(G, smem, budget, slice_ns);
  }
}

}  // namespace sc
