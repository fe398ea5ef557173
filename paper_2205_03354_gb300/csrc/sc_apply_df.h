// Pair-arithmetic (two FP32) evaluation of FP64 Laplacian compositions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/stencilcomp.h"

namespace sc {

// True when s is a symmetric star stencil with the same integer weight at
// every point of a given distance (a Laplacian), radius 1 or 2; returns its
// centre, distance-1 and distance-2 numerators.
bool star_int_form(const sc_stencil *s, float *c0, float *c1, float *c2);

// True when the packed pair passes cover this case: dims_y[0] even, 16-byte
// aligned x / t / y, periodic (R 1 or 2) or ghosted (R 2) boundary mode, and
// a scale whose exponent lies in [-800, 800].
bool df_supported(int ndim, int R, const int64_t *dims_y, int bc, double scale, const void *x, const void *t,
                  const void *y);

// t = A_int x (pairs, folded rows), y = scale * B_int t (doubles); both passes stream the
// same boundary mode (periodic, or ghosted with input ring R).  *flag is set
// when an input value cannot be split into normal floats.
int df_composition_enqueue(int ndim, int R, const void *x, void *t, void *y, const int64_t *dims_t,
                           const int64_t *dims_y, int bc, const float *ca, const float *cb, double scale,
                           int *flag, cudaStream_t st, int planes = 0);

}  // namespace sc
