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

// t = A_int x (pairs), y = scale * B_int t (doubles); both passes stream the
// same boundary mode (periodic, or ghosted with input ring R).  *flag is set
// when an input value cannot be split into normal floats.
int df_composition_enqueue(int ndim, int R, const void *x, void *t, void *y, const int64_t *dims_t,
                           const int64_t *dims_y, int bc, const float *ca, const float *cb, double scale,
                           int *flag, cudaStream_t st, int planes = 0);

}  // namespace sc
