// Host-side interface of the apply dispatch, shared by the solver and
// serving translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/stencilcomp.h"

namespace sc {

struct ApplyReq {
  const sc_stencil *s;
  int dtype;
  int bc;
  const int64_t *dims;
  int64_t h_num, h_den;
  const void *x;
  void *y;
  const int *guard = nullptr;  // if set: the kernel only works when *guard != 0
  int planes = 0;              // output planes per CTA (0: occupancy model)
};

size_t composition_work_bytes(const sc_stencil *B, const sc_stencil *A, int dtype, int bc, const int64_t *dims);
int composition_enqueue(const sc_stencil *B, const sc_stencil *A, int dtype, int bc, const int64_t *dims,
                        int64_t h_num, int64_t h_den, const void *x, void *y, void *work, cudaStream_t st,
                        int arith, int planes = 0);

// Fused single-pass nested apply (FP32 axis-stencil factors, sc_fused.cu).
bool fused_supported(const sc_stencil *B, const sc_stencil *A, int dtype, int bc, const int64_t *dims);
int fused_enqueue(const sc_stencil *B, const sc_stencil *A, int dtype, int bc, const int64_t *dims, int64_t hn,
                  int64_t hd, const void *x, void *y, int planes, cudaStream_t st);

int validate_apply(const sc_stencil *s, int dtype, int bc, const int64_t *dims, int64_t h_num,
                   int64_t h_den);
// Enqueues y = A x on `st` (no validation of pointers).
int apply_enqueue(const ApplyReq &q, cudaStream_t st);
size_t grid_elems(const sc_stencil *s, int bc, const int64_t *dims, bool input);
// Elements of a grid of `dims` extended by `ext` on every side of every axis.
size_t grid_elems_ext(int ndim, const int64_t *dims, int ext);
// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
bool spans_overlap(const void *a, size_t na, const void *b, size_t nb);
// SC_EINVAL unless x (input extent for radius `r_in` under `bc`), y (the
// output grid) and, when given, the work space are pairwise disjoint.
int check_disjoint(int ndim, int bc, const int64_t *dims, int r_in, size_t es, const void *x, const void *y,
                   const void *work = nullptr, size_t work_bytes = 0);
int num_sms();
// Planes per CTA for a streamed launch of `tiles_xy` tiles per plane over
// `nplanes` planes with halo R, given `slots` = resident CTAs per SM x SMs:
// minimises ceil(CTAs / slots) * (H + 2R), i.e. whole waves of CTAs that each
// stream as long a run as the wave count allows.
int wave_planes(long long tiles_xy, int nplanes, int R, long long slots, int hmin);
// Testing/tuning knob: fixes the number of output planes per CTA (0 = auto).

}  // namespace sc
