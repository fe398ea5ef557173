// Internal helpers shared by the library's translation units (not part of the
// public ABI).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/stencilcomp.h"

namespace sc {

// Raises a kernel's dynamic shared-memory limit once per device (the
// attribute is per device; concurrent callers may both set it, which is
// harmless).  `done` holds one bit per device ordinal.
template <typename K>
inline void set_smem_limit_once(K *kern, size_t bytes, std::atomic<unsigned long long> &done) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load(std::memory_order_acquire) & bit)) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    done.fetch_or(bit, std::memory_order_acq_rel);
  }
}

// Records a reason for the calling thread and returns the status unchanged.
int fail(int status, const char *fmt, ...);
void clear_error();

typedef unsigned __int128 u128;
typedef __int128 i128;

// Correctly rounded (ties-to-even) conversion of the exact ratio
// (neg ? -1 : 1) * n / d to a binary floating value with `mant_bits`
// significand bits (53 for double, 24 for float).  n, d > 0, both < 2^127.
double round_ratio(bool neg, u128 n, u128 d, int mant_bits);

// Exact weights of stencil s at spacing h = h_num/h_den, correctly rounded.
int weights_f64(const sc_stencil *s, int64_t h_num, int64_t h_den, double *out);
int weights_f32(const sc_stencil *s, int64_t h_num, int64_t h_den, float *out);

}  // namespace sc
