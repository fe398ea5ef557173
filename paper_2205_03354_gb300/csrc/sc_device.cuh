// Device-side building blocks shared by the apply, vector and solver kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sc {

// ---- cp.async (global -> shared, bypassing registers) ----------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte copy; src_bytes = 0 writes zeros (zero fill) and reads nothing.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes));
}
template <int N>
__device__ __forceinline__ void cp_async_elem(void *dst, const void *src, int src_bytes) {
  static_assert(N == 4 || N == 8, "element copy is 4 or 8 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(dst)), "l"(src),
               "n"(N), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// ---- boundary index maps ----------------------------------------------------
enum { BC_PERIODIC = 0, BC_GHOSTED = 1, BC_ZERO = 2 };

// Maps an output-grid coordinate g (may lie up to R outside [0, n)) to an
// input-array index, or -1 when the value is zero.  Periodic needs n >= R.
__device__ __forceinline__ int map_coord(int g, int n, int bc, int R) {
  if (bc == BC_PERIODIC) {
    if (g < 0) g += n;
    else if (g >= n) g -= n;
    return (g >= 0 && g < n) ? g : -1;  // beyond one wrap: never read by a stored output
  }
  if (bc == BC_GHOSTED) {
    int i = g + R;
    return (i >= 0 && i < n + 2 * R) ? i : -1;
  }
  return (g >= 0 && g < n) ? g : -1;
}

// ---- deterministic block reduction of doubles ------------------------------
// Fixed summation order for a given blockDim: warp tree, then warp 0 sums the
// per-warp partials in index order.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red /* >= NT/32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < NT / 32 ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

}  // namespace sc
