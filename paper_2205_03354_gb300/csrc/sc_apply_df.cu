// FP64 Laplacian passes in double-float arithmetic (pairs of FP32 numbers).
//
// GB300 issues two FP64 FMAs per clock per SM against 128 FP32 FMAs, so an
// FP64 stencil apply is bound by the FP64 pipe at a few percent of HBM
// bandwidth.  For the factors of the composed operators used here -- a
// Laplacian L = s * L_int, L_int with small integer weights c0 (centre),
// c1 (distance 1) and c2 (distance 2, fourth order) on every axis, s =
// 1/(den h^2) -- the nested form y = s^2 L_int(L_int x) (Eq. C=B(A)) can be
// evaluated on the FP32 pipe instead:
//   * a double x is split exactly into hi + lo + rest with integer bit
//     operations (hi: the leading 24 significand bits, lo: the next 29 bits
//     rounded to 24; |rest| <= 2^-48 |x|);
//   * sums are carried as unevaluated pairs (hi, lo) with error-free
//     transformations (Knuth's TwoSum, Dekker's Fast2Sum, TwoProduct via
//     FMA); products by the integer weights are exact up to the pair format;
//   * the scaled result s^2 z is rebuilt as a double exactly from its pair
//     with integer bit operations and one FP64 addition.
// Relative error per pass is a few units of 2^-48 of sum_k |w_k x_k|, inside
// the FP64 apply tolerance (npts * 2^-52 of the same sum).  Inputs whose
// magnitude lies outside [2^-74, 2^100] (and are not zero) cannot be split
// into normal floats: such a value raises a flag in device memory, and the
// native FP64 passes that follow the emulated ones (launched unconditionally,
// each CTA returning at once while the flag is clear) recompute the result.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "sc_apply_df.h"
#include "sc_apply_host.h"
#include "sc_device.cuh"
#include "sc_internal.h"

namespace sc {

struct F2 {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  F2 r;
  r.h = a + b;
  r.l = b - (r.h - a);
  return r;
}
// Neumaier-style accumulation of pairs: running (s, c), s the leading sum,
// c the collected rounding errors and low parts.
struct Acc {
  float s, c;
};
__device__ __forceinline__ void acc_add(Acc &a, F2 v) {
  float s, e;
  two_sum(a.s, v.h, s, e);
  a.s = s;
  a.c += e + v.l;
}
__device__ __forceinline__ F2 acc_get(const Acc &a) { return fast_two_sum(a.s, a.c); }
// pair times a small integer k (|k| < 2^24, exact as a float)
__device__ __forceinline__ F2 mul_int(F2 a, float k) {
  const float p = a.h * k;
  float e = fmaf(a.h, k, -p);
  e = fmaf(a.l, k, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ F2 mul_pair(F2 a, F2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ F2 add_pair(F2 a, F2 b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e += a.l + b.l;
  return fast_two_sum(s, e);
}

// Exact split of a double into two floats (|x - hi - lo| <= 2^-48 |x|);
// sets bad when |x| is outside [2^-74, 2^100] and not zero.
__device__ __forceinline__ F2 split_double(double x, int &bad) {
  const unsigned long long b = __double_as_longlong(x);
  const unsigned hi32 = unsigned(b >> 32), lo32 = unsigned(b);
  const int e = int((hi32 >> 20) & 0x7ffu);
  const unsigned sgn = hi32 & 0x80000000u;
  F2 r;
  if (e == 0 && ((hi32 & 0xfffffu) | lo32) == 0u) {  // +-0
    r.h = 0.0f;
    r.l = 0.0f;
    return r;
  }
  if (e < 1023 - 74 || e > 1023 + 100) {  // denormal, tiny, huge, inf, nan
    bad = 1;
    r.h = 0.0f;
    r.l = 0.0f;
    return r;
  }
  const unsigned mh = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  r.h = __int_as_float(int(sgn | (unsigned(e - 1023 + 127) << 23) | mh));
  // remaining 29 bits, weight 2^(e - 1075): convert, then scale exactly
  const unsigned rem = lo32 & 0x1fffffffu;
  float l = __uint2float_rn(rem);                             // rounds 29 -> 24 bits
  l *= __int_as_float(int(unsigned(e - 1075 + 127) << 23));  // 2^(e-1075) is a normal float
  r.l = sgn ? -l : l;
  return r;
}

// Float -> double by bit re-biasing (no FP64 instruction).
__device__ __forceinline__ double f2d_bits(float f, int extra_exp) {
  const unsigned u = __float_as_uint(f);
  if ((u & 0x7fffffffu) == 0u) return 0.0;
  if ((u & 0x7f800000u) == 0u) return ldexp(double(f), extra_exp);  // subnormal: rare, FP64 path
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const long long e = (long long)((u >> 23) & 0xffu) - 127 + 1023 + extra_exp;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)e << 52) | m));
}

template <int NDIM>
struct DfCfg;
template <>
struct DfCfg<2> {
  static constexpr int VX = 4, TX = 256, TY = 1;
};
template <>
struct DfCfg<3> {
  static constexpr int VX = 4, TX = 16, TY = 16;
};

// One Laplacian pass t = L_int(x) in pair arithmetic over a streamed tile.
// IN_PAIR: x is stored as float pairs (else doubles, split on arrival);
// OUT_PAIR: t is stored as float pairs (else as the double scale * t).
template <int NDIM, int R, bool IN_PAIR, bool OUT_PAIR>
struct DfPass {
  using C = DfCfg<NDIM>;
  static constexpr int VX = C::VX, TX = C::TX, TY = C::TY, NTHR = TX * TY;
  static constexpr int BX = TX * VX, BY = NDIM == 3 ? TY : 1;
  static constexpr int RP = NDIM == 3 ? R : 0;
  static constexpr int HX = 2;  // stored x halo: R <= 2, two 8-byte elements per 16-byte chunk
  static constexpr int PXS = BX + 2 * HX, PYS = BY + 2 * RP, PLANE = PXS * PYS;
  static constexpr int PF = 2;            // planes in flight ahead of the one consumed
  static constexpr int NR = R + 1 + PF;   // ring: R planes kept back for the in-plane terms
  static constexpr int NQ = 2 * R + 1;    // register queue of centre values
  static constexpr int NCHUNK = PLANE / 2;
  static constexpr size_t SMEM = size_t(NR) * PLANE * 8;
};

struct DfGeom {
  int nx, ny, nz;  // output dims (nz = 1 in 2D)
  int bc;          // BC_PERIODIC or BC_GHOSTED (input ring R)
  int H;
  long long in_sy, in_ss, out_sy, out_ss;
  float c0, c1, c2;  // integer weights: centre (all axes), distance 1, distance 2
  F2 scale;          // OUT double: scale' in [1, 2) as a pair ...
  int scale_exp;     // ... times 2^scale_exp
};

template <int NDIM, int R, bool IN_PAIR, bool OUT_PAIR>
__global__ void __launch_bounds__(DfPass<NDIM, R, IN_PAIR, OUT_PAIR>::NTHR)
    df_lap_kernel(const void *__restrict__ xin, void *__restrict__ yout, DfGeom g, int *__restrict__ bad_flag) {
  using K = DfPass<NDIM, R, IN_PAIR, OUT_PAIR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // ring of planes, 8 bytes per element (a double, or a float pair once split)
  unsigned long long *ring = reinterpret_cast<unsigned long long *>(smem_raw);
  const int tx = threadIdx.x % K::TX, ty = threadIdx.x / K::TX;
  const int x0 = blockIdx.x * K::BX;
  const int y0 = NDIM == 3 ? blockIdx.y * K::BY : 0;
  const int z0 = (NDIM == 3 ? blockIdx.z : blockIdx.y) * g.H;
  const int ns = NDIM == 3 ? g.nz : g.ny;
  const int zend = min(z0 + g.H, ns);
  const int NT = (zend - z0) + 2 * R;
  const unsigned long long *src = static_cast<const unsigned long long *>(xin);
  int bad = 0;

  auto load_plane = [&](int t) {
    const int zs = z0 - R + t;
    const int iz = map_coord(zs, ns, g.bc, R);
    unsigned long long *buf = ring + (t % K::NR) * K::PLANE;
    const long long pbase = (long long)iz * (NDIM == 3 ? g.in_ss : g.in_sy);
    for (int c = threadIdx.x; c < K::NCHUNK; c += K::NTHR) {
      const int e = c * 2, r = e / K::PXS, cc = e - r * K::PXS;
      const int ix = map_coord(x0 - K::HX + cc, g.nx, g.bc, R);
      int iy = 0;
      if (NDIM == 3) iy = map_coord(y0 - K::RP + r, g.ny, g.bc, R);
      const bool ok = (iz >= 0) & (ix >= 0) & (iy >= 0);
      const unsigned long long *s = ok ? src + pbase + (long long)iy * g.in_sy + ix : src;
      cp_async16(buf + e, s, ok ? 16 : 0);
    }
  };

  F2 q[K::NQ][K::VX];
#pragma unroll
  for (int k = 0; k < K::PF; ++k) {
    if (k < NT) load_plane(k);
    cp_async_commit();
  }
  const int xo = x0 + tx * K::VX;
  const int yy = y0 + ty;
  const int col = tx * K::VX + K::HX;         // smem column of the first owned point
  const int row = NDIM == 3 ? ty + K::RP : 0;  // smem row of the owned points
  for (int tb = 0; tb < NT; tb += K::NQ) {
#pragma unroll
    for (int s = 0; s < K::NQ; ++s) {
      const int t = tb + s;
      if (t >= NT) break;
      cp_async_wait<K::PF - 1>();
      __syncthreads();
      if (t + K::PF < NT) load_plane(t + K::PF);
      cp_async_commit();
      unsigned long long *pl = ring + (t % K::NR) * K::PLANE;
      if (!IN_PAIR) {  // split the arrived doubles into pairs, in place
        for (int e = threadIdx.x; e < K::PLANE; e += K::NTHR) {
          const F2 v = split_double(__longlong_as_double((long long)pl[e]), bad);
          pl[e] = (unsigned long long)__float_as_uint(v.h) | ((unsigned long long)__float_as_uint(v.l) << 32);
        }
        __syncthreads();
      }
      const F2 *pf = reinterpret_cast<const F2 *>(pl);
      // centre values of this plane into the queue
#pragma unroll
      for (int v = 0; v < K::VX; ++v) q[s][v] = pf[row * K::PXS + col + v];
      if (t >= 2 * R) {
        // output plane z0 + t - 2R: in-plane terms from the plane R back,
        // streaming-axis terms from the queue
        const F2 *pc = reinterpret_cast<const F2 *>(ring + ((t - R) % K::NR) * K::PLANE);
        const int j = z0 + t - 2 * R;
        const int sc_ = ((s - R) % K::NQ + K::NQ) % K::NQ;
        F2 seg[K::VX + 2 * R];
#pragma unroll
        for (int i = 0; i < K::VX + 2 * R; ++i) seg[i] = pc[row * K::PXS + col - R + i];
        F2 out[K::VX];
#pragma unroll
        for (int v = 0; v < K::VX; ++v) {
          Acc a1{0.0f, 0.0f}, a2{0.0f, 0.0f};
          acc_add(a1, seg[v + R - 1]);
          acc_add(a1, seg[v + R + 1]);
          acc_add(a1, q[((s - R - 1) % K::NQ + K::NQ) % K::NQ][v]);
          acc_add(a1, q[((s - R + 1) % K::NQ + K::NQ) % K::NQ][v]);
          if (NDIM == 3) {
            acc_add(a1, pc[(row - 1) * K::PXS + col + v]);
            acc_add(a1, pc[(row + 1) * K::PXS + col + v]);
          }
          F2 t1 = mul_int(acc_get(a1), g.c1);
          F2 tc = mul_int(q[sc_][v], g.c0);
          F2 r = add_pair(t1, tc);
          if (R == 2) {
            acc_add(a2, seg[v + R - 2]);
            acc_add(a2, seg[v + R + 2]);
            acc_add(a2, q[((s - R - 2) % K::NQ + K::NQ) % K::NQ][v]);
            acc_add(a2, q[((s - R + 2) % K::NQ + K::NQ) % K::NQ][v]);
            if (NDIM == 3) {
              acc_add(a2, pc[(row - 2) * K::PXS + col + v]);
              acc_add(a2, pc[(row + 2) * K::PXS + col + v]);
            }
            r = add_pair(r, mul_int(acc_get(a2), g.c2));
          }
          out[v] = r;
        }
        if (j < zend && (NDIM == 2 || yy < g.ny)) {
          const long long base = (long long)j * (NDIM == 3 ? g.out_ss : g.out_sy) +
                                 (NDIM == 3 ? (long long)yy * g.out_sy : 0) + xo;
#pragma unroll
          for (int v = 0; v < K::VX; ++v) {
            if (xo + v >= g.nx) continue;
            if (OUT_PAIR) {
              reinterpret_cast<F2 *>(yout)[base + v] = out[v];
            } else {
              const F2 z = mul_pair(out[v], g.scale);  // |scale| in [1, 2): no overflow
              // exact: the pair's 48 significant bits fit a double
              const double d = f2d_bits(z.h, g.scale_exp) + f2d_bits(z.l, g.scale_exp);
              static_cast<double *>(yout)[base + v] = d;
            }
          }
        }
      }
    }
  }
  cp_async_wait<0>();
  if (bad) atomicOr(bad_flag, 1);
}

// ---------------------------------------------------------------------------

// Integer form of a symmetric star stencil: centre c0 (all axes), c1 at
// distance 1 and c2 at distance 2 on every axis; false if s is not of that
// form (then the native passes are used).
bool star_int_form(const sc_stencil *s, float *c0, float *c1, float *c2) {
  if (s->radius < 1 || s->radius > 2) return false;
  long long v0 = 0, v1 = 0, v2 = 0;
  bool h1 = false, h2 = false, h0 = false;
  int n1 = 0, n2 = 0;
  for (int k = 0; k < s->npts; ++k) {
    const int dx = s->off[k][0], dy = s->off[k][1], dz = s->off[k][2];
    const int nzc = (dx != 0) + (dy != 0) + (dz != 0);
    if (nzc > 1) return false;
    const int d = std::abs(dx) + std::abs(dy) + std::abs(dz);
    const long long v = s->num[k];
    if (d == 0) {
      v0 = v;
      h0 = true;
    } else if (d == 1) {
      if (h1 && v != v1) return false;
      v1 = v;
      h1 = true;
      ++n1;
    } else {
      if (h2 && v != v2) return false;
      v2 = v;
      h2 = true;
      ++n2;
    }
  }
  if (!h1 || n1 != 2 * s->ndim || (h2 && n2 != 2 * s->ndim)) return false;
  if (std::llabs(v0) >= (1LL << 20) || std::llabs(v1) >= (1LL << 20) || std::llabs(v2) >= (1LL << 20)) return false;
  *c0 = h0 ? float(v0) : 0.0f;
  *c1 = float(v1);
  *c2 = h2 ? float(v2) : 0.0f;
  return true;
}

template <int NDIM, int R, bool IN_PAIR, bool OUT_PAIR>
static int launch_df(const void *x, void *y, const int64_t *dims, int bc, float c0, float c1, float c2,
                     double scale, int *flag, cudaStream_t st, int planes) {
  using K = DfPass<NDIM, R, IN_PAIR, OUT_PAIR>;
  DfGeom g;
  std::memset(&g, 0, sizeof(g));
  g.nx = int(dims[0]);
  g.ny = int(dims[1]);
  g.nz = NDIM == 3 ? int(dims[2]) : 1;
  g.bc = bc == SC_BC_GHOSTED ? BC_GHOSTED : BC_PERIODIC;
  const int sh = bc == SC_BC_GHOSTED ? 2 * R : 0;
  g.in_sy = g.nx + sh;
  g.in_ss = (long long)(g.nx + sh) * (g.ny + sh);
  g.out_sy = g.nx;
  g.out_ss = (long long)g.nx * g.ny;
  g.c0 = c0;
  g.c1 = c1;
  g.c2 = c2;
  if (!OUT_PAIR) {  // scale = m * 2^e, m in [1, 2), m as an exact pair of floats
    int e = 0;
    const double m = std::frexp(scale, &e) * 2.0;
    g.scale_exp = e - 1;
    const float mh = float(m);
    g.scale.h = mh;
    g.scale.l = float(m - double(mh));
  }
  const int ns = NDIM == 3 ? g.nz : g.ny;
  const long long txy = (long long)((g.nx + K::BX - 1) / K::BX) * (NDIM == 3 ? (g.ny + K::BY - 1) / K::BY : 1);
  auto kern = df_lap_kernel<NDIM, R, IN_PAIR, OUT_PAIR>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(K::SMEM));
    attr = true;
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, K::NTHR, K::SMEM);
  g.H = planes > 0 ? std::min(planes, ns)
                   : wave_planes(txy, ns, R, (long long)std::max(occ, 1) * num_sms(), std::max(4 * R, 8));
  dim3 grid((g.nx + K::BX - 1) / K::BX, NDIM == 3 ? (g.ny + K::BY - 1) / K::BY : (ns + g.H - 1) / g.H,
            NDIM == 3 ? (ns + g.H - 1) / g.H : 1);
  kern<<<grid, K::NTHR, K::SMEM, st>>>(x, y, g, flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SC_ECUDA, "pair-arithmetic apply launch: %s", cudaGetErrorString(e));
  return SC_OK;
}

template <int NDIM, int R>
static int df_two_passes(const void *x, void *t, void *y, const int64_t *dims_t, const int64_t *dims_y, int bc,
                         const float *ca, const float *cb, double scale, int *flag, cudaStream_t st, int planes) {
  if (int rc = launch_df<NDIM, R, false, true>(x, t, dims_t, bc, ca[0], ca[1], ca[2], 1.0, flag, st, planes))
    return rc;
  return launch_df<NDIM, R, true, false>(t, y, dims_y, bc, cb[0], cb[1], cb[2], scale, flag, st, planes);
}

int df_composition_enqueue(int ndim, int R, const void *x, void *t, void *y, const int64_t *dims_t,
                           const int64_t *dims_y, int bc, const float *ca, const float *cb, double scale,
                           int *flag, cudaStream_t st, int planes) {
  if (ndim == 2)
    return R == 1 ? df_two_passes<2, 1>(x, t, y, dims_t, dims_y, bc, ca, cb, scale, flag, st, planes)
                  : df_two_passes<2, 2>(x, t, y, dims_t, dims_y, bc, ca, cb, scale, flag, st, planes);
  return R == 1 ? df_two_passes<3, 1>(x, t, y, dims_t, dims_y, bc, ca, cb, scale, flag, st, planes)
                : df_two_passes<3, 2>(x, t, y, dims_t, dims_y, bc, ca, cb, scale, flag, st, planes);
}

}  // namespace sc
