// FP64 Laplacian passes in double-float arithmetic (pairs of FP32 numbers),
// two grid points per packed f32x2 instruction.
//
// GB300 issues two FP64 FMAs per clock per SM against 128 FP32 FMAs, so an
// FP64 stencil apply is bound by the FP64 pipe at a few percent of HBM
// bandwidth.  For the factors of the composed operators used here -- a
// Laplacian L = s * L_int, L_int with small integer weights c0 (centre),
// c1 (distance 1) and c2 (distance 2, fourth order) on every axis, s =
// 1/(den h^2) -- the nested form y = s^2 L_int(L_int x) (Eq. C=B(A)) is
// evaluated on the FP32 pipe instead:
//   * a double x is split exactly into hi + lo + rest with integer bit
//     operations (hi: the leading 24 significand bits, lo: the next 29 bits
//     rounded to 24; |rest| <= 2^-48 |x|);
//   * sums are carried as unevaluated pairs (hi, lo) with error-free
//     transformations (Knuth's TwoSum, Dekker's Fast2Sum, TwoProduct via
//     FMA) in Neumaier's running-compensation order; products by the integer
//     weights are exact up to the pair format;
//   * the scaled result s^2 z is rebuilt as a double exactly from its pair
//     with integer bit operations and one FP64 addition.
// Relative error per pass is a few units of 2^-48 of sum_k |w_k x_k|, inside
// the FP64 apply tolerance (npts * 2^-52 of the same sum).  Inputs whose
// magnitude lies outside [2^-74, 2^100] (and are not zero) cannot be split
// into normal floats: such a value raises a flag in device memory, and the
// native FP64 passes that follow the emulated ones (launched unconditionally,
// each CTA returning at once while the flag is clear) recompute the result.
//
// Packing.  sm_103a executes add/sub/mul/fma.rn.f32x2 on register pairs with
// the rounding of the scalar instructions, one issue slot for two lanes.  The
// x axis of a row of length n (even) is folded in half: cell c in [0, n/2)
// holds the points c (lane a) and c + n/2 (lane b).  Every x offset of a
// stencil then maps a cell to a cell with both lanes in step, so one thread
// evaluates two points with one instruction stream.  The intermediate of the
// two passes is kept in this folded layout in HBM, one 16-byte cell
// {hi_a, hi_b, lo_a, lo_b} per pair of points, so the second pass copies it
// with 16-byte cp.async and no rearrangement.  Halo cells left of cell 0 and
// right of cell n/2 - 1 are the cells n/2 away with their lanes swapped
// (periodic rows; for the ghosted intermediate the lane that is swapped in
// feeds only points outside the output).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "sc_apply_df.h"
#include "sc_apply_host.h"
#include "sc_device.cuh"
#include "sc_internal.h"

namespace sc {

typedef unsigned long long f2x;  // two FP32 values, lane a in the low half

__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2x pk2(float a, float b) {
  f2x d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ void upk2(f2x d, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(d));
}

// Two double-float numbers (lanes a and b): value = h + l per lane.
struct P2 {
  f2x h, l;
};
// Neumaier accumulation: s the running sum, c the collected rounding errors
// and low parts (unnormalised).
struct Acc2 {
  f2x s, c;
};
__device__ __forceinline__ void acc_add2(Acc2 &A, f2x vh, f2x vl) {
  const f2x s = add2(A.s, vh);  // TwoSum(A.s, vh) = (s, e)
  const f2x bb = sub2(s, A.s);
  const f2x e = add2(sub2(A.s, sub2(s, bb)), sub2(vh, bb));
  A.s = s;
  A.c = add2(A.c, add2(e, vl));
}
// Rounded packed products are formed as fma(a, b, Z), Z a zero pair that the
// kernel receives as an argument.  Measured on sm_103a: products taken with
// mul.rn.f32x2 and then consumed by the error-free transformations below did
// not reproduce the scalar mul.rn.f32 results once ptxas optimisation was on
// (bit-exact at -O0 and with scalar products), so the kernels take no packed
// mul and the product's rounding is fixed by the FMA.
__device__ __forceinline__ f2x rmul2(f2x a, f2x b, f2x Z) { return fma2(a, b, Z); }

// A *= k for an integer k exact in FP32 (kk = (k, k), nk = (-k, -k)):
// TwoProduct of the leading sum, the compensation scaled with one rounding.
__device__ __forceinline__ void acc_scale2(Acc2 &A, f2x kk, f2x nk, f2x Z) {
  const f2x p = rmul2(A.s, kk, Z);
  const f2x e = fma2(A.s, kk, rmul2(A.s, nk, Z));  // A.s k - RN(A.s k), exact
  A.c = fma2(A.c, kk, e);
  A.s = p;
}
// (a_h + a_l) + (b_h + b_l) as an unnormalised accumulator: TwoSum of the
// leading parts, the low parts and the rounding error collected.
__device__ __forceinline__ Acc2 pair_sum2(f2x ah, f2x al, f2x bh, f2x bl) {
  const f2x s = add2(ah, bh);
  const f2x bb = sub2(s, ah);
  const f2x e = add2(sub2(ah, sub2(s, bb)), sub2(bh, bb));
  return Acc2{s, add2(e, add2(al, bl))};
}
// A -= B (TwoSum of A.s and -B.s, compensations subtracted)
__device__ __forceinline__ void acc_sub2(Acc2 &A, const Acc2 &B) {
  const f2x s = sub2(A.s, B.s);
  const f2x bb = sub2(s, A.s);
  const f2x e = sub2(sub2(A.s, sub2(s, bb)), add2(B.s, bb));
  A.s = s;
  A.c = add2(A.c, sub2(e, B.c));
}
__device__ __forceinline__ P2 acc_get2(const Acc2 &A) {  // Fast2Sum(s, c)
  P2 r;
  r.h = add2(A.s, A.c);
  r.l = sub2(A.c, sub2(r.h, A.s));
  return r;
}

// Exact split of a double into two floats (|x - hi - lo| <= 2^-48 |x|) with
// integer operations; (0, 0) for +-0, and (0, 0) with bad set when |x| is
// outside [2^-74, 2^100].
__device__ __forceinline__ void split_double(double x, float &h, float &l, int &bad) {
  const unsigned long long b = __double_as_longlong(x);
  const unsigned hi = unsigned(b >> 32), lo = unsigned(b);
  const unsigned t = hi & 0x7fffffffu;
  const bool ok = (t - (949u << 20)) < (175u << 20);  // biased exponent in [949, 1123]
  // float exponent e - 896 in [53, 227]; hi = leading 24 significand bits
  const unsigned hb = __funnelshift_l(lo, t - (896u << 20), 3) | (hi & 0x80000000u);
  // the next 29 bits, weight 2^(e - 1075) (a normal float for e >= 949)
  const float w = __uint_as_float((hb & 0xff800000u) - (52u << 23));
  const float lf = __uint2float_rn(lo & 0x1fffffffu) * w;
  h = ok ? __uint_as_float(hb) : 0.0f;
  l = ok ? lf : 0.0f;
  bad |= int(!ok & ((t | lo) != 0u));
}

// Float -> double times 2^extra by re-biasing the exponent (no FP64
// instruction); ebias = (1023 - 127 + extra) << 20.  Zero maps to zero; a
// subnormal float sets bad (the native passes then recompute the result).
__device__ __forceinline__ double f2d_bits(float f, unsigned ebias, int &bad) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7fffffffu, sg = u & 0x80000000u;
  const unsigned hi = a ? (sg | (a >> 3)) + ebias : sg;
  bad |= int(a != 0u && a < 0x00800000u);
  return __hiloint2double(int(hi), int(u << 29));
}

template <int NDIM>
struct PkCfg;
template <>
struct PkCfg<2> {
  static constexpr int TX = 128, TY = 1, VP = 2, PF = 2;
};
template <>
struct PkCfg<3> {
  static constexpr int TX = 16, TY = 16, VP = 2, PF = 2;
};

// PASS 1: doubles -> folded pair intermediate; PASS 2: folded pairs -> doubles.
template <int NDIM, int R, int PASS>
struct PkPass {
  using C = PkCfg<NDIM>;
  static constexpr int TX = C::TX, TY = C::TY, VP = C::VP, PF = C::PF, NTHR = TX * TY;
  static constexpr int D = TX * VP;  // cells per tile row
  static constexpr int HX = 2;       // x halo in cells (R <= 2)
  static constexpr int RP = NDIM == 3 ? R : 0;
  static constexpr int BY = NDIM == 3 ? TY : 1;
  static constexpr int PYS = BY + 2 * RP;
  static constexpr int KS = D + 2 * HX;  // cells per smem row
  static constexpr int FPLANE = KS * PYS;
  // folded planes in smem: R behind the consumed one, the consumed one, PF
  // in flight.  Pass 1 copies each double (8 bytes) straight into its lane
  // of the cell and the copying thread splits the cell in place; pass 2
  // copies whole 16-byte cells.
  static constexpr int NF = R + 1 + PF;
  static constexpr int NQ = 2 * R + 1;                     // register queue of centre cells
  static constexpr int NCPT = (FPLANE + NTHR - 1) / NTHR;  // cells copied per thread
  static constexpr size_t SMEM = size_t(NF) * FPLANE * 16;
};

enum { PK_C1_POW2 = 1, PK_C2_POW2 = 2, PK_C2_MINUS1 = 4 };

struct PkGeom {
  int nx, ny, nz;   // output grid (nz = 1 in 2D)
  int nf, nc;       // folded row length (even) and its cells nf / 2
  int off_out;      // pass 2: output x = fold position - off_out
  int bc;           // BC_PERIODIC or BC_GHOSTED (input ring R) on y/z (and on x of pass 1)
  int H;            // output planes per CTA
  long long in_sy, in_ss;    // input strides (pass 1: doubles, pass 2: cells)
  long long out_sy, out_ss;  // output strides (pass 1: cells, pass 2: doubles)
  float c0, c1, c2;          // integer weights
  float zero;                // 0.0f (see rmul2)
  int flags;                 // PK_* properties of the weights
  float sh, sl;              // pass 2: scale mantissa in [1, 2) as an exact float pair ...
  int sexp;                  // ... times 2^sexp
};

template <int NDIM, int R, int PASS>
__global__ void __launch_bounds__(PkPass<NDIM, R, PASS>::NTHR, NDIM == 3 ? 3 : 4)
    pk_lap_kernel(const void *__restrict__ xin, void *__restrict__ yout, PkGeom g, int *__restrict__ bad_flag) {
  using K = PkPass<NDIM, R, PASS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2 *fold = reinterpret_cast<ulonglong2 *>(smem_raw);
  const int tid = threadIdx.x;
  const int tx = tid % K::TX, ty = tid / K::TX;
  const int k0 = blockIdx.x * K::D;  // first cell of the tile
  const int y0 = NDIM == 3 ? blockIdx.y * K::BY : 0;
  const int z0 = (NDIM == 3 ? blockIdx.z : blockIdx.y) * g.H;
  const int ns = NDIM == 3 ? g.nz : g.ny;
  const int zend = min(z0 + g.H, ns);
  const int NT = (zend - z0) + 2 * R;
  const long long in_ps = NDIM == 3 ? g.in_ss : g.in_sy;
  int bad = 0;

  // In-plane source offsets of this thread's cells (fixed for the CTA);
  // -1: zero fill.  Pass 1: one double per lane; pass 2: one 16-byte cell,
  // noting the cells whose lanes are swapped.
  constexpr int NSRC = PASS == 1 ? 2 : 1;
  int src_off[K::NCPT][NSRC];
  unsigned swap_mask = 0;
#pragma unroll
  for (int i = 0; i < K::NCPT; ++i) {
    const int ch = tid + i * K::NTHR;
#pragma unroll
    for (int l = 0; l < NSRC; ++l) src_off[i][l] = -1;
    if (ch >= K::FPLANE) continue;
    const int r = ch / K::KS, c = ch - r * K::KS;
    int iy = 0;
    if (NDIM == 3) iy = map_coord(y0 - K::RP + r, g.ny, g.bc, R);
    if (iy < 0) continue;
    if (PASS == 1) {
      const int p = k0 - K::HX + c;  // fold position of lane a; lane b is nc further
#pragma unroll
      for (int l = 0; l < NSRC; ++l) {
        const int ix = map_coord(p + l * g.nc, g.nf, g.bc, R);
        if (ix >= 0) src_off[i][l] = int((long long)iy * g.in_sy + ix);
      }
    } else {
      int gc = k0 - K::HX + c;
      bool sw = false;
      if (gc < 0) {
        gc += g.nc;
        sw = true;
      } else if (gc >= g.nc) {
        gc -= g.nc;
        sw = true;
      }
      if (gc >= 0 && gc < g.nc) {
        src_off[i][0] = int((long long)iy * g.in_sy + gc);
        if (sw) swap_mask |= 1u << i;
      }
    }
  }

  auto load_plane = [&](int t) {
    const int iz = map_coord(z0 - R + t, ns, g.bc, R);
    const long long pb = (long long)iz * in_ps;
#pragma unroll
    for (int i = 0; i < K::NCPT; ++i) {
      const int ch = tid + i * K::NTHR;
      if (ch >= K::FPLANE) continue;
      ulonglong2 *dst = fold + size_t(t % K::NF) * K::FPLANE + ch;
#pragma unroll
      for (int l = 0; l < NSRC; ++l) {
        const bool ok = iz >= 0 && src_off[i][l] >= 0;
        if (PASS == 1) {
          const unsigned long long *src = static_cast<const unsigned long long *>(xin) + (ok ? pb + src_off[i][l] : 0);
          cp_async_elem<8>(reinterpret_cast<unsigned long long *>(dst) + l, src, ok ? 8 : 0);
        } else {
          const ulonglong2 *src = static_cast<const ulonglong2 *>(xin) + (ok ? pb + src_off[i][l] : 0);
          cp_async16(dst, src, ok ? 16 : 0);
        }
      }
    }
  };

  const f2x kc0 = pk2(g.c0, g.c0), nc0 = pk2(-g.c0, -g.c0);
  const f2x kc1 = pk2(g.c1, g.c1), nc1 = pk2(-g.c1, -g.c1);
  const f2x kc2 = pk2(g.c2, g.c2), nc2 = pk2(-g.c2, -g.c2);
  const f2x Z = pk2(g.zero, g.zero);
  const int row = NDIM == 3 ? ty + K::RP : 0;
  // owned cells tx + v TX (v < VP): consecutive lanes read consecutive
  // 16-byte cells, free of shared-memory bank conflicts
  const int col = tx + K::HX;  // smem cell of the first owned cell
  const int yy = y0 + ty;
  P2 q[K::NQ][K::VP];

#pragma unroll
  for (int k = 0; k < K::PF; ++k) {
    if (k < NT) load_plane(k);
    cp_async_commit();
  }
  for (int tb = 0; tb < NT; tb += K::NQ) {
#pragma unroll
    for (int s = 0; s < K::NQ; ++s) {
      const int t = tb + s;
      if (t >= NT) break;
      cp_async_wait<K::PF - 1>();
      ulonglong2 *fp = fold + size_t(t % K::NF) * K::FPLANE;
      // own copies have landed: split pass 1's doubles into pairs in place,
      // swap the lanes of pass 2's wrapped cells
      if (PASS == 1) {
#pragma unroll
        for (int i = 0; i < K::NCPT; ++i) {
          const int ch = tid + i * K::NTHR;
          if (ch >= K::FPLANE) continue;
          const ulonglong2 v = fp[ch];
          float ha, la, hb, lb;
          split_double(__longlong_as_double((long long)v.x), ha, la, bad);
          split_double(__longlong_as_double((long long)v.y), hb, lb, bad);
          fp[ch] = make_ulonglong2(pk2(ha, hb), pk2(la, lb));
        }
      } else if (swap_mask) {
#pragma unroll
        for (int i = 0; i < K::NCPT; ++i)
          if (swap_mask & (1u << i)) {
            ulonglong2 v = fp[tid + i * K::NTHR];
            float a, b;
            upk2(v.x, a, b);
            v.x = pk2(b, a);
            upk2(v.y, a, b);
            v.y = pk2(b, a);
            fp[tid + i * K::NTHR] = v;
          }
      }
      __syncthreads();
      if (t + K::PF < NT) load_plane(t + K::PF);
      cp_async_commit();
      // centre cells of this plane into the queue
#pragma unroll
      for (int v = 0; v < K::VP; ++v) {
        const ulonglong2 c = fp[row * K::KS + col + v * K::TX];
        q[s][v].h = c.x;
        q[s][v].l = c.y;
      }
      if (t < 2 * R) continue;
      // output plane z0 + t - 2R: in-plane terms from the plane R back,
      // streaming-axis terms from the queue
      const ulonglong2 *pc = fold + size_t((t - R) % K::NF) * K::FPLANE;
      const int j = z0 + t - 2 * R;
      P2 out[K::VP];
#pragma unroll
      for (int v = 0; v < K::VP; ++v) {
        const P2 &zm1 = q[(s - R - 1 + 2 * K::NQ) % K::NQ][v];
        const P2 &zp1 = q[(s - R + 1 + 2 * K::NQ) % K::NQ][v];
        const P2 &ctr = q[(s - R + 2 * K::NQ) % K::NQ][v];
        const ulonglong2 *pr = pc + row * K::KS + col + v * K::TX;  // this cell, plane t - R
        // distance-1 sum as a tree of pair sums (short dependency chains)
        const ulonglong2 xm1 = pr[-1], xp1 = pr[1];
        Acc2 A = pair_sum2(xm1.x, xm1.y, xp1.x, xp1.y);
        Acc2 Az = pair_sum2(zm1.h, zm1.l, zp1.h, zp1.l);
        if (NDIM == 3) {
          const ulonglong2 a = pr[-K::KS], b = pr[K::KS];
          const Acc2 Ay = pair_sum2(a.x, a.y, b.x, b.y);
          acc_add2(Az, Ay.s, Ay.c);
        }
        acc_add2(A, Az.s, Az.c);
        if (g.flags & PK_C1_POW2) {  // exact scaling
          A.s = rmul2(A.s, kc1, Z);
          A.c = rmul2(A.c, kc1, Z);
        } else {
          acc_scale2(A, kc1, nc1, Z);
        }
        {  // centre: TwoProduct of c0 * hi, plus c0 * lo
          const f2x p = rmul2(ctr.h, kc0, Z);
          f2x e = fma2(ctr.h, kc0, rmul2(ctr.h, nc0, Z));
          e = fma2(ctr.l, kc0, e);
          acc_add2(A, p, e);
        }
        if (R == 2) {
          const P2 &zm2 = q[(s - R - 2 + 2 * K::NQ) % K::NQ][v];
          const P2 &zp2 = q[(s - R + 2 + 2 * K::NQ) % K::NQ][v];
          const ulonglong2 xm2 = pr[-2], xp2 = pr[2];
          Acc2 B = pair_sum2(xm2.x, xm2.y, xp2.x, xp2.y);
          Acc2 Bz = pair_sum2(zm2.h, zm2.l, zp2.h, zp2.l);
          if (NDIM == 3) {
            const ulonglong2 a = pr[-2 * K::KS], b = pr[2 * K::KS];
            const Acc2 By = pair_sum2(a.x, a.y, b.x, b.y);
            acc_add2(Bz, By.s, By.c);
          }
          acc_add2(B, Bz.s, Bz.c);
          if (g.flags & PK_C2_MINUS1) {
            acc_sub2(A, B);
          } else {
            if (g.flags & PK_C2_POW2) {
              B.s = rmul2(B.s, kc2, Z);
              B.c = rmul2(B.c, kc2, Z);
            } else {
              acc_scale2(B, kc2, nc2, Z);
            }
            acc_add2(A, B.s, B.c);
          }
        }
        out[v] = acc_get2(A);
      }
      if (j >= zend || (NDIM == 3 && yy >= g.ny)) continue;
      const long long obase = (long long)j * (NDIM == 3 ? g.out_ss : g.out_sy) + (NDIM == 3 ? (long long)yy * g.out_sy : 0);
      if (PASS == 1) {
#pragma unroll
        for (int v = 0; v < K::VP; ++v) {
          const int cell = k0 + tx + v * K::TX;
          if (cell < g.nc) reinterpret_cast<ulonglong2 *>(yout)[obase + cell] = make_ulonglong2(out[v].h, out[v].l);
        }
      } else {
        const f2x sh = pk2(g.sh, g.sh), nsh = pk2(-g.sh, -g.sh), sl = pk2(g.sl, g.sl);
        const unsigned ebias = unsigned(1023 - 127 + g.sexp) << 20;
        double da[K::VP], db[K::VP];
#pragma unroll
        for (int v = 0; v < K::VP; ++v) {
          // z = out * scale (TwoProduct, |scale| in [1, 2): no overflow), then
          // the pair's 48 significant bits rebuilt exactly as a double
          const f2x p = rmul2(out[v].h, sh, Z);
          f2x e = fma2(out[v].h, sh, rmul2(out[v].h, nsh, Z));
          e = fma2(out[v].h, sl, e);
          e = fma2(out[v].l, sh, e);
          const f2x zh = add2(p, e);
          const f2x zl = sub2(e, sub2(zh, p));
          float ha, hb, la, lb;
          upk2(zh, ha, hb);
          upk2(zl, la, lb);
          da[v] = f2d_bits(ha, ebias, bad) + f2d_bits(la, ebias, bad);
          db[v] = f2d_bits(hb, ebias, bad) + f2d_bits(lb, ebias, bad);
        }
        double *yo = static_cast<double *>(yout) + obase;
        const int xa = k0 + tx - g.off_out, xb = xa + g.nc;
#pragma unroll
        for (int v = 0; v < K::VP; ++v) {
          if (k0 + tx + v * K::TX >= g.nc) continue;
          const int o = v * K::TX;
          if (xa + o >= 0 && xa + o < g.nx) yo[xa + o] = da[v];
          if (xb + o >= 0 && xb + o < g.nx) yo[xb + o] = db[v];
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


template <int NDIM, int R, int PASS>
static int launch_pk(const void *x, void *y, const int64_t *dims, int bc, const float *c, double scale, int *flag,
                     cudaStream_t st, int planes) {
  using K = PkPass<NDIM, R, PASS>;
  PkGeom g;
  std::memset(&g, 0, sizeof(g));
  g.nx = int(dims[0]);
  g.ny = int(dims[1]);
  g.nz = NDIM == 3 ? int(dims[2]) : 1;
  g.bc = bc == SC_BC_GHOSTED ? BC_GHOSTED : BC_PERIODIC;
  const int sh = bc == SC_BC_GHOSTED ? 2 * R : 0;
  // pass 1 folds its output rows (length nx); pass 2 folds its input rows
  // (length nx + 2R when ghosted) and writes the points that are outputs
  g.nf = PASS == 1 ? g.nx : g.nx + sh;
  g.nc = g.nf / 2;
  g.off_out = PASS == 1 ? 0 : sh / 2;
  const long long in_rows = (long long)g.ny + sh;
  if (PASS == 1) {
    g.in_sy = g.nx + sh;
    g.in_ss = (long long)(g.nx + sh) * in_rows;
    g.out_sy = g.nc;
    g.out_ss = (long long)g.nc * g.ny;
  } else {
    g.in_sy = g.nc;
    g.in_ss = (long long)g.nc * in_rows;
    g.out_sy = g.nx;
    g.out_ss = (long long)g.nx * g.ny;
  }
  g.c0 = c[0];
  g.c1 = c[1];
  g.c2 = c[2];
  auto pow2 = [](float v) {  // +-2^k: products are exact
    int e = 0;
    return v != 0.0f && std::fabs(std::frexp(v, &e)) == 0.5f;
  };
  g.flags = (pow2(c[1]) ? PK_C1_POW2 : 0) | (pow2(c[2]) ? PK_C2_POW2 : 0) | (c[2] == -1.0f ? PK_C2_MINUS1 : 0);
  if (PASS == 2) {  // scale = m * 2^e, m in [1, 2), m as an exact pair of floats
    int e = 0;
    const double m = std::frexp(scale, &e) * 2.0;
    g.sexp = e - 1;
    g.sh = float(m);
    g.sl = float(m - double(g.sh));
  }
  const int ns = NDIM == 3 ? g.nz : g.ny;
  const int gx = (g.nc + K::D - 1) / K::D;
  const long long txy = (long long)gx * (NDIM == 3 ? (g.ny + K::BY - 1) / K::BY : 1);
  auto kern = pk_lap_kernel<NDIM, R, PASS>;
  static std::atomic<unsigned long long> smem_set{0};
  set_smem_limit_once(kern, K::SMEM, smem_set);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, K::NTHR, K::SMEM);
  g.H = planes > 0 ? std::min(planes, ns)
                   : wave_planes(txy, ns, R, (long long)std::max(occ, 1) * num_sms(), std::max(4 * R, 8));
  dim3 grid(gx, NDIM == 3 ? (g.ny + K::BY - 1) / K::BY : (ns + g.H - 1) / g.H, NDIM == 3 ? (ns + g.H - 1) / g.H : 1);
  kern<<<grid, K::NTHR, K::SMEM, st>>>(x, y, g, flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SC_ECUDA, "pair-arithmetic apply launch: %s", cudaGetErrorString(e));
  return SC_OK;
}

template <int NDIM, int R>
static int pk_two_passes(const void *x, void *t, void *y, const int64_t *dims_t, const int64_t *dims_y, int bc,
                         const float *ca, const float *cb, double scale, int *flag, cudaStream_t st, int planes) {
  if (int rc = launch_pk<NDIM, R, 1>(x, t, dims_t, bc, ca, 1.0, flag, st, planes)) return rc;
  return launch_pk<NDIM, R, 2>(t, y, dims_y, bc, cb, scale, flag, st, planes);
}

bool df_supported(int ndim, int R, const int64_t *dims_y, int bc, double scale, const void *x, const void *t,
                  const void *y) {
  if (ndim < 2 || ndim > 3 || R < 1 || R > 2) return false;
  if (bc != SC_BC_PERIODIC && !(bc == SC_BC_GHOSTED && R == 2)) return false;
  if (dims_y[0] % 2 != 0 || dims_y[0] < 4) return false;
  if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(t) | reinterpret_cast<uintptr_t>(y)) & 15) != 0)
    return false;
  // the result's exponent stays inside the double range after re-biasing
  int e = 0;
  std::frexp(scale, &e);
  if (!(scale > 0.0) || e < -800 || e > 800) return false;
  // in-plane offsets are 32-bit
  const long long sh = bc == SC_BC_GHOSTED ? 4 * R : 0;
  const long long plane = ndim == 3 ? (dims_y[0] + sh) * (dims_y[1] + sh) : dims_y[0] + sh;
  return plane < (1LL << 31);
}

int df_composition_enqueue(int ndim, int R, const void *x, void *t, void *y, const int64_t *dims_t,
                           const int64_t *dims_y, int bc, const float *ca, const float *cb, double scale,
                           int *flag, cudaStream_t st, int planes) {
  if (ndim == 2)
    return R == 1 ? pk_two_passes<2, 1>(x, t, y, dims_t, dims_y, bc, ca, cb, scale, flag, st, planes)
                  : pk_two_passes<2, 2>(x, t, y, dims_t, dims_y, bc, ca, cb, scale, flag, st, planes);
  return R == 1 ? pk_two_passes<3, 1>(x, t, y, dims_t, dims_y, bc, ca, cb, scale, flag, st, planes)
                : pk_two_passes<3, 2>(x, t, y, dims_t, dims_y, bc, ca, cb, scale, flag, st, planes);
}

}  // namespace sc
