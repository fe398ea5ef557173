// Fused nested apply y = B(A x) in one pass (Eq. C=B(A), double-sum form),
// for factors that are sums of 1D stencils along the axes (STAR: every
// Laplacian), radius R <= 2, in FP32.
//
// The nested form needs 2 x (2 d R + 1) multiply-adds per point against the
// flat composed stencil's (4R+1)^d-ish support, but evaluated as two passes it
// writes and re-reads the intermediate t = A x through HBM, doubling the
// traffic of a bandwidth-bound operation.  Here t never leaves the SM:
//
// 3D.  A CTA owns BX x BY outputs of every z plane and streams H output
// planes.  Input planes of x pass through a shared-memory ring (cp.async, the
// boundary condition applied at load time).  Each thread owns a VX x VY block
// of the t region -- the tile grown by the outer factor's radius (rounded up
// to whole blocks) -- and keeps two register queues along z: its x values of
// the last 2R+1 input planes and its t values of the last 2R+1 t planes.
// When input plane p arrives, t(p - R) is formed from the queue (z terms)
// and the ring (in-plane terms) and written to a small shared ring of t
// planes; after a barrier, the threads whose block lies inside the tile form
// y(p - 2R) from their t queue and the t ring.  Each point of t is computed
// once per CTA (the halo blocks once more by the neighbouring CTA), each x and
// y value crosses HBM once.
//
// 2D.  A warp owns 4 * 32 consecutive t columns (the 120-wide output tile and
// 4 halo columns each side) and streams rows; x rows are read straight from
// global memory into registers (prefetched two rows ahead), in-row neighbours
// come from the adjacent lanes by warp shuffles, and the row-direction terms
// from the register queues.  No shared memory, no block barriers.
//
// Rounding: each factor's sum is formed in FP32 with FP32 weights (each
// correctly rounded from the exact rational), so the error is that of the
// two-pass nested evaluation, (2 n_A + 2) eps (|B| o |A|)|x| plus the weights'
// rounding, whatever the summation order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <type_traits>
#include <vector>

#include "sc_apply_host.h"
#include "sc_device.cuh"
#include "sc_internal.h"

namespace sc {

// Weights of a Laplacian-like factor: a sum of the same symmetric 1D
// stencil along every axis -- centre c (all axes' centre terms) and w[d - 1]
// at offsets -+d on each axis.  Held in registers by the kernels.
template <int R>
struct StarW {
  float c;
  float w[R];
};

template <int R>
struct FusedW {
  StarW<R> A, B;
};

// ---------------------------------------------------------------------------
// 3D
// ---------------------------------------------------------------------------

template <int R>
struct Fused3 {
  static constexpr int VX = 4, VY = 2;
  static constexpr int BX = 64, BY = 16;
  static constexpr int HXT = 4;                          // t halo columns (>= R, whole blocks)
  static constexpr int HYT = 2;                          // t halo rows (>= R, whole blocks)
  static constexpr int NBX = (BX + 2 * HXT) / VX;        // block columns of the t region
  static constexpr int NBY = (BY + 2 * HYT) / VY;        // block rows of the t region
  static constexpr int NTB = NBX * NBY;                  // t blocks (t warps, one block per thread)
  static constexpr int NTW = (NTB + 31) / 32;
  static constexpr int NYBX = BX / VX, NYBY = BY / VY;   // y blocks (y warps, one block per thread)
  static constexpr int NYW = NYBX * NYBY / 32;
  static constexpr int NTHR = 32 * (NTW + NYW);
  static constexpr int HXX = HXT + 4;                    // x halo columns (>= HXT + R, chunk multiple)
  static constexpr int XL = BX + 2 * HXX;                // x columns loaded per row
  // row pitches: two block rows apart is 8 banks apart, so a quarter warp
  // whose blocks wrap from the end of one block row to the next reads 32
  // distinct banks
  static constexpr int XC = XL % 16 == 4 ? XL : XL + ((4 - XL % 16) + 16) % 16;
  static constexpr int XR = BY + 2 * (HYT + R);          // x ring rows
  static constexpr int TL = BX + 2 * HXT;                // t columns
  static constexpr int TC = TL % 16 == 4 ? TL : TL + ((4 - TL % 16) + 16) % 16;
  static constexpr int TR = BY + 2 * HYT;                // t ring rows
  // ring depths equal the queue depth, so that every ring slot is a
  // compile-time index of the step loop unrolled over NQ steps
  static constexpr int NQ = 2 * R + 1;                   // queue depth
  static constexpr int NXS = NQ;                         // x ring planes
  static constexpr int PF = NXS - R - 1;                 // x planes in flight
  static constexpr int NTS = NQ;                         // t ring planes (>= R + 2)
  static constexpr int XPL = XC * XR, TPL = TC * TR;
  static constexpr int NCR = XL / 4;                     // 16-byte chunks per loaded row
  static constexpr int NCH = NCR * XR;                   // chunks per x plane
  static constexpr int CPT = (NCH + NTHR - 1) / NTHR;
  static constexpr size_t SMEM = size_t(NXS * XPL + NTS * TPL) * sizeof(float);
  static_assert(HXT >= R && HYT >= R && HXX >= HXT + R, "halo too small for the radius");
  static_assert(XL % 4 == 0 && XC % 16 == 4 && TC % 16 == 4, "pitches");
  static_assert(NYBX * NYBY % 32 == 0, "y blocks fill whole warps");
  static_assert(PF >= 1 && NTS >= R + 2, "ring depths");
};

struct FusedGeom {
  int nx, ny, nz;  // output grid
  int bc;          // BC_PERIODIC / BC_GHOSTED (ring 2R) / BC_ZERO
  int H;           // output planes per CTA
  int vec;         // 16-byte chunk copies legal
  long long in_sy, in_ss, out_sy, out_ss;
};

__device__ __forceinline__ float4 ld4s(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float f4at(const float4 &v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// f(integral_constant<int, I>) for I = B .. E-1 (compile-time step index).
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F &&f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// Packed FP32 pairs (sm_103a add/fma.rn.f32x2: two lanes per issue slot,
// each rounded as the scalar instruction would be).
typedef unsigned long long fpair;
__device__ __forceinline__ fpair fp_pk(float a, float b) {
  fpair d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ void fp_upk(fpair d, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(d));
}
__device__ __forceinline__ fpair fp_add(fpair a, fpair b) {
  fpair d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ fpair fp_mul(fpair a, fpair b) {
  fpair d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ fpair fp_fma(fpair a, fpair b, fpair c) {
  fpair d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// One STAR factor on a block of VY rows x 4 columns of plane k.  Q: the
// block's queue (slot C holds plane k, slots C -+ d planes k -+ d); row0:
// the block's first row in the ring (row pitch P).  The R rows above and
// below the block are read from the ring once, and each row's R left / right
// neighbours with one 4- or 8-byte load per side; everything else comes from
// the queue.  Every index is a compile-time constant, so nothing is copied.
// Arithmetic in packed FP32 pairs, points (0, 1) and (2, 3) of a row.
template <int R, int NQ, int VY, int C, int P>
__device__ __forceinline__ void star_block(const StarW<R> W, const float (&Q)[NQ][VY][4], const float *row0,
                                           float (&out)[VY][4]) {
  static_assert(R == 1 || R == 2, "radius 1 or 2");
  float4 up[R], dn[R];  // up[d - 1]: row -d; dn[d - 1]: row VY - 1 + d
#pragma unroll
  for (int d = 1; d <= R; ++d) {
    up[d - 1] = ld4s(row0 - d * P);
    dn[d - 1] = ld4s(row0 + (VY - 1 + d) * P);
  }
  const fpair wc = fp_pk(W.c, W.c);
  static_for<0, VY>([&](auto vc) {
    constexpr int VYI = decltype(vc)::value;
    const float *row = row0 + VYI * P;
    // the row with R neighbours each side: ext[R + i] is column i
    float ext[4 + 2 * R];
    if constexpr (R == 1) {
      ext[0] = row[-1];
      ext[5] = row[4];
    } else {
      const float2 a = *reinterpret_cast<const float2 *>(row - 2);
      const float2 b = *reinterpret_cast<const float2 *>(row + 4);
      ext[0] = a.x;
      ext[1] = a.y;
      ext[6] = b.x;
      ext[7] = b.y;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) ext[R + i] = Q[C][VYI][i];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int v = 2 * j;
      fpair s = fp_mul(wc, fp_pk(ext[R + v], ext[R + v + 1]));
#pragma unroll
      for (int d = 1; d <= R; ++d) {
        const fpair xm = fp_pk(ext[R + v - d], ext[R + v + 1 - d]);
        const fpair xp = fp_pk(ext[R + v + d], ext[R + v + 1 + d]);
        fpair ym, yp;
        if (VYI - d >= 0)
          ym = fp_pk(Q[C][(VYI - d) & (VY - 1)][v], Q[C][(VYI - d) & (VY - 1)][v + 1]);
        else
          ym = fp_pk(f4at(up[(d - VYI - 1) & (R - 1)], v), f4at(up[(d - VYI - 1) & (R - 1)], v + 1));
        if (VYI + d < VY)
          yp = fp_pk(Q[C][(VYI + d) & (VY - 1)][v], Q[C][(VYI + d) & (VY - 1)][v + 1]);
        else
          yp = fp_pk(f4at(dn[(VYI + d - VY) & (R - 1)], v), f4at(dn[(VYI + d - VY) & (R - 1)], v + 1));
        const fpair zm = fp_pk(Q[(C - d + NQ) % NQ][VYI][v], Q[(C - d + NQ) % NQ][VYI][v + 1]);
        const fpair zp = fp_pk(Q[(C + d) % NQ][VYI][v], Q[(C + d) % NQ][VYI][v + 1]);
        const fpair sum = fp_add(fp_add(fp_add(xm, xp), fp_add(ym, yp)), fp_add(zm, zp));
        s = fp_fma(fp_pk(W.w[d - 1], W.w[d - 1]), sum, s);
      }
      fp_upk(s, out[VYI][v], out[VYI][v + 1]);
    }
  });
}

// t warps (the first NTW): thread i < NTB owns t block (i % NBX, i / NBX)
// and keeps the x queue; y warps: thread j owns the output block
// (j % NYBX, j / NYBX) and keeps the t queue.  Step s (one barrier): x plane
// p_s = z0 - 2R + s has landed; t warps form t(p_s - R) while y warps form
// y(p_{s-1} - 2R) from the t planes written in earlier steps.
template <int R>
__global__ void __launch_bounds__(Fused3<R>::NTHR, 2)
    fused3_kernel(const float *__restrict__ x, float *__restrict__ y, FusedGeom g,
                  const __grid_constant__ FusedW<R> W) {
  using K = Fused3<R>;
  const StarW<R> WA = W.A, WB = W.B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *xr = reinterpret_cast<float *>(smem_raw);  // NXS planes of XC x XR
  float *tr = xr + K::NXS * K::XPL;                  // NTS planes of TC x TR
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * K::BX, y0 = blockIdx.y * K::BY, z0 = blockIdx.z * g.H;
  const int zend = min(z0 + g.H, g.nz);
  const int NT = (zend - z0) + 4 * R;  // input planes z0 - 2R .. zend + 2R - 1
  const int RING = 2 * R;               // ghost ring of a ghosted input
  const bool twarp = tid < 32 * K::NTW;

  // t warps: block (bc, br) of the t region; y warps: output block (bc, br)
  // of the tile, i.e. t block (bc + HXT/VX, br + HYT/VY)
  int bc, br;
  if (twarp) {
    bc = tid % K::NBX;
    br = tid / K::NBX;
  } else {
    const int j = tid - 32 * K::NTW;
    bc = j % K::NYBX + K::HXT / K::VX;
    br = j / K::NYBX + K::HYT / K::VY;
  }
  const bool towner = twarp && tid < K::NTB;
  const int xcol = K::HXX - K::HXT + K::VX * bc, xrow = R + K::VY * br;
  const int tcol = K::VX * bc, trow = K::VY * br;

  // 16-byte chunks of an x plane this thread copies: in-plane source offsets
  int coff[K::CPT], soff[K::CPT];
#pragma unroll
  for (int k = 0; k < K::CPT; ++k) {
    const int c = tid + k * K::NTHR;
    int o = -2;  // -2: no chunk, -1: zero fill
    soff[k] = 0;
    if (c < K::NCH) {
      const int r = c / K::NCR, cc = 4 * (c - r * K::NCR);
      const int ix = map_coord(x0 - K::HXX + cc, g.nx, g.bc, RING);
      const int iy = map_coord(y0 - K::HYT - R + r, g.ny, g.bc, RING);
      o = (ix >= 0 && iy >= 0) ? int((long long)iy * g.in_sy + ix) : -1;
      soff[k] = r * K::XC + cc;
    }
    coff[k] = o;
  }
  auto load_plane = [&](int s, int slot) {
    const int iz = map_coord(z0 - 2 * R + s, g.nz, g.bc, RING);
    float *dst = xr + slot * K::XPL;
    const long long pb = (long long)iz * g.in_ss;
    if (g.vec) {
#pragma unroll
      for (int k = 0; k < K::CPT; ++k) {
        if (coff[k] == -2) continue;
        const bool ok = iz >= 0 && coff[k] >= 0;
        cp_async16(dst + soff[k], ok ? x + pb + coff[k] : x, ok ? 16 : 0);
      }
    } else {
      for (int e = tid; e < K::XL * K::XR; e += K::NTHR) {
        const int r = e / K::XL, cc = e - r * K::XL;
        const int ix = map_coord(x0 - K::HXX + cc, g.nx, g.bc, RING);
        const int iy = map_coord(y0 - K::HYT - R + r, g.ny, g.bc, RING);
        const bool ok = iz >= 0 && ix >= 0 && iy >= 0;
        cp_async_elem<4>(dst + r * K::XC + cc, ok ? x + pb + (long long)iy * g.in_sy + ix : x, ok ? 4 : 0);
      }
    }
  };

  float q[K::NQ][K::VY][4];  // t warps: x of the block; y warps: t of the block

#pragma unroll
  for (int k = 0; k < K::PF; ++k) {
    if (k < NT) load_plane(k, k);
    cp_async_commit();
  }
  for (int sb = 0; sb <= NT; sb += K::NQ) {
    static_for<0, K::NQ>([&](auto uc) {
      constexpr int u = decltype(uc)::value;
      const int s = sb + u;
      if (s > NT) return;
      cp_async_wait<K::PF - 1>();
      __syncthreads();
      if (s + K::PF < NT) load_plane(s + K::PF, (u + K::PF) % K::NXS);
      cp_async_commit();
      if (twarp) {
        if (!towner || s >= NT) return;
        // ---- x(p_s) into the queue; t(q), q = p_s - R, once 2R planes are queued ----
        const float *xp = xr + u * K::XPL;
#pragma unroll
        for (int vy = 0; vy < K::VY; ++vy) {
          const float4 v = ld4s(xp + (xrow + vy) * K::XC + xcol);
          q[u][vy][0] = v.x;
          q[u][vy][1] = v.y;
          q[u][vy][2] = v.z;
          q[u][vy][3] = v.w;
        }
        if (s < 2 * R) return;
        const float *xc = xr + ((u - R + K::NQ) % K::NXS) * K::XPL;
        float *tw = tr + ((u - R + K::NQ) % K::NTS) * K::TPL + trow * K::TC + tcol;
        constexpr int CS = (u - R + K::NQ) % K::NQ;
        float out[K::VY][4];
        star_block<R, K::NQ, K::VY, CS, K::XC>(WA, q, xc + xrow * K::XC + xcol, out);
#pragma unroll
        for (int vy = 0; vy < K::VY; ++vy)
          *reinterpret_cast<float4 *>(tw + vy * K::TC) = make_float4(out[vy][0], out[vy][1], out[vy][2], out[vy][3]);
      } else {
        // ---- t(q'), q' = p_{s-1} - R, into the queue; y(q' - R) once 2R t planes are queued ----
        const int s1 = s - 1;
        if (s1 < 2 * R) return;
        constexpr int u1 = (u + K::NQ - 1) % K::NQ;
        const float *tq = tr + ((u1 - R + K::NQ) % K::NTS) * K::TPL;
#pragma unroll
        for (int vy = 0; vy < K::VY; ++vy) {
          const float4 v = ld4s(tq + (trow + vy) * K::TC + tcol);
          q[u1][vy][0] = v.x;
          q[u1][vy][1] = v.y;
          q[u1][vy][2] = v.z;
          q[u1][vy][3] = v.w;
        }
        if (s1 < 4 * R) return;
        const int j = z0 + s1 - 4 * R;
        const float *tc = tr + ((u1 - 2 * R + 2 * K::NQ) % K::NTS) * K::TPL + trow * K::TC + tcol;
        constexpr int CS = (u + K::NQ - 1 - R + K::NQ) % K::NQ;
        const int xo = x0 - K::HXT + tcol;
        float outb[K::VY][4];
        star_block<R, K::NQ, K::VY, CS, K::TC>(WB, q, tc, outb);
#pragma unroll
        for (int vy = 0; vy < K::VY; ++vy) {
          const float(&out)[4] = outb[vy];
          const int yy = y0 - K::HYT + trow + vy;
          if (yy < g.ny && j < zend) {
            float *dst = y + (long long)j * g.out_ss + (long long)yy * g.out_sy + xo;
            if (g.vec && xo + 4 <= g.nx) {
              __stcs(reinterpret_cast<float4 *>(dst), make_float4(out[0], out[1], out[2], out[3]));
            } else {
#pragma unroll
              for (int v = 0; v < 4; ++v)
                if (xo + v < g.nx) dst[v] = out[v];
            }
          }
        }
      }
    });
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// 2D
// ---------------------------------------------------------------------------

template <int R>
struct Fused2 {
  static constexpr int WARPS = 4;           // independent tiles per CTA
  static constexpr int NTHR = 32 * WARPS;
  static constexpr int TW = 128;            // t columns per warp (4 per lane)
  static constexpr int HXT = 4;             // t halo columns each side (one lane)
  static constexpr int BX = TW - 2 * HXT;   // 120 output columns per warp
  static constexpr int NQ = 2 * R + 1;
  static constexpr int PF = NQ;             // rows loaded ahead (slot of row s: s mod NQ)
  static_assert(HXT >= R, "halo too small for the radius");
};

struct Row4 {
  float v[4];
};

// The run of 4 values of input row `row` at the lane's columns (ix4: index
// of the run's first column for 16-byte loads, ixs: per-column indices
// otherwise; -1 outside the grid), boundary applied, zero outside.
__device__ __forceinline__ Row4 load_row4(const float *__restrict__ x, const FusedGeom &g, int ix4,
                                          const int (&ixs)[4], int row, int ring) {
  Row4 r;
  const int iy = map_coord(row, g.ny, g.bc, ring);
  r.v[0] = r.v[1] = r.v[2] = r.v[3] = 0.0f;
  if (iy < 0) return r;
  const float *rp = x + (long long)iy * g.in_sy;
  if (g.vec) {
    if (ix4 >= 0) {
      const float4 v = __ldcs(reinterpret_cast<const float4 *>(rp + ix4));
      r.v[0] = v.x;
      r.v[1] = v.y;
      r.v[2] = v.z;
      r.v[3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (ixs[i] >= 0) r.v[i] = __ldg(rp + ixs[i]);
  }
  return r;
}

// One STAR factor on a run of 4 values of row k: in-row terms from the
// neighbouring lanes, streaming-axis terms from the queue Q (slot C: row k,
// slots C -+ d: rows k -+ d).  Compile-time slots, nothing copied.
template <int R, int NQ, int C>
__device__ __forceinline__ void star_row2(const StarW<R> W, const float (&Q)[NQ][4], float (&out)[4]) {
  float lf[R], rt[R];  // lf[i]: column -R + i of the run, rt[i]: column 4 + i
#pragma unroll
  for (int i = 0; i < R; ++i) {
    lf[i] = __shfl_up_sync(0xffffffffu, Q[C][4 - R + i], 1);
    rt[i] = __shfl_down_sync(0xffffffffu, Q[C][i], 1);
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float s = W.c * Q[C][v];
#pragma unroll
    for (int d = 1; d <= R; ++d) {
      const float xm = v - d >= 0 ? Q[C][(v - d) & 3] : lf[(v - d + R) & (2 * R - 1)];
      const float xp = v + d < 4 ? Q[C][(v + d) & 3] : rt[(v + d - 4) & (2 * R - 1)];
      s = fmaf(W.w[d - 1], (xm + xp) + (Q[(C - d + NQ) % NQ][v] + Q[(C + d) % NQ][v]), s);
    }
    out[v] = s;
  }
}

template <int R>
__global__ void __launch_bounds__(Fused2<R>::NTHR)
    fused2_kernel(const float *__restrict__ x, float *__restrict__ y, FusedGeom g,
                  const __grid_constant__ FusedW<R> W) {
  using K = Fused2<R>;
  const StarW<R> WA = W.A, WB = W.B;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = blockIdx.x * K::WARPS + warp;
  const int x0 = tile * K::BX;
  if (x0 >= g.nx) return;  // whole warp: no shuffle partner is left behind
  const int c0 = x0 - K::HXT;
  const int z0 = blockIdx.y * g.H;
  const int zend = min(z0 + g.H, g.ny);
  const int NT = (zend - z0) + 4 * R;
  const int ring = 2 * R;
  const int xo = x0 + 4 * (lane - 1);
  const bool yowner = lane >= 1 && lane <= 30 && xo < x0 + K::BX;

  // the lane's columns: one 16-byte run (chunk-aligned: wholly in or out)
  const int c = c0 + 4 * lane;
  const int ix4 = map_coord(c, g.nx, g.bc, ring);
  int ixs[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) ixs[i] = map_coord(c + i, g.nx, g.bc, ring);
  float xq[K::NQ][4], tq[K::NQ][4];
  Row4 pre[K::PF];
#pragma unroll
  for (int k = 0; k < K::PF; ++k) pre[k] = load_row4(x, g, ix4, ixs, z0 - 2 * R + k, ring);

  for (int sb = 0; sb < NT; sb += K::NQ) {
    static_for<0, K::NQ>([&](auto uc) {
      constexpr int u = decltype(uc)::value;
      const int s = sb + u;
      if (s >= NT) return;
      // row s arrives in slot u, row s + PF is requested into the same slot
#pragma unroll
      for (int i = 0; i < 4; ++i) xq[u][i] = pre[u].v[i];
      if (s + K::PF < NT) pre[u] = load_row4(x, g, ix4, ixs, z0 - 2 * R + s + K::PF, ring);
      if (s < 2 * R) return;
      star_row2<R, K::NQ, (u - R + K::NQ) % K::NQ>(WA, xq, tq[u]);  // t(q), q = p - R
      if (s < 4 * R) return;
      float out[4];
      star_row2<R, K::NQ, (u - R + K::NQ) % K::NQ>(WB, tq, out);  // y(r), r = q - R
      const int j = z0 + s - 4 * R;
      if (yowner && j < zend) {
        float *dst = y + (long long)j * g.out_sy + xo;
        if (g.vec && xo + 4 <= g.nx) {
          __stcs(reinterpret_cast<float4 *>(dst), make_float4(out[0], out[1], out[2], out[3]));
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (xo + v < g.nx) dst[v] = out[v];
        }
      }
    });
  }
}

}  // namespace sc

namespace sc {

// Weights of a factor that is the same symmetric 1D stencil of radius <= R
// along every axis (a Laplacian); false for anything else.
template <int R>
static bool star_weights(const sc_stencil *s, int64_t hn, int64_t hd, StarW<R> &W) {
  std::vector<float> w(s->npts);
  if (weights_f32(s, hn, hd, w.data())) return false;
  float ax[3][2 * R + 1];
  bool seen[3][2 * R + 1];
  std::memset(ax, 0, sizeof(ax));
  std::memset(seen, 0, sizeof(seen));
  W.c = 0.0f;
  for (int k = 0; k < s->npts; ++k) {
    const int o[3] = {s->off[k][0], s->off[k][1], s->ndim == 3 ? s->off[k][2] : 0};
    int nz = 0, a = -1;
    for (int i = 0; i < 3; ++i)
      if (o[i]) {
        ++nz;
        a = i;
      }
    if (nz == 0) {
      W.c = w[k];
      continue;
    }
    if (nz > 1 || o[a] < -R || o[a] > R) return false;
    ax[a][o[a] + R] = w[k];
    seen[a][o[a] + R] = true;
  }
  for (int d = 1; d <= R; ++d) {
    W.w[d - 1] = ax[0][R + d];
    for (int a = 0; a < s->ndim; ++a)
      if (ax[a][R + d] != W.w[d - 1] || ax[a][R - d] != W.w[d - 1] || seen[a][R + d] != seen[0][R + d] ||
          seen[a][R - d] != seen[0][R + d])
        return false;
  }
  return true;
}

template <int R>
static int fused_launch(const sc_stencil *B, const sc_stencil *A, int bc, const int64_t *dims, int64_t hn,
                        int64_t hd, const float *x, float *y, int planes, cudaStream_t st) {
  FusedW<R> W;
  if (!star_weights<R>(A, hn, hd, W.A) || !star_weights<R>(B, hn, hd, W.B))
    return fail(SC_EINVAL, "fused apply: factors are not axis stencils of radius <= %d", R);
  const int nd = A->ndim;
  FusedGeom g;
  g.nx = int(dims[0]);
  g.ny = int(dims[1]);
  g.nz = nd == 3 ? int(dims[2]) : 1;
  g.bc = bc;
  const int sh = bc == SC_BC_GHOSTED ? 4 * R : 0;
  g.in_sy = g.nx + sh;
  g.in_ss = (long long)(g.nx + sh) * (g.ny + sh);
  g.out_sy = g.nx;
  g.out_ss = (long long)g.nx * g.ny;
  const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ya = reinterpret_cast<uintptr_t>(y);
  g.vec = (xa % 16 == 0) && (ya % 16 == 0) && (g.nx % 4 == 0) && (bc != SC_BC_GHOSTED || (2 * R) % 4 == 0);
  int occ = 0;
  cudaError_t e;
  if (nd == 3) {
    using K = Fused3<R>;
    auto kern = fused3_kernel<R>;
    static std::atomic<unsigned long long> smem_set{0};
    set_smem_limit_once(kern, K::SMEM, smem_set);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, K::NTHR, K::SMEM);
    const long long tiles = (long long)((g.nx + K::BX - 1) / K::BX) * ((g.ny + K::BY - 1) / K::BY);
    g.H = planes > 0 ? std::min(planes, g.nz)
                     : wave_planes(tiles, g.nz, 2 * R, (long long)std::max(occ, 1) * num_sms(), 16);
    dim3 grid((g.nx + K::BX - 1) / K::BX, (g.ny + K::BY - 1) / K::BY, (g.nz + g.H - 1) / g.H);
    kern<<<grid, K::NTHR, K::SMEM, st>>>(x, y, g, W);
  } else {
    using K = Fused2<R>;
    auto kern = fused2_kernel<R>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, K::NTHR, 0);
    const int ntile = (g.nx + K::BX - 1) / K::BX;
    const long long ctas_x = (ntile + K::WARPS - 1) / K::WARPS;
    g.H = planes > 0 ? std::min(planes, g.ny)
                     : wave_planes(ctas_x, g.ny, 2 * R, (long long)std::max(occ, 1) * num_sms(), 32);
    dim3 grid(unsigned(ctas_x), (g.ny + g.H - 1) / g.H);
    kern<<<grid, K::NTHR, 0, st>>>(x, y, g, W);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SC_ECUDA, "fused apply launch: %s", cudaGetErrorString(e));
  return SC_OK;
}

bool fused_supported(const sc_stencil *B, const sc_stencil *A, int dtype, int bc, const int64_t *dims) {
  if (dtype != SC_F32 || A->ndim != B->ndim || A->radius != B->radius) return false;
  const int R = A->radius;
  if (R < 1 || R > 2) return false;
  StarW<2> W;
  if (!star_weights<2>(A, 1, 1, W) || !star_weights<2>(B, 1, 1, W)) return false;
  if (bc == SC_BC_PERIODIC) {
    // one wrap must cover every halo a tile reads: 3D columns
    // [x0 - 8, x0 + 72), rows [y0 - 4, y0 + 20), planes [z0 - 4, zend + 4);
    // 2D columns [x0 - 4, x0 + 124), rows [z0 - 4, zend + 4)
    if (A->ndim == 3) return dims[0] >= 72 && dims[1] >= 24 && dims[2] >= 8;
    return dims[0] >= 128 && dims[1] >= 8;
  }
  return true;
}

int fused_enqueue(const sc_stencil *B, const sc_stencil *A, int dtype, int bc, const int64_t *dims, int64_t hn,
                  int64_t hd, const void *x, void *y, int planes, cudaStream_t st) {
  if (!fused_supported(B, A, dtype, bc, dims))
    return fail(SC_EINVAL, "fused apply: needs FP32 axis-stencil factors of equal radius 1 or 2 "
                           "(periodic grids of at least 72 x 24 x 8 in 3D, 128 x 8 in 2D)");
  const float *xf = static_cast<const float *>(x);
  float *yf = static_cast<float *>(y);
  return A->radius == 1 ? fused_launch<1>(B, A, bc, dims, hn, hd, xf, yf, planes, st)
                        : fused_launch<2>(B, A, bc, dims, hn, hd, xf, yf, planes, st);
}

}  // namespace sc
