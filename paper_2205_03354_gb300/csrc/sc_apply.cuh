// Flat composed-stencil apply, y_i = sum_k w_k x_{i+k} (Def. 2.1 evaluated
// at every grid point), as a device routine that streams one tile.
//
// Tile scheme ("scatter along the streaming axis"):
//  * the streaming axis S is y in 2D and z in 3D; a "plane" is the slab
//    orthogonal to it (a row in 2D, an xy tile in 3D);
//  * a CTA owns BX (x) by BY (y, 3D only) outputs of every plane and walks
//    H output planes; the NT = H + 2R input planes it needs are staged one by
//    one into a NSTAGE-deep shared-memory ring by cp.async, each with its
//    in-plane halo, the boundary condition applied at load time;
//  * each thread owns VX x VY outputs per plane and keeps 2R+1 register
//    accumulators per output (one for each pending output plane); when an
//    input plane arrives, its in-plane neighbourhood is read once from shared
//    memory and scattered into every pending output it reaches, so each
//    input value is touched once per thread and each output is stored once;
//  * the support of the stencil is a compile-time class (CROSS2 for every
//    Lap o Lap composition, BOX for anything within a small box), so the
//    point loop unrolls completely and zero weights cost nothing.
#pragma once
#include "sc_device.cuh"

namespace sc {

enum { CLS_BOX = 0, CLS_CROSS2 = 1, CLS_STAR = 2 };

// Is (dx, dy, dz) in the support class?  STAR(R): at most one nonzero
// component (a sum of 1D stencils along the axes, e.g. a Laplacian).
// CROSS2(R): STAR(R) plus the points with exactly two nonzero components
// both |.| <= R/2 -- the support of Lap o Lap for a Laplacian whose 1D
// stencils have radius R/2.  BOX(R): everything within radius R.
template <int CLS, int R>
__host__ __device__ constexpr bool in_support(int dx, int dy, int dz) {
  return CLS == CLS_BOX
             ? true
             : CLS == CLS_STAR
             ? (dx != 0) + (dy != 0) + (dz != 0) <= 1
             : ((dx != 0) + (dy != 0) + (dz != 0) <= 1
                    ? true
                    : ((dx != 0) + (dy != 0) + (dz != 0) == 2 && (dx < 0 ? -dx : dx) <= R / 2 &&
                       (dy < 0 ? -dy : dy) <= R / 2 && (dz < 0 ? -dz : dz) <= R / 2));
}

template <typename T, int NDIM, int R>
struct BoxWeights {
  static constexpr int W = 2 * R + 1;
  static constexpr int N = NDIM == 3 ? W * W * W : W * W;
  T w[N];
};

// Tile shape per (dtype, ndim, family); VX * sizeof(T) is a multiple of 16
// bytes.  Family 0: standalone streaming applies; family 1: the solver's
// tiles.  They are the same today (8 outputs per thread in 2D measured slower
// than 4); the split lets the two be tuned separately.
template <typename T, int NDIM, int FAM>
struct TileCfg;
template <>
struct TileCfg<float, 2, 0> {
  static constexpr int VX = 4, VY = 1, TX = 128, TY = 1;
};
template <>
struct TileCfg<double, 2, 0> {
  static constexpr int VX = 2, VY = 1, TX = 128, TY = 1;
};
// 2D solver tiles: TY warps stream TY independent row ranges of one
// TX * VX wide column (see FlatApply::WS), so narrow grids keep every lane
// busy and a small problem splits into many short tiles.
template <>
struct TileCfg<float, 2, 1> {
  static constexpr int VX = 2, VY = 1, TX = 32, TY = 4;
};
template <>
struct TileCfg<double, 2, 1> {
  static constexpr int VX = 2, VY = 1, TX = 32, TY = 4;
};
template <int FAM>
struct TileCfg<float, 3, FAM> {
  static constexpr int VX = 4, VY = 2, TX = 16, TY = 8;
};
template <int FAM>
struct TileCfg<double, 3, FAM> {
  static constexpr int VX = 2, VY = 2, TX = 32, TY = 4;
};

struct ApplyGeom {
  int nx, ny, nz;     // output (interior) dims; ny = 1 unused in 2D, nz = 1 in 2D
  int bc;             // BC_PERIODIC / BC_GHOSTED / BC_ZERO
  int H;              // output planes per CTA
  int vec;            // 1: 16-byte chunk loads are legal (alignment checked on host)
  long long in_sy;    // input row stride (elements)
  long long in_ss;    // input plane stride along the streaming axis (3D)
  long long out_sy;   // output row stride
  long long out_ss;   // output plane stride (3D)
};

template <typename T, int NDIM, int R, int CLS, int FAM = 0>
struct FlatApply {
  using Cfg = TileCfg<T, NDIM, FAM>;
  static constexpr int VX = Cfg::VX, VY = Cfg::VY, TX = Cfg::TX, TY = Cfg::TY;
  static constexpr int NTHR = TX * TY;
  static constexpr int BX = TX * VX;
  static constexpr int BY = NDIM == 3 ? TY * VY : 1;
  static constexpr int RP = NDIM == 3 ? R : 0;  // in-plane halo rows
  static constexpr int CH = 16 / sizeof(T);     // elements per 16-byte chunk
  static constexpr int HX = ((R + CH - 1) / CH) * CH;  // stored x halo (chunk multiple)
  static constexpr int PXS = BX + 2 * HX;       // smem row length
  static constexpr int PYS = BY + 2 * RP;       // smem rows per plane
  static constexpr int PLANE = PXS * PYS;
  // planes in the ring: streaming applies (family 0) keep 2 in flight; the
  // solver's short tiles (family 1) are L2-latency bound and keep more
  static constexpr int NSTAGE = FAM == 0 ? 3 : (NDIM == 2 ? 8 : 6);
  // the solver family keeps the R input planes behind the consumed one in the
  // ring, so that an epilogue reads each output's own input value from shared
  // memory; loads run NSTAGE - 1 - KEEP planes ahead
  static constexpr int KEEP = FAM == 1 ? R : 0;
  static constexpr int PD = NSTAGE - 1 - KEEP;
  static_assert(PD >= 1, "ring too short for the kept planes");
  static constexpr int NS = 2 * R + 1;          // pending output planes
  // Warp streams (2D solver family): warp w of the CTA streams output rows
  // [z0 + w H, z0 + (w + 1) H) of the tile's column with its own ring,
  // synchronising with __syncwarp; a tile spans TY * H rows.
  static constexpr bool WS = NDIM == 2 && FAM == 1;
  static constexpr int NSTREAM = WS ? TY : 1;
  static constexpr int LANES = WS ? TX : NTHR;  // threads sharing one ring
  static constexpr int NCHUNK = PLANE / CH;
  static constexpr int CPT = (NCHUNK + LANES - 1) / LANES;  // chunks per thread
  static constexpr size_t SMEM = size_t(NSTREAM) * NSTAGE * PLANE * sizeof(T);

  static __device__ __forceinline__ int lid() { return WS ? int(threadIdx.x) % TX : int(threadIdx.x); }
  static __device__ __forceinline__ void ring_sync() {
    if (WS)
      __syncwarp();
    else
      __syncthreads();
  }

  static __device__ __forceinline__ int wsidx(int ds, int dp, int dx) {
    return NDIM == 3 ? ((ds + R) * (2 * R + 1) + (dp + R)) * (2 * R + 1) + (dx + R)
                     : (ds + R) * (2 * R + 1) + (dx + R);
  }
  static __host__ __device__ constexpr bool supp(int dx, int dp, int ds) {
    return NDIM == 3 ? in_support<CLS, R>(dx, dp, ds) : (dp == 0 && in_support<CLS, R>(dx, ds, 0));
  }

  // Stages input plane `zs` (output coordinate along S, may be outside the
  // grid) of the tile (x0, y0) into `buf`: 16-byte cp.async.cg chunks (L2,
  // zero-filled outside the grid) when aligned, else element loads.
  static __device__ __forceinline__ void load_plane(const T *__restrict__ x, const ApplyGeom &g,
                                                    int x0, int y0, int zs, T *buf,
                                                    const int *coff) {
    const int ns = NDIM == 3 ? g.nz : g.ny;
    const int iz = map_coord(zs, ns, g.bc, R);
    const long long pbase = (long long)iz * (NDIM == 3 ? g.in_ss : g.in_sy);
    if (g.vec) {
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int c = lid() + k * LANES;
        if (c < NCHUNK) {
          const int o = coff[k];
          const bool ok = (iz >= 0) & (o >= 0);
          const T *src = ok ? x + pbase + o : x;
          cp_async16(buf + c * CH, src, ok ? 16 : 0);
        }
      }
    } else {
      for (int e = lid(); e < PLANE; e += LANES) {
        const int r = e / PXS, cc = e - r * PXS;
        const int gx = x0 - HX + cc;
        int ix = map_coord(gx, g.nx, g.bc, R);
        int iy = 0;
        if (NDIM == 3) iy = map_coord(y0 - RP + r, g.ny, g.bc, R);
        const bool ok = (iz >= 0) & (ix >= 0) & (iy >= 0);
        // plain L2 loads (not L1): persistent solvers rewrite x between tiles
        buf[e] = ok ? __ldcg(x + pbase + (long long)iy * g.in_sy + ix) : T(0);
      }
    }
  }

  // In-plane source offsets of this thread's 16-byte chunks (-1: zero fill).
  static __device__ __forceinline__ void chunk_offsets(const ApplyGeom &g, int x0, int y0,
                                                       int *coff) {
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int c = lid() + k * LANES;
      int o = -1;
      if (c < NCHUNK) {
        const int e = c * CH;
        const int r = e / PXS, cc = e - r * PXS;
        const int ix = map_coord(x0 - HX + cc, g.nx, g.bc, R);  // chunk-aligned
        int iy = 0;
        if (NDIM == 3) iy = map_coord(y0 - RP + r, g.ny, g.bc, R);
        if (ix >= 0 && iy >= 0) o = int((long long)iy * g.in_sy + ix);
      }
      coff[k] = o;
    }
  }

  // One tile: outputs [x0, x0+BX) x [y0, y0+BY) x planes [z0, z0+H).  WT
  // holds the dense weight box (member array w), EPI consumes every
  // completed run of VX outputs: epi(plane, row, first column, values).
  template <class WT, class EPI>
  static __device__ __forceinline__ void run_tile(const T *__restrict__ x, const ApplyGeom &g,
                                                  const WT &W, int x0, int y0, int z0, T *smem,
                                                  EPI &epi) {
    int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    if (WS) {  // this warp's row range and ring
      z0 += ty * g.H;
      smem += size_t(ty) * NSTAGE * PLANE;
      ty = 0;
    }
    const int ns = NDIM == 3 ? g.nz : g.ny;
    const int zend = min(z0 + g.H, ns);
    const int NT = zend > z0 ? (zend - z0) + 2 * R : 0;
    int coff[CPT];
    if (g.vec) chunk_offsets(g, x0, y0, coff);

    T acc[NS][VY][VX];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int a = 0; a < VY; ++a)
#pragma unroll
        for (int b = 0; b < VX; ++b) acc[s][a][b] = T(0);

#pragma unroll
    for (int k = 0; k < PD; ++k) {
      if (k < NT) load_plane(x, g, x0, y0, z0 - R + k, smem + k * PLANE, coff);
      cp_async_commit();
    }

    const int xo = x0 + tx * VX;  // first owned output column
    for (int tb = 0; tb < NT; tb += NS) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int t = tb + s;
        if (t >= NT) break;
        cp_async_wait<PD - 1>();
        ring_sync();
        {
          const int tl = t + PD;
          if (tl < NT) load_plane(x, g, x0, y0, z0 - R + tl, smem + (tl % NSTAGE) * PLANE, coff);
          cp_async_commit();
        }
        const T *pl = smem + (t % NSTAGE) * PLANE;
        // --- scatter this input plane into the pending outputs ---
#pragma unroll
        for (int ry = -RP; ry < VY + RP; ++ry) {
          T seg[VX + 2 * R];
          const T *row = pl + (ty * VY + ry + RP) * PXS + tx * VX + (HX - R);
#pragma unroll
          for (int i = 0; i < VX + 2 * R; ++i) seg[i] = row[i];
#pragma unroll
          for (int vy = 0; vy < VY; ++vy) {
            const int dp = ry - vy;
            if (dp < -RP || dp > RP) continue;
#pragma unroll
            for (int ds = -R; ds <= R; ++ds) {
              const int slot = ((s - R - ds) % NS + NS) % NS;
#pragma unroll
              for (int dx = -R; dx <= R; ++dx) {
                if (!supp(dx, dp, ds)) continue;
                const T w = W.w[wsidx(ds, dp, dx)];
#pragma unroll
                for (int vx = 0; vx < VX; ++vx)
                  acc[slot][vy][vx] = fma(w, seg[vx + dx + R], acc[slot][vy][vx]);
              }
            }
          }
        }
        // --- output plane z0 + t - 2R is complete ---
        {
          const int sc_ = ((s - 2 * R) % NS + NS) % NS;
          const int j = z0 + t - 2 * R;
          if (t >= 2 * R && j < zend) {
            // input plane j (consumed R steps ago) is still in the ring when KEEP
            const T *pj = smem + ((t - R) % NSTAGE) * PLANE;
#pragma unroll
            for (int vy = 0; vy < VY; ++vy) {
              const int yy = NDIM == 3 ? y0 + ty * VY + vy : 0;
              if (NDIM == 3 && yy >= g.ny) continue;
              const T *ctr = KEEP ? pj + (ty * VY + vy + RP) * PXS + tx * VX + HX : nullptr;
              epi(j, yy, xo, acc[sc_][vy], ctr);
            }
          }
#pragma unroll
          for (int vy = 0; vy < VY; ++vy)
#pragma unroll
            for (int vx = 0; vx < VX; ++vx) acc[sc_][vy][vx] = T(0);
        }
      }
    }
    cp_async_wait<0>();
    __syncthreads();  // the ring may be reused by the caller
  }
};

// Stores the outputs: y = acc (a plain apply).
template <typename T, int NDIM, int VX>
struct StoreEpi {
  T *__restrict__ y;
  const ApplyGeom *g;
  __device__ __forceinline__ void operator()(int j, int yy, int xo, const T (&v)[VX], const T *) const {
    T *dst = y + (long long)j * (NDIM == 3 ? g->out_ss : g->out_sy) +
             (NDIM == 3 ? (long long)yy * g->out_sy : 0) + xo;
    if (g->vec && xo + VX <= g->nx && (sizeof(T) * VX) % 16 == 0) {
#pragma unroll
      for (int c = 0; c < VX; c += 16 / int(sizeof(T))) {
        if (sizeof(T) == 4) {
          *reinterpret_cast<float4 *>(dst + c) = make_float4(float(v[c]), float(v[(c + 1) % VX]),
                                                              float(v[(c + 2) % VX]), float(v[(c + 3) % VX]));
        } else {
          *reinterpret_cast<double2 *>(dst + c) = make_double2(double(v[c]), double(v[(c + 1) % VX]));
        }
      }
    } else {
#pragma unroll
      for (int vx = 0; vx < VX; ++vx)
        if (xo + vx < g->nx) dst[vx] = v[vx];
    }
  }
};

}  // namespace sc
