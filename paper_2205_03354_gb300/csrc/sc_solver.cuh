// Persistent batched conjugate-gradient engine.
//
// One cooperative launch solves a batch of independent SPD systems
//     (a I + b B) x = rhs,   B = a composed stencil (Lap o Lap) on a 2D or 3D grid,
// of uneven sizes.  Every problem owns a contiguous group of CTAs; a group
// advances its own CG iteration with group barriers (global-memory counters,
// bounded spins), so small problems never wait for large ones.
//
// Per CG iteration (inner precision TI = float or double):
//   A:  q = (a I + b B) p              tile apply; partial p.q per tile
//   B:  d += alpha p, rh -= alpha q    chunked vector pass; partial rh.rh
//   C:  p = rh + beta p                chunked vector pass
// with a group barrier after each phase.  Reductions are deterministic: every
// tile/chunk writes its partial to a fixed slot and the slots are summed in
// index order (by every CTA of a small group, by the last CTA to arrive in a
// large one), so a problem's result does not depend on its group size or on
// the rest of the batch.
//
// Mixed precision (TI = float): FP32 stencil applies and vector updates; the
// FP64 solution x, right-hand side and true residual r = rhs - A x are kept in
// FP64 and refreshed by reliable updates (Sleijpen & van der Vorst 1996):
// whenever the FP32 recurrence residual has dropped by the factor `delta`
// since the last refresh, or meets the tolerance, x += d in FP64, the FP64
// residual is recomputed with an FP64 apply and becomes the new FP32
// residual (the search direction is kept).  Convergence is only declared on
// the FP64 true residual.
#pragma once
#include "../../include/stencilcomp.h"
#include "sc_apply.cuh"

namespace sc {

enum { ST_RUNNING = 0, ST_DONE = 1 };

struct SolveState {
  long long iters;   // inner iterations so far
  long long outer;   // reliable updates (FP64 residual refreshes)
  double rr;         // current recurrence residual^2 (inner precision)
  double rmax;       // |rh| at the last refresh (mixed)
  double bnorm;      // |rhs|_2
  double rel;        // last true relative residual
  double sumb;       // sum(rhs) (mean fix)
  int status;        // SC_OK while running / final status
  int phase;         // 0 = not started, 1 = iterating, 2 = finished
  double beta;       // pending beta for phase C
};

struct SolveProb {
  int ndim, nx, ny, nz, bc;
  long long npts;
  int H_in, H_64;            // planes per apply tile (inner, FP64 tile shapes)
  int ntiles_in, ntiles_64;  // tile counts
  int nchunks;               // vector-phase chunks
  int chunk;                 // elements per chunk: CG_STEP * 2^k, fixed by the problem size
  int nslot;                 // partial slots per reduction value
  int cta0, ncta;            // CTA group
  double a, b;               // operator a I + b B
  int mixed, mean_fix;
  int vec_in, vec_64;        // 16-byte tile loads legal (alignment checked on host)
  int vec_v;                 // 16-byte vector-phase loads legal (aligned vectors, npts % 4 == 0)
  double rtol, delta;
  long long maxit;
  const double *w64;         // dense weight box of B (FP64)
  const void *wT;            // the same in the inner type
  double *x, *rhs, *r;       // FP64 vectors
  void *rh, *p, *q, *d;      // inner vectors (FP64 path: rh == r, d == x)
  double *part;              // 3 * nslot partial sums
  double *scal;              // 4 published scalars
  unsigned *bar;             // [0] arrival counter, [1] release generation
  SolveState *st;
};

constexpr int CG_NTHR = 128;
constexpr int CG_STEP = CG_NTHR * 4;      // elements per vector-phase step (4 per thread)
constexpr int CG_CHUNK = CG_STEP * 8;     // largest chunk used for sizing scratch (see P.chunk)
constexpr long long SPIN_LIMIT = 1LL << 24;  // ~1-2 s with the back-off below
// group reductions whose CTAs x partials x values stay below this read all
// partials in every CTA instead of waiting for a published result
constexpr long long ALLREAD_MAX = 16384;

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Group barrier that also reduces `nval` partial arrays (part[k*nslot + i],
// i < nused) in index order; the sums are returned in out[0..nval-1] in every
// CTA of the group.  Returns false when a wait timed out (the problem is then
// marked SC_ETIMEOUT and every CTA of the group leaves).
//
// The partial slots are double-buffered by the parity of the reduction's
// sequence number: the phase before reduction k writes buffer k & 1 and the
// reduction reads it.  In the small-group protocol every CTA reads the slots
// after the arrival count alone, so a CTA that finished reading may already
// write the next phase's partials while a slower one still reads; those go to
// the other buffer, and no CTA can write buffer k & 1 again before every CTA
// has arrived at reduction k + 1, i.e. finished reading reduction k.
struct GroupCtx {
  const SolveProb *P;
  int rank;
  unsigned target;  // arrival count to wait for
  unsigned gen;     // release generation
  double *red;      // shared scratch (>= CG_NTHR/32 doubles)
  int *flag;        // shared int
  long long spin_limit = SPIN_LIMIT;
  unsigned nred = 0;  // reductions completed in this launch (selects the slot buffer)
};

// The partial slots the next reduction of this group reads (3 * nslot values).
__device__ __forceinline__ double *cur_part(const GroupCtx &G) {
  return G.P->part + (G.nred & 1u) * 3LL * G.P->nslot;
}

__device__ __forceinline__ double fixed_sum(const double *a, int n, double *red) {
  // thread t adds slots t, t + 128, ... in order; 8 loads in flight
  double s = 0.0;
  int i = threadIdx.x;
  for (; i + 7 * CG_NTHR < n; i += 8 * CG_NTHR) {
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __ldcg(a + i + k * CG_NTHR);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
  }
  for (; i < n; i += CG_NTHR) s += __ldcg(a + i);
  return block_sum<CG_NTHR>(s, red);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// With deadline != 0 the reducing CTA also reads the global timer and
// publishes out[3] = 1.0 when it is past the deadline, so that every CTA of
// the group takes the same stop decision.
__device__ inline bool group_reduce(GroupCtx &G, int nval, int nused, double *out,
                             unsigned long long deadline = 0ull) {
  const SolveProb &P = *G.P;
  const double *part = cur_part(G);
  __shared__ double s_out[4];
  __syncthreads();
  bool ok = true;
  if (P.ncta == 1) {
    for (int k = 0; k < nval; ++k) {
      __threadfence_block();
      double v = fixed_sum(part + (long long)k * P.nslot, nused, G.red);
      if (threadIdx.x == 0) s_out[k] = v;
    }
    if (deadline && threadIdx.x == 0) s_out[3] = global_ns() >= deadline ? 1.0 : 0.0;
    __syncthreads();
  } else if (deadline == 0ull && (long long)P.ncta * nused * nval <= ALLREAD_MAX) {
    // small group: every CTA waits for the arrival count alone and then sums
    // the partials itself in the same fixed order (the same bits in every
    // CTA), one publish round trip shorter than the path below
    G.target += P.ncta;
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&P.bar[0], 1u);
      long long spins = 0;
      *G.flag = 0;
      while (ld_acquire(&P.bar[0]) < G.target) {
        if (++spins > G.spin_limit) {
          *G.flag = -1;
          break;
        }
        __nanosleep(32);
      }
    }
    __syncthreads();
    if (*G.flag == -1) {
      ok = false;
      if (threadIdx.x == 0) {
        P.st->status = SC_ETIMEOUT;
        P.st->phase = 2;
      }
    } else {
      __threadfence();
      for (int k = 0; k < nval; ++k) {
        const double v = fixed_sum(part + (long long)k * P.nslot, nused, G.red);
        if (threadIdx.x == 0) s_out[k] = v;
      }
    }
    __syncthreads();
  } else {
    G.target += P.ncta;
    G.gen += 1;
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned old = atomicAdd(&P.bar[0], 1u);
      *G.flag = (old == G.target - 1) ? 1 : 0;
    }
    __syncthreads();
    if (*G.flag) {  // last to arrive: reduce in fixed order and publish
      __threadfence();
      for (int k = 0; k < nval; ++k) {
        double v = fixed_sum(part + (long long)k * P.nslot, nused, G.red);
        if (threadIdx.x == 0) P.scal[k] = v;
      }
      if (deadline && threadIdx.x == 0) P.scal[3] = global_ns() >= deadline ? 1.0 : 0.0;
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(&P.bar[1], G.gen);
      }
    } else if (threadIdx.x == 0) {
      long long spins = 0;
      while (ld_acquire(&P.bar[1]) < G.gen) {
        if (++spins > G.spin_limit) {
          *G.flag = -1;
          break;
        }
        __nanosleep(64);
      }
    }
    __syncthreads();
    if (*G.flag == -1) {
      ok = false;
      if (threadIdx.x == 0) {
        P.st->status = SC_ETIMEOUT;
        P.st->phase = 2;
      }
    }
    if (threadIdx.x == 0 && ok) {
      __threadfence();
      for (int k = 0; k < nval; ++k) s_out[k] = __ldcg(P.scal + k);
      if (deadline) s_out[3] = __ldcg(P.scal + 3);
    }
    __syncthreads();
  }
  for (int k = 0; k < nval; ++k) out[k] = s_out[k];
  if (deadline) out[3] = s_out[3];
  G.nred += 1;
  __syncthreads();
  return ok;
}

template <typename T, int NDIM, int R>
struct WBox {
  T w[BoxWeights<T, NDIM, R>::N];
};

// Epilogue of the CG apply: q = a p + b (B p), partial p.q.
template <typename T, int NDIM, int VX>
struct CgApplyEpi {
  const T *__restrict__ p;
  T *__restrict__ q;
  long long sy, ss;
  int nx;
  T a, b;
  T dot;  // this thread's partial p.q, accumulated in the inner type (FP32
          // inner iterations accumulate in FP32; the group sum is FP64)
  // ctr: p at the VX outputs, from the tile's shared-memory ring
  __device__ __forceinline__ void operator()(int j, int yy, int xo, const T (&v)[VX], const T *ctr) {
    const long long base = (long long)j * (NDIM == 3 ? ss : sy) + (NDIM == 3 ? (long long)yy * sy : 0);
#pragma unroll
    for (int vx = 0; vx < VX; ++vx) {
      if (xo + vx < nx) {
        const long long i = base + xo + vx;
        const T pv = ctr[vx];
        const T qv = a * pv + b * v[vx];
        q[i] = qv;
        dot = fma(pv, qv, dot);
      }
    }
  }
};

// Epilogue of the FP64 residual: r = rhs - (a x + b (B x)), partial r.r.
template <int NDIM, int VX>
struct ResidEpi {
  const double *__restrict__ x;
  const double *__restrict__ rhs;
  double *__restrict__ r;
  long long sy, ss;
  int nx;
  double a, b, dot;
  // ctr: x at the VX outputs, from the tile's shared-memory ring
  __device__ __forceinline__ void operator()(int j, int yy, int xo, const double (&v)[VX], const double *ctr) {
    const long long base = (long long)j * (NDIM == 3 ? ss : sy) + (NDIM == 3 ? (long long)yy * sy : 0);
#pragma unroll
    for (int vx = 0; vx < VX; ++vx) {
      if (xo + vx < nx) {
        const long long i = base + xo + vx;
        const double rv = __ldcg(rhs + i) - fma(b, v[vx], a * ctr[vx]);
        r[i] = rv;
        dot += rv * rv;
      }
    }
  }
};

template <typename T, int NDIM, int R>
__device__ __forceinline__ ApplyGeom cg_geom(const SolveProb &P, int H) {
  ApplyGeom g;
  g.nx = P.nx;
  g.ny = P.ny;
  g.nz = NDIM == 3 ? P.nz : 1;
  g.bc = P.bc;
  g.H = H;
  g.vec = sizeof(T) == 8 ? P.vec_64 : P.vec_in;
  g.in_sy = P.nx;
  g.in_ss = (long long)P.nx * P.ny;
  g.out_sy = P.nx;
  g.out_ss = (long long)P.nx * P.ny;
  return g;
}

template <typename K>
__device__ __forceinline__ void tile_origin(const SolveProb &P, int tile, int H, int ndim, int &x0,
                                            int &y0, int &z0) {
  const int tx = (P.nx + K::BX - 1) / K::BX;
  if (ndim == 3) {
    const int ty = (P.ny + K::BY - 1) / K::BY;
    x0 = (tile % tx) * K::BX;
    y0 = ((tile / tx) % ty) * K::BY;
    z0 = (tile / (tx * ty)) * H;
  } else {
    x0 = (tile % tx) * K::BX;
    y0 = 0;
    z0 = (tile / tx) * H * K::NSTREAM;
  }
}

// The problem's weight boxes, staged in shared memory once per launch.
struct CgWeights {
  double w64[125];
  float w32[125];
};

// Phase A: q = A p over the group's tiles.
template <typename T, int NDIM, int R>
__device__ void phase_apply(const SolveProb &P, int rank, unsigned char *smem, double *red,
                            const CgWeights &cw, double *part) {
  using K = FlatApply<T, NDIM, R, CLS_CROSS2, 1>;
  const ApplyGeom g = cg_geom<T, NDIM, R>(P, P.H_in);
  const WBox<T, NDIM, R> &W = *reinterpret_cast<const WBox<T, NDIM, R> *>(
      sizeof(T) == 8 ? static_cast<const void *>(cw.w64) : static_cast<const void *>(cw.w32));
  for (int tile = rank; tile < P.ntiles_in; tile += P.ncta) {
    int x0, y0, z0;
    tile_origin<K>(P, tile, P.H_in, NDIM, x0, y0, z0);
    CgApplyEpi<T, NDIM, K::VX> epi{static_cast<const T *>(P.p), static_cast<T *>(P.q), g.out_sy,
                                   g.out_ss, P.nx, T(P.a), T(P.b), T(0)};
    K::run_tile(static_cast<const T *>(P.p), g, W, x0, y0, z0, reinterpret_cast<T *>(smem), epi);
    const double s = block_sum<CG_NTHR>(double(epi.dot), red);
    if (threadIdx.x == 0) part[tile] = s;
  }
}

// FP64 residual r = rhs - A x over the FP64 tiles; partial r.r in slot 0 and
// (when mean_fix) partial sum(x) in slot 1.
template <int NDIM, int R>
__device__ void phase_resid(const SolveProb &P, int rank, unsigned char *smem, double *red,
                            const CgWeights &cw, double *part) {
  using K = FlatApply<double, NDIM, R, CLS_CROSS2, 1>;
  const ApplyGeom g = cg_geom<double, NDIM, R>(P, P.H_64);
  const WBox<double, NDIM, R> &W = *reinterpret_cast<const WBox<double, NDIM, R> *>(cw.w64);
  for (int tile = rank; tile < P.ntiles_64; tile += P.ncta) {
    int x0, y0, z0;
    tile_origin<K>(P, tile, P.H_64, NDIM, x0, y0, z0);
    ResidEpi<NDIM, K::VX> epi{P.x, P.rhs, P.r, g.out_sy, g.out_ss, P.nx, P.a, P.b, 0.0};
    K::run_tile(P.x, g, W, x0, y0, z0, reinterpret_cast<double *>(smem), epi);
    const double s = block_sum<CG_NTHR>(epi.dot, red);
    if (threadIdx.x == 0) part[tile] = s;
  }
}

// Vector phases over fixed chunks of P.chunk elements (chunk c is always
// handled by group rank c % ncta, in a fixed element order).  KIND:
//  0: init     rh = TI(r), p = rh, d = 0 (mixed); partials rh.rh, rhs.rhs, sum(rhs)
//  1: update   d += alpha p, rh -= alpha q; partial rh.rh
//  2: direction p = rh + beta p
//  3: refresh  x += d, d = 0 (mixed)
//  4: to-inner rh = TI(r); partial rh.rh
//  5: sum(x)   partial
//  6: shift    x += c
// Each thread moves 4 consecutive elements per step (16-byte loads for FP32,
// two for FP64) and keeps up to 4 steps in flight; all loads go through L2.

template <typename T>
__device__ __forceinline__ void ld4(const T *p, T (&v)[4]) {
  if (sizeof(T) == 4) {
    const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
    v[0] = T(t.x); v[1] = T(t.y); v[2] = T(t.z); v[3] = T(t.w);
  } else {
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = T(a.x); v[1] = T(a.y); v[2] = T(b.x); v[3] = T(b.y);
  }
}
template <typename T>
__device__ __forceinline__ void st4(T *p, const T (&v)[4]) {
  if (sizeof(T) == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(float(v[0]), float(v[1]), float(v[2]), float(v[3]));
  } else {
    reinterpret_cast<double2 *>(p)[0] = make_double2(double(v[0]), double(v[1]));
    reinterpret_cast<double2 *>(p)[1] = make_double2(double(v[2]), double(v[3]));
  }
}

template <typename TI, int KIND>
__device__ __forceinline__ void vec_elems(const SolveProb &P, long long i, int n, double s1, double &a0,
                                          double &a1, double &a2) {
  // scalar fallback for ragged or unaligned data, n <= 4 elements from i
  TI *rh = static_cast<TI *>(P.rh), *p = static_cast<TI *>(P.p), *q = static_cast<TI *>(P.q),
     *d = static_cast<TI *>(P.d);
  for (int k = 0; k < n; ++k, ++i) {
    if (KIND == 0) {
      const TI v = TI(__ldcg(P.r + i));
      rh[i] = v;
      p[i] = v;
      if (P.mixed) d[i] = TI(0);
      const double bv = __ldcg(P.rhs + i);
      a0 += double(v) * double(v);
      a1 += bv * bv;
      a2 += bv;
    } else if (KIND == 1) {
      const TI al = TI(s1);
      const TI pv = __ldcg(p + i);
      d[i] = __ldcg(d + i) + al * pv;
      const TI v = __ldcg(rh + i) - al * __ldcg(q + i);
      rh[i] = v;
      a0 += double(v * v);
    } else if (KIND == 2) {
      p[i] = __ldcg(rh + i) + TI(s1) * __ldcg(p + i);
    } else if (KIND == 3) {
      P.x[i] = __ldcg(P.x + i) + double(__ldcg(d + i));
      d[i] = TI(0);
    } else if (KIND == 4) {
      const TI v = TI(__ldcg(P.r + i));
      rh[i] = v;
      a0 += double(v) * double(v);
    } else if (KIND == 5) {
      a0 += __ldcg(P.x + i);
    } else {
      P.x[i] = __ldcg(P.x + i) + s1;
    }
  }
}

template <typename TI, int KIND>
__device__ void phase_vec(const SolveProb &P, int rank, double s1, double *red, double *part) {
  TI *rh = static_cast<TI *>(P.rh), *p = static_cast<TI *>(P.p), *q = static_cast<TI *>(P.q),
     *d = static_cast<TI *>(P.d);
  for (int c = rank; c < P.nchunks; c += P.ncta) {
    const long long e0 = (long long)c * P.chunk;
    const long long e1 = min(e0 + P.chunk, P.npts);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    TI acc_t = TI(0);  // the update's partial rh.rh in the inner type (FP32 accumulation)
    if ((KIND == 1 || KIND == 2) && P.vec_v && e1 - e0 == P.chunk && P.chunk >= 2 * CG_STEP) {
      // the per-iteration updates: two steps' loads issued before any store
      // (the vectors may alias as far as the compiler knows, so it would not
      // hoist them itself); chunks are CG_STEP * 2^k
      const int nsteps = P.chunk / CG_STEP;
      for (int k = 0; k < nsteps; k += 2) {
        const long long i0 = e0 + 4LL * (k * CG_NTHR + threadIdx.x), i1 = i0 + 4LL * CG_NTHR;
        if (KIND == 1) {
          TI pv[2][4], dv[2][4], rv[2][4], qv[2][4];
          ld4(p + i0, pv[0]);
          ld4(p + i1, pv[1]);
          ld4(d + i0, dv[0]);
          ld4(d + i1, dv[1]);
          ld4(rh + i0, rv[0]);
          ld4(rh + i1, rv[1]);
          ld4(q + i0, qv[0]);
          ld4(q + i1, qv[1]);
          const TI al = TI(s1);
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              dv[h][j] = dv[h][j] + al * pv[h][j];
              rv[h][j] = rv[h][j] - al * qv[h][j];
              acc_t = fma(rv[h][j], rv[h][j], acc_t);
            }
          st4(d + i0, dv[0]);
          st4(d + i1, dv[1]);
          st4(rh + i0, rv[0]);
          st4(rh + i1, rv[1]);
        } else {
          TI pv[2][4], rv[2][4];
          ld4(p + i0, pv[0]);
          ld4(p + i1, pv[1]);
          ld4(rh + i0, rv[0]);
          ld4(rh + i1, rv[1]);
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j) pv[h][j] = rv[h][j] + TI(s1) * pv[h][j];
          st4(p + i0, pv[0]);
          st4(p + i1, pv[1]);
        }
      }
    } else if (P.vec_v && e1 - e0 == P.chunk) {
      const int nsteps = P.chunk / CG_STEP;
#pragma unroll 4
      for (int k = 0; k < nsteps; ++k) {
        const long long i = e0 + 4LL * (k * CG_NTHR + threadIdx.x);
        if (KIND == 0) {
          double r[4], b[4];
          ld4(P.r + i, r);
          ld4(P.rhs + i, b);
          TI v[4], z[4] = {TI(0), TI(0), TI(0), TI(0)};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            v[j] = TI(r[j]);
            a0 += double(v[j]) * double(v[j]);
            a1 += b[j] * b[j];
            a2 += b[j];
          }
          st4(rh + i, v);
          st4(p + i, v);
          if (P.mixed) st4(d + i, z);
        } else if (KIND == 1) {
          TI pv[4], dv[4], rv[4], qv[4];
          ld4(p + i, pv);
          ld4(d + i, dv);
          ld4(rh + i, rv);
          ld4(q + i, qv);
          const TI al = TI(s1);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            dv[j] = dv[j] + al * pv[j];
            rv[j] = rv[j] - al * qv[j];
            acc_t = fma(rv[j], rv[j], acc_t);
          }
          st4(d + i, dv);
          st4(rh + i, rv);
        } else if (KIND == 2) {
          TI pv[4], rv[4];
          ld4(p + i, pv);
          ld4(rh + i, rv);
#pragma unroll
          for (int j = 0; j < 4; ++j) pv[j] = rv[j] + TI(s1) * pv[j];
          st4(p + i, pv);
        } else if (KIND == 3) {
          double xv[4];
          TI dv[4], z[4] = {TI(0), TI(0), TI(0), TI(0)};
          ld4(P.x + i, xv);
          ld4(d + i, dv);
#pragma unroll
          for (int j = 0; j < 4; ++j) xv[j] += double(dv[j]);
          st4(P.x + i, xv);
          st4(d + i, z);
        } else if (KIND == 4) {
          double r[4];
          ld4(P.r + i, r);
          TI v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            v[j] = TI(r[j]);
            a0 += double(v[j]) * double(v[j]);
          }
          st4(rh + i, v);
        } else if (KIND == 5) {
          double xv[4];
          ld4(P.x + i, xv);
#pragma unroll
          for (int j = 0; j < 4; ++j) a0 += xv[j];
        } else {
          double xv[4];
          ld4(P.x + i, xv);
#pragma unroll
          for (int j = 0; j < 4; ++j) xv[j] += s1;
          st4(P.x + i, xv);
        }
      }
    } else {
      for (long long i = e0 + 4LL * threadIdx.x; i < e1; i += 4LL * CG_NTHR)
        vec_elems<TI, KIND>(P, i, int(min(4LL, e1 - i)), s1, a0, a1, a2);
    }
    if (KIND == 0 || KIND == 1 || KIND == 4 || KIND == 5) {
      const double t0 = block_sum<CG_NTHR>(a0 + double(acc_t), red);
      if (threadIdx.x == 0) part[c] = t0;
      if (KIND == 0) {
        const double t1 = block_sum<CG_NTHR>(a1, red);
        if (threadIdx.x == 0) part[P.nslot + c] = t1;
        const double t2 = block_sum<CG_NTHR>(a2, red);
        if (threadIdx.x == 0) part[2 * P.nslot + c] = t2;
      }
    }
  }
}

__device__ __forceinline__ bool finite_pos(double v) { return v > 0.0 && v < 1.0e300; }

// Runs one problem for at most `budget` inner iterations.
// Runs one problem for at most `budget` inner iterations and, when slice_ns
// is nonzero, for about that long (the global timer is compared once per
// iteration by the reducing CTA, so the whole group stops together); the
// state is saved for the next launch.
template <typename TI, int NDIM, int R>
__device__ void cg_run(GroupCtx &G, unsigned char *smem, long long budget,
                       unsigned long long slice_ns) {
  const SolveProb &P = *G.P;
  const unsigned long long deadline = slice_ns ? global_ns() + slice_ns : 0ull;
  __shared__ CgWeights cw;
  {
    constexpr int NB = NDIM == 3 ? 125 : 25;
    for (int i = threadIdx.x; i < NB; i += CG_NTHR) {
      cw.w64[i] = P.w64[i];
      cw.w32[i] = P.mixed ? static_cast<const float *>(P.wT)[i] : 0.0f;
    }
    __syncthreads();
  }
  SolveState &S = *P.st;
  double red_out[4];
  double *red = G.red;
  // scalars live in registers, identical in every CTA of the group
  long long iters = S.iters, outer = S.outer;
  double rr = S.rr, rmax = S.rmax, bnorm = S.bnorm, rel = S.rel, sumb = S.sumb, beta = S.beta;
  int phase = S.phase;
  int status = SC_OK;
  const double tol = P.rtol;

  if (phase == 0) {
    // r = rhs - A x0 (FP64); rh = r; p = rh
    phase_resid<NDIM, R>(P, G.rank, smem, red, cw, cur_part(G));
    if (!group_reduce(G, 1, P.ntiles_64, red_out)) return;
    phase_vec<TI, 0>(P, G.rank, 0.0, red, cur_part(G));
    if (!group_reduce(G, 3, P.nchunks, red_out)) return;
    rr = red_out[0];
    bnorm = sqrt(red_out[1]);
    sumb = red_out[2];
    rmax = sqrt(rr);
    rel = bnorm > 0 ? sqrt(rr) / bnorm : 0.0;
    beta = 0.0;
    phase = 1;
    if (bnorm == 0.0 || sqrt(rr) <= tol * bnorm) phase = 3;  // already converged
  }

  long long done = 0;
  while (phase == 1 && done < budget) {
    if (iters >= P.maxit) {
      status = SC_ENOTCONV;
      phase = 3;
      break;
    }
    // A: q = A p, p.q
    phase_apply<TI, NDIM, R>(P, G.rank, smem, red, cw, cur_part(G));
    if (!group_reduce(G, 1, P.ntiles_in, red_out)) return;
    const double pq = red_out[0];
    if (!finite_pos(pq) || !(rr == rr)) {
      status = SC_EBREAKDOWN;
      phase = 3;
      break;
    }
    const double alpha = rr / pq;
    // B: d += alpha p, rh -= alpha q, rh.rh
    phase_vec<TI, 1>(P, G.rank, alpha, red, cur_part(G));
    if (!group_reduce(G, 1, P.nchunks, red_out)) return;
    double rr_new = red_out[0];
    ++iters;
    ++done;
    const double rn = sqrt(rr_new);
    if (!(rn == rn)) {
      status = SC_EBREAKDOWN;
      phase = 3;
      break;
    }
    // refresh: mixed -- every `delta` decrease or at the tolerance; FP64 --
    // at the tolerance.  The FP64 true residual replaces the recurrence one;
    // convergence is only declared on it.
    const bool refresh = P.mixed ? (rn <= P.delta * rmax || rn <= tol * bnorm) : (rn <= tol * bnorm);
    if (refresh) {
      if (P.mixed) {  // x += d in FP64
        phase_vec<TI, 3>(P, G.rank, 0.0, red, cur_part(G));
        if (!group_reduce(G, 0, 0, red_out)) return;
      }
      phase_resid<NDIM, R>(P, G.rank, smem, red, cw, cur_part(G));
      if (!group_reduce(G, 1, P.ntiles_64, red_out)) return;
      ++outer;
      rel = bnorm > 0 ? sqrt(red_out[0]) / bnorm : 0.0;
      if (rel <= tol) {
        phase = 3;
        break;
      }
      if (P.mixed) {
        phase_vec<TI, 4>(P, G.rank, 0.0, red, cur_part(G));
        if (!group_reduce(G, 1, P.nchunks, red_out)) return;
        rr_new = red_out[0];
      } else {
        rr_new = red_out[0];  // r (== rh) now holds the true residual
      }
      rmax = sqrt(rr_new);
    }
    beta = rr_new / rr;
    rr = rr_new;
    // C: p = rh + beta p
    phase_vec<TI, 2>(P, G.rank, beta, red, cur_part(G));
    if (!group_reduce(G, 0, 0, red_out, deadline)) return;
    if (deadline && red_out[3] != 0.0) break;
  }

  if (phase == 3) {
    // finish: FP64 x (mixed: fold d), optional mean fix, true residual
    if (P.mixed) {
      phase_vec<TI, 3>(P, G.rank, 0.0, red, cur_part(G));
      if (!group_reduce(G, 0, 0, red_out)) return;
    }
    if (P.mean_fix) {
      phase_vec<TI, 5>(P, G.rank, 0.0, red, cur_part(G));
      if (!group_reduce(G, 1, P.nchunks, red_out)) return;
      const double c = (sumb - red_out[0]) / double(P.npts);
      phase_vec<TI, 6>(P, G.rank, c, red, cur_part(G));
      if (!group_reduce(G, 0, 0, red_out)) return;
    }
    phase_resid<NDIM, R>(P, G.rank, smem, red, cw, cur_part(G));
    if (!group_reduce(G, 1, P.ntiles_64, red_out)) return;
    rel = bnorm > 0 ? sqrt(red_out[0]) / bnorm : 0.0;
    if (status == SC_OK && !(rel <= tol)) {
      // the recurrence met the tolerance but the true residual did not:
      // report it honestly
      status = (rel == rel) ? SC_ENOTCONV : SC_EBREAKDOWN;
    }
    phase = 2;
  }
  if (G.rank == 0 && threadIdx.x == 0) {
    S.iters = iters;
    S.outer = outer;
    S.rr = rr;
    S.rmax = rmax;
    S.bnorm = bnorm;
    S.rel = rel;
    S.sumb = sumb;
    S.beta = beta;
    S.phase = phase;
    if (phase == 2) S.status = status;
  }
}

}  // namespace sc
