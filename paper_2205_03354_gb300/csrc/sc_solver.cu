// Solver entry points: the biharmonic plate problem (Sec. 3.3), semi-implicit
// Cahn-Hilliard steps (Sec. 4) and their batched form, on top of the
// persistent CG engine of sc_solver.cuh and a host-driven plain CG.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "sc_apply_host.h"
#include "sc_internal.h"
#include "sc_cg_kernels.h"
#include "sc_solver.cuh"
#include "sc_solver_host.h"
#include "sc_stats_kernels.h"

namespace sc {

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// out = ring of g (padded array), interior set to zero.
__global__ void k_ring_copy(const double *__restrict__ g, double *__restrict__ out, int ndim,
                            long long px, long long py, long long pz, int R) {
  const long long n = px * py * pz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long ix = i % px, iy = (i / px) % py, iz = i / (px * py);
    bool inner = ix >= R && ix < px - R && iy >= R && iy < py - R;
    if (ndim == 3) inner = inner && iz >= R && iz < pz - R;
    out[i] = inner ? 0.0 : g[i];
  }
}

// y = f - y
__global__ void k_sub_from(double *__restrict__ y, const double *__restrict__ f, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = f[i] - y[i];
}

// y = u + c * y
__global__ void k_u_plus_cy(double *__restrict__ y, const double *__restrict__ u, double c, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(c, y[i], u[i]);
}

// g = f'(u)
__global__ void k_fprime(const double *__restrict__ u, double *__restrict__ g, long long n, int chem,
                         double rho, double ca, double cb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double c = u[i];
    g[i] = chem == 0 ? c * c * c - c : 2.0 * rho * (c - ca) * (c - cb) * (2.0 * c - ca - cb);
  }
}

// g = sum_j b_j f'(u^(n-j)) over the history (u0 = u^n, h1 = u^(n-1), h2 = u^(n-2))
__global__ void k_fprime_hist(const double *__restrict__ u0, const double *__restrict__ h1,
                              const double *__restrict__ h2, int order, double b0, double b1, double b2,
                              double *__restrict__ g, long long n, int chem, double rho, double ca, double cb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    auto fp = [&](double c) {
      return chem == 0 ? c * c * c - c : 2.0 * rho * (c - ca) * (c - cb) * (2.0 * c - ca - cb);
    };
    double v = b0 * fp(u0[i]);
    if (order > 1) v += b1 * fp(h1[i]);
    if (order > 2) v += b2 * fp(h2[i]);
    g[i] = v;
  }
}

// y = sum_j al_j u^(n-j) + c y   (y holds Lap g on entry)
__global__ void k_sbdf_rhs(double *__restrict__ y, const double *__restrict__ u0, const double *__restrict__ h1,
                           const double *__restrict__ h2, int order, double a0, double a1, double a2, double c,
                           long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double v = a0 * u0[i];
    if (order > 1) v += a1 * h1[i];
    if (order > 2) v += a2 * h2[i];
    y[i] = fma(c, y[i], v);
  }
}

// ---- plain CG helpers (one kernel per operation) --------------------------
constexpr int PL_NTHR = 256;
constexpr int PL_CHUNK = PL_NTHR * 16;
static_assert(PL_NTHR == STATS_NTHR && PL_CHUNK == STATS_CHUNK, "statistics kernel shape");

__global__ void k_dot_part(const double *__restrict__ a, const double *__restrict__ b, long long n,
                           double *__restrict__ part) {
  __shared__ double red[PL_NTHR / 32];
  const long long e0 = (long long)blockIdx.x * PL_CHUNK, e1 = min(e0 + PL_CHUNK, n);
  double s = 0.0;
  for (long long i = e0 + threadIdx.x; i < e1; i += PL_NTHR) s += a[i] * b[i];
  s = block_sum<PL_NTHR>(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// scal[slot] = sum(part[0..n)) in index order
__global__ void k_sum_final(const double *__restrict__ part, int n, double *__restrict__ scal, int slot) {
  __shared__ double red[PL_NTHR / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += PL_NTHR) s += part[i];
  s = block_sum<PL_NTHR>(s, red);
  if (threadIdx.x == 0) scal[slot] = s;
}

// scalar slots: 0 rr, 1 pq, 2 rr_new, 3 alpha, 4 beta, 5 bnorm^2, 6 converged flag, 7 breakdown
__global__ void k_alpha(double *s) {
  const double pq = s[1];
  if (!(pq > 0.0) || !(pq < 1e300)) {
    s[7] = 1.0;
    s[3] = 0.0;
  } else {
    s[3] = s[0] / pq;
  }
}
__global__ void k_beta(double *s, double tol) {
  s[4] = s[2] / s[0];
  s[0] = s[2];
  if (sqrt(s[2]) <= tol * sqrt(s[5])) s[6] = 1.0;
  if (!(s[2] == s[2])) s[7] = 1.0;
}
__global__ void k_xr_update(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                            const double *__restrict__ q, const double *__restrict__ s, long long n) {
  const double al = s[3];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] += al * p[i];
    r[i] -= al * q[i];
  }
}
__global__ void k_p_update(double *__restrict__ p, const double *__restrict__ r, const double *__restrict__ s,
                           long long n) {
  const double be = s[4];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = r[i] + be * p[i];
}
// q = a p + b q
__global__ void k_axpby(double *__restrict__ q, const double *__restrict__ p, double a, double b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    q[i] = fma(b, q[i], a * p[i]);
}
__global__ void k_add_const(double *__restrict__ x, const double *__restrict__ s, int num, int den_slot,
                            long long n) {
  const double c = (s[num] - s[den_slot]) / double(n);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += c;
}

// ---- Cahn-Hilliard statistics ---------------------------------------------
__global__ void k_ch_stats_part(const double *__restrict__ u, int ndim, int nx, int ny, int nz, double h,
                                double kappa, int chem, double rho, double ca, double cb,
                                double *__restrict__ pm, double *__restrict__ pe) {
  __shared__ double red[PL_NTHR / 32];
  const long long n = (long long)nx * ny * (ndim == 3 ? nz : 1);
  const long long e0 = (long long)blockIdx.x * PL_CHUNK, e1 = min(e0 + PL_CHUNK, n);
  double m = 0.0, e = 0.0;
  for (long long i = e0 + threadIdx.x; i < e1; i += PL_NTHR) {
    const int ix = int(i % nx), iy = int((i / nx) % ny), iz = ndim == 3 ? int(i / ((long long)nx * ny)) : 0;
    const double c = u[i];
    m += c;
    const double f = chem == 0 ? (c * c - 1.0) * (c * c - 1.0) / 4.0
                               : rho * (c - ca) * (c - ca) * (c - cb) * (c - cb);
    double g2 = 0.0;
    const long long bz = (long long)iz * nx * ny;
    double d = (u[bz + (long long)iy * nx + (ix + 1 == nx ? 0 : ix + 1)] - c) / h;
    g2 += d * d;
    d = (u[bz + (long long)(iy + 1 == ny ? 0 : iy + 1) * nx + ix] - c) / h;
    g2 += d * d;
    if (ndim == 3) {
      d = (u[(long long)(iz + 1 == nz ? 0 : iz + 1) * nx * ny + (long long)iy * nx + ix] - c) / h;
      g2 += d * d;
    }
    e += f + 0.5 * kappa * g2;
  }
  m = block_sum<PL_NTHR>(m, red);
  if (threadIdx.x == 0) pm[blockIdx.x] = m;
  e = block_sum<PL_NTHR>(e, red);
  if (threadIdx.x == 0) pe[blockIdx.x] = e;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------



// Tile-size scale of the persistent solver per (ndim, precision class):
// the tile targets below are multiplied by it.  Set by sc_autotune_solver or
// sc_solver_tile_scale_set; 1 by default.  Stored as the scale's log2 + 8.
static std::atomic<int> g_tile_log2[2][2] = {{{8}, {8}}, {{8}, {8}}};
constexpr int TILE_LOG2_MIN = -2, TILE_LOG2_MAX = 2;  // scales 1/4 .. 4

static double tile_scale(int ndim, bool mixed) {
  return std::ldexp(1.0, g_tile_log2[ndim == 3][mixed ? 1 : 0].load(std::memory_order_relaxed) - 8);
}

template <typename T, int NDIM, int R>
static void tiles_for(const ProbSpec &sp, int &H, int &ntiles, double scale = -1.0) {
  using K = FlatApply<T, NDIM, R, CLS_CROSS2, 1>;
  const long long nx = sp.n[0], ny = sp.n[1], nz = NDIM == 3 ? sp.n[2] : 1;
  const long long txy = ((nx + K::BX - 1) / K::BX) * (NDIM == 3 ? (ny + K::BY - 1) / K::BY : 1);
  const long long planes = NDIM == 3 ? nz : ny;
  const long long npts = nx * ny * nz;
  const long long ns = K::NSTREAM;  // 2D: row streams per tile, h rows each
  // 3D: about one tile per 2048 points, at most ~1024 tiles.  2D: one per
  // 1024 points (short row streams keep small grids parallel), at most one
  // round of the CTAs a 2D launch keeps resident (4 per SM).  FP64 tiles
  // are 4x smaller: a warp retires one FP64 FMA instruction per 64 clocks
  if (scale <= 0.0) scale = tile_scale(NDIM, sp.mixed);
  const long long per =
      std::max<long long>(16, (long long)((NDIM == 3 ? 2048 : 1024) / (sizeof(T) == 8 ? 4 : 1) * scale));
  const long long target =
      NDIM == 3 ? std::max<long long>(1, std::min<long long>(npts / per, 1024))
                : std::max<long long>(1, std::min<long long>(npts / per, 4LL * num_sms()));
  long long h = (txy * planes + target * ns - 1) / (target * ns);
  // at least 2 rows per 2D stream / 4 planes per 3D tile (the 2R halo is
  // re-read by the neighbouring stream or tile), at most 128
  h = std::max<long long>(NDIM == 2 ? 2 : 4, std::min<long long>(h, 128));
  h = std::min<long long>(h, (planes + ns - 1) / ns);
  H = int(h);
  ntiles = int(txy * ((planes + h * ns - 1) / (h * ns)));
}

static size_t smem_bytes_cg() {
  size_t m = 0;
  m = std::max(m, FlatApply<float, 2, 2, CLS_CROSS2, 1>::SMEM);
  m = std::max(m, FlatApply<float, 3, 2, CLS_CROSS2, 1>::SMEM);
  m = std::max(m, FlatApply<double, 2, 2, CLS_CROSS2, 1>::SMEM);
  m = std::max(m, FlatApply<double, 3, 2, CLS_CROSS2, 1>::SMEM);
  return m;
}

// Lays out one problem's work space; with base == nullptr only sizes.
void layout(const ProbSpec &sp, Carver &cv, SolveProb &P, ProbAux &aux) {
  std::memset(&P, 0, sizeof(P));
  const long long npts = sp.n[0] * sp.n[1] * (sp.ndim == 3 ? sp.n[2] : 1);
  P.ndim = sp.ndim;
  P.nx = int(sp.n[0]);
  P.ny = int(sp.n[1]);
  P.nz = sp.ndim == 3 ? int(sp.n[2]) : 1;
  P.bc = sp.bc;
  P.npts = npts;
  if (sp.ndim == 2) {
    tiles_for<float, 2, 2>(sp, P.H_in, P.ntiles_in);
    if (!sp.mixed) tiles_for<double, 2, 2>(sp, P.H_in, P.ntiles_in);
    tiles_for<double, 2, 2>(sp, P.H_64, P.ntiles_64);
  } else {
    tiles_for<float, 3, 2>(sp, P.H_in, P.ntiles_in);
    if (!sp.mixed) tiles_for<double, 3, 2>(sp, P.H_in, P.ntiles_in);
    tiles_for<double, 3, 2>(sp, P.H_64, P.ntiles_64);
  }
  // chunk = CG_STEP * 2^k: the smallest with at most 1024 chunks
  P.chunk = CG_STEP;
  while ((npts + P.chunk - 1) / P.chunk > 1024) P.chunk *= 2;
  P.nchunks = int((npts + P.chunk - 1) / P.chunk);
  // the plain path reduces in blocks of PL_CHUNK points through the same slots;
  // the slots also cover the most tiles any tile scale gives, so that a work
  // space sized once serves every tuning choice
  int most = 0;
  {
    int hh, nt;
    const double smin = std::ldexp(1.0, TILE_LOG2_MIN);
    if (sp.ndim == 2) {
      tiles_for<float, 2, 2>(sp, hh, nt, smin);
      most = std::max(most, nt);
      tiles_for<double, 2, 2>(sp, hh, nt, smin);
      most = std::max(most, nt);
    } else {
      tiles_for<float, 3, 2>(sp, hh, nt, smin);
      most = std::max(most, nt);
      tiles_for<double, 3, 2>(sp, hh, nt, smin);
      most = std::max(most, nt);
    }
  }
  P.nslot = std::max({P.ntiles_in, P.ntiles_64, P.nchunks, int((npts + 4095) / 4096), most});
  P.a = sp.a;
  P.b = sp.b;
  P.mixed = sp.mixed;
  P.mean_fix = sp.mean_fix;
  P.rtol = sp.rtol;
  P.delta = 0.1;
  P.maxit = sp.maxit;
  const size_t ti = sp.mixed ? 4 : 8;
  P.x = sp.x;
  P.rhs = static_cast<double *>(cv.take(npts * 8));
  P.r = static_cast<double *>(cv.take(npts * 8));
  if (sp.mixed) {
    P.rh = cv.take(npts * ti);
    P.d = cv.take(npts * ti);
  } else {
    P.rh = P.r;
    P.d = P.x;
  }
  P.p = cv.take(npts * ti);
  P.q = cv.take(npts * ti);
  // two buffers of 3 * nslot partials, alternating by reduction parity
  P.part = static_cast<double *>(cv.take(size_t(6) * P.nslot * 8));
  P.scal = static_cast<double *>(cv.take(8 * 8));
  P.bar = static_cast<unsigned *>(cv.take(16));
  P.st = static_cast<SolveState *>(cv.take(sizeof(SolveState)));
  const int nbox = sp.ndim == 3 ? 125 : 25;
  P.w64 = static_cast<const double *>(cv.take(nbox * 8));
  P.wT = cv.take(nbox * 8);
  aux.nbox = nbox;
  // scratch for problem set-up (ring copy of the padded grid)
  long long padded = 1;
  for (int a = 0; a < sp.ndim; ++a) padded *= sp.n[a] + 2 * sp.R;
  aux.scratch = static_cast<double *>(cv.take(std::max<long long>(padded, npts) * 8));
  if (sp.solver == SC_SOLVER_PCG) {
    const long long N = sp.n[0];
    aux.z = static_cast<double *>(cv.take(npts * 8));
    aux.u0 = static_cast<float *>(cv.take(npts * 4));
    aux.u1 = static_cast<float *>(cv.take(npts * 4));
    aux.S = static_cast<float *>(cv.take(N * N * 4));
    aux.lam1 = static_cast<double *>(cv.take(N * 8));
    aux.part = static_cast<double *>(cv.take(3 * pcg_parts(npts) * 8));
    aux.out = static_cast<double *>(cv.take(32 * 8));  // dot results, then the inner loop's scalars
    const long long K0 = pcg_low_modes(sp.ndim, N);
    aux.Sl = static_cast<double *>(cv.take(K0 * N * 8));
    aux.SlT = static_cast<double *>(cv.take(K0 * N * 8));
    aux.wa = static_cast<double *>(cv.take((sp.ndim == 3 ? N * N : N) * K0 * 8));
    aux.wb = static_cast<double *>(cv.take(N * K0 * K0 * 8));
    aux.wc = static_cast<double *>(cv.take(K0 * K0 * K0 * 8));
    aux.zl = static_cast<double *>(cv.take(npts * 8));
  }
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Fills the dense weight boxes of B (composed Lap o Lap, exact weights) and
// the state on the device (asynchronously from pageable host buffers).
int upload_prob(const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t st) {
  sc_stencil L, B;
  int rc = sc_laplacian(sp.ndim, sp.order, &L);
  if (!rc) rc = sc_compose_stencil(&L, &L, &B);
  if (rc) return rc;
  std::vector<double> w(B.npts);
  if ((rc = weights_f64(&B, sp.h_num, sp.h_den, w.data()))) return rc;
  const int R = 2, Wd = 2 * R + 1;
  std::vector<double> box(aux.nbox, 0.0);
  std::vector<float> boxf(aux.nbox * 2, 0.0f);  // room for a double box too
  for (int k = 0; k < B.npts; ++k) {
    const int dx = B.off[k][0], dy = B.off[k][1], dz = B.off[k][2];
    const int idx = sp.ndim == 3 ? ((dz + R) * Wd + (dy + R)) * Wd + (dx + R) : (dy + R) * Wd + (dx + R);
    box[idx] = w[k];
  }
  cudaMemcpyAsync(const_cast<double *>(P.w64), box.data(), aux.nbox * 8, cudaMemcpyHostToDevice, st);
  if (P.mixed) {
    std::vector<float> wf(B.npts);
    if ((rc = weights_f32(&B, sp.h_num, sp.h_den, wf.data()))) return rc;
    for (int k = 0; k < B.npts; ++k) {
      const int dx = B.off[k][0], dy = B.off[k][1], dz = B.off[k][2];
      const int idx = sp.ndim == 3 ? ((dz + R) * Wd + (dy + R)) * Wd + (dx + R) : (dy + R) * Wd + (dx + R);
      boxf[idx] = wf[k];
    }
    cudaMemcpyAsync(const_cast<void *>(P.wT), boxf.data(), aux.nbox * 4, cudaMemcpyHostToDevice, st);
  } else {
    cudaMemcpyAsync(const_cast<void *>(P.wT), box.data(), aux.nbox * 8, cudaMemcpyHostToDevice, st);
  }
  SolveState s0;
  std::memset(&s0, 0, sizeof(s0));
  cudaMemcpyAsync(P.st, &s0, sizeof(s0), cudaMemcpyHostToDevice, st);
  // 16-byte tile loads need aligned vectors and rows
  const bool al = aligned16(P.x) && aligned16(P.p) && aligned16(P.r);
  P.vec_in = al && (P.nx % (P.mixed ? 4 : 2) == 0);
  P.vec_64 = al && (P.nx % 2 == 0);
  P.vec_v = al && aligned16(P.rhs) && aligned16(P.q) && aligned16(P.rh) && aligned16(P.d) && (P.npts % 4 == 0);
  cudaError_t e = cudaStreamSynchronize(st);  // host buffers above are locals
  if (e != cudaSuccess) return fail(SC_ECUDA, "upload: %s", cudaGetErrorString(e));
  return SC_OK;
}

static int grid1d(long long n) { return int(std::min<long long>((n + 255) / 256, 8LL * num_sms())); }

// Right-hand side of the plate problem: rhs = g - A(ring), x = 0.
int setup_bvp(const sc_bvp *bp, const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t st) {
  const int R = sp.R;
  long long p[3] = {1, 1, 1};
  for (int a = 0; a < sp.ndim; ++a) p[a] = sp.n[a] + 2 * R;
  const long long np = p[0] * p[1] * p[2];
  k_ring_copy<<<grid1d(np), 256, 0, st>>>(bp->ghost_dev, aux.scratch, sp.ndim, p[0], p[1], p[2], R);
  sc_stencil L, B;
  sc_laplacian(sp.ndim, sp.order, &L);
  sc_compose_stencil(&L, &L, &B);
  ApplyReq q{&B, SC_F64, SC_BC_GHOSTED, sp.n, sp.h_num, sp.h_den, aux.scratch, P.rhs};
  if (int rc = apply_enqueue(q, st)) return rc;
  k_sub_from<<<grid1d(P.npts), 256, 0, st>>>(P.rhs, bp->f_dev, P.npts);
  cudaMemsetAsync(P.x, 0, P.npts * 8, st);
  return SC_OK;
}

// Right-hand side of a Cahn-Hilliard step: rhs = u + dt M Lap(f'(u)).
int setup_ch(const sc_ch *cp, const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t st) {
  k_fprime<<<grid1d(P.npts), 256, 0, st>>>(P.x, aux.scratch, P.npts, cp->chem, cp->rho, cp->ca, cp->cb);
  sc_stencil L;
  sc_laplacian(sp.ndim, sp.order, &L);
  ApplyReq q{&L, SC_F64, SC_BC_PERIODIC, sp.n, sp.h_num, sp.h_den, aux.scratch, P.rhs};
  if (int rc = apply_enqueue(q, st)) return rc;
  k_u_plus_cy<<<grid1d(P.npts), 256, 0, st>>>(P.rhs, P.x, cp->dt * cp->M, P.npts);
  return SC_OK;
}

// Assigns CTA groups for problems[first..last) and launches one cooperative
// persistent kernel for them.
// CTA groups for problems hp[idx]: proportional to size, at least one each,
// at most the problem's number of work units; returns the CTA -> problem map.
static int assign_groups(std::vector<SolveProb> &hp, const std::vector<int> &idx, int G, unsigned *dbars,
                         std::vector<int> &map) {
  double wsum = 0.0;
  for (int i : idx) wsum += double(hp[i].npts);
  int used = 0;
  std::vector<int> nc(idx.size());
  for (size_t k = 0; k < idx.size(); ++k) {
    const SolveProb &P = hp[idx[k]];
    const int units = std::max({P.ntiles_in, P.ntiles_64, P.nchunks});
    int c = int(std::floor(double(G - int(idx.size())) * double(P.npts) / wsum)) + 1;
    c = std::max(1, std::min(c, units));
    nc[k] = c;
    used += c;
  }
  if (used > G || G > 32 * num_sms()) return fail(SC_EINVAL, "internal: CTA assignment exceeds the grid");
  map.assign(used, -1);
  int c0 = 0;
  for (size_t k = 0; k < idx.size(); ++k) {
    SolveProb &P = hp[idx[k]];
    P.cta0 = c0;
    P.ncta = nc[k];
    P.bar = dbars + 2 * idx[k];
    for (int j = 0; j < nc[k]; ++j) map[c0 + j] = idx[k];
    c0 += nc[k];
  }
  return SC_OK;
}

// the persistent kernel variants live in sc_cg_f32.cu, sc_cg_f64.cu and
// sc_cg_both.cu (separate translation units, compiled in parallel)
template <typename TI>
static CgKernel cg_kernel_for(int dims);
template <>
CgKernel cg_kernel_for<float>(int dims) {
  return cg_kernel_f32(dims);
}
template <>
CgKernel cg_kernel_for<double>(int dims) {
  return cg_kernel_f64(dims);
}
template <>
CgKernel cg_kernel_for<void>(int dims) {
  return cg_kernel_both(dims);
}

// Which dimensionalities occur among hp[idx] (bit 0: 2D, bit 1: 3D).
static int dims_mask(const std::vector<SolveProb> &hp, const std::vector<int> &idx) {
  int m = 0;
  for (int i : idx) m |= hp[i].ndim == 2 ? 1 : 2;
  return m ? m : 1;
}

template <typename TI>
static size_t cg_smem_setup(int dims) {
  const size_t smem = smem_bytes_cg();
  static std::atomic<unsigned long long> smem_set[4];
  set_smem_limit_once(cg_kernel_for<TI>(dims), smem, smem_set[dims]);
  return smem;
}

// Cooperative launch of the persistent kernel over descriptors already on
// the device (capturable in a CUDA graph).
template <typename TI>
static int enqueue_cg(const SolveProb *dprobs, const int *dmap, int grid, cudaStream_t st, long long budget,
                      unsigned long long slice_ns, int dims) {
  auto kern = cg_kernel_for<TI>(dims);
  const size_t smem = cg_smem_setup<TI>(dims);
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(CG_NTHR);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, dprobs, dmap, budget, slice_ns);
  if (e != cudaSuccess) return fail(SC_ECUDA, "cooperative launch: %s", cudaGetErrorString(e));
  return SC_OK;
}

// Assigns CTA groups for problems hp[idx] and launches one cooperative
// persistent kernel for them (synchronous).
template <typename TI>
static int launch_group(std::vector<SolveProb> &hp, const std::vector<int> &idx, SolveProb *dprobs,
                        int *dmap, unsigned *dbars, cudaStream_t st, long long budget,
                        double slice_ms) {
  const int dims = dims_mask(hp, idx);
  auto kern = cg_kernel_for<TI>(dims);
  const size_t smem = cg_smem_setup<TI>(dims);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, CG_NTHR, smem);
  if (nb < 1) return fail(SC_ECUDA, "persistent CG kernel does not fit on an SM");
  const int G = nb * num_sms();
  std::vector<int> map;
  if (int rc = assign_groups(hp, idx, G, dbars, map)) return rc;
  cudaMemcpyAsync(dprobs, hp.data(), hp.size() * sizeof(SolveProb), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dmap, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(dbars, 0, hp.size() * 2 * sizeof(unsigned), st);
  const unsigned long long slice_ns = slice_ms > 0.0 ? (unsigned long long)(slice_ms * 1e6) : 0ull;
  if (int rc = enqueue_cg<TI>(dprobs, dmap, int(map.size()), st, budget, slice_ns, dims)) return rc;
  // pageable sources above: finish before the vectors go out of scope
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SC_ECUDA, "persistent CG: %s", cudaGetErrorString(e));
  return SC_OK;
}

int max_group_ctas(bool mixed, int dims) {
  const size_t smem = smem_bytes_cg();
  int nb = 0;
  if (mixed)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cg_kernel_for<float>(dims), CG_NTHR, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cg_kernel_for<double>(dims), CG_NTHR, smem);
  return std::max(1, nb) * num_sms();
}

// Runs every problem to completion (waves of at most one CTA per problem
// beyond the grid size).
int run_persistent(std::vector<SolveProb> &hp, SolveProb *dprobs, int *dmap, unsigned *dbars,
                   cudaStream_t st, long long budget, double slice_ms) {
  bool has[2] = {false, false};
  for (const SolveProb &P : hp) has[P.mixed ? 1 : 0] = true;
  if (has[0] && has[1]) {
    // both precision classes share one launch (each problem picks its path)
    std::vector<int> all(hp.size());
    for (size_t i = 0; i < hp.size(); ++i) all[i] = int(i);
    const int dims = dims_mask(hp, all);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cg_kernel_for<void>(dims), CG_NTHR, smem_bytes_cg());
    const int G = std::max(1, nb) * num_sms();
    for (size_t w0 = 0; w0 < all.size(); w0 += size_t(G)) {
      std::vector<int> idx(all.begin() + w0, all.begin() + std::min(all.size(), w0 + size_t(G)));
      if (int rc = launch_group<void>(hp, idx, dprobs, dmap, dbars, st, budget, slice_ms)) return rc;
    }
    return SC_OK;
  }
  for (int mixed = 0; mixed < 2; ++mixed) {
    std::vector<int> all;
    for (size_t i = 0; i < hp.size(); ++i)
      if (hp[i].mixed == mixed) all.push_back(int(i));
    if (all.empty()) continue;
    const int G = max_group_ctas(mixed, dims_mask(hp, all));
    for (size_t w0 = 0; w0 < all.size(); w0 += size_t(G)) {
      std::vector<int> idx(all.begin() + w0, all.begin() + std::min(all.size(), w0 + size_t(G)));
      int rc = mixed ? launch_group<float>(hp, idx, dprobs, dmap, dbars, st, budget, slice_ms)
                     : launch_group<double>(hp, idx, dprobs, dmap, dbars, st, budget, slice_ms);
      if (rc) return rc;
    }
  }
  return SC_OK;
}

// Host-driven FP64 CG, one kernel per operation (the plain comparison path).
static int run_plain(const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t st,
                     double *scal_host) {
  const long long n = P.npts;
  const int nblk = int((n + PL_CHUNK - 1) / PL_CHUNK);
  double *part = P.part;  // >= nchunks slots (PL_CHUNK == CG_CHUNK)
  double *s = P.scal;
  sc_stencil L, B;
  sc_laplacian(sp.ndim, sp.order, &L);
  sc_compose_stencil(&L, &L, &B);
  const int g = grid1d(n);
  auto apply_op = [&](const double *in, double *out) -> int {
    ApplyReq q{&B, SC_F64, sp.bc, sp.n, sp.h_num, sp.h_den, in, out};
    if (int rc = apply_enqueue(q, st)) return rc;
    if (P.a != 0.0 || P.b != 1.0) k_axpby<<<g, 256, 0, st>>>(out, in, P.a, P.b, n);
    return SC_OK;
  };
  auto dot = [&](const double *a, const double *b, int slot) {
    k_dot_part<<<nblk, PL_NTHR, 0, st>>>(a, b, n, part);
    k_sum_final<<<1, PL_NTHR, 0, st>>>(part, nblk, s, slot);
  };
  double *p = static_cast<double *>(P.p), *q = static_cast<double *>(P.q), *r = P.r;
  cudaMemsetAsync(s, 0, 8 * 8, st);
  // r = rhs - A x
  if (int rc = apply_op(P.x, r)) return rc;
  k_sub_from<<<g, 256, 0, st>>>(r, P.rhs, n);
  cudaMemcpyAsync(p, r, n * 8, cudaMemcpyDeviceToDevice, st);
  dot(r, r, 0);
  dot(P.rhs, P.rhs, 5);
  double hs[8];
  cudaMemcpyAsync(hs, s, sizeof(hs), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  long long it = 0;
  int status = SC_OK;
  const double tol = sp.rtol;
  const double bn2 = hs[5];
  bool conv = std::sqrt(hs[0]) <= tol * std::sqrt(bn2);
  double rel = 0.0;
  for (;;) {
    while (!conv) {
      if (it >= sp.maxit) {
        status = SC_ENOTCONV;
        break;
      }
      if (int rc = apply_op(p, q)) return rc;
      dot(p, q, 1);
      k_alpha<<<1, 1, 0, st>>>(s);
      k_xr_update<<<g, 256, 0, st>>>(P.x, r, p, q, s, n);
      dot(r, r, 2);
      k_beta<<<1, 1, 0, st>>>(s, tol);
      k_p_update<<<g, 256, 0, st>>>(p, r, s, n);
      ++it;
      if ((it & 7) == 0 || it >= sp.maxit) {
        cudaMemcpyAsync(hs, s, sizeof(hs), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        if (hs[7] != 0.0) {
          status = SC_EBREAKDOWN;
          break;
        }
        conv = hs[6] != 0.0;
      }
    }
    if (status != SC_OK) break;
    // the recurrence met the tolerance: check the true residual
    if (int rc = apply_op(P.x, r)) return rc;
    k_sub_from<<<g, 256, 0, st>>>(r, P.rhs, n);
    dot(r, r, 0);
    cudaMemcpyAsync(hs, s, sizeof(hs), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    rel = bn2 > 0 ? std::sqrt(hs[0]) / std::sqrt(bn2) : 0.0;
    if (rel <= tol || it >= sp.maxit) break;
    // restart from the true residual
    cudaMemcpyAsync(p, r, n * 8, cudaMemcpyDeviceToDevice, st);
    double zero = 0.0;
    cudaMemcpyAsync(s + 6, &zero, 8, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
    conv = false;
  }
  if (P.mean_fix) {
    k_dot_part<<<nblk, PL_NTHR, 0, st>>>(P.rhs, aux.ones, n, part);
    k_sum_final<<<1, PL_NTHR, 0, st>>>(part, nblk, s, 0);
    k_dot_part<<<nblk, PL_NTHR, 0, st>>>(P.x, aux.ones, n, part);
    k_sum_final<<<1, PL_NTHR, 0, st>>>(part, nblk, s, 1);
    k_add_const<<<g, 256, 0, st>>>(P.x, s, 0, 1, n);
  }
  // true residual of the returned x
  if (int rc = apply_op(P.x, r)) return rc;
  k_sub_from<<<g, 256, 0, st>>>(r, P.rhs, n);
  dot(r, r, 2);
  cudaMemcpyAsync(hs, s, sizeof(hs), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SC_ECUDA, "plain CG: %s", cudaGetErrorString(e));
  const double bn = std::sqrt(hs[5]);
  scal_host[0] = double(it);
  scal_host[1] = bn > 0 ? std::sqrt(hs[2]) / bn : 0.0;
  if (status == SC_OK && !(scal_host[1] <= tol)) status = SC_ENOTCONV;
  scal_host[2] = double(status);
  return SC_OK;
}

// ---------------------------------------------------------------------------
// problem specs from the public structs
// ---------------------------------------------------------------------------

double kappa_estimate(const ProbSpec &sp, double h) {
  const double d = sp.ndim;
  if (sp.bc == SC_BC_PERIODIC) {  // I + s B, eigenvalues 1 .. 1 + s (4d/h^2)^2
    const double lm = 4.0 * d / (h * h);
    return 1.0 + sp.b * lm * lm;
  }
  const double lmax = 4.0 * d / (h * h), lmin = d * M_PI * M_PI;  // Dirichlet-like Laplacian
  return (lmax / lmin) * (lmax / lmin);
}

static int choose_prec(int req, double kappa) {
  if (req == SC_PREC_F64 || req == SC_PREC_MIXED) return req;
  return kappa * std::ldexp(1.0, -24) <= 1e-2 ? SC_PREC_MIXED : SC_PREC_F64;
}

int bvp_spec(const sc_bvp *b, ProbSpec &sp) {
  if (!b) return fail(SC_EINVAL, "null problem");
  if (b->ndim != 2 && b->ndim != 3) return fail(SC_EINVAL, "ndim must be 2 or 3");
  if (b->order != 2) return fail(SC_EINVAL, "the solvers support the order-2 Laplacian (13/25-point Lap o Lap)");
  for (int a = 0; a < b->ndim; ++a)
    if (b->n[a] != b->n[0] || b->n[a] < 1 || b->n[a] > 65536) return fail(SC_EINVAL, "n must be equal per axis, 1..65536");
  if (!(b->rtol > 0.0) || b->maxit < 0) return fail(SC_EINVAL, "bad rtol/maxit");
  if (b->solver != SC_SOLVER_PERSISTENT && b->solver != SC_SOLVER_PLAIN && b->solver != SC_SOLVER_PCG)
    return fail(SC_EINVAL, "bad solver");
  if (b->prec < 0 || b->prec > 2) return fail(SC_EINVAL, "bad prec");
  if (!b->f_dev || !b->ghost_dev || !b->x_dev) return fail(SC_EINVAL, "null device pointer");
  std::memset(&sp, 0, sizeof(sp));
  sp.ndim = b->ndim;
  sp.order = b->order;
  sp.R = 2;
  for (int a = 0; a < 3; ++a) sp.n[a] = a < b->ndim ? b->n[a] : 1;
  sp.bc = SC_BC_ZERO;
  sp.h_num = 1;
  sp.h_den = b->n[0] + 1;
  sp.a = 0.0;
  sp.b = 1.0;
  sp.rtol = b->rtol;
  sp.maxit = b->maxit;
  sp.x = b->x_dev;
  sp.mean_fix = 0;
  const int prec = choose_prec(b->prec, kappa_estimate(sp, 1.0 / double(b->n[0] + 1)));
  sp.mixed = prec == SC_PREC_MIXED && b->solver == SC_SOLVER_PERSISTENT;
  sp.solver = b->solver;
  return SC_OK;
}

int ch_spec(const sc_ch *c, int item, double *u, ProbSpec &sp) {
  std::memset(&sp, 0, sizeof(sp));
  sp.ndim = c->ndim;
  sp.order = c->order;
  sp.R = 2;
  for (int a = 0; a < 3; ++a) sp.n[a] = a < c->ndim ? c->n[a] : 1;
  sp.bc = SC_BC_PERIODIC;
  sp.h_num = c->h_num;
  sp.h_den = c->h_den;
  sp.a = 1.0;
  sp.b = c->dt * c->M * c->kappa;
  sp.rtol = c->rtol;
  sp.maxit = c->maxit;
  const long long npts = sp.n[0] * sp.n[1] * sp.n[2];
  sp.x = u + (long long)item * npts;
  sp.mean_fix = 1;
  const int prec = choose_prec(c->prec, kappa_estimate(sp, double(c->h_num) / double(c->h_den)));
  sp.mixed = prec == SC_PREC_MIXED && c->solver == SC_SOLVER_PERSISTENT;
  sp.solver = c->solver;
  (void)item;
  return SC_OK;
}

static int ch_validate(const sc_ch *c) {
  if (!c) return fail(SC_EINVAL, "null problem");
  if (c->ndim != 2 && c->ndim != 3) return fail(SC_EINVAL, "ndim must be 2 or 3");
  if (c->order != 2) return fail(SC_EINVAL, "the solvers support the order-2 Laplacian");
  for (int a = 0; a < c->ndim; ++a)
    if (c->n[a] != c->n[0] || c->n[a] < 4 || c->n[a] > 65536) return fail(SC_EINVAL, "n must be equal per axis, 4..65536");
  if (c->batch < 1 || c->batch > 4096) return fail(SC_EINVAL, "batch out of range");
  if (c->h_num <= 0 || c->h_den <= 0) return fail(SC_EINVAL, "h must be positive");
  if (!(c->dt > 0.0) || !(c->M > 0.0) || !(c->kappa > 0.0)) return fail(SC_EINVAL, "dt, M, kappa must be positive");
  if (c->chem != 0 && c->chem != 1) return fail(SC_EINVAL, "chem must be 0 or 1");
  if (!(c->rtol > 0.0) || c->maxit < 0) return fail(SC_EINVAL, "bad rtol/maxit");
  if (c->solver != SC_SOLVER_PERSISTENT && c->solver != SC_SOLVER_PLAIN) return fail(SC_EINVAL, "bad solver");
  if (c->prec < 0 || c->prec > 2) return fail(SC_EINVAL, "bad prec");
  return SC_OK;
}

int ch_single_spec(const sc_ch *c, double *u, ProbSpec &sp) {
  if (int rc = ch_validate(c)) return rc;
  if (c->batch != 1) return fail(SC_EINVAL, "a served Cahn-Hilliard request holds one field");
  return ch_spec(c, 0, u, sp);
}

// Work space of a set of problems: per-problem areas + batch descriptors.
size_t batch_bytes(const std::vector<ProbSpec> &sps) {
  Carver cv(nullptr, 0);
  for (const ProbSpec &sp : sps) {
    SolveProb P;
    ProbAux aux;
    layout(sp, cv, P, aux);
    cv.take(std::max<long long>(P.npts, 1) * 8);  // ones vector (plain mean fix)
  }
  cv.take(sps.size() * sizeof(SolveProb));
  cv.take(sizeof(int) * size_t(32) * num_sms());  // CTA map (max grid)
  cv.take(sps.size() * 2 * sizeof(unsigned));
  return cv.off + 256;
}

__global__ void k_fill(double *x, double v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

// Sets up, solves and reports a set of problems.  setup(i, P, aux) enqueues
// the right-hand side (and initial guess) of problem i.
template <class SETUP>
int solve_set(std::vector<ProbSpec> &sps, void *work, size_t work_bytes, sc_solve_info *infos,
              cudaStream_t st, SETUP setup) {
  auto t0 = std::chrono::steady_clock::now();
  if (!work) return fail(SC_EINVAL, "null work space");
  const size_t need = batch_bytes(sps);
  if (work_bytes < need) return fail(SC_ENOMEM, "work space %zu < %zu bytes", work_bytes, need);
  Carver cv(work, work_bytes);
  std::vector<SolveProb> hp(sps.size());
  std::vector<ProbAux> aux(sps.size());
  for (size_t i = 0; i < sps.size(); ++i) {
    layout(sps[i], cv, hp[i], aux[i]);
    aux[i].ones = static_cast<double *>(cv.take(std::max<long long>(hp[i].npts, 1) * 8));
  }
  SolveProb *dprobs = static_cast<SolveProb *>(cv.take(sps.size() * sizeof(SolveProb)));
  int *dmap = static_cast<int *>(cv.take(sizeof(int) * size_t(32) * num_sms()));
  unsigned *dbars = static_cast<unsigned *>(cv.take(sps.size() * 2 * sizeof(unsigned)));
  for (size_t i = 0; i < sps.size(); ++i) {
    if (int rc = upload_prob(sps[i], hp[i], aux[i], st)) return rc;
    if (int rc = setup(int(i), hp[i], aux[i])) return rc;
  }
  std::vector<double> plain_res(3 * sps.size(), 0.0);
  bool any_persistent = false;
  for (size_t i = 0; i < sps.size(); ++i) {
    if (sps[i].solver == SC_SOLVER_PLAIN) {
      k_fill<<<grid1d(hp[i].npts), 256, 0, st>>>(aux[i].ones, 1.0, hp[i].npts);
      if (int rc = run_plain(sps[i], hp[i], aux[i], st, &plain_res[3 * i])) return rc;
    } else if (sps[i].solver == SC_SOLVER_PCG) {
      if (int rc = run_pcg(sps[i], hp[i], aux[i], st, &plain_res[3 * i])) return rc;
    } else {
      any_persistent = true;
    }
  }
  if (any_persistent) {
    std::vector<SolveProb> sub;
    std::vector<int> back;
    for (size_t i = 0; i < sps.size(); ++i)
      if (sps[i].solver == SC_SOLVER_PERSISTENT) {
        sub.push_back(hp[i]);
        back.push_back(int(i));
      }
    if (int rc = run_persistent(sub, dprobs, dmap, dbars, st, LLONG_MAX, 0.0)) return rc;
    for (size_t k = 0; k < sub.size(); ++k) hp[back[k]] = sub[k];
  }
  std::vector<SolveState> hs(sps.size());
  for (size_t i = 0; i < sps.size(); ++i)
    if (sps[i].solver == SC_SOLVER_PERSISTENT)
      cudaMemcpyAsync(&hs[i], hp[i].st, sizeof(SolveState), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SC_ECUDA, "solve: %s", cudaGetErrorString(e));
  const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (size_t i = 0; i < sps.size(); ++i) {
    sc_solve_info &in = infos[i];
    std::memset(&in, 0, sizeof(in));
    in.prec = sps[i].mixed ? SC_PREC_MIXED : SC_PREC_F64;
    in.seconds = sec;
    if (sps[i].solver != SC_SOLVER_PERSISTENT) {
      in.iters = (long long)plain_res[3 * i];
      in.rel_res = plain_res[3 * i + 1];
      in.status = int(plain_res[3 * i + 2]);
    } else {
      in.iters = hs[i].iters;
      in.outer = hs[i].outer;
      in.rel_res = hs[i].rel;
      in.status = hs[i].phase == 2 ? hs[i].status : SC_ETIMEOUT;
    }
  }
  clear_error();
  return SC_OK;
}

// out[i] = *probs[i].st for i < n (one contiguous read-back).
__global__ void k_gather_states(const SolveProb *__restrict__ probs, int n, SolveState *__restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = *probs[i].st;
}

int gather_states(const SolveProb *dprobs, int n, SolveState *dout, SolveState *host, cudaStream_t st) {
  if (n <= 0) return SC_OK;
  k_gather_states<<<(n + 127) / 128, 128, 0, st>>>(dprobs, n, dout);
  cudaMemcpyAsync(host, dout, size_t(n) * sizeof(SolveState), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SC_ECUDA, "state read-back: %s", cudaGetErrorString(e));
  return SC_OK;
}

// Resets every problem's solver state (a graph node in the multi-step run).
__global__ void k_reset_states(const SolveProb *__restrict__ probs, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    SolveState *s = probs[i].st;
    s->iters = 0;
    s->outer = 0;
    s->rr = 0.0;
    s->rmax = 0.0;
    s->bnorm = 0.0;
    s->rel = 0.0;
    s->sumb = 0.0;
    s->status = 0;
    s->phase = 0;
    s->beta = 0.0;
  }
}

// Appends every problem's final state of this step to out[step * n + i].
__global__ void k_record_states(const SolveProb *__restrict__ probs, int n, SolveState *__restrict__ out,
                                int *__restrict__ step) {
  const int i = threadIdx.x;
  const int k = *step;
  for (int j = i; j < n; j += blockDim.x) out[(long long)k * n + j] = *probs[j].st;
  __syncthreads();
  if (i == 0) *step = k + 1;
}

// A group of two CTAs of which only one is launched: its barrier can never
// be released, so the bounded wait must run out and report SC_ETIMEOUT.
// Both group-reduction protocols in turn (the small-group one, then the
// publishing one, selected by a far-off deadline); the status is
// SC_ETIMEOUT only if each gave up after its spin limit.
__global__ void k_barrier_timeout_probe(SolveProb *P, long long spin_limit) {
  __shared__ double red[CG_NTHR / 32];
  __shared__ int flag;
  GroupCtx G{P, 0, 0u, 0u, red, &flag, spin_limit};
  double out[4];
  if (threadIdx.x == 0) P->part[0] = 1.0;
  const bool ok_small = group_reduce(G, 1, 1, out);
  const bool ok_publish = group_reduce(G, 1, 1, out, ~0ull);
  if (threadIdx.x == 0) P->st->status = (!ok_small && !ok_publish) ? SC_ETIMEOUT : SC_OK;
}

// Times `iters` inner iterations of the persistent engine on the problem
// set for every tile scale and keeps the fastest for the classes present.
template <class SETUP>
static int tune_solver_set(std::vector<ProbSpec> &sps, void *work, size_t work_bytes, int iters, cudaStream_t st,
                           SETUP setup, sc_solver_tuning *out) {
  if (!work) return fail(SC_EINVAL, "null work space");
  if (iters < 1 || iters > 100000) return fail(SC_EINVAL, "iters must be 1..100000");
  for (const ProbSpec &sp : sps)
    if (sp.solver != SC_SOLVER_PERSISTENT) return fail(SC_EINVAL, "the tuner times the persistent solver");
  const size_t need = batch_bytes(sps);
  if (work_bytes < need) return fail(SC_ENOMEM, "work space %zu < %zu bytes", work_bytes, need);
  bool cls[2][2] = {{false, false}, {false, false}};
  for (const ProbSpec &sp : sps) cls[sp.ndim == 3][sp.mixed ? 1 : 0] = true;
  int saved[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) saved[a][b] = g_tile_log2[a][b].load();
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best_ms = 1e300;
  int best = 0;
  std::memset(out, 0, sizeof(*out));
  for (int lg = TILE_LOG2_MIN; lg <= TILE_LOG2_MAX; ++lg) {
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        if (cls[a][b]) g_tile_log2[a][b].store(lg + 8);
    Carver cv(work, work_bytes);
    std::vector<SolveProb> hp(sps.size());
    std::vector<ProbAux> aux(sps.size());
    for (size_t i = 0; i < sps.size(); ++i) {
      layout(sps[i], cv, hp[i], aux[i]);
      aux[i].ones = static_cast<double *>(cv.take(std::max<long long>(hp[i].npts, 1) * 8));
    }
    SolveProb *dprobs = static_cast<SolveProb *>(cv.take(sps.size() * sizeof(SolveProb)));
    int *dmap = static_cast<int *>(cv.take(sizeof(int) * size_t(32) * num_sms()));
    unsigned *dbars = static_cast<unsigned *>(cv.take(sps.size() * 2 * sizeof(unsigned)));
    int rc = SC_OK;
    for (size_t i = 0; i < sps.size() && !rc; ++i) {
      rc = upload_prob(sps[i], hp[i], aux[i], st);
      if (!rc) rc = setup(int(i), hp[i], aux[i]);
    }
    float ms = 0.0f;
    if (!rc) {
      cudaEventRecord(e0, st);
      rc = run_persistent(hp, dprobs, dmap, dbars, st, iters, 0.0);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    if (rc) {
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) g_tile_log2[a][b].store(saved[a][b]);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc;
    }
    out->ms[lg - TILE_LOG2_MIN] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = lg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) g_tile_log2[a][b].store(cls[a][b] ? best + 8 : saved[a][b]);
  out->log2_scale = best;
  clear_error();
  return SC_OK;
}

}  // namespace sc

using namespace sc;

extern "C" {

int sc_selftest_barrier_timeout(void *work_dev, size_t work_bytes, int64_t spin_limit, int32_t *status_out,
                                sc_stream_t stream) {
  if (!work_dev || !status_out || spin_limit < 1 || spin_limit > (1LL << 24))
    return fail(SC_EINVAL, "bad argument");
  if (work_bytes < 4096) return fail(SC_ENOMEM, "work space too small");
  cudaStream_t st = (cudaStream_t)stream;
  char *w = static_cast<char *>(work_dev);
  SolveProb P;
  std::memset(&P, 0, sizeof(P));
  P.ncta = 2;  // a second member that never arrives
  P.nslot = 8;
  P.part = reinterpret_cast<double *>(w + 1024);
  P.scal = reinterpret_cast<double *>(w + 1536);
  P.bar = reinterpret_cast<unsigned *>(w + 1792);
  P.st = reinterpret_cast<SolveState *>(w + 2048);
  SolveProb *dP = reinterpret_cast<SolveProb *>(w);
  cudaMemsetAsync(w + 1024, 0, 2048, st);
  cudaMemcpyAsync(dP, &P, sizeof(P), cudaMemcpyHostToDevice, st);
  k_barrier_timeout_probe<<<1, CG_NTHR, 0, st>>>(dP, spin_limit);
  SolveState s;
  cudaMemcpyAsync(&s, P.st, sizeof(s), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SC_ECUDA, "self-test: %s", cudaGetErrorString(e));
  *status_out = s.status;
  clear_error();
  return SC_OK;
}

size_t sc_ch_run_work_bytes(const sc_ch *c, int64_t nsteps) {
  if (ch_validate(c) || nsteps < 1) return 0;
  const size_t base = sc_ch_work_bytes(c);
  return base + size_t(nsteps) * c->batch * sizeof(SolveState) + 1024;
}

int sc_ch_run(const sc_ch *c, double *u_dev, int64_t nsteps, int32_t use_graph, void *work_dev,
              size_t work_bytes, sc_solve_info *infos, sc_stream_t stream) {
  if (int rc = ch_validate(c)) return rc;
  if (!u_dev || !infos || !work_dev || nsteps < 1) return fail(SC_EINVAL, "bad argument");
  if (c->solver != SC_SOLVER_PERSISTENT) return fail(SC_EINVAL, "sc_ch_run uses the persistent solver");
  const size_t need = sc_ch_run_work_bytes(c, nsteps);
  if (work_bytes < need) return fail(SC_ENOMEM, "work space %zu < %zu bytes", work_bytes, need);
  auto t0 = std::chrono::steady_clock::now();
  // The run goes on a private non-blocking stream ordered after the caller's
  // (the legacy default stream cannot be captured into a graph).
  cudaStream_t cst = (cudaStream_t)stream, st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
    return fail(SC_ECUDA, "stream creation failed");
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } guard{st};
  {
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, cst);
    cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
  }
  std::vector<ProbSpec> sps(c->batch);
  for (int i = 0; i < c->batch; ++i) ch_spec(c, i, u_dev, sps[i]);
  Carver cv(work_dev, work_bytes);
  std::vector<SolveProb> hp(sps.size());
  std::vector<ProbAux> aux(sps.size());
  for (size_t i = 0; i < sps.size(); ++i) {
    layout(sps[i], cv, hp[i], aux[i]);
    aux[i].ones = static_cast<double *>(cv.take(std::max<long long>(hp[i].npts, 1) * 8));
  }
  SolveProb *dprobs = static_cast<SolveProb *>(cv.take(sps.size() * sizeof(SolveProb)));
  int *dmap = static_cast<int *>(cv.take(sizeof(int) * size_t(32) * num_sms()));
  unsigned *dbars = static_cast<unsigned *>(cv.take(sps.size() * 2 * sizeof(unsigned)));
  SolveState *dinfo = static_cast<SolveState *>(cv.take(size_t(nsteps) * sps.size() * sizeof(SolveState)));
  int *dstep = static_cast<int *>(cv.take(sizeof(int)));
  for (size_t i = 0; i < sps.size(); ++i)
    if (int rc = upload_prob(sps[i], hp[i], aux[i], st)) return rc;
  const bool mixed = hp[0].mixed != 0;
  std::vector<int> idx(sps.size()), map;
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = int(i);
  const int dims = dims_mask(hp, idx);
  const int G = max_group_ctas(mixed, dims);
  if (int rc = assign_groups(hp, idx, G, dbars, map)) return rc;
  cudaMemcpyAsync(dprobs, hp.data(), hp.size() * sizeof(SolveProb), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dmap, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(dstep, 0, sizeof(int), st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SC_ECUDA, "set-up: %s", cudaGetErrorString(e));
  const int n = int(sps.size());
  auto enqueue_step = [&]() -> int {
    for (int i = 0; i < n; ++i)
      if (int rc = setup_ch(c, sps[i], hp[i], aux[i], st)) return rc;
    k_reset_states<<<(n + 127) / 128, 128, 0, st>>>(dprobs, n);
    cudaMemsetAsync(dbars, 0, size_t(n) * 2 * sizeof(unsigned), st);
    int rc = mixed ? enqueue_cg<float>(dprobs, dmap, int(map.size()), st, LLONG_MAX, 0ull, dims)
                   : enqueue_cg<double>(dprobs, dmap, int(map.size()), st, LLONG_MAX, 0ull, dims);
    if (rc) return rc;
    k_record_states<<<1, 128, 0, st>>>(dprobs, n, dinfo, dstep);
    return SC_OK;
  };
  // first step directly (also initialises every kernel's attributes)
  if (int rc = enqueue_step()) return rc;
  if (nsteps > 1) {
    if (use_graph) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) return fail(SC_ECUDA, "begin capture: %s", cudaGetErrorString(e));
      int rc = enqueue_step();
      e = cudaStreamEndCapture(st, &graph);
      if (rc) return rc;
      if (e != cudaSuccess) return fail(SC_ECUDA, "end capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&exec, graph, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(SC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
      }
      for (int64_t k = 1; k < nsteps && e == cudaSuccess; ++k) e = cudaGraphLaunch(exec, st);
      cudaError_t e2 = cudaStreamSynchronize(st);
      cudaGraphExecDestroy(exec);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(SC_ECUDA, "graph replay: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    } else {
      for (int64_t k = 1; k < nsteps; ++k)
        if (int rc = enqueue_step()) return rc;
    }
  }
  std::vector<SolveState> hs(size_t(nsteps) * n);
  cudaMemcpyAsync(hs.data(), dinfo, hs.size() * sizeof(SolveState), cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SC_ECUDA, "multi-step run: %s", cudaGetErrorString(e));
  const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (size_t k = 0; k < hs.size(); ++k) {
    sc_solve_info &in = infos[k];
    std::memset(&in, 0, sizeof(in));
    in.prec = mixed ? SC_PREC_MIXED : SC_PREC_F64;
    in.seconds = sec;
    in.iters = hs[k].iters;
    in.outer = hs[k].outer;
    in.rel_res = hs[k].rel;
    in.status = hs[k].phase == 2 ? hs[k].status : SC_ETIMEOUT;
  }
  clear_error();
  return SC_OK;
}

size_t sc_bvp_batch_work_bytes(const sc_bvp *probs, int32_t count) {
  if (!probs || count < 1) return 0;
  std::vector<ProbSpec> sps(count);
  for (int i = 0; i < count; ++i)
    if (bvp_spec(&probs[i], sps[i])) return 0;
  return batch_bytes(sps);
}

size_t sc_bvp_work_bytes(const sc_bvp *p) { return sc_bvp_batch_work_bytes(p, 1); }

int sc_autotune_solver(const sc_bvp *probs, int32_t count, int32_t iters, void *work_dev, size_t work_bytes,
                       sc_solver_tuning *out, sc_stream_t stream) {
  if (!probs || count < 1 || !out) return fail(SC_EINVAL, "bad arguments");
  std::vector<ProbSpec> sps(count);
  for (int i = 0; i < count; ++i)
    if (int rc = bvp_spec(&probs[i], sps[i])) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  return tune_solver_set(sps, work_dev, work_bytes, iters, st, [&](int i, SolveProb &P, ProbAux &aux) {
    return setup_bvp(&probs[i], sps[i], P, aux, st);
  }, out);
}

int sc_autotune_ch(const sc_ch *c, double *u_dev, int32_t iters, void *work_dev, size_t work_bytes,
                   sc_solver_tuning *out, sc_stream_t stream) {
  if (int rc = ch_validate(c)) return rc;
  if (!u_dev || !out) return fail(SC_EINVAL, "null pointer");
  std::vector<ProbSpec> sps(c->batch);
  for (int i = 0; i < c->batch; ++i) ch_spec(c, i, u_dev, sps[i]);
  cudaStream_t st = (cudaStream_t)stream;
  return tune_solver_set(sps, work_dev, work_bytes, iters, st, [&](int i, SolveProb &P, ProbAux &aux) {
    return setup_ch(c, sps[i], P, aux, st);
  }, out);
}

int sc_solver_tile_scale_set(int32_t ndim, int32_t prec, int32_t log2_scale) {
  if (ndim != 2 && ndim != 3) return fail(SC_EINVAL, "ndim must be 2 or 3");
  if (prec != SC_PREC_F64 && prec != SC_PREC_MIXED) return fail(SC_EINVAL, "prec must be F64 or MIXED");
  if (log2_scale < TILE_LOG2_MIN || log2_scale > TILE_LOG2_MAX) return fail(SC_EINVAL, "log2_scale out of range");
  g_tile_log2[ndim == 3][prec == SC_PREC_MIXED].store(log2_scale + 8);
  clear_error();
  return SC_OK;
}

int sc_solver_tile_scale_get(int32_t ndim, int32_t prec, int32_t *log2_scale) {
  if ((ndim != 2 && ndim != 3) || (prec != SC_PREC_F64 && prec != SC_PREC_MIXED) || !log2_scale)
    return fail(SC_EINVAL, "bad arguments");
  *log2_scale = g_tile_log2[ndim == 3][prec == SC_PREC_MIXED].load() - 8;
  clear_error();
  return SC_OK;
}

int sc_solve_biharmonic_batch(const sc_bvp *probs, int32_t count, void *work_dev, size_t work_bytes,
                              sc_solve_info *infos, sc_stream_t stream) {
  if (!probs || count < 1 || !infos) return fail(SC_EINVAL, "bad batch arguments");
  std::vector<ProbSpec> sps(count);
  for (int i = 0; i < count; ++i)
    if (int rc = bvp_spec(&probs[i], sps[i])) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  return solve_set(sps, work_dev, work_bytes, infos, st,
                   [&](int i, SolveProb &P, ProbAux &aux) { return setup_bvp(&probs[i], sps[i], P, aux, st); });
}

int sc_solve_biharmonic(const sc_bvp *p, void *work_dev, size_t work_bytes, sc_solve_info *info,
                        sc_stream_t stream) {
  return sc_solve_biharmonic_batch(p, 1, work_dev, work_bytes, info, stream);
}

size_t sc_ch_work_bytes(const sc_ch *c) {
  if (ch_validate(c)) return 0;
  std::vector<ProbSpec> sps(c->batch);
  for (int i = 0; i < c->batch; ++i) ch_spec(c, i, nullptr, sps[i]);
  return batch_bytes(sps);
}

int sc_ch_step_sbdf(const sc_ch *c, int32_t order, double *u_dev, double *hist_dev, void *work_dev,
                    size_t work_bytes, sc_solve_info *infos, sc_stream_t stream) {
  if (int rc = ch_validate(c)) return rc;
  if (order < 1 || order > 3) return fail(SC_EINVAL, "order must be 1, 2 or 3");
  if (!u_dev || !infos || (order > 1 && !hist_dev)) return fail(SC_EINVAL, "null pointer");
  // SBDF coefficients of the form (I + g dt M kappa B) u+ = sum al_j u^(n-j) + g dt M Lap sum b_j f'
  static const double AL[4][3] = {{0, 0, 0}, {1, 0, 0}, {4.0 / 3.0, -1.0 / 3.0, 0}, {18.0 / 11.0, -9.0 / 11.0, 2.0 / 11.0}};
  static const double BE[4][3] = {{0, 0, 0}, {1, 0, 0}, {2, -1, 0}, {3, -3, 1}};
  static const double GA[4] = {0, 1.0, 2.0 / 3.0, 6.0 / 11.0};
  const double gdt = GA[order] * c->dt;
  std::vector<ProbSpec> sps(c->batch);
  const double h = double(c->h_num) / double(c->h_den);
  for (int i = 0; i < c->batch; ++i) {
    ch_spec(c, i, u_dev, sps[i]);
    sps[i].b = gdt * c->M * c->kappa;
    const int prec = choose_prec(c->prec, kappa_estimate(sps[i], h));
    sps[i].mixed = prec == SC_PREC_MIXED && c->solver == SC_SOLVER_PERSISTENT;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long long npts = c->n[0] * c->n[1] * (c->ndim == 3 ? c->n[2] : 1);
  const long long per = npts * c->batch;  // history slice j at hist_dev + (j - 1) * per
  return solve_set(sps, work_dev, work_bytes, infos, st, [&](int i, SolveProb &P, ProbAux &aux) -> int {
    const ProbSpec &sp = sps[i];
    double *u0 = sp.x;
    double *h1 = order > 1 ? hist_dev + (long long)i * npts : nullptr;
    double *h2 = order > 2 ? hist_dev + per + (long long)i * npts : nullptr;
    k_fprime_hist<<<grid1d(npts), 256, 0, st>>>(u0, h1, h2, order, BE[order][0], BE[order][1], BE[order][2],
                                                aux.scratch, npts, c->chem, c->rho, c->ca, c->cb);
    sc_stencil L;
    sc_laplacian(sp.ndim, sp.order, &L);
    ApplyReq q{&L, SC_F64, SC_BC_PERIODIC, sp.n, sp.h_num, sp.h_den, aux.scratch, P.rhs};
    if (int rc = apply_enqueue(q, st)) return rc;
    k_sbdf_rhs<<<grid1d(npts), 256, 0, st>>>(P.rhs, u0, h1, h2, order, AL[order][0], AL[order][1], AL[order][2],
                                             gdt * c->M, npts);
    // the history for the next step: u^(n-1) -> slot 2, u^n -> slot 1
    if (order > 2) cudaMemcpyAsync(h2, h1, size_t(npts) * 8, cudaMemcpyDeviceToDevice, st);
    if (order > 1) cudaMemcpyAsync(h1, u0, size_t(npts) * 8, cudaMemcpyDeviceToDevice, st);
    return SC_OK;
  });
}

int sc_ch_step(const sc_ch *c, double *u_dev, void *work_dev, size_t work_bytes, sc_solve_info *infos,
               sc_stream_t stream) {
  if (int rc = ch_validate(c)) return rc;
  if (!u_dev || !infos) return fail(SC_EINVAL, "null pointer");
  std::vector<ProbSpec> sps(c->batch);
  for (int i = 0; i < c->batch; ++i) ch_spec(c, i, u_dev, sps[i]);
  cudaStream_t st = (cudaStream_t)stream;
  return solve_set(sps, work_dev, work_bytes, infos, st,
                   [&](int i, SolveProb &P, ProbAux &aux) { return setup_ch(c, sps[i], P, aux, st); });
}

int sc_ch_stats(const sc_ch *c, const double *u_dev, double *mass_host, double *energy_host, void *work_dev,
                size_t work_bytes, sc_stream_t stream) {
  if (int rc = ch_validate(c)) return rc;
  if (!u_dev || !mass_host || !energy_host || !work_dev) return fail(SC_EINVAL, "null pointer");
  const long long npts = c->n[0] * c->n[1] * (c->ndim == 3 ? c->n[2] : 1);
  const int nblk = int((npts + PL_CHUNK - 1) / PL_CHUNK);
  if (work_bytes < size_t(2 * nblk + 2) * 8) return fail(SC_ENOMEM, "work space too small");
  double *pm = static_cast<double *>(work_dev), *pe = pm + nblk, *out = pe + nblk;
  cudaStream_t st = (cudaStream_t)stream;
  const double h = double(c->h_num) / double(c->h_den);
  const double hd = c->ndim == 3 ? h * h * h : h * h;
  for (int b = 0; b < c->batch; ++b) {
    k_ch_stats_part<<<nblk, PL_NTHR, 0, st>>>(u_dev + (long long)b * npts, c->ndim, int(c->n[0]), int(c->n[1]),
                                               c->ndim == 3 ? int(c->n[2]) : 1, h, c->kappa, c->chem, c->rho,
                                               c->ca, c->cb, pm, pe);
    k_sum_final<<<1, PL_NTHR, 0, st>>>(pm, nblk, out, 0);
    k_sum_final<<<1, PL_NTHR, 0, st>>>(pe, nblk, out, 1);
    double hs[2];
    cudaMemcpyAsync(hs, out, 16, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SC_ECUDA, "stats: %s", cudaGetErrorString(e));
    mass_host[b] = hs[0];
    energy_host[b] = hs[1] * hd;
  }
  clear_error();
  return SC_OK;
}

}  // extern "C"
