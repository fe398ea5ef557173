// sc_apply_composed: host dispatch of the flat composed-stencil apply.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "sc_apply.cuh"
#include "sc_apply_df.h"
#include "sc_apply_host.h"
#include "sc_internal.h"

namespace sc {

template <typename T, int NDIM, int R, int CLS>
__global__ void __launch_bounds__(FlatApply<T, NDIM, R, CLS>::NTHR)
    flat_apply_kernel(const T *__restrict__ x, T *__restrict__ y, ApplyGeom g,
                      const __grid_constant__ BoxWeights<T, NDIM, R> W, const int *__restrict__ guard) {
  using K = FlatApply<T, NDIM, R, CLS>;
  if (guard && __ldcg(guard) == 0) return;  // conditional fallback pass: nothing to redo
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smem = reinterpret_cast<T *>(smem_raw);
  const int x0 = blockIdx.x * K::BX;
  const int y0 = NDIM == 3 ? blockIdx.y * K::BY : 0;
  const int z0 = (NDIM == 3 ? blockIdx.z : blockIdx.y) * g.H;
  StoreEpi<T, NDIM, K::VX> epi{y, &g};
  K::run_tile(x, g, W, x0, y0, z0, smem, epi);
}

// SM count of the current device, cached per device ordinal (0: not read yet)
int num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  cudaGetDevice(&dev);
  std::atomic<int> &c = cache[dev & 63];
  int n = c.load(std::memory_order_relaxed);
  if (n <= 0) {
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
    c.store(n, std::memory_order_relaxed);
  }
  return n;
}

int wave_planes(long long tiles_xy, int nplanes, int R, long long slots, int hmin) {
  // Each SM runs up to occ = slots / SMs CTAs at a time; a CTA streams H + 2R
  // planes.  Time ~ rounds * (H + 2R) with rounds = ceil(ceil(CTAs/SMs)/occ):
  // a last round with a single CTA per SM costs as much as a full one.
  // Grids that leave more than a quarter of the slots empty are only taken
  // when nothing larger exists (small problems).
  if (nplanes <= 1) return 1;
  const long long sms = num_sms();
  const long long occ = std::max<long long>(1, slots / sms);
  long long best_h = -1, small_h = nplanes;
  double best = 1e300;
  for (long long zb = 1; zb <= nplanes; ++zb) {
    const long long h = (nplanes + zb - 1) / zb;
    if (h < hmin && zb > 1) break;
    small_h = h;
    const long long ctas = tiles_xy * ((nplanes + h - 1) / h);
    if (4 * ctas >= 3 * slots) {
      const long long per_sm = (ctas + sms - 1) / sms;
      const long long rounds = (per_sm + occ - 1) / occ;
      const double cost = double(rounds) * double(h + 2 * R);
      if (cost < best * 0.999) {
        best = cost;
        best_h = h;
      }
    }
    if (h == hmin) break;
  }
  return int(best_h > 0 ? best_h : small_h);
}

// Output planes per CTA (see wave_planes).
template <typename KERN>
static int choose_h(KERN kern, int nthr, size_t smem, long long tiles_per_plane, int nplanes, int R,
                    int override_h) {
  if (override_h > 0) return std::min(override_h, nplanes);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nthr, smem);
  const long long slots = (long long)std::max(occ, 1) * num_sms();
  return wave_planes(tiles_per_plane, nplanes, R, slots, std::max(4 * R, 8));
}


template <typename T, int NDIM, int R, int CLS>
static int launch_flat(const ApplyReq &q, const T *wts_sparse, cudaStream_t st) {
  using K = FlatApply<T, NDIM, R, CLS>;
  BoxWeights<T, NDIM, R> W;
  for (int i = 0; i < BoxWeights<T, NDIM, R>::N; ++i) W.w[i] = T(0);
  const int Wd = 2 * R + 1;
  for (int k = 0; k < q.s->npts; ++k) {
    const int dx = q.s->off[k][0], dy = q.s->off[k][1], dz = q.s->off[k][2];
    int idx;
    if (NDIM == 3)
      idx = ((dz + R) * Wd + (dy + R)) * Wd + (dx + R);
    else
      idx = (dy + R) * Wd + (dx + R);
    W.w[idx] = wts_sparse[k];
  }
  ApplyGeom g;
  g.nx = int(q.dims[0]);
  g.ny = int(q.dims[1]);
  g.nz = NDIM == 3 ? int(q.dims[2]) : 1;
  g.bc = q.bc;
  const int sh = q.bc == SC_BC_GHOSTED ? 2 * q.s->radius : 0;
  // strides are those of the arrays (ghosted input carries the ring of the
  // stencil's own radius, which may be smaller than the class radius R)
  g.in_sy = g.nx + sh;
  g.in_ss = (long long)(g.nx + sh) * (g.ny + sh);
  g.out_sy = g.nx;
  g.out_ss = (long long)g.nx * g.ny;
  const int ns = NDIM == 3 ? g.nz : g.ny;
  const long long tiles = (long long)((g.nx + K::BX - 1) / K::BX) *
                          (NDIM == 3 ? (g.ny + K::BY - 1) / K::BY : 1);
  auto kern = flat_apply_kernel<T, NDIM, R, CLS>;
  static std::atomic<unsigned long long> smem_set{0};
  set_smem_limit_once(kern, K::SMEM, smem_set);
  g.H = choose_h(kern, K::NTHR, K::SMEM, tiles, ns, R, q.planes);
  const uintptr_t xa = reinterpret_cast<uintptr_t>(q.x), ya = reinterpret_cast<uintptr_t>(q.y);
  bool vec = (xa % 16 == 0) && (ya % 16 == 0) && (g.nx % K::CH == 0);
  if (q.bc == SC_BC_GHOSTED) vec = vec && (q.s->radius == R) && ((R - K::HX) % K::CH == 0) &&
                                    ((g.nx + sh) % K::CH == 0);
  if (q.bc == SC_BC_PERIODIC) vec = vec && (g.nx >= K::HX);
  g.vec = vec ? 1 : 0;
  if (q.bc == SC_BC_GHOSTED && q.s->radius != R)
    return fail(SC_EINVAL, "ghosted apply needs the class radius to equal the stencil radius");
  dim3 grid((g.nx + K::BX - 1) / K::BX, NDIM == 3 ? (g.ny + K::BY - 1) / K::BY : (ns + g.H - 1) / g.H,
            NDIM == 3 ? (ns + g.H - 1) / g.H : 1);
  kern<<<grid, K::NTHR, K::SMEM, st>>>(static_cast<const T *>(q.x), static_cast<T *>(q.y), g, W, q.guard);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SC_ECUDA, "apply launch: %s", cudaGetErrorString(e));
  return SC_OK;
}


template <typename T>
static int dispatch(const ApplyReq &q, cudaStream_t st) {
  std::vector<T> w(q.s->npts);
  int rc = (sizeof(T) == 8) ? weights_f64(q.s, q.h_num, q.h_den, reinterpret_cast<double *>(w.data()))
                            : weights_f32(q.s, q.h_num, q.h_den, reinterpret_cast<float *>(w.data()));
  if (rc) return rc;
  const int nd = q.s->ndim;
  bool c2 = true, c4 = true, star = true;
  for (int k = 0; k < q.s->npts; ++k) {
    const int dx = q.s->off[k][0], dy = q.s->off[k][1], dz = q.s->off[k][2];
    star = star && in_support<CLS_STAR, 4>(dx, dy, dz);
    c2 = c2 && std::max({std::abs(dx), std::abs(dy), std::abs(dz)}) <= 2 &&
         in_support<CLS_CROSS2, 2>(dx, dy, dz);
    c4 = c4 && std::max({std::abs(dx), std::abs(dy), std::abs(dz)}) <= 4 &&
         in_support<CLS_CROSS2, 4>(dx, dy, dz);
  }
  const int r = q.s->radius;
  // the ghosted layout has a ring of the stencil's radius; the class radius
  // must equal it for the strides to match
  if (nd == 2) {
    if (star && r == 1) return launch_flat<T, 2, 1, CLS_STAR>(q, w.data(), st);
    if (star && r == 2) return launch_flat<T, 2, 2, CLS_STAR>(q, w.data(), st);
    if (c2 && (q.bc != SC_BC_GHOSTED || r == 2)) return launch_flat<T, 2, 2, CLS_CROSS2>(q, w.data(), st);
    if (c4 && (q.bc != SC_BC_GHOSTED || r == 4)) return launch_flat<T, 2, 4, CLS_CROSS2>(q, w.data(), st);
    if (r <= 1 && (q.bc != SC_BC_GHOSTED || r == 1)) return launch_flat<T, 2, 1, CLS_BOX>(q, w.data(), st);
    if (r <= 2 && (q.bc != SC_BC_GHOSTED || r == 2)) return launch_flat<T, 2, 2, CLS_BOX>(q, w.data(), st);
    if (r <= 4 && (q.bc != SC_BC_GHOSTED || r == 4)) return launch_flat<T, 2, 4, CLS_BOX>(q, w.data(), st);
  } else {
    if (star && r == 1) return launch_flat<T, 3, 1, CLS_STAR>(q, w.data(), st);
    if (star && r == 2) return launch_flat<T, 3, 2, CLS_STAR>(q, w.data(), st);
    if (c2 && (q.bc != SC_BC_GHOSTED || r == 2)) return launch_flat<T, 3, 2, CLS_CROSS2>(q, w.data(), st);
    if (c4 && (q.bc != SC_BC_GHOSTED || r == 4)) return launch_flat<T, 3, 4, CLS_CROSS2>(q, w.data(), st);
    if (r <= 1 && (q.bc != SC_BC_GHOSTED || r == 1)) return launch_flat<T, 3, 1, CLS_BOX>(q, w.data(), st);
    if (r <= 2 && (q.bc != SC_BC_GHOSTED || r == 2)) return launch_flat<T, 3, 2, CLS_BOX>(q, w.data(), st);
  }
  return fail(SC_EINVAL, "stencil support is not covered by a compiled apply class "
                         "(2D: radius <= 4; 3D: Lap o Lap supports of radius <= 4 or any radius <= 2)");
}

int validate_apply(const sc_stencil *s, int dtype, int bc, const int64_t *dims, int64_t h_num,
                   int64_t h_den) {
  if (!s || !dims) return fail(SC_EINVAL, "null argument");
  if (s->ndim != 2 && s->ndim != 3) return fail(SC_EINVAL, "apply needs a 2D or 3D stencil");
  if (s->npts < 1 || s->npts > SC_MAX_PTS) return fail(SC_EINVAL, "bad npts");
  if (s->radius > SC_MAX_APPLY_RADIUS) return fail(SC_EINVAL, "radius %d > %d", s->radius, SC_MAX_APPLY_RADIUS);
  if (dtype != SC_F64 && dtype != SC_F32) return fail(SC_EINVAL, "unknown dtype");
  if (bc != SC_BC_PERIODIC && bc != SC_BC_GHOSTED && bc != SC_BC_ZERO) return fail(SC_EINVAL, "unknown bc");
  if (h_num <= 0 || h_den <= 0) return fail(SC_EINVAL, "h must be positive");
  for (int a = 0; a < s->ndim; ++a) {
    if (dims[a] < 1 || dims[a] > (1 << 30)) return fail(SC_EINVAL, "dims[%d] out of range", a);
    if (bc == SC_BC_PERIODIC && dims[a] < 4) return fail(SC_EINVAL, "periodic grids need n >= 4");
  }
  long long tot = 1;
  for (int a = 0; a < s->ndim; ++a) tot *= dims[a];
  if (tot > (1LL << 34)) return fail(SC_EINVAL, "grid too large");
  return SC_OK;
}

int apply_enqueue(const ApplyReq &q, cudaStream_t st) {
  return q.dtype == SC_F64 ? dispatch<double>(q, st) : dispatch<float>(q, st);
}

size_t grid_elems(const sc_stencil *s, int bc, const int64_t *dims, bool input) {
  size_t n = 1;
  const int sh = (input && bc == SC_BC_GHOSTED) ? 2 * s->radius : 0;
  for (int a = 0; a < s->ndim; ++a) n *= size_t(dims[a] + sh);
  return n;
}


// xp = x surrounded by a zero ring of width R (all dims).
template <typename T>
__global__ void k_pad_zero(const T *__restrict__ x, T *__restrict__ xp, int ndim, long long nx, long long ny,
                           long long nz, int R) {
  const long long px = nx + 2 * R, py = ny + 2 * R, pz = ndim == 3 ? nz + 2 * R : 1;
  const long long n = px * py * pz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long ix = i % px - R, iy = (i / px) % py - R, iz = ndim == 3 ? i / (px * py) - R : 0;
    const bool in = ix >= 0 && ix < nx && iy >= 0 && iy < ny && iz >= 0 && iz < (ndim == 3 ? nz : 1);
    xp[i] = in ? x[(iz * ny + iy) * nx + ix] : T(0);
  }
}

static size_t elems_ext(int ndim, const int64_t *dims, int ext) {
  size_t n = 1;
  for (int a = 0; a < ndim; ++a) n *= size_t(dims[a] + 2 * ext);
  return n;
}

size_t grid_elems_ext(int ndim, const int64_t *dims, int ext) { return elems_ext(ndim, dims, ext); }

bool spans_overlap(const void *a, size_t na, const void *b, size_t nb) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  return na && nb && a0 < b0 + nb && b0 < a0 + na;
}

int check_disjoint(int ndim, int bc, const int64_t *dims, int r_in, size_t es, const void *x, const void *y,
                   const void *work, size_t work_bytes) {
  const size_t xb = elems_ext(ndim, dims, bc == SC_BC_GHOSTED ? r_in : 0) * es;
  const size_t yb = elems_ext(ndim, dims, 0) * es;
  if (spans_overlap(x, xb, y, yb)) return fail(SC_EINVAL, "x and y must not overlap");
  if (work && (spans_overlap(work, work_bytes, x, xb) || spans_overlap(work, work_bytes, y, yb)))
    return fail(SC_EINVAL, "the work space must not overlap x or y");
  return SC_OK;
}

size_t composition_work_bytes(const sc_stencil *B, const sc_stencil *A, int dtype, int bc, const int64_t *dims) {
  const size_t es = dtype == SC_F64 ? 8 : 4;
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  size_t b = up(elems_ext(A->ndim, dims, B->radius) * es);
  if (bc == SC_BC_ZERO) b += up(elems_ext(A->ndim, dims, A->radius + B->radius) * es);
  return b + 256;  // + the out-of-range flag of the pair-arithmetic path
}

// y = B(A x): the inner stencil on the grid extended by B's radius into a
// temporary, then the outer stencil (Eq. C=B(A), nested form).
int composition_enqueue(const sc_stencil *B, const sc_stencil *A, int dtype, int bc, const int64_t *dims,
                        int64_t h_num, int64_t h_den, const void *x, void *y, void *work, cudaStream_t st,
                        int arith, int planes) {
  const int nd = A->ndim, rA = A->radius, rB = B->radius;
  const size_t es = dtype == SC_F64 ? 8 : 4;
  char *w = static_cast<char *>(work);
  void *t = w;
  const size_t tb = (elems_ext(nd, dims, rB) * es + 255) & ~size_t(255);
  int64_t dext[3] = {1, 1, 1};
  for (int a = 0; a < nd; ++a) dext[a] = dims[a] + 2 * rB;
  const size_t xpb = bc == SC_BC_ZERO ? (elems_ext(nd, dims, rA + rB) * es + 255) & ~size_t(255) : 0;
  int *flag = reinterpret_cast<int *>(w + tb + xpb);
  // pair arithmetic for FP64 Laplacian compositions (see sc_apply_df.cu)
  float ca[3], cb[3];
  bool pair = arith == SC_ARITH_PAIR && dtype == SC_F64 && rA == rB && star_int_form(A, ca, ca + 1, ca + 2) &&
              star_int_form(B, cb, cb + 1, cb + 2) && A->hpow == B->hpow;
  double scale = 1.0;
  if (pair) {
    // exact rational 1 / (den_A den_B h^(pA + pB)), rounded once
    sc_stencil one;
    std::memset(&one, 0, sizeof(one));
    one.ndim = nd;
    one.npts = 1;
    one.hpow = A->hpow + B->hpow;
    one.den = 1;
    one.num[0] = 1;
    double unit = 0.0;
    if (int rc = weights_f64(&one, h_num, h_den, &unit)) return rc;
    scale = unit / (double(A->den) * double(B->den));  // den products are small integers: exact
    if (!(double(A->den) * double(B->den) < 9007199254740992.0)) return fail(SC_EOVERFLOW, "denominator");
    const void *xin = bc == SC_BC_ZERO ? static_cast<const void *>(w + tb) : x;
    pair = df_supported(nd, rA, dims, bc == SC_BC_PERIODIC ? SC_BC_PERIODIC : SC_BC_GHOSTED, scale, xin, t, y);
  }
  if (pair) cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (bc == SC_BC_PERIODIC) {
    if (pair) {
      if (int rc = df_composition_enqueue(nd, rA, x, t, y, dims, dims, SC_BC_PERIODIC, ca, cb, scale, flag, st,
                                          planes))
        return rc;
    }
    ApplyReq qa{A, dtype, SC_BC_PERIODIC, dims, h_num, h_den, x, t, pair ? flag : nullptr, pair ? 0 : planes};
    if (int rc = apply_enqueue(qa, st)) return rc;
    ApplyReq qb{B, dtype, SC_BC_PERIODIC, dims, h_num, h_den, t, y, pair ? flag : nullptr, pair ? 0 : planes};
    return apply_enqueue(qb, st);
  }
  const void *xin = x;
  if (bc == SC_BC_ZERO) {
    void *xp = w + tb;
    const size_t n = elems_ext(nd, dims, rA + rB);
    const int g = int(std::min<size_t>((n + 255) / 256, 8 * size_t(num_sms())));
    if (dtype == SC_F64)
      k_pad_zero<double><<<g, 256, 0, st>>>(static_cast<const double *>(x), static_cast<double *>(xp), nd,
                                             dims[0], dims[1], nd == 3 ? dims[2] : 1, rA + rB);
    else
      k_pad_zero<float><<<g, 256, 0, st>>>(static_cast<const float *>(x), static_cast<float *>(xp), nd,
                                            dims[0], dims[1], nd == 3 ? dims[2] : 1, rA + rB);
    xin = xp;
  }
  // x (n + 2(rA + rB)) -> t (n + 2 rB) -> y (n)
  if (pair) {
    if (int rc = df_composition_enqueue(nd, rA, xin, t, y, dext, dims, SC_BC_GHOSTED, ca, cb, scale, flag, st,
                                        planes))
      return rc;
  }
  ApplyReq qa{A, dtype, SC_BC_GHOSTED, dext, h_num, h_den, xin, t, pair ? flag : nullptr, pair ? 0 : planes};
  if (int rc = apply_enqueue(qa, st)) return rc;
  ApplyReq qb{B, dtype, SC_BC_GHOSTED, dims, h_num, h_den, t, y, pair ? flag : nullptr, pair ? 0 : planes};
  return apply_enqueue(qb, st);
}

// t *= m (pointwise coefficient between the factors of a composition)
template <typename T>
__global__ void k_scale_pointwise(T *__restrict__ t, const T *__restrict__ m, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    t[i] *= m[i];
}

}  // namespace sc

using namespace sc;

extern "C" {

int sc_apply_varcoef(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, const int64_t *dims,
                     int64_t h_num, int64_t h_den, const void *m_dev, const void *x_dev, void *y_dev,
                     void *work_dev, size_t work_bytes, sc_stream_t stream) {
  if (int rc = validate_apply(outer, dtype, SC_BC_PERIODIC, dims, h_num, h_den)) return rc;
  if (int rc = validate_apply(inner, dtype, SC_BC_PERIODIC, dims, h_num, h_den)) return rc;
  if (outer->ndim != inner->ndim) return fail(SC_EINVAL, "outer and inner dimensions differ");
  if (!m_dev || !x_dev || !y_dev || !work_dev) return fail(SC_EINVAL, "null device pointer");
  const size_t es = dtype == SC_F64 ? 8 : 4;
  const long long n = (long long)grid_elems_ext(outer->ndim, dims, 0);
  if (work_bytes < size_t(n) * es) return fail(SC_ENOMEM, "work space %zu < %zu bytes", work_bytes, size_t(n) * es);
  if (int rc = check_disjoint(outer->ndim, SC_BC_PERIODIC, dims, 0, es, x_dev, y_dev, work_dev, size_t(n) * es))
    return rc;
  if (spans_overlap(m_dev, size_t(n) * es, work_dev, size_t(n) * es) ||
      spans_overlap(m_dev, size_t(n) * es, y_dev, size_t(n) * es))
    return fail(SC_EINVAL, "m must not overlap y or the work space");
  cudaStream_t st = (cudaStream_t)stream;
  ApplyReq qa{inner, dtype, SC_BC_PERIODIC, dims, h_num, h_den, x_dev, work_dev};
  if (int rc = apply_enqueue(qa, st)) return rc;
  const int g = int(std::min<long long>((n + 255) / 256, 8LL * num_sms()));
  if (dtype == SC_F64)
    k_scale_pointwise<double><<<g, 256, 0, st>>>(static_cast<double *>(work_dev), static_cast<const double *>(m_dev), n);
  else
    k_scale_pointwise<float><<<g, 256, 0, st>>>(static_cast<float *>(work_dev), static_cast<const float *>(m_dev), n);
  ApplyReq qb{outer, dtype, SC_BC_PERIODIC, dims, h_num, h_den, work_dev, y_dev};
  int rc = apply_enqueue(qb, st);
  if (!rc) clear_error();
  return rc;
}


int sc_apply_composed(const sc_stencil *s, int32_t dtype, int32_t bc, const int64_t *dims,
                      int64_t h_num, int64_t h_den, const void *x_dev, void *y_dev,
                      sc_stream_t stream) {
  if (int rc = validate_apply(s, dtype, bc, dims, h_num, h_den)) return rc;
  if (!x_dev || !y_dev) return fail(SC_EINVAL, "null device pointer");
  if (int rc = check_disjoint(s->ndim, bc, dims, s->radius, dtype == SC_F64 ? 8 : 4, x_dev, y_dev)) return rc;
  ApplyReq q{s, dtype, bc, dims, h_num, h_den, x_dev, y_dev};
  int rc = apply_enqueue(q, (cudaStream_t)stream);
  if (!rc) clear_error();
  return rc;
}

size_t sc_apply_composition_work_bytes(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype,
                                        int32_t bc, const int64_t *dims) {
  if (validate_apply(outer, dtype, bc, dims, 1, 1) || validate_apply(inner, dtype, bc, dims, 1, 1)) return 0;
  if (outer->ndim != inner->ndim) return 0;
  return composition_work_bytes(outer, inner, dtype, bc, dims);
}

int sc_apply_composition(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                         const int64_t *dims, int64_t h_num, int64_t h_den, const void *x_dev, void *y_dev,
                         void *work_dev, size_t work_bytes, int32_t arith, sc_stream_t stream) {
  if (arith != SC_ARITH_NATIVE && arith != SC_ARITH_PAIR) return fail(SC_EINVAL, "unknown arith %d", arith);
  if (int rc = validate_apply(outer, dtype, bc, dims, h_num, h_den)) return rc;
  if (int rc = validate_apply(inner, dtype, bc, dims, h_num, h_den)) return rc;
  if (outer->ndim != inner->ndim) return fail(SC_EINVAL, "outer and inner dimensions differ");
  if (outer->radius + inner->radius > SC_MAX_APPLY_RADIUS)
    return fail(SC_EINVAL, "composed radius %d > %d", outer->radius + inner->radius, SC_MAX_APPLY_RADIUS);
  if (!x_dev || !y_dev || !work_dev) return fail(SC_EINVAL, "null device pointer");
  const size_t need = composition_work_bytes(outer, inner, dtype, bc, dims);
  if (work_bytes < need) return fail(SC_ENOMEM, "work space %zu < %zu bytes", work_bytes, need);
  if (int rc = check_disjoint(outer->ndim, bc, dims, outer->radius + inner->radius, dtype == SC_F64 ? 8 : 4,
                              x_dev, y_dev, work_dev, need))
    return rc;
  int rc = composition_enqueue(outer, inner, dtype, bc, dims, h_num, h_den, x_dev, y_dev, work_dev,
                               (cudaStream_t)stream, arith);
  if (!rc) clear_error();
  return rc;
}

size_t sc_apply_host_work_bytes(const sc_stencil *s, int32_t dtype, int32_t bc, const int64_t *dims) {
  if (validate_apply(s, dtype, bc, dims, 1, 1)) return 0;
  const size_t es = dtype == SC_F64 ? 8 : 4;
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  return up(grid_elems(s, bc, dims, true) * es) + up(grid_elems(s, bc, dims, false) * es);
}

int sc_apply_composed_host(const sc_stencil *s, int32_t dtype, int32_t bc, const int64_t *dims,
                           int64_t h_num, int64_t h_den, const void *x_host, void *y_host,
                           void *work_dev, size_t work_bytes, sc_stream_t stream) {
  if (int rc = validate_apply(s, dtype, bc, dims, h_num, h_den)) return rc;
  if (!x_host || !y_host || !work_dev) return fail(SC_EINVAL, "null pointer");
  const size_t need = sc_apply_host_work_bytes(s, dtype, bc, dims);
  if (work_bytes < need) return fail(SC_ENOMEM, "work space %zu < %zu bytes", work_bytes, need);
  const size_t es = dtype == SC_F64 ? 8 : 4;
  const size_t nin = grid_elems(s, bc, dims, true) * es, nout = grid_elems(s, bc, dims, false) * es;
  char *xd = static_cast<char *>(work_dev);
  char *yd = xd + ((nin + 255) & ~size_t(255));
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(xd, x_host, nin, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(SC_ECUDA, "host-to-device copy failed");
  ApplyReq q{s, dtype, bc, dims, h_num, h_den, xd, yd};
  if (int rc = apply_enqueue(q, st)) return rc;
  if (cudaMemcpyAsync(y_host, yd, nout, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(SC_ECUDA, "device-to-host copy failed");
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SC_ECUDA, "apply: %s", cudaGetErrorString(e));
  clear_error();
  return SC_OK;
}

}  // extern "C"
