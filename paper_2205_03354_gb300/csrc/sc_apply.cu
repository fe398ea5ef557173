// sc_apply_composed: host dispatch of the flat composed-stencil apply.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sc_apply.cuh"
#include "sc_apply_host.h"
#include "sc_internal.h"

namespace sc {

template <typename T, int NDIM, int R, int CLS>
__global__ void __launch_bounds__(FlatApply<T, NDIM, R, CLS>::NTHR)
    flat_apply_kernel(const T *__restrict__ x, T *__restrict__ y, ApplyGeom g,
                      const __grid_constant__ BoxWeights<T, NDIM, R> W) {
  using K = FlatApply<T, NDIM, R, CLS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smem = reinterpret_cast<T *>(smem_raw);
  const int x0 = blockIdx.x * K::BX;
  const int y0 = NDIM == 3 ? blockIdx.y * K::BY : 0;
  const int z0 = (NDIM == 3 ? blockIdx.z : blockIdx.y) * g.H;
  StoreEpi<T, NDIM, K::VX> epi{y, &g};
  K::run_tile(x, g, W, x0, y0, z0, smem, epi);
}

static int g_num_sms = 0;
int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 152;
  }
  return g_num_sms;
}

// Output planes per CTA: enough CTAs for several waves of resident blocks,
// long enough runs to amortise the 2R halo planes.
static int choose_h(long long tiles_per_plane, int nplanes, int R, int override_h) {
  if (override_h > 0) return std::min(override_h, nplanes);
  const long long target = 8LL * num_sms();
  long long h = (tiles_per_plane * nplanes + target - 1) / target;
  h = std::max<long long>(h, 4 * R);
  h = std::min<long long>(h, 256);
  h = std::min<long long>(h, nplanes);
  return int(std::max<long long>(h, 1));
}

static int g_h_override = 0;

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
  g.H = choose_h(tiles, ns, R, g_h_override);
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
  auto kern = flat_apply_kernel<T, NDIM, R, CLS>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(K::SMEM));
    attr_set = true;
  }
  kern<<<grid, K::NTHR, K::SMEM, st>>>(static_cast<const T *>(q.x), static_cast<T *>(q.y), g, W);
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
  bool c2 = true, c4 = true;
  for (int k = 0; k < q.s->npts; ++k) {
    const int dx = q.s->off[k][0], dy = q.s->off[k][1], dz = q.s->off[k][2];
    c2 = c2 && std::max({std::abs(dx), std::abs(dy), std::abs(dz)}) <= 2 &&
         in_support<CLS_CROSS2, 2>(dx, dy, dz);
    c4 = c4 && std::max({std::abs(dx), std::abs(dy), std::abs(dz)}) <= 4 &&
         in_support<CLS_CROSS2, 4>(dx, dy, dz);
  }
  const int r = q.s->radius;
  // the ghosted layout has a ring of the stencil's radius; the class radius
  // must equal it for the strides to match
  if (nd == 2) {
    if (c2 && (q.bc != SC_BC_GHOSTED || r == 2)) return launch_flat<T, 2, 2, CLS_CROSS2>(q, w.data(), st);
    if (c4 && (q.bc != SC_BC_GHOSTED || r == 4)) return launch_flat<T, 2, 4, CLS_CROSS2>(q, w.data(), st);
    if (r <= 1 && (q.bc != SC_BC_GHOSTED || r == 1)) return launch_flat<T, 2, 1, CLS_BOX>(q, w.data(), st);
    if (r <= 2 && (q.bc != SC_BC_GHOSTED || r == 2)) return launch_flat<T, 2, 2, CLS_BOX>(q, w.data(), st);
    if (r <= 4 && (q.bc != SC_BC_GHOSTED || r == 4)) return launch_flat<T, 2, 4, CLS_BOX>(q, w.data(), st);
  } else {
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

void set_apply_planes_override(int h) { g_h_override = h; }

}  // namespace sc

using namespace sc;

extern "C" {

int sc_apply_composed(const sc_stencil *s, int32_t dtype, int32_t bc, const int64_t *dims,
                      int64_t h_num, int64_t h_den, const void *x_dev, void *y_dev,
                      sc_stream_t stream) {
  if (int rc = validate_apply(s, dtype, bc, dims, h_num, h_den)) return rc;
  if (!x_dev || !y_dev) return fail(SC_EINVAL, "null device pointer");
  if (x_dev == y_dev) return fail(SC_EINVAL, "x and y must not overlap");
  ApplyReq q{s, dtype, bc, dims, h_num, h_den, x_dev, y_dev};
  int rc = apply_enqueue(q, (cudaStream_t)stream);
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
