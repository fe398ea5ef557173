// sc_ch_stats_noalloc: the mass / free-energy statistics of sc_ch_stats for
// callers that must not allocate device memory.
//
// Some host programs own every device allocation themselves -- for example
// an application that hands all device memory to its own pool allocator, or
// a latency-critical loop in which cudaMalloc (which can synchronise the
// whole device) is not acceptable -- and cannot supply the work buffer that
// sc_ch_stats needs for its partial sums.  This variant keeps that scratch in
// a fixed-size array in device global memory that is part of the library
// itself, so a call allocates nothing.
//
// Properties a caller must know:
//  * the array is loaded with the library and stays resident on every GPU
//    that uses it until the process exits (STATS_SCRATCH doubles, 64 KiB);
//  * host code cannot use the array's name as a device address, so the first
//    call on each device looks the address up with cudaGetSymbolAddress
//    while that device is current and keeps it for later calls; make that
//    first call outside any stream capture;
//  * the kept address belongs to the device's context at the first call: a
//    process that calls cudaDeviceReset on a device gets a new context in
//    which the array may sit elsewhere, so it must call sc_noalloc_forget()
//    after the reset (the next call then looks the address up again);
//  * every call on a device shares the one array and it keeps the previous
//    call's contents: each call writes every slot it later reads, so nothing
//    has to start at zero, but two calls that can run on the GPU at the same
//    time (different streams, or different host threads) race on it and must
//    be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "sc_internal.h"
#include "sc_stats_kernels.h"

namespace sc {

// Largest field (grid points per batch item) the fixed scratch can reduce.
constexpr long long NOALLOC_MAX_POINTS = 1LL << 24;
constexpr int NOALLOC_MAX_PARTS = int(NOALLOC_MAX_POINTS / STATS_CHUNK);  // 4096
constexpr int STATS_SCRATCH = 2 * NOALLOC_MAX_PARTS + 8;

static __device__ __align__(256) double g_stats_scratch[STATS_SCRATCH];

constexpr int MAX_DEVICES = 64;
static std::mutex g_mu;
static double *g_scratch_ptr[MAX_DEVICES];

// Device address of g_stats_scratch on the current device (looked up once
// per device).
static int scratch_address(double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SC_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(SC_EINVAL, "device ordinal %d not supported", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_stats_scratch);
    if (e != cudaSuccess || !p)
      return fail(SC_ECUDA, "cudaGetSymbolAddress of the statistics scratch: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return SC_OK;
}

}  // namespace sc

using namespace sc;

extern "C" {

void sc_noalloc_forget(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (int d = 0; d < MAX_DEVICES; ++d) g_scratch_ptr[d] = nullptr;
}

int sc_ch_stats_noalloc(const sc_ch *c, const double *u_dev, double *mass_host, double *energy_host,
                        sc_stream_t stream) {
  if (!c || !u_dev || !mass_host || !energy_host) return fail(SC_EINVAL, "null pointer");
  if (c->ndim != 2 && c->ndim != 3) return fail(SC_EINVAL, "ndim must be 2 or 3");
  if (c->batch < 1) return fail(SC_EINVAL, "batch must be positive");
  if (c->h_num <= 0 || c->h_den <= 0) return fail(SC_EINVAL, "h must be positive");
  if (c->chem != 0 && c->chem != 1) return fail(SC_EINVAL, "chem must be 0 or 1");
  long long npts = 1;
  for (int a = 0; a < c->ndim; ++a) {
    if (c->n[a] < 1) return fail(SC_EINVAL, "n must be positive");
    npts *= c->n[a];
    if (npts > NOALLOC_MAX_POINTS)
      return fail(SC_EINVAL,
                  "field too large for the fixed scratch of sc_ch_stats_noalloc: at most %lld grid points "
                  "per field (use sc_ch_stats with a work buffer)",
                  NOALLOC_MAX_POINTS);
  }
  double *scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;
  const int nblk = int((npts + STATS_CHUNK - 1) / STATS_CHUNK);
  double *pm = scratch, *pe = scratch + NOALLOC_MAX_PARTS, *out = scratch + 2 * NOALLOC_MAX_PARTS;
  cudaStream_t st = (cudaStream_t)stream;
  const double h = double(c->h_num) / double(c->h_den);
  const double hd = c->ndim == 3 ? h * h * h : h * h;
  for (int b = 0; b < c->batch; ++b) {
    k_ch_stats_part<<<nblk, STATS_NTHR, 0, st>>>(u_dev + (long long)b * npts, c->ndim, int(c->n[0]),
                                                  int(c->n[1]), c->ndim == 3 ? int(c->n[2]) : 1, h, c->kappa,
                                                  c->chem, c->rho, c->ca, c->cb, pm, pe);
    k_sum_final<<<1, STATS_NTHR, 0, st>>>(pm, nblk, out, 0);
    k_sum_final<<<1, STATS_NTHR, 0, st>>>(pe, nblk, out, 1);
    double hs[2];
    cudaError_t e = cudaMemcpyAsync(hs, out, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SC_ECUDA, "statistics: %s", cudaGetErrorString(e));
    mass_host[b] = hs[0];
    energy_host[b] = hs[1] * hd;
  }
  clear_error();
  return SC_OK;
}

}  // extern "C"
