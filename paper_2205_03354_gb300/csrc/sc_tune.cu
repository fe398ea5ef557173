// Autotuner of the composed-stencil apply: evaluation schedule (flat
// composed weights, nested native B(A x), nested FP32-pair for FP64
// Laplacian factors) and halo-blocking depth (output planes per CTA, which
// sets how often the 2R halo planes are re-read), timed on the caller's data
// and stream; the winner is cached per problem shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "sc_apply_host.h"
#include "sc_internal.h"

namespace sc {

typedef std::tuple<int, int, int, long long, long long, long long, long long, long long> TuneKey;

static std::mutex g_tune_mu;
static std::map<TuneKey, sc_tune_choice> g_tune;

static long long fingerprint(const sc_stencil *s) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](long long v) {
    h ^= (unsigned long long)v;
    h *= 1099511628211ull;
  };
  mix(s->ndim);
  mix(s->npts);
  mix(s->hpow);
  mix(s->den);
  for (int k = 0; k < s->npts; ++k) {
    mix(s->off[k][0]);
    mix(s->off[k][1]);
    mix(s->off[k][2]);
    mix(s->num[k]);
  }
  return (long long)h;
}

static TuneKey key_of(const sc_stencil *B, const sc_stencil *A, int dtype, int bc, const int64_t *dims) {
  return TuneKey(A->ndim, dtype, bc, dims[0], dims[1], A->ndim == 3 ? dims[2] : 1, fingerprint(B),
                 fingerprint(A));
}

static int run_choice(const sc_stencil *B, const sc_stencil *A, const sc_stencil *C, int dtype, int bc,
                      const int64_t *dims, int64_t hn, int64_t hd, const void *x, void *y, void *work,
                      const sc_tune_choice &c, cudaStream_t st) {
  if (c.eval == SC_EVAL_FLAT) {
    ApplyReq q{C, dtype, bc, dims, hn, hd, x, y, nullptr, c.planes};
    return apply_enqueue(q, st);
  }
  if (c.eval == SC_EVAL_FUSED && fused_supported(B, A, dtype, bc, dims))
    return fused_enqueue(B, A, dtype, bc, dims, hn, hd, x, y, c.planes, st);
  return composition_enqueue(B, A, dtype, bc, dims, hn, hd, x, y, work, st,
                             c.eval == SC_EVAL_PAIR ? SC_ARITH_PAIR : SC_ARITH_NATIVE, c.planes);
}

}  // namespace sc

using namespace sc;

extern "C" {

int sc_autotune_apply(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                      const int64_t *dims, int64_t h_num, int64_t h_den, const void *x_dev, void *y_dev,
                      void *work_dev, size_t work_bytes, sc_tune_choice *out, sc_stream_t stream) {
  if (int rc = validate_apply(outer, dtype, bc, dims, h_num, h_den)) return rc;
  if (int rc = validate_apply(inner, dtype, bc, dims, h_num, h_den)) return rc;
  if (outer->ndim != inner->ndim) return fail(SC_EINVAL, "outer and inner dimensions differ");
  if (!x_dev || !y_dev || !work_dev) return fail(SC_EINVAL, "bad device pointers");
  const size_t need = composition_work_bytes(outer, inner, dtype, bc, dims);
  if (work_bytes < need) return fail(SC_ENOMEM, "work space too small");
  if (int rc = check_disjoint(outer->ndim, bc, dims, outer->radius + inner->radius, dtype == SC_F64 ? 8 : 4,
                              x_dev, y_dev, work_dev, need))
    return rc;
  sc_stencil C;
  if (int rc = sc_compose_stencil(outer, inner, &C)) return rc;
  if (C.radius > SC_MAX_APPLY_RADIUS) return fail(SC_EINVAL, "composed radius too large");
  cudaStream_t st = (cudaStream_t)stream;
  const int nd = outer->ndim;
  const int nplanes = int(nd == 3 ? dims[2] : dims[1]);
  std::vector<sc_tune_choice> cands;
  const int evals[4] = {SC_EVAL_FLAT, SC_EVAL_NESTED, SC_EVAL_PAIR, SC_EVAL_FUSED};
  for (int e : evals) {
    if (e == SC_EVAL_PAIR && dtype != SC_F64) continue;
    if (e == SC_EVAL_FUSED && !fused_supported(outer, inner, dtype, bc, dims)) continue;
    // planes per CTA: the occupancy model (0) and a spread of fixed depths
    const int ps[5] = {0, 16, 32, 64, 128};
    for (int p : ps) {
      if (p > nplanes) continue;
      sc_tune_choice c;
      std::memset(&c, 0, sizeof(c));
      c.eval = e;
      c.planes = p;
      cands.push_back(c);
    }
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  sc_tune_choice best;
  std::memset(&best, 0, sizeof(best));
  best.ms = 1e300;
  for (sc_tune_choice &c : cands) {
    // one warm-up, then the median of three timed runs
    int rc = run_choice(outer, inner, &C, dtype, bc, dims, h_num, h_den, x_dev, y_dev, work_dev, c, st);
    if (rc) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return rc;
    }
    float t[3];
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(a, st);
      run_choice(outer, inner, &C, dtype, bc, dims, h_num, h_den, x_dev, y_dev, work_dev, c, st);
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      cudaEventElapsedTime(&t[r], a, b);
    }
    std::sort(t, t + 3);
    c.ms = t[1];
    if (c.ms < best.ms) best = c;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SC_ECUDA, "autotune: %s", cudaGetErrorString(e));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key_of(outer, inner, dtype, bc, dims)] = best;
  }
  if (out) *out = best;
  clear_error();
  return SC_OK;
}

int sc_apply_tuned(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                   const int64_t *dims, int64_t h_num, int64_t h_den, const void *x_dev, void *y_dev,
                   void *work_dev, size_t work_bytes, sc_stream_t stream) {
  if (int rc = validate_apply(outer, dtype, bc, dims, h_num, h_den)) return rc;
  if (int rc = validate_apply(inner, dtype, bc, dims, h_num, h_den)) return rc;
  if (outer->ndim != inner->ndim) return fail(SC_EINVAL, "outer and inner dimensions differ");
  if (!x_dev || !y_dev) return fail(SC_EINVAL, "bad device pointers");
  if (int rc = check_disjoint(outer->ndim, bc, dims, outer->radius + inner->radius, dtype == SC_F64 ? 8 : 4,
                              x_dev, y_dev))
    return rc;
  sc_tune_choice c;
  std::memset(&c, 0, sizeof(c));
  bool have = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key_of(outer, inner, dtype, bc, dims));
    if (it != g_tune.end()) {
      c = it->second;
      have = true;
    }
  }
  if (!have) c.eval = SC_EVAL_FLAT;  // untuned: the composed weights, model depth
  if (c.eval != SC_EVAL_FLAT && (!work_dev || work_bytes < composition_work_bytes(outer, inner, dtype, bc, dims)))
    return fail(SC_ENOMEM, "work space too small for the tuned schedule");
  if (c.eval != SC_EVAL_FLAT)
    if (int rc = check_disjoint(outer->ndim, bc, dims, outer->radius + inner->radius, dtype == SC_F64 ? 8 : 4,
                                x_dev, y_dev, work_dev, composition_work_bytes(outer, inner, dtype, bc, dims)))
      return rc;
  sc_stencil C;
  if (int rc = sc_compose_stencil(outer, inner, &C)) return rc;
  int rc = run_choice(outer, inner, &C, dtype, bc, dims, h_num, h_den, x_dev, y_dev, work_dev, c,
                      (cudaStream_t)stream);
  if (!rc) clear_error();
  return rc;
}

size_t sc_apply_tuned_host_work_bytes(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype,
                                      int32_t bc, const int64_t *dims) {
  if (!outer || !inner || !dims) return 0;
  if (validate_apply(outer, dtype, bc, dims, 1, 1) || validate_apply(inner, dtype, bc, dims, 1, 1)) return 0;
  if (outer->ndim != inner->ndim) return 0;
  const size_t es = dtype == SC_F64 ? 8 : 4;
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  const int nd = outer->ndim, rin = bc == SC_BC_GHOSTED ? outer->radius + inner->radius : 0;
  return up(grid_elems_ext(nd, dims, rin) * es) + up(grid_elems_ext(nd, dims, 0) * es) +
         composition_work_bytes(outer, inner, dtype, bc, dims);
}

// Per-device copy streams and the events that order consecutive host-buffer
// applies (created on first use, kept until exit).
struct HostPipe {
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t in_done = nullptr, comp_done = nullptr, out_done = nullptr;
  bool primed = false;  // comp_done / out_done recorded at least once
};
static std::mutex g_pipe_mu;
static HostPipe g_pipe[64];

int sc_apply_tuned_host(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                        const int64_t *dims, int64_t h_num, int64_t h_den, const void *x_host, void *y_host,
                        void *work_dev, size_t work_bytes, sc_stream_t stream) {
  if (int rc = validate_apply(outer, dtype, bc, dims, h_num, h_den)) return rc;
  if (int rc = validate_apply(inner, dtype, bc, dims, h_num, h_den)) return rc;
  if (outer->ndim != inner->ndim) return fail(SC_EINVAL, "outer and inner dimensions differ");
  if (!x_host || !y_host || !work_dev) return fail(SC_EINVAL, "null pointer");
  const size_t need = sc_apply_tuned_host_work_bytes(outer, inner, dtype, bc, dims);
  if (work_bytes < need) return fail(SC_ENOMEM, "work space %zu < %zu bytes", work_bytes, need);
  const size_t es = dtype == SC_F64 ? 8 : 4;
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  const int nd = outer->ndim, rin = bc == SC_BC_GHOSTED ? outer->radius + inner->radius : 0;
  const size_t xb = grid_elems_ext(nd, dims, rin) * es, yb = grid_elems_ext(nd, dims, 0) * es;
  char *xd = static_cast<char *>(work_dev), *yd = xd + up(xb), *wd = yd + up(yb);
  const size_t wb = work_bytes - up(xb) - up(yb);
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe &hp = g_pipe[dev & 63];
  if (!hp.in) {
    if (cudaStreamCreateWithFlags(&hp.in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp.out, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&hp.in_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&hp.comp_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&hp.out_done, cudaEventDisableTiming) != cudaSuccess)
      return fail(SC_ECUDA, "copy stream or event creation failed");
  }
  cudaStream_t st = (cudaStream_t)stream;
  // copy-in: after the previous apply has read the previous input
  if (hp.primed) cudaStreamWaitEvent(hp.in, hp.comp_done, 0);
  if (cudaMemcpyAsync(xd, x_host, xb, cudaMemcpyHostToDevice, hp.in) != cudaSuccess)
    return fail(SC_ECUDA, "host-to-device copy failed");
  cudaEventRecord(hp.in_done, hp.in);
  // apply: after the copy-in, and after the previous result has left yd
  cudaStreamWaitEvent(st, hp.in_done, 0);
  if (hp.primed) cudaStreamWaitEvent(st, hp.out_done, 0);
  if (int rc = sc_apply_tuned(outer, inner, dtype, bc, dims, h_num, h_den, xd, yd, wd, wb, stream)) return rc;
  cudaEventRecord(hp.comp_done, st);
  // copy-out, and the caller's stream waits for it
  cudaStreamWaitEvent(hp.out, hp.comp_done, 0);
  if (cudaMemcpyAsync(y_host, yd, yb, cudaMemcpyDeviceToHost, hp.out) != cudaSuccess)
    return fail(SC_ECUDA, "device-to-host copy failed");
  cudaEventRecord(hp.out_done, hp.out);
  cudaStreamWaitEvent(st, hp.out_done, 0);
  hp.primed = true;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SC_ECUDA, "host apply: %s", cudaGetErrorString(e));
  clear_error();
  return SC_OK;
}

int sc_tuned_choice(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                    const int64_t *dims, sc_tune_choice *out) {
  if (!outer || !inner || !dims || !out) return fail(SC_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key_of(outer, inner, dtype, bc, dims));
  if (it == g_tune.end()) return fail(SC_EINVAL, "shape not tuned");
  *out = it->second;
  clear_error();
  return SC_OK;
}

int sc_tune_set(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                const int64_t *dims, const sc_tune_choice *in) {
  if (!outer || !inner || !dims || !in) return fail(SC_EINVAL, "null argument");
  if (int rc = validate_apply(outer, dtype, bc, dims, 1, 1)) return rc;
  if (int rc = validate_apply(inner, dtype, bc, dims, 1, 1)) return rc;
  if (outer->ndim != inner->ndim) return fail(SC_EINVAL, "outer and inner dimensions differ");
  if (in->eval < SC_EVAL_FLAT || in->eval > SC_EVAL_FUSED) return fail(SC_EINVAL, "unknown eval %d", in->eval);
  if (in->planes < 0 || in->planes > 4096) return fail(SC_EINVAL, "planes %d out of range", in->planes);
  sc_stencil C;
  if (int rc = sc_compose_stencil(outer, inner, &C)) return rc;
  if (C.radius > SC_MAX_APPLY_RADIUS) return fail(SC_EINVAL, "composed radius too large");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key_of(outer, inner, dtype, bc, dims)] = *in;
  clear_error();
  return SC_OK;
}

}  // extern "C"
