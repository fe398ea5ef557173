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

// ---- host-buffer apply: slab pipeline -------------------------------------
//
// The grid is cut along its slowest axis into K slabs of S output planes.
// Slab k needs the input planes [z0 - Rc, z1 + Rc) (Rc: the composed
// radius): they are copied into a device staging buffer (the 2 Rc planes it
// shares with slab k - 1 from that slab's staging buffer, device to device;
// the rest from the host), the in-plane boundary ring is filled around them
// (periodic: wrapped copies, zero: zeros; a ghosted input already has it),
// the tuned schedule runs on the slab as a ghosted grid of S planes, and the
// S output planes go back to the host.  Two buffer sets alternate, so the
// copy-in of slab k + 1, the apply of slab k and the copy-out of slab k - 1
// run at once on three streams.  Grids too short for two slabs go through
// one buffer set whole (K = 1: copy-in, apply, copy-out).

struct HostPlan {
  int nd = 0, Rc = 0, bc = 0;
  bool slabs = false;    // false: the whole grid in one piece
  long long N = 0;       // output planes along the slowest axis
  long long S = 0;       // planes per slab (the last may be shorter)
  int K = 0;             // slabs
  size_t es = 0;
  long long pin = 0;     // elements per staged input plane
  long long ppad = 0;    // elements per ring-filled plane (slabs, non-ghosted)
  long long pout = 0;    // elements per output plane
  // byte offsets in the work space: staging[2], ring-filled[2], apply work;
  // the output buffers y[2] (ybytes each) sit at the END of the caller's
  // work space, so that a following call of another shape on the same space
  // stages its input clear of the outputs still being copied out
  size_t off_stage[2] = {0, 0}, off_pad[2] = {0, 0}, off_work = 0, ybytes = 0, ynum = 0;
  size_t work_bytes = 0, total = 0;
  int64_t sdims[3] = {0, 0, 0};  // slab dims (full-length slab) for the apply work size
};

static size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

// Work-space plan of a host-buffer apply (sizes only; no validation).
static HostPlan host_plan(const sc_stencil *outer, const sc_stencil *inner, int dtype, int bc, const int64_t *dims) {
  HostPlan p;
  p.nd = outer->ndim;
  p.Rc = outer->radius + inner->radius;
  p.bc = bc;
  p.es = dtype == SC_F64 ? 8 : 4;
  const int nd = p.nd, Rc = p.Rc;
  const bool ghost = bc == SC_BC_GHOSTED;
  p.N = dims[nd - 1];
  long long inner_out = 1, inner_ring = 1;
  for (int a = 0; a < nd - 1; ++a) {
    inner_out *= dims[a];
    inner_ring *= dims[a] + 2 * Rc;
  }
  p.pout = inner_out;
  // slabs of at least 4 Rc planes, about 8 of them; in-plane wraps must be
  // single (periodic extents >= Rc)
  const long long smin = 4LL * Rc;
  bool ok = p.N >= 2 * smin && inner_ring < (1LL << 31);
  for (int a = 0; a < nd - 1; ++a)
    if (bc == SC_BC_PERIODIC && dims[a] < Rc) ok = false;
  if (ok) {
    p.slabs = true;
    p.S = std::max(smin, (p.N + 7) / 8);
    p.K = int((p.N + p.S - 1) / p.S);
    if (p.K < 2) p.slabs = false;
  }
  if (p.slabs) {
    p.pin = ghost ? inner_ring : inner_out;
    p.ppad = ghost ? 0 : inner_ring;
    const size_t stage = up256(size_t(p.S + 2 * Rc) * p.pin * p.es);
    const size_t pad = up256(size_t(p.S + 2 * Rc) * p.ppad * p.es);
    const size_t ys = up256(size_t(p.S) * p.pout * p.es);
    for (int a = 0; a < nd - 1; ++a) p.sdims[a] = dims[a];
    p.sdims[nd - 1] = p.S;
    p.work_bytes = composition_work_bytes(outer, inner, dtype, SC_BC_GHOSTED, p.sdims);
    size_t o = 0;
    p.off_stage[0] = o;
    o += stage;
    p.off_stage[1] = o;
    o += stage;
    p.off_pad[0] = o;
    o += pad;
    p.off_pad[1] = o;
    o += pad;
    p.off_work = o;
    o += up256(p.work_bytes);
    p.ybytes = ys;
    p.ynum = 2;
    p.total = o + 2 * ys;
  } else {
    p.S = p.N;
    p.K = 1;
    p.pin = ghost ? inner_ring : inner_out;
    const size_t xb = up256(grid_elems_ext(nd, dims, ghost ? Rc : 0) * p.es);
    const size_t yb = up256(grid_elems_ext(nd, dims, 0) * p.es);
    p.work_bytes = composition_work_bytes(outer, inner, dtype, bc, dims);
    p.off_stage[0] = p.off_stage[1] = 0;
    p.off_work = xb;
    p.ybytes = yb;
    p.ynum = 1;
    p.total = xb + up256(p.work_bytes) + yb;
  }
  return p;
}

// Ring fill of a staged slab: pad[z][gy][gx] = stage[z][gy - Rc][gx - Rc]
// wrapped (periodic) or zero outside (zero boundary); 2D rows have no gy.
template <typename T>
__global__ void k_ring_fill(const T *__restrict__ stage, T *__restrict__ pad, int nx, int ny, int nplanes, int Rc,
                            int periodic, int nd) {
  const int px = nx + 2 * Rc, py = nd == 3 ? ny + 2 * Rc : 1;
  const int plane = px * py;
  const long long in_plane = (long long)nx * (nd == 3 ? ny : 1);
  for (int z = blockIdx.y; z < nplanes; z += gridDim.y) {
    const T *src = stage + (long long)z * in_plane;
    T *dst = pad + (long long)z * plane;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += gridDim.x * blockDim.x) {
      const int gy = i / px, gx = i - gy * px;
      int sx = gx - Rc, sy = nd == 3 ? gy - Rc : 0;
      bool ok;
      if (periodic) {
        sx += sx < 0 ? nx : (sx >= nx ? -nx : 0);
        if (nd == 3) sy += sy < 0 ? ny : (sy >= ny ? -ny : 0);
        ok = true;
      } else {
        ok = sx >= 0 && sx < nx && (nd != 3 || (sy >= 0 && sy < ny));
      }
      dst[i] = ok ? src[(long long)sy * nx + sx] : T(0);
    }
  }
}

static int ring_fill(const HostPlan &p, const int64_t *dims, const void *stage, void *pad, int nplanes,
                     cudaStream_t st) {
  const int px = int(dims[0] + 2 * p.Rc), py = p.nd == 3 ? int(dims[1] + 2 * p.Rc) : 1;
  const int plane = px * py;
  dim3 grid(unsigned(std::min((plane + 255) / 256, 256)), unsigned(std::min(nplanes, 65535)));
  const int periodic = p.bc == SC_BC_PERIODIC;
  const int ny = p.nd == 3 ? int(dims[1]) : 1;
  if (p.es == 8)
    k_ring_fill<double><<<grid, 256, 0, st>>>(static_cast<const double *>(stage), static_cast<double *>(pad),
                                                int(dims[0]), ny, nplanes, p.Rc, periodic, p.nd);
  else
    k_ring_fill<float><<<grid, 256, 0, st>>>(static_cast<const float *>(stage), static_cast<float *>(pad),
                                              int(dims[0]), ny, nplanes, p.Rc, periodic, p.nd);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SC_OK : fail(SC_ECUDA, "ring fill launch: %s", cudaGetErrorString(e));
}

// One piece of a slab's staging: `n` planes into staging plane `dst` from
// host plane `src` (kind 0), from the previous slab's staging plane `src`
// (kind 1), or zeros (kind 2).
struct StageRun {
  int kind;
  long long src, dst, n;
};

static void stage_runs(const HostPlan &p, int k, long long z0, long long z1, std::vector<StageRun> &runs) {
  runs.clear();
  const bool ghost = p.bc == SC_BC_GHOSTED;
  for (long long q = z0 - p.Rc; q < z1 + p.Rc; ++q) {
    StageRun r{0, 0, q - (z0 - p.Rc), 1};
    if (k > 0 && q < z0 + p.Rc) {
      r.kind = 1;
      r.src = q - (z0 - p.S - p.Rc);  // slab k - 1 started S planes earlier
    } else if (ghost) {
      r.src = q + p.Rc;
    } else if (p.bc == SC_BC_PERIODIC) {
      r.src = q < 0 ? q + p.N : (q >= p.N ? q - p.N : q);
    } else if (q < 0 || q >= p.N) {
      r.kind = 2;
    } else {
      r.src = q;
    }
    if (!runs.empty()) {
      StageRun &b = runs.back();
      if (b.kind == r.kind && b.dst + b.n == r.dst && (r.kind == 2 || b.src + b.n == r.src)) {
        ++b.n;
        continue;
      }
    }
    runs.push_back(r);
  }
}

// Per-device copy streams and the events that order the slabs (alternating
// buffer sets 0 / 1) within a call and across consecutive calls.
struct HostPipe {
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t in_done[2] = {nullptr, nullptr}, comp_done[2] = {nullptr, nullptr}, out_done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  unsigned next = 0;                    // buffer set of the next slab
  uintptr_t y_lo = 0, y_hi = 0;         // output buffers of the previous call
};
static std::mutex g_pipe_mu;
static HostPipe g_pipe[64];

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
  return host_plan(outer, inner, dtype, bc, dims).total;
}

int sc_apply_tuned_host(const sc_stencil *outer, const sc_stencil *inner, int32_t dtype, int32_t bc,
                        const int64_t *dims, int64_t h_num, int64_t h_den, const void *x_host, void *y_host,
                        void *work_dev, size_t work_bytes, sc_stream_t stream) {
  if (int rc = validate_apply(outer, dtype, bc, dims, h_num, h_den)) return rc;
  if (int rc = validate_apply(inner, dtype, bc, dims, h_num, h_den)) return rc;
  if (outer->ndim != inner->ndim) return fail(SC_EINVAL, "outer and inner dimensions differ");
  if (!x_host || !y_host || !work_dev) return fail(SC_EINVAL, "null pointer");
  const HostPlan p = host_plan(outer, inner, dtype, bc, dims);
  if (work_bytes < p.total) return fail(SC_ENOMEM, "work space %zu < %zu bytes", work_bytes, p.total);
  // slab k's output reaches y_host while later slabs still read x_host
  if (int rc = check_disjoint(p.nd, bc, dims, p.Rc, p.es, x_host, y_host)) return rc;
  sc_stencil C;
  if (int rc = sc_compose_stencil(outer, inner, &C)) return rc;
  if (C.radius > SC_MAX_APPLY_RADIUS) return fail(SC_EINVAL, "composed radius too large");
  sc_tune_choice c;
  std::memset(&c, 0, sizeof(c));
  c.eval = SC_EVAL_FLAT;  // untuned: the composed weights, model depth (as sc_apply_tuned)
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key_of(outer, inner, dtype, bc, dims));
    if (it != g_tune.end()) c = it->second;
  }
  char *w = static_cast<char *>(work_dev);
  char *ybase = w + ((work_bytes - p.ynum * p.ybytes) & ~size_t(255));  // >= the apply work's end
  const char *xh = static_cast<const char *>(x_host);
  char *yh = static_cast<char *>(y_host);
  const size_t es = p.es;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe &hp = g_pipe[dev & 63];
  if (!hp.in) {
    bool ok = cudaStreamCreateWithFlags(&hp.in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&hp.out, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
      ok = cudaEventCreateWithFlags(&hp.in_done[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&hp.comp_done[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&hp.out_done[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return fail(SC_ECUDA, "copy stream or event creation failed");
  }
  cudaStream_t st = (cudaStream_t)stream;
  // Call boundary: the previous call's applies must have read their inputs
  // before this call's copy-ins overwrite staging space, and its copy-outs
  // must have left the output buffers before this call writes over them (or
  // stages into them, when the layouts overlap).
  const uintptr_t front_lo = reinterpret_cast<uintptr_t>(w), front_hi = front_lo + p.off_work;
  const bool clash = hp.y_lo < front_hi && front_lo < hp.y_hi;
  for (int b = 0; b < 2; ++b) {
    if (!hp.used[b]) continue;
    cudaStreamWaitEvent(hp.in, hp.comp_done[b], 0);
    if (clash) cudaStreamWaitEvent(hp.in, hp.out_done[b], 0);
    cudaStreamWaitEvent(st, hp.out_done[b], 0);
  }
  // an error after the first enqueue leaves nothing of this call in flight
  auto drain = [&](int rc) {
    cudaStreamSynchronize(hp.in);
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(hp.out);
    hp.y_lo = hp.y_hi = 0;
    return rc;
  };
  std::vector<StageRun> runs;
  int last = 0;
  for (int k = 0; k < p.K; ++k) {
    const int b = int(hp.next++ & 1u);
    last = b;
    const long long z0 = k * p.S, z1 = std::min(p.N, z0 + p.S), nz = z1 - z0;
    char *stg = w + p.off_stage[b], *ys = ybase + (p.ynum == 2 ? b * p.ybytes : 0);
    // copy-in (after the apply that last read this staging buffer)
    if (hp.used[b]) cudaStreamWaitEvent(hp.in, hp.comp_done[b], 0);
    if (!p.slabs) {
      const size_t xb = grid_elems_ext(p.nd, dims, bc == SC_BC_GHOSTED ? p.Rc : 0) * es;
      if (cudaMemcpyAsync(stg, xh, xb, cudaMemcpyHostToDevice, hp.in) != cudaSuccess)
        return drain(fail(SC_ECUDA, "host-to-device copy failed"));
    } else {
      stage_runs(p, k, z0, z1, runs);
      const size_t pb = size_t(p.pin) * es;
      const char *prev = w + p.off_stage[b ^ 1];
      for (const StageRun &r : runs) {
        cudaError_t e;
        if (r.kind == 0)
          e = cudaMemcpyAsync(stg + r.dst * pb, xh + r.src * pb, r.n * pb, cudaMemcpyHostToDevice, hp.in);
        else if (r.kind == 1)
          e = cudaMemcpyAsync(stg + r.dst * pb, prev + r.src * pb, r.n * pb, cudaMemcpyDeviceToDevice, hp.in);
        else
          e = cudaMemsetAsync(stg + r.dst * pb, 0, r.n * pb, hp.in);
        if (e != cudaSuccess) return drain(fail(SC_ECUDA, "slab copy-in failed: %s", cudaGetErrorString(e)));
      }
    }
    cudaEventRecord(hp.in_done[b], hp.in);
    // apply (after the copy-in, and after the copy-out that last read this
    // output buffer)
    cudaStreamWaitEvent(st, hp.in_done[b], 0);
    if (hp.used[b]) cudaStreamWaitEvent(st, hp.out_done[b], 0);
    int rc;
    if (!p.slabs) {
      rc = run_choice(outer, inner, &C, dtype, bc, dims, h_num, h_den, stg, ys, w + p.off_work, c, st);
    } else {
      int64_t sd[3];
      for (int a = 0; a < 3; ++a) sd[a] = p.sdims[a];
      sd[p.nd - 1] = nz;
      const void *xin = stg;
      if (bc != SC_BC_GHOSTED) {
        if ((rc = ring_fill(p, dims, stg, w + p.off_pad[b], int(nz + 2 * p.Rc), st))) return drain(rc);
        xin = w + p.off_pad[b];
      }
      rc = run_choice(outer, inner, &C, dtype, SC_BC_GHOSTED, sd, h_num, h_den, xin, ys, w + p.off_work, c, st);
    }
    if (rc) return drain(rc);
    cudaEventRecord(hp.comp_done[b], st);
    // copy-out
    cudaStreamWaitEvent(hp.out, hp.comp_done[b], 0);
    const size_t ob = size_t(nz) * p.pout * es;
    if (cudaMemcpyAsync(yh + size_t(z0) * p.pout * es, ys, ob, cudaMemcpyDeviceToHost, hp.out) != cudaSuccess)
      return drain(fail(SC_ECUDA, "device-to-host copy failed"));
    cudaEventRecord(hp.out_done[b], hp.out);
    hp.used[b] = true;
  }
  // the caller's stream completes once the last output plane is in host memory
  cudaStreamWaitEvent(st, hp.out_done[last], 0);
  hp.y_lo = reinterpret_cast<uintptr_t>(ybase);
  hp.y_hi = reinterpret_cast<uintptr_t>(ybase + p.ynum * p.ybytes);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return drain(fail(SC_ECUDA, "host apply: %s", cudaGetErrorString(e)));
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
