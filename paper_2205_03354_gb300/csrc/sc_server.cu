// Serving loop: continuous batching of plate-problem solves and
// Cahn-Hilliard steps on one GPU.
//
// A scheduler thread alternates between (1) admitting queued requests into
// free space of the caller's device arena (copy fields in, build the
// right-hand side: b = g - A(ring) for a plate problem, u + dt M Lap f'(u)
// for a Cahn-Hilliard step), (2) one time slice of the persistent CG engine
// over every resident request, and (3) retiring converged requests (result
// to the caller's host buffer, arena space back to the free list).  Requests
// that arrive while others run join at the next slice boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sc_apply_host.h"
#include "sc_internal.h"
#include "sc_solver.cuh"
#include "sc_solver_host.h"

namespace sc {

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit free list over [0, size).
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_total() const {
    size_t m = 0;
    for (auto &kv : free_) m += kv.second;
    return m;
  }
  size_t largest() const {
    size_t m = 0;
    for (auto &kv : free_) m = std::max(m, kv.second);
    return m;
  }

 private:
  std::map<size_t, size_t> free_;
};

struct Req {
  uint64_t id;
  sc_request rq;
  ProbSpec sp;
  size_t bytes = 0, off = 0;
  SolveProb P;
  ProbAux aux;
  double *f = nullptr, *g = nullptr, *x = nullptr;  // x: plate solution or Cahn-Hilliard field
  double t_submit = 0, t_admit = 0, t_done = 0;
  bool done = false;
  sc_result res;
};

static long long npts_of(const sc_request *r) {
  long long n = 1;
  for (int a = 0; a < r->ndim; ++a) n *= r->n[a];
  return n;
}
static long long padded_of(const sc_request *r, int R) {
  long long n = 1;
  for (int a = 0; a < r->ndim; ++a) n *= r->n[a] + 2 * R;
  return n;
}

// The solver a plate request runs on (the size rule of sc_request.solver).
constexpr long long PCG_MIN_POINTS = 1LL << 16;
static int plate_solver(const sc_request *r, long long min_pts) {
  if (r->solver == SC_SOLVER_PERSISTENT || r->solver == SC_SOLVER_PCG) return r->solver;
  return npts_of(r) >= min_pts ? SC_SOLVER_PCG : SC_SOLVER_PERSISTENT;
}

// Plate problem view of a request (device pointers filled in at admission).
static sc_bvp as_bvp(const sc_request *r, const double *f, const double *g, double *x,
                     long long min_pts = PCG_MIN_POINTS) {
  sc_bvp b;
  std::memset(&b, 0, sizeof(b));
  b.ndim = r->ndim;
  b.order = r->order;
  for (int a = 0; a < 3; ++a) b.n[a] = r->n[a];
  b.prec = r->prec;
  b.solver = plate_solver(r, min_pts);
  b.rtol = r->rtol;
  b.maxit = r->maxit;
  b.f_dev = f;
  b.ghost_dev = g;
  b.x_dev = x;
  return b;
}

// Cahn-Hilliard step view of a request (one field, persistent solver).
static sc_ch as_ch(const sc_request *r) {
  sc_ch c;
  std::memset(&c, 0, sizeof(c));
  c.ndim = r->ndim;
  c.order = r->order;
  for (int a = 0; a < 3; ++a) c.n[a] = r->n[a];
  c.batch = 1;
  c.h_num = r->h_num;
  c.h_den = r->h_den;
  c.dt = r->dt;
  c.M = r->M;
  c.kappa = r->kappa;
  c.chem = r->chem;
  c.rho = r->rho;
  c.ca = r->ca;
  c.cb = r->cb;
  c.prec = r->prec;
  c.solver = SC_SOLVER_PERSISTENT;
  c.rtol = r->rtol;
  c.maxit = r->maxit;
  return c;
}

// The request's spec with device pointers placed at x (f, g for a plate).
static int request_spec(const sc_request *r, double *f, double *g, double *x, ProbSpec &sp,
                        long long min_pts) {
  if (r->kind == SC_REQ_CH) {
    sc_ch c = as_ch(r);
    return ch_single_spec(&c, x, sp);
  }
  if (r->kind != SC_REQ_PLATE) return fail(SC_EINVAL, "unknown request kind %d", r->kind);
  if (r->solver != -1 && r->solver != SC_SOLVER_PERSISTENT && r->solver != SC_SOLVER_PCG)
    return fail(SC_EINVAL, "request solver must be -1, SC_SOLVER_PERSISTENT or SC_SOLVER_PCG");
  sc_bvp b = as_bvp(r, f, g, x, min_pts);
  return bvp_spec(&b, sp);
}

static int request_layout(const sc_request *r, ProbSpec &sp, size_t *bytes, long long min_pts) {
  // validation with placeholder pointers (never dereferenced)
  static double dummy;
  if (int rc = request_spec(r, &dummy, &dummy, &dummy, sp, min_pts)) return rc;
  Carver cv(nullptr, 0);
  if (r->kind == SC_REQ_PLATE) {
    cv.take(npts_of(r) * 8);          // f
    cv.take(padded_of(r, sp.R) * 8);  // ghost field
  }
  cv.take(npts_of(r) * 8);  // x / u
  SolveProb P;
  ProbAux aux;
  layout(sp, cv, P, aux);
  *bytes = cv.off + 256;
  return SC_OK;
}

}  // namespace sc

struct sc_server {
  sc_server_cfg cfg;
  int device = 0;
  cudaStream_t st = nullptr;
  char *arena_base = nullptr;  // after the descriptor head
  size_t arena_size = 0;
  sc::Arena arena;
  sc::SolveProb *dprobs = nullptr;
  int *dmap = nullptr;
  unsigned *dbars = nullptr;
  sc::SolveState *dstates = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<sc::Req *> pending;
  std::vector<sc::Req *> active;
  std::deque<sc::Req *> pcg_pending;  // plate requests for the preconditioned solver
  sc::Req *pcg_active = nullptr;
  long long min_pts = 1LL << 16;
  cudaStream_t st2 = nullptr;
  std::thread pcg_worker;
  std::unordered_map<uint64_t, sc::Req *> all;
  uint64_t next_id = 1;
  bool stop = false;
  int worker_error = 0;
  long long slices = 0;  // time slices run (the failure hook counts them)
  std::thread worker;
};

namespace sc {

static void retire(sc_server *S, Req *r, const SolveState &st) {
  cudaMemcpy(r->rq.x_host, r->x, npts_of(&r->rq) * 8, cudaMemcpyDeviceToHost);
  r->t_done = now_s();
  std::memset(&r->res, 0, sizeof(r->res));
  r->res.status = st.phase == 2 ? st.status : SC_ETIMEOUT;
  r->res.prec = r->sp.mixed ? SC_PREC_MIXED : SC_PREC_F64;
  r->res.iters = st.iters;
  r->res.rel_res = st.rel;
  r->res.queue_s = r->t_admit - r->t_submit;
  r->res.latency_s = r->t_done - r->t_submit;
}

// Copies a request's fields into its arena space and enqueues its
// right-hand side on `st` (synchronous for the host buffers it reads).
static int setup_request(sc_server *S, Req *r, cudaStream_t st) {
  Carver cv(S->arena_base + r->off, r->bytes);
  const long long n = npts_of(&r->rq);
  const bool plate = r->rq.kind == SC_REQ_PLATE;
  if (plate) {
    const long long np = padded_of(&r->rq, r->sp.R);
    r->f = static_cast<double *>(cv.take(n * 8));
    r->g = static_cast<double *>(cv.take(np * 8));
    cudaMemcpyAsync(r->f, r->rq.f_host, n * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(r->g, r->rq.ghost_host, np * 8, cudaMemcpyHostToDevice, st);
  }
  r->x = static_cast<double *>(cv.take(n * 8));
  if (!plate) cudaMemcpyAsync(r->x, r->rq.u_host, n * 8, cudaMemcpyHostToDevice, st);
  r->sp.x = r->x;
  layout(r->sp, cv, r->P, r->aux);
  int rc = upload_prob(r->sp, r->P, r->aux, st);
  if (!rc && plate) {
    sc_bvp b = as_bvp(&r->rq, r->f, r->g, r->x, S->min_pts);
    rc = setup_bvp(&b, r->sp, r->P, r->aux, st);
  } else if (!rc) {
    sc_ch c = as_ch(&r->rq);
    rc = setup_ch(&c, r->sp, r->P, r->aux, st);
  }
  r->t_admit = now_s();
  return rc;
}

// Second scheduler: plate requests for the preconditioned solver, one at a
// time in arrival order (skipping those that do not fit yet), on st2.
static void pcg_loop(sc_server *S) {
  cudaSetDevice(S->device);
  for (;;) {
    Req *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&] { return S->stop || !S->pcg_pending.empty(); });
      if (S->stop) return;
      for (auto it = S->pcg_pending.begin(); it != S->pcg_pending.end(); ++it) {
        size_t off;
        if (S->arena.alloc((*it)->bytes, &off)) {
          r = *it;
          r->off = off;
          S->pcg_pending.erase(it);
          S->pcg_active = r;
          break;
        }
      }
    }
    if (!r) continue;
    int rc = setup_request(S, r, S->st2);
    double res[3] = {0.0, 0.0, double(SC_OK)};
    if (!rc) rc = run_pcg(r->sp, r->P, r->aux, S->st2, res);
    if (!rc) {
      cudaError_t e = cudaMemcpyAsync(r->rq.x_host, r->x, npts_of(&r->rq) * 8, cudaMemcpyDeviceToHost, S->st2);
      if (e == cudaSuccess) e = cudaStreamSynchronize(S->st2);
      if (e != cudaSuccess) rc = fail(SC_ECUDA, "result copy: %s", cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(&r->res, 0, sizeof(r->res));
    r->t_done = now_s();
    r->res.status = rc ? rc : int(res[2]);
    r->res.prec = SC_PREC_F64;
    r->res.iters = (long long)res[0];
    r->res.rel_res = res[1];
    r->res.queue_s = r->t_admit - r->t_submit;
    r->res.latency_s = r->t_done - r->t_submit;
    r->done = true;
    if (rc == SC_ECUDA && !S->worker_error) S->worker_error = rc;
    S->arena.release(r->off, r->bytes);
    S->pcg_active = nullptr;
    S->cv_done.notify_all();
  }
}

static void worker_loop(sc_server *S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<Req *> admit;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->active.empty() && S->pending.empty())
        S->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&] { return S->stop || !S->pending.empty(); });
      if (S->stop) return;
      // admit in arrival order, skipping requests that do not fit yet
      int look = 0;
      for (auto it = S->pending.begin(); it != S->pending.end() && look < 256;) {
        ++look;
        if (int(S->active.size() + admit.size()) >= S->cfg.max_active) break;
        Req *r = *it;
        size_t off;
        if (S->arena.alloc(r->bytes, &off)) {
          r->off = off;
          admit.push_back(r);
          it = S->pending.erase(it);
        } else {
          ++it;
        }
      }
    }
    // set up admitted requests (outside the lock)
    for (Req *r : admit) {
      const int rc = setup_request(S, r, S->st);
      std::lock_guard<std::mutex> lk(S->mu);
      if (rc) {
        std::memset(&r->res, 0, sizeof(r->res));
        r->res.status = rc;
        r->t_done = now_s();
        r->res.latency_s = r->t_done - r->t_submit;
        r->done = true;
        S->arena.release(r->off, r->bytes);
        S->cv_done.notify_all();
      } else {
        S->active.push_back(r);
      }
    }
    std::vector<Req *> act;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      act = S->active;
    }
    if (act.empty()) continue;
    std::vector<SolveProb> hp(act.size());
    for (size_t i = 0; i < act.size(); ++i) hp[i] = act[i]->P;
    ++S->slices;
    // the test hook stands in for a launch that returned an error: nothing
    // is launched for that slice
    int rc = (S->cfg.fail_slice > 0 && S->slices == S->cfg.fail_slice)
                 ? fail(SC_ECUDA, "time slice %lld failed (injected by the test hook)", S->slices)
                 : run_persistent(hp, S->dprobs, S->dmap, S->dbars, S->st, LLONG_MAX, S->cfg.slice_ms);
    std::vector<SolveState> hs(act.size());
    if (!rc) rc = gather_states(S->dprobs, int(act.size()), S->dstates, hs.data(), S->st);
    cudaError_t e = cudaStreamSynchronize(S->st);
    if (rc || e != cudaSuccess) {
      // every resident request ends with the error and gives its arena
      // space back; later submissions are refused with the same error
      std::lock_guard<std::mutex> lk(S->mu);
      if (!S->worker_error) S->worker_error = rc ? rc : SC_ECUDA;
      const double t = now_s();
      for (Req *r : act) {
        std::memset(&r->res, 0, sizeof(r->res));
        r->res.status = S->worker_error;
        r->res.queue_s = r->t_admit - r->t_submit;
        r->res.latency_s = t - r->t_submit;
        r->done = true;
        S->arena.release(r->off, r->bytes);
      }
      S->active.clear();
      S->cv_done.notify_all();
      continue;
    }
    std::vector<Req *> finished;
    for (size_t i = 0; i < act.size(); ++i)
      if (hs[i].phase == 2) {
        retire(S, act[i], hs[i]);
        finished.push_back(act[i]);
      }
    if (!finished.empty()) {
      std::lock_guard<std::mutex> lk(S->mu);
      for (Req *r : finished) {
        r->done = true;
        S->arena.release(r->off, r->bytes);
        S->active.erase(std::find(S->active.begin(), S->active.end(), r));
      }
      S->cv_done.notify_all();
    }
  }
}

}  // namespace sc

using namespace sc;

extern "C" {

size_t sc_request_bytes(const sc_request *req) {
  if (!req) return 0;
  ProbSpec sp;
  size_t b = 0;
  if (request_layout(req, sp, &b, PCG_MIN_POINTS)) return 0;
  return b;
}

int sc_server_create(const sc_server_cfg *cfg, sc_server **out) {
  if (!cfg || !out || !cfg->arena_dev) return fail(SC_EINVAL, "null argument");
  if (cfg->max_active < 1 || cfg->max_active > 4096) return fail(SC_EINVAL, "max_active must be 1..4096");
  if (!(cfg->slice_ms > 0.0)) return fail(SC_EINVAL, "slice_ms must be positive");
  if (cfg->fail_slice < 0) return fail(SC_EINVAL, "fail_slice must be >= 0");
  if (cfg->pcg_min_points < 0) return fail(SC_EINVAL, "pcg_min_points must be >= 0");
  // the CTA -> problem map must hold the largest grid any persistent-kernel
  // variant can launch: bound it by the hardware limit of resident CTAs
  const int G = 32 * num_sms();
  Carver head(nullptr, 0);
  head.take(size_t(cfg->max_active) * sizeof(SolveProb));
  head.take(size_t(G) * sizeof(int));
  head.take(size_t(cfg->max_active) * 2 * sizeof(unsigned));
  head.take(size_t(cfg->max_active) * sizeof(SolveState));
  const size_t hbytes = (head.off + 255) & ~size_t(255);
  if (cfg->arena_bytes <= hbytes + 4096) return fail(SC_ENOMEM, "arena smaller than the server's descriptors");
  sc_server *S = new sc_server();
  S->cfg = *cfg;
  if (cfg->pcg_min_points > 0) S->min_pts = cfg->pcg_min_points;
  cudaGetDevice(&S->device);
  if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete S;
    return fail(SC_ECUDA, "stream creation failed");
  }
  if (cudaStreamCreateWithFlags(&S->st2, cudaStreamNonBlocking) != cudaSuccess) {
    cudaStreamDestroy(S->st);
    delete S;
    return fail(SC_ECUDA, "stream creation failed");
  }
  Carver hc(cfg->arena_dev, cfg->arena_bytes);
  S->dprobs = static_cast<SolveProb *>(hc.take(size_t(cfg->max_active) * sizeof(SolveProb)));
  S->dmap = static_cast<int *>(hc.take(size_t(G) * sizeof(int)));
  S->dbars = static_cast<unsigned *>(hc.take(size_t(cfg->max_active) * 2 * sizeof(unsigned)));
  S->dstates = static_cast<SolveState *>(hc.take(size_t(cfg->max_active) * sizeof(SolveState)));
  S->arena_base = static_cast<char *>(cfg->arena_dev) + hbytes;
  S->arena_size = cfg->arena_bytes - hbytes;
  S->arena.reset(S->arena_size);
  S->worker = std::thread(worker_loop, S);
  S->pcg_worker = std::thread(pcg_loop, S);
  *out = S;
  clear_error();
  return SC_OK;
}

int sc_server_destroy(sc_server *S) {
  if (!S) return fail(SC_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  if (S->pcg_worker.joinable()) S->pcg_worker.join();
  cudaStreamSynchronize(S->st);
  cudaStreamSynchronize(S->st2);
  cudaStreamDestroy(S->st);
  cudaStreamDestroy(S->st2);
  for (auto &kv : S->all) delete kv.second;
  delete S;
  clear_error();
  return SC_OK;
}

int sc_submit(sc_server *S, const sc_request *req, uint64_t *ticket) {
  if (!S || !req || !ticket) return fail(SC_EINVAL, "null argument");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->worker_error) return fail(S->worker_error, "the server stopped after a failed time slice");
  }
  if (!req->x_host) return fail(SC_EINVAL, "null host buffer");
  if (req->kind == SC_REQ_PLATE && (!req->f_host || !req->ghost_host)) return fail(SC_EINVAL, "null host buffer");
  if (req->kind == SC_REQ_CH && !req->u_host) return fail(SC_EINVAL, "null host buffer");
  Req *r = new Req();
  r->rq = *req;
  if (int rc = request_layout(req, r->sp, &r->bytes, S->min_pts)) {
    delete r;
    return rc;
  }
  if (r->bytes > S->arena_size) {
    delete r;
    return fail(SC_ENOMEM, "request needs %zu bytes, arena holds %zu", r->bytes, S->arena_size);
  }
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    S->all[r->id] = r;
    if (r->sp.solver == SC_SOLVER_PCG)
      S->pcg_pending.push_back(r);
    else
      S->pending.push_back(r);
    *ticket = r->id;
  }
  S->cv_work.notify_all();
  clear_error();
  return SC_OK;
}

int sc_poll(sc_server *S, uint64_t ticket, sc_result *out) {
  if (!S || !out) return fail(SC_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return fail(SC_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  Req *r = it->second;
  if (!r->done) return SC_EPENDING;
  *out = r->res;
  delete r;
  S->all.erase(it);
  clear_error();
  return SC_OK;
}

int sc_server_status(sc_server *S, int32_t *worker_error, size_t *free_bytes, size_t *arena_bytes,
                     int32_t *active, int32_t *pending) {
  if (!S) return fail(SC_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (worker_error) *worker_error = S->worker_error;
  if (free_bytes) *free_bytes = S->arena.free_total();
  if (arena_bytes) *arena_bytes = S->arena_size;
  if (active) *active = int32_t(S->active.size() + (S->pcg_active ? 1 : 0));
  if (pending) *pending = int32_t(S->pending.size() + S->pcg_pending.size());
  clear_error();
  return SC_OK;
}

int sc_server_drain(sc_server *S, double timeout_s) {
  if (!S) return fail(SC_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(S->mu);
  const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [&] {
                                        return S->pending.empty() && S->active.empty() && S->pcg_pending.empty() &&
                                               !S->pcg_active;
                                      });
  if (!ok) return fail(SC_ETIMEOUT, "requests still in flight after %.3f s", timeout_s);
  clear_error();
  return SC_OK;
}

}  // extern "C"
