// Preconditioned CG for the plate problem (Sec. 3.3) on large grids.
//
// Unpreconditioned CG on the composed 13/25-point operator needs O(N^2)
// iterations (its condition number grows like h^-4: about 4.5e5 iterations
// at 2048^2).  With the boundary data read by odd reflection the composed
// operator would be exactly L_D^2, L_D the second-order Dirichlet Laplacian,
// which the orthonormal sine transform (DST-I) S diagonalises along every
// axis: L_D = S Lambda S with Lambda = sum_a (2 - 2 cos(pi k_a / (N+1))) / h^2.
// The exact-ghost operator A (zero ghost ring, the data moved to the
// right-hand side) differs from L_D^2 only in rows next to the boundary, so
// M^-1 = S Lambda^-2 S is a preconditioner under which CG needs tens of
// iterations (measured 10-31 from N = 32 to 512 in 2D).
//
// The preconditioner runs in FP32: each axis transform is a dense product
// with S (a cuBLAS GEMM, batched over the other axes, with FP32 accuracy
// emulated on the BF16 tensor cores), then the diagonal scaling, then the
// transforms again; the lowest K0^d modes are transformed in FP64.  Everything else --
// x, r, p, the products A p, the dot products -- stays in FP64, and because
// an FP32 preconditioner is not exactly the same linear map at every use, the
// update of the search direction uses the flexible (Polak-Ribiere) form
// beta = z_new . (r_new - r_old) / (z_old . r_old), with r_new - r_old =
// -alpha A p.  Convergence is declared on the FP64 true residual.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "sc_apply_host.h"
#include "sc_device.cuh"
#include "sc_internal.h"
#include "sc_solver.cuh"
#include "sc_solver_host.h"

namespace sc {

// ---------------------------------------------------------------------------
// Dense products of the transforms (cuBLAS), row-major, strided batches:
// C[b] = A[b] (M x K) * B[b] (K x N)
// ---------------------------------------------------------------------------

template <typename T>
struct GemmArgs {
  const T *A, *B;
  T *C;
  int M, N, K;
  long long lda, ldb, ldc;
  long long sa, sb, sc;  // batch strides (0: shared operand)
};

// One cuBLAS handle per host thread and device (the server's scheduler
// threads and callers' threads never share one), destroyed at thread exit.
struct BlasHandles {
  cublasHandle_t h[64] = {};
  ~BlasHandles() {
    for (cublasHandle_t &x : h)
      if (x) cublasDestroy(x);
  }
};

static cublasHandle_t blas_handle() {
  thread_local BlasHandles hs;
  int dev = 0;
  cudaGetDevice(&dev);
  cublasHandle_t &h = hs.h[dev & 63];
  if (!h && cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) h = nullptr;
  return h;
}

// The FP32 transforms run with FP32 accuracy emulated on the BF16 tensor
// cores (each operand split into three BF16 parts, nine products, FP32
// accumulation; cuBLAS picks the emulation where it is faster and the native
// pipe otherwise; a library without that compute type runs the native one).
// The FP64 low-mode products stay native FP64: the fixed-point emulation left
// an algebraic error of 1e-8 in the 2048^2 plate solution at a residual of
// 1e-10 (native: below 1e-9).
template <typename T>
static int gemm(const GemmArgs<T> &g, int batch, cudaStream_t st) {
  static std::atomic<int> emulate{1};
  cublasHandle_t h = blas_handle();
  if (!h) return fail(SC_ECUDA, "cuBLAS handle creation failed");
  if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return fail(SC_ECUDA, "cuBLAS stream");
  const cudaDataType_t dt = sizeof(T) == 8 ? CUDA_R_64F : CUDA_R_32F;
  const T one = T(1), zero = T(0);
  // row-major C = A B is column-major C^T = B^T A^T
  for (int pass = 0; pass < 2; ++pass) {
    const bool em = emulate.load(std::memory_order_relaxed) != 0;
    if (pass == 1 && em) break;
    cublasComputeType_t ct =
        sizeof(T) == 8 ? CUBLAS_COMPUTE_64F : (em ? CUBLAS_COMPUTE_32F_EMULATED_16BFX9 : CUBLAS_COMPUTE_32F);
    const cublasStatus_t s = cublasGemmStridedBatchedEx(
        h, CUBLAS_OP_N, CUBLAS_OP_N, g.N, g.M, g.K, &one, g.B, dt, int(g.ldb), g.sb, g.A, dt, int(g.lda), g.sa,
        &zero, g.C, dt, int(g.ldc), g.sc, batch, ct, CUBLAS_GEMM_DEFAULT);
    if (s == CUBLAS_STATUS_SUCCESS) return SC_OK;
    if (!em || sizeof(T) == 8 || (s != CUBLAS_STATUS_NOT_SUPPORTED && s != CUBLAS_STATUS_INVALID_VALUE))
      return fail(SC_ECUDA, "cuBLAS GEMM failed (status %d)", int(s));
    emulate.store(0);  // retry with the native compute type
  }
  return fail(SC_ECUDA, "cuBLAS GEMM failed");
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

// S[j][k] = sqrt(2 / (N + 1)) sin(pi (j + 1)(k + 1) / (N + 1)), the
// orthonormal DST-I (S S = I).  The angle is reduced exactly in integers.
__global__ void k_dst_matrix(float *S, int N) {
  const long long n2 = (long long)N * N;
  const double c = sqrt(2.0 / double(N + 1));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = i / N + 1, k = i % N + 1;
    const long long m = (j * k) % (2LL * (N + 1));
    S[i] = float(c * sinpi(double(m) / double(N + 1)));
  }
}

// Sl[k][j] = S[k][j] for k < K0 (FP64) and SlT its transpose.
__global__ void k_dst_low(double *Sl, double *SlT, int N, int K0) {
  const long long n = (long long)K0 * N;
  const double c = sqrt(2.0 / double(N + 1));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long k = i / N, j = i % N;
    const long long m = ((k + 1) * (j + 1)) % (2LL * (N + 1));
    const double v = c * sinpi(double(m) / double(N + 1));
    Sl[i] = v;
    SlT[j * K0 + k] = v;
  }
}

// C[k...] /= (sum_a lam1[k_a])^2 on the K0^ndim low block.
__global__ void k_low_scale(double *__restrict__ C, const double *__restrict__ lam1, int K0, int ndim) {
  const long long n = ndim == 3 ? (long long)K0 * K0 * K0 : (long long)K0 * K0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double l = lam1[i % K0] + lam1[(i / K0) % K0];
    if (ndim == 3) l += lam1[i / ((long long)K0 * K0)];
    C[i] /= l * l;
  }
}

// z = double(u) + zl
__global__ void k_add_f32(const float *__restrict__ u, const double *__restrict__ zl, double *__restrict__ z,
                          long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    z[i] = double(u[i]) + zl[i];
}

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = float(a[i]);
}
__global__ void k_to_f64(const float *__restrict__ a, double *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = double(a[i]);
}

// u /= (sum_a lam1[k_a])^2 on the N^ndim grid (k_a the index along axis a),
// except on the low block (every k_a < K0), which is set to zero: those
// modes are handled in FP64.
// u /= Lambda^2 mode by mode in FP32 (the transforms around it are FP32),
// zero on the low block that the FP64 products handle.  Blocks stride over
// the grid rows (ky, kz), threads over kx: no 64-bit index division.
__global__ void k_inv_lambda2(float *__restrict__ u, const double *__restrict__ lam1, int N, int ndim, int K0) {
  const long long rows = ndim == 3 ? (long long)N * N : N;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int ky = int(row % N), kz = ndim == 3 ? int(row / N) : 0;
    const float lyz = float(lam1[ky] + (ndim == 3 ? lam1[kz] : 0.0));
    const bool low_yz = ky < K0 && kz < K0;
    float *ur = u + row * N;
    for (int kx = threadIdx.x; kx < N; kx += blockDim.x) {
      const float l = float(lam1[kx]) + lyz;
      ur[kx] = (low_yz && kx < K0) ? 0.0f : ur[kx] / (l * l);
    }
  }
}

// Scalars of the inner CG loop, kept on the device so that an iteration
// needs no host round trip (and can be replayed from a CUDA graph).
struct PcgScal {
  double rz;       // z . r of the current direction
  double alpha, beta;
  double rn;       // ||r|| of the recurrence
  double stop;     // the recurrence stops at rn <= stop
  long long it, maxit;
  int active;      // 0: converged, failed or out of iterations: kernels skip
  int status;      // SC_OK, SC_ENOTCONV or SC_EBREAKDOWN
};

static_assert(sizeof(PcgScal) <= 24 * sizeof(double), "the scalars follow 8 result slots in a 32-double block");

__global__ void k_pcg_scal_init(PcgScal *sc, double rz, double stop, long long it, long long maxit) {
  sc->rz = rz;
  sc->alpha = sc->beta = 0.0;
  sc->rn = 0.0;
  sc->stop = stop;
  sc->it = it;
  sc->maxit = maxit;
  sc->active = 1;
  sc->status = SC_OK;
}
// alpha = rz / (p . q)
__global__ void k_pcg_alpha(PcgScal *sc, const double *__restrict__ out) {
  if (!sc->active) return;
  if (sc->it >= sc->maxit) {
    sc->status = SC_ENOTCONV;
    sc->active = 0;
    return;
  }
  const double pq = out[0], rz = sc->rz;
  if (!(pq > 0.0) || !(rz == rz)) {
    sc->status = SC_EBREAKDOWN;
    sc->active = 0;
    return;
  }
  sc->alpha = rz / pq;
}
// out = {r.r, z.r, z.q}: the flexible direction update z_new . (r_new -
// r_old) = -alpha z_new . q, and the recurrence's stopping test
__global__ void k_pcg_beta(PcgScal *sc, const double *__restrict__ out) {
  if (!sc->active) return;
  ++sc->it;
  const double rn = sqrt(out[0]);
  sc->rn = rn;
  if (!(rn == rn)) {
    sc->status = SC_EBREAKDOWN;
    sc->active = 0;
    return;
  }
  sc->beta = -sc->alpha * out[2] / sc->rz;
  sc->rz = out[1];
  if (rn <= sc->stop) sc->active = 0;
}
// x += alpha p, r -= alpha q
__global__ void k_pcg_xr(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                         const double *__restrict__ q, const PcgScal *__restrict__ sc, long long n) {
  if (!sc->active) return;
  const double a = sc->alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    r[i] = fma(-a, q[i], r[i]);
  }
}
// p = z + beta p
__global__ void k_pcg_p(double *__restrict__ p, const double *__restrict__ z, const PcgScal *__restrict__ sc,
                        long long n) {
  if (!sc->active) return;
  const double b = sc->beta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(b, p[i], z[i]);
}
// r = b - A x for the plate operator (zero ghost ring) with the sum of the
// products carried in double-double: each product w x is split exactly by
// an FMA (TwoProduct) and the running sum by Knuth's TwoSum, so the only
// rounding is that of the final difference.  The composed weights are exact
// integers times (N+1)^4 here, so A x itself is exact up to the final
// rounding; the plain FP64 sum loses about log10(sum |w x| / |A x|) digits
// (12 at 2048^2), which puts a 1e-10 relative residual out of its reach.
struct DdStencil {
  int npts;
  int off[25][3];
  double w[25];
};
__global__ void k_resid_dd(const double *__restrict__ x, const double *__restrict__ b, double *__restrict__ r,
                           int nx, int ny, int nz, const __grid_constant__ DdStencil S) {
  const long long n = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = int(i % nx), iy = int((i / nx) % ny), iz = int(i / ((long long)nx * ny));
    double hi = 0.0, lo = 0.0;
    for (int k = 0; k < S.npts; ++k) {
      const int jx = ix + S.off[k][0], jy = iy + S.off[k][1], jz = iz + S.off[k][2];
      if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
      const double v = __ldg(x + ((long long)jz * ny + jy) * nx + jx);
      const double p = S.w[k] * v, pe = fma(S.w[k], v, -p);
      const double s = hi + p, bb = s - hi;
      lo += ((hi - (s - bb)) + (p - bb)) + pe;
      hi = s;
    }
    const double bi = b[i], s = bi - hi, bb = s - bi;
    const double e = (bi - (s - bb)) + (-hi - bb);
    r[i] = s + (e - lo);
  }
}

// p = z + b p
// Up to three dot products in one pass: part[k * nblk + blk] = sum over the
// block's chunk of u_k . v_k (fixed order), then k_pcg_sum adds the parts.
constexpr int PD_NTHR = 256, PD_CHUNK = PD_NTHR * 16;
__global__ void k_pcg_dots(const double *__restrict__ u0, const double *__restrict__ v0,
                           const double *__restrict__ u1, const double *__restrict__ v1,
                           const double *__restrict__ u2, const double *__restrict__ v2, int nd,
                           long long n, double *__restrict__ part) {
  __shared__ double red[PD_NTHR / 32];
  const long long e0 = (long long)blockIdx.x * PD_CHUNK, e1 = min(e0 + PD_CHUNK, n);
  const double *us[3] = {u0, u1, u2}, *vs[3] = {v0, v1, v2};
  for (int k = 0; k < nd; ++k) {
    double s = 0.0;
    for (long long i = e0 + threadIdx.x; i < e1; i += PD_NTHR) s = fma(us[k][i], vs[k][i], s);
    s = block_sum<PD_NTHR>(s, red);
    if (threadIdx.x == 0) part[(long long)k * gridDim.x + blockIdx.x] = s;
  }
}
__global__ void k_pcg_sum(const double *__restrict__ part, int nblk, int nd, double *__restrict__ out) {
  __shared__ double red[PD_NTHR / 32];
  for (int k = 0; k < nd; ++k) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += PD_NTHR) s += part[(long long)k * nblk + i];
    s = block_sum<PD_NTHR>(s, red);
    if (threadIdx.x == 0) out[k] = s;
  }
}

}  // namespace sc

namespace sc {

long long pcg_parts(long long n) { return (n + PD_CHUNK - 1) / PD_CHUNK; }

static const double *b_dev(const SolveProb &P) { return P.rhs; }

static int grid_for(long long n) { return int(std::min<long long>((n + 255) / 256, 8LL * num_sms())); }

// u <- u transformed by S along every axis (ping-pong through w; the result
// ends in u).  Grid layout [z][y][x], N points per axis.
static int dst_all(float *u, float *w, const float *S, int N, int ndim, cudaStream_t st) {
  const long long N2 = (long long)N * N;
  // x axis: rows of N values times S (S symmetric): C = U S
  if (int rc = gemm(GemmArgs<float>{u, S, w, int(ndim == 3 ? N2 : N), N, N, N, N, N, 0, 0, 0}, 1, st)) return rc;
  if (ndim == 2)  // y axis: C = S W
    return gemm(GemmArgs<float>{S, w, u, N, N, N, N, N, N, 0, 0, 0}, 1, st);
  // y axis, one z plane per batch: C_z = S W_z
  if (int rc = gemm(GemmArgs<float>{S, w, u, N, N, N, N, N, N, 0, N2, N2}, N, st)) return rc;
  // z axis: C = S U viewed as N x N^2
  if (int rc = gemm(GemmArgs<float>{S, u, w, N, int(N2), N, N, N2, N2, 0, 0, 0}, 1, st)) return rc;
  cudaMemcpyAsync(u, w, size_t(N2) * N * sizeof(float), cudaMemcpyDeviceToDevice, st);
  return SC_OK;
}

// 16^ndim lowest modes: a 2048^2 plate converges in 85 iterations with it
// (81 with 64^2 FP64 modes, at twice the FP64 product time per iteration).
int pcg_low_modes(int ndim, long long N) {
  (void)ndim;
  return int(std::min<long long>(N, 16));
}

// zl = S_low^T Lambda^-2 S_low r over the K0^ndim lowest modes, in FP64.
static int precond_low(const double *r, const ProbAux &aux, int N, int K0, int ndim, cudaStream_t st) {
  const long long N2 = (long long)N * N, K2 = (long long)K0 * K0;
  typedef GemmArgs<double> G;
  if (ndim == 2) {
    const G g1{r, aux.SlT, aux.wa, N, K0, N, N, K0, K0, 0, 0, 0};            // (y, kx)
    const G g2{aux.Sl, aux.wa, aux.wb, K0, K0, N, N, K0, K0, 0, 0, 0};       // (ky, kx)
    const G g3{aux.SlT, aux.wb, aux.wa, N, K0, K0, K0, K0, K0, 0, 0, 0};     // (y, kx)
    const G g4{aux.wa, aux.Sl, aux.zl, N, N, K0, K0, N, N, 0, 0, 0};         // (y, x)
    if (int rc = gemm(g1, 1, st)) return rc;
    if (int rc = gemm(g2, 1, st)) return rc;
    k_low_scale<<<grid_for(K2), 256, 0, st>>>(aux.wb, aux.lam1, K0, 2);
    if (int rc = gemm(g3, 1, st)) return rc;
    return gemm(g4, 1, st);
  }
  const G g1{r, aux.SlT, aux.wa, int(N2), K0, N, N, K0, K0, 0, 0, 0};                    // (z, y, kx)
  const G g2{aux.Sl, aux.wa, aux.wb, K0, K0, N, N, K0, K0, 0, (long long)N * K0, K2};    // (z, ky, kx)
  const G g3{aux.Sl, aux.wb, aux.wc, K0, int(K2), N, N, K2, K2, 0, 0, 0};                // (kz, ky, kx)
  const G g4{aux.SlT, aux.wc, aux.wb, N, int(K2), K0, K0, K2, K2, 0, 0, 0};              // (z, ky, kx)
  const G g5{aux.SlT, aux.wb, aux.wa, N, K0, K0, K0, K0, K0, 0, K2, (long long)N * K0};  // (z, y, kx)
  const G g6{aux.wa, aux.Sl, aux.zl, int(N2), N, K0, K0, N, N, 0, 0, 0};                 // (z, y, x)
  if (int rc = gemm(g1, 1, st)) return rc;
  if (int rc = gemm(g2, N, st)) return rc;
  if (int rc = gemm(g3, 1, st)) return rc;
  k_low_scale<<<grid_for(K2 * K0), 256, 0, st>>>(aux.wc, aux.lam1, K0, 3);
  if (int rc = gemm(g4, 1, st)) return rc;
  if (int rc = gemm(g5, N, st)) return rc;
  return gemm(g6, 1, st);
}

// z = M^-1 r = S Lambda^-2 S r: the lowest modes in FP64, the rest in FP32.
static int precond(const double *r, double *z, const ProbAux &aux, int N, int ndim, long long n,
                   cudaStream_t st) {
  const int g = grid_for(n);
  const int K0 = pcg_low_modes(ndim, N);
  if (int rc = precond_low(r, aux, N, K0, ndim, st)) return rc;
  k_to_f32<<<g, 256, 0, st>>>(r, aux.u0, n);
  if (int rc = dst_all(aux.u0, aux.u1, aux.S, N, ndim, st)) return rc;
  k_inv_lambda2<<<int(std::min<long long>(ndim == 3 ? (long long)N * N : N, 16LL * num_sms())), 256, 0, st>>>(
      aux.u0, aux.lam1, N, ndim, K0);
  if (int rc = dst_all(aux.u0, aux.u1, aux.S, N, ndim, st)) return rc;
  k_add_f32<<<g, 256, 0, st>>>(aux.u0, aux.zl, z, n);
  return SC_OK;
}

// Dot products (u_k . v_k, k < nd) to the host.
static int dots(const double *u0, const double *v0, const double *u1, const double *v1, const double *u2,
                const double *v2, int nd, long long n, const ProbAux &aux, cudaStream_t st, double *host) {
  const int nblk = int(pcg_parts(n));
  k_pcg_dots<<<nblk, PD_NTHR, 0, st>>>(u0, v0, u1, v1, u2, v2, nd, n, aux.part);
  k_pcg_sum<<<1, PD_NTHR, 0, st>>>(aux.part, nblk, nd, aux.out);
  cudaMemcpyAsync(host, aux.out, size_t(nd) * 8, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SC_ECUDA, "preconditioned CG: %s", cudaGetErrorString(e));
  return SC_OK;
}

// A non-blocking stream per host thread and device for the solve (the
// caller's stream may be the legacy default stream, which cannot be
// captured into a graph), with the event that orders it after the caller's
// earlier work.
struct PcgStreams {
  cudaStream_t s[64] = {};
  cudaEvent_t e[64] = {};
  ~PcgStreams() {
    for (int i = 0; i < 64; ++i) {
      if (e[i]) cudaEventDestroy(e[i]);
      if (s[i]) cudaStreamDestroy(s[i]);
    }
  }
};

static int solve_stream(cudaStream_t caller, cudaStream_t *out) {
  thread_local PcgStreams ps;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaStream_t &s = ps.s[dev & 63];
  cudaEvent_t &e = ps.e[dev & 63];
  if (!s && (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess))
    return fail(SC_ECUDA, "preconditioned CG: stream creation failed");
  cudaEventRecord(e, caller);
  cudaStreamWaitEvent(s, e, 0);
  *out = s;
  return SC_OK;
}

static int pcg_on(const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t st, double *res);

int run_pcg(const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t caller, double *res) {
  // the whole solve runs on the thread's own stream, and nothing of it is
  // left in flight when this returns, on success or on error
  cudaStream_t st = nullptr;
  if (int rc = solve_stream(caller, &st)) return rc;
  const int rc = pcg_on(sp, P, aux, st, res);
  cudaStreamSynchronize(st);
  return rc;
}

static int pcg_on(const ProbSpec &sp, SolveProb &P, const ProbAux &aux, cudaStream_t st, double *res) {
  const int N = int(sp.n[0]), nd = sp.ndim;
  const long long n = P.npts;
  const int g = grid_for(n);
  // operator, transform and eigenvalues
  sc_stencil L, B;
  sc_laplacian(nd, sp.order, &L);
  sc_compose_stencil(&L, &L, &B);
  auto apply = [&](const double *in, double *out) {
    ApplyReq q{&B, SC_F64, SC_BC_ZERO, sp.n, sp.h_num, sp.h_den, in, out};
    return apply_enqueue(q, st);
  };
  DdStencil dd;
  std::memset(&dd, 0, sizeof(dd));
  if (B.npts > 25) return fail(SC_EINVAL, "internal: operator too wide for the residual kernel");
  dd.npts = B.npts;
  {
    std::vector<double> w(B.npts);
    if (int rc = weights_f64(&B, sp.h_num, sp.h_den, w.data())) return rc;
    for (int k = 0; k < B.npts; ++k) {
      for (int a = 0; a < 3; ++a) dd.off[k][a] = B.off[k][a];
      dd.w[k] = w[k];
    }
  }
  // r = b - A x with an accurate sum (see k_resid_dd)
  auto resid = [&](const double *xx, double *rr) {
    k_resid_dd<<<g, 256, 0, st>>>(xx, b_dev(P), rr, int(sp.n[0]), int(sp.n[1]), nd == 3 ? int(sp.n[2]) : 1, dd);
  };
  k_dst_matrix<<<grid_for((long long)N * N), 256, 0, st>>>(aux.S, N);
  {
    const int K0 = pcg_low_modes(nd, N);
    k_dst_low<<<grid_for((long long)K0 * N), 256, 0, st>>>(aux.Sl, aux.SlT, N, K0);
  }
  {
    const double h = double(sp.h_num) / double(sp.h_den);
    std::vector<double> lam(N);
    for (int k = 1; k <= N; ++k) {
      const double s = std::sin(M_PI * double(k) / (2.0 * double(N + 1)));
      lam[k - 1] = 4.0 * s * s / (h * h);  // (2 - 2 cos(pi k / (N+1))) / h^2
    }
    cudaMemcpyAsync(aux.lam1, lam.data(), size_t(N) * 8, cudaMemcpyHostToDevice, st);
    cudaError_t e = cudaStreamSynchronize(st);  // lam is a local
    if (e != cudaSuccess) return fail(SC_ECUDA, "preconditioned CG set-up: %s", cudaGetErrorString(e));
  }
  double *x = P.x, *b = P.rhs, *r = P.r, *p = static_cast<double *>(P.p), *q = static_cast<double *>(P.q),
         *z = aux.z;
  PcgScal *dsc = reinterpret_cast<PcgScal *>(aux.out + 8);
  const int nblk = int(pcg_parts(n));
  auto dots_enq = [&](const double *u0, const double *v0, const double *u1, const double *v1, const double *u2,
                      const double *v2, int ndot) {
    k_pcg_dots<<<nblk, PD_NTHR, 0, st>>>(u0, v0, u1, v1, u2, v2, ndot, n, aux.part);
    k_pcg_sum<<<1, PD_NTHR, 0, st>>>(aux.part, nblk, ndot, aux.out);
  };
  // One inner iteration, enqueued with no host synchronisation; once the
  // recurrence has stopped, its own kernels return at once.
  auto iteration = [&]() -> int {
    if (int rc = apply(p, q)) return rc;
    dots_enq(p, q, nullptr, nullptr, nullptr, nullptr, 1);
    k_pcg_alpha<<<1, 1, 0, st>>>(dsc, aux.out);
    k_pcg_xr<<<g, 256, 0, st>>>(x, r, p, q, dsc, n);
    if (int rc = precond(r, z, aux, N, nd, n, st)) return rc;
    dots_enq(r, r, z, r, z, q, 3);
    k_pcg_beta<<<1, 1, 0, st>>>(dsc, aux.out);
    k_pcg_p<<<g, 256, 0, st>>>(p, z, dsc, n);
    return SC_OK;
  };
  // The iteration as a CUDA graph, captured after the first batch has run
  // (so that every library set-up is done) and replayed from then on; a
  // stream that cannot be captured keeps launching the iteration directly.
  struct Exec {
    cudaGraphExec_t e = nullptr;
    ~Exec() {
      if (e) cudaGraphExecDestroy(e);
    }
  } graph;
  bool tried = false;
  auto try_capture = [&]() {
    tried = true;
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    const int rc = iteration();
    const cudaError_t e = cudaStreamEndCapture(st, &gr);
    if (rc == SC_OK && e == cudaSuccess && gr && cudaGraphInstantiate(&graph.e, gr, 0) != cudaSuccess)
      graph.e = nullptr;
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    clear_error();
  };
  constexpr int BATCH = 4;  // iterations between reads of the scalars
  double hs[3];
  if (int rc = dots(b, b, nullptr, nullptr, nullptr, nullptr, 1, n, aux, st, hs)) return rc;
  const double bn = std::sqrt(hs[0]), tol = sp.rtol;
  long long it = 0;
  int status = SC_OK;
  double rel = 0.0;
  // x0 = 0 (set by the plate set-up); each pass starts from the true residual
  for (int pass = 0; bn > 0 && pass < 8; ++pass) {
    resid(x, r);
    if (int rc = precond(r, z, aux, N, nd, n, st)) return rc;
    cudaMemcpyAsync(p, z, size_t(n) * 8, cudaMemcpyDeviceToDevice, st);
    if (int rc = dots(r, z, r, r, nullptr, nullptr, 2, n, aux, st, hs)) return rc;
    const double rz = hs[0], rn = std::sqrt(hs[1]);
    rel = rn / bn;
    if (rel <= tol) break;  // the true residual meets the tolerance
    // the recurrence is driven a little below the tolerance: on the largest
    // grids the recomputed residual differs from it by rounding of the same
    // order (the operator's weights scale as h^-4)
    k_pcg_scal_init<<<1, 1, 0, st>>>(dsc, rz, 0.25 * tol * bn, it, sp.maxit);
    for (;;) {
      for (int k = 0; k < BATCH; ++k) {
        if (graph.e) {
          if (cudaGraphLaunch(graph.e, st) != cudaSuccess) return fail(SC_ECUDA, "preconditioned CG graph launch");
        } else if (int rc = iteration()) {
          return rc;
        }
      }
      PcgScal hsc;
      cudaMemcpyAsync(&hsc, dsc, sizeof(hsc), cudaMemcpyDeviceToHost, st);
      const cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return fail(SC_ECUDA, "preconditioned CG: %s", cudaGetErrorString(e));
      it = hsc.it;
      if (!hsc.active) {
        status = hsc.status;
        break;
      }
      if (!tried) try_capture();
    }
    if (status != SC_OK) break;
  }
  // true residual of the returned x
  resid(x, r);
  double rr;
  if (int rc = dots(r, r, nullptr, nullptr, nullptr, nullptr, 1, n, aux, st, &rr)) return rc;
  rel = bn > 0 ? std::sqrt(rr) / bn : 0.0;
  if (status == SC_OK && !(rel <= tol)) status = (rel == rel) ? SC_ENOTCONV : SC_EBREAKDOWN;
  res[0] = double(it);
  res[1] = rel;
  res[2] = double(status);
  return SC_OK;
}

}  // namespace sc
