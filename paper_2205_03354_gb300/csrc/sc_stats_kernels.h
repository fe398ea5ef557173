// Declarations of the Cahn-Hilliard statistics kernels defined in
// sc_solver.cu, for other translation units that launch them.
#pragma once
#include <cuda_runtime.h>

namespace sc {

constexpr int STATS_NTHR = 256;          // block size of both kernels
constexpr int STATS_CHUNK = 256 * 16;    // grid points per partial sum

__global__ void k_ch_stats_part(const double *__restrict__ u, int ndim, int nx, int ny, int nz, double h,
                                double kappa, int chem, double rho, double ca, double cb,
                                double *__restrict__ pm, double *__restrict__ pe);
__global__ void k_sum_final(const double *__restrict__ part, int n, double *__restrict__ scal, int slot);

}  // namespace sc
