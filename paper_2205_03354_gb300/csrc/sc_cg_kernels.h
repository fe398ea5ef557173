// Entry points of the persistent CG kernel variants (sc_cg_f32.cu,
// sc_cg_f64.cu, sc_cg_both.cu).
#pragma once
#include "sc_solver.cuh"

namespace sc {

typedef void (*CgKernel)(const SolveProb *, const int *, long long, unsigned long long);

// dims: 1 = 2D problems only, 2 = 3D only, 3 = both
CgKernel cg_kernel_f32(int dims);   // FP32 inner iterations (mixed precision)
CgKernel cg_kernel_f64(int dims);   // FP64 throughout
CgKernel cg_kernel_both(int dims);  // either, chosen per problem

}  // namespace sc
