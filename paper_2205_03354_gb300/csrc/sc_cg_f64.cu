// Persistent CG kernel variants with FP64 iterations.
#include "sc_cg_kernels.cuh"

namespace sc {

CgKernel cg_kernel_f64(int dims) {
  return dims == 1 ? cg_persistent_kernel<double, 2, 1>
                   : dims == 2 ? cg_persistent_kernel<double, 2, 2> : cg_persistent_kernel<double, 2, 3>;
}

}  // namespace sc
