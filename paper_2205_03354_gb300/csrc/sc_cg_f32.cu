// Persistent CG kernel variants with FP32 inner iterations (mixed precision).
#include "sc_cg_kernels.cuh"

namespace sc {

CgKernel cg_kernel_f32(int dims) {
  return dims == 1 ? cg_persistent_kernel<float, 2, 1>
                   : dims == 2 ? cg_persistent_kernel<float, 2, 2> : cg_persistent_kernel<float, 2, 3>;
}

}  // namespace sc
