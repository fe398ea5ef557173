// Persistent CG kernel variants serving both precision classes in one launch.
#include "sc_cg_kernels.cuh"

namespace sc {

CgKernel cg_kernel_both(int dims) {
  return dims == 1 ? cg_persistent_both<2, 1> : dims == 2 ? cg_persistent_both<2, 2> : cg_persistent_both<2, 3>;
}

}  // namespace sc
