// Kernel instantiations of the hierarchical sum for one input dtype.
#include "sr_reduce_kernels.cuh"

namespace sr {
bool kernels_i32(bool comp, bool fp64, bool bulk, int vec, int unroll, KernelSet* k) {
    (void)comp;  // integer sums are exact: no compensation
    return pick_kernels<kDtI32, false>(fp64, bulk, vec, unroll, k);
}
}  // namespace sr
