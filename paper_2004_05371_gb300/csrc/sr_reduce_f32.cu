// Kernel instantiations of the hierarchical sum for one input dtype.
#include "sr_reduce_kernels.cuh"

namespace sr {
bool kernels_f32(bool comp, bool fp64, bool bulk, int vec, int unroll, KernelSet* k) {
    return comp ? pick_kernels<kDtF32, true>(fp64, bulk, vec, unroll, k)
                : pick_kernels<kDtF32, false>(fp64, bulk, vec, unroll, k);
}
}  // namespace sr
