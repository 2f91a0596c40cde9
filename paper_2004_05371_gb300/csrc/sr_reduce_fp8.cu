// Kernel instantiations of the hierarchical sum for one input dtype.
#include "sr_reduce_kernels.cuh"

namespace sr {
bool kernels_fp8(bool comp, bool fp64, bool bulk, int vec, int unroll, KernelSet* k) {
    return comp ? pick_kernels<kDtFP8, true>(fp64, bulk, vec, unroll, k)
                : pick_kernels<kDtFP8, false>(fp64, bulk, vec, unroll, k);
}
}  // namespace sr
