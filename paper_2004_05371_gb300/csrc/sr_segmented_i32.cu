// Segmented-sum kernel instantiations for one input dtype.
#include "sr_segmented_kernels.cuh"

namespace sr {
bool seg_kernels_i32(bool comp, int vec, int unroll, bool dense, bool bulk, const void** main, const void** fin) {
    (void)comp;  // integer sums are exact: no compensation
    return pick_seg_kernels<kDtI32, false>(vec, unroll, dense, bulk, main, fin);
}
}  // namespace sr
