// Segmented-sum kernel instantiations for one input dtype.
#include "sr_segmented_kernels.cuh"

namespace sr {
bool seg_kernels_f32(bool comp, int vec, int unroll, bool dense, bool bulk, const void** main, const void** fin) {
    return comp ? pick_seg_kernels<kDtF32, true>(vec, unroll, dense, bulk, main, fin)
                : pick_seg_kernels<kDtF32, false>(vec, unroll, dense, bulk, main, fin);
}
}  // namespace sr
