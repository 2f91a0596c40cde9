// Segmented-sum kernels for one input dtype: the dense variant (SR_F_DENSE_SEGMENTS).
#include "sr_segmented_kernels.cuh"

namespace sr {
const void* seg_dense_f32(bool comp, int vec, int unroll) {
    return comp ? pick_seg_dense<kDtF32, true>(vec, unroll) : pick_seg_dense<kDtF32, false>(vec, unroll);
}
}  // namespace sr
