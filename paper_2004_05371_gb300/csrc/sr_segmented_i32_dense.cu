// Segmented-sum kernels for one input dtype: the dense variant (SR_F_DENSE_SEGMENTS).
// Integer sums are exact: no compensated form.
#include "sr_segmented_kernels.cuh"

namespace sr {
const void* seg_dense_i32(bool comp, int vec, int unroll) {
    (void)comp;
    return pick_seg_dense<kDtI32, false>(vec, unroll);
}
}  // namespace sr
