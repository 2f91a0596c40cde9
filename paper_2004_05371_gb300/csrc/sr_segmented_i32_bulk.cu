// Segmented-sum kernels for one input dtype: the TMA form (SR_F_BULK).
// Integer sums are exact: no compensated form.
#include "sr_segmented_kernels.cuh"

namespace sr {
const void* seg_tma_i32(bool comp, int vec, int unroll) {
    (void)comp;
    return pick_seg_tma<kDtI32, false>(vec, unroll);
}
}  // namespace sr
