// Segmented-sum kernels for one input dtype: the TMA form (SR_F_BULK).
#include "sr_segmented_kernels.cuh"

namespace sr {
const void* seg_tma_fp8(bool comp, int vec, int unroll) {
    return comp ? pick_seg_tma<kDtFP8, true>(vec, unroll) : pick_seg_tma<kDtFP8, false>(vec, unroll);
}
}  // namespace sr
