// Segmented-sum kernels for one input dtype: the TMA form (SR_F_BULK).
#include "sr_segmented_kernels.cuh"

namespace sr {
const void* seg_tma_bf16(bool comp, int vec, int unroll) {
    return comp ? pick_seg_tma<kDtBF16, true>(vec, unroll) : pick_seg_tma<kDtBF16, false>(vec, unroll);
}
}  // namespace sr
