// Segmented-sum kernels of every input dtype: the adaptive form
// (SR_F_ADAPTIVE_SEGMENTS), one cooperative launch for mixed layouts.
#include "sr_segmented_kernels.cuh"

namespace sr {
const void* seg_adapt_f32(bool comp, int vec, int unroll) {
    return comp ? pick_seg_adapt<kDtF32, true>(vec, unroll) : pick_seg_adapt<kDtF32, false>(vec, unroll);
}
const void* seg_adapt_i32(bool comp, int vec, int unroll) {
    (void)comp;  // integer sums are exact
    return pick_seg_adapt<kDtI32, false>(vec, unroll);
}
const void* seg_adapt_bf16(bool comp, int vec, int unroll) {
    return comp ? pick_seg_adapt<kDtBF16, true>(vec, unroll) : pick_seg_adapt<kDtBF16, false>(vec, unroll);
}
const void* seg_adapt_fp8(bool comp, int vec, int unroll) {
    return comp ? pick_seg_adapt<kDtFP8, true>(vec, unroll) : pick_seg_adapt<kDtFP8, false>(vec, unroll);
}
}  // namespace sr
