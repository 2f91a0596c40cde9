// Segmented-sum kernels for one input dtype: the LDG form and the second
// kernel of the two-kernel finish.
#include "sr_segmented_kernels.cuh"

namespace sr {
const void* seg_ldg_fp8(bool comp, int vec, int unroll, const void** fin) {
    *fin = comp ? (const void*)seg_finish_kernel<kDtFP8, true> : (const void*)seg_finish_kernel<kDtFP8, false>;
    return comp ? pick_seg_ldg<kDtFP8, true>(vec, unroll) : pick_seg_ldg<kDtFP8, false>(vec, unroll);
}
}  // namespace sr
