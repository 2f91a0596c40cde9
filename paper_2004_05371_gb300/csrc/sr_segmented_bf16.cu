// Segmented-sum kernels for one input dtype: the LDG form and the second
// kernel of the two-kernel finish.
#include "sr_segmented_kernels.cuh"

namespace sr {
const void* seg_ldg_bf16(bool comp, int vec, int unroll, const void** fin) {
    *fin = comp ? (const void*)seg_finish_kernel<kDtBF16, true> : (const void*)seg_finish_kernel<kDtBF16, false>;
    return comp ? pick_seg_ldg<kDtBF16, true>(vec, unroll) : pick_seg_ldg<kDtBF16, false>(vec, unroll);
}
}  // namespace sr
