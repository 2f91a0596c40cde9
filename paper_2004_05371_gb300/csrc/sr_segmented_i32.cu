// Segmented-sum kernels for one input dtype: the LDG form and the second
// kernel of the two-kernel finish.  Integer sums are exact: no compensated form.
#include "sr_segmented_kernels.cuh"

namespace sr {
const void* seg_ldg_i32(bool comp, int vec, int unroll, const void** fin) {
    (void)comp;
    *fin = (const void*)seg_finish_kernel<kDtI32, false>;
    return pick_seg_ldg<kDtI32, false>(vec, unroll);
}
}  // namespace sr
