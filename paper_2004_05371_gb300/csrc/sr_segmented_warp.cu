// Segmented-sum kernels of every input dtype: the warp-per-segment form
// (SR_F_WARP_SEGMENTS) and the lane-per-segment form (SR_F_LANE_SEGMENTS).
#include "sr_segmented_kernels.cuh"

namespace sr {
const void* seg_warp_f32(bool comp, int vec, int unroll) {
    return comp ? pick_seg_warp<kDtF32, true>(vec, unroll) : pick_seg_warp<kDtF32, false>(vec, unroll);
}
const void* seg_warp_i32(bool comp, int vec, int unroll) {
    (void)comp;  // integer sums are exact
    return pick_seg_warp<kDtI32, false>(vec, unroll);
}
const void* seg_warp_bf16(bool comp, int vec, int unroll) {
    return comp ? pick_seg_warp<kDtBF16, true>(vec, unroll) : pick_seg_warp<kDtBF16, false>(vec, unroll);
}
const void* seg_warp_fp8(bool comp, int vec, int unroll) {
    return comp ? pick_seg_warp<kDtFP8, true>(vec, unroll) : pick_seg_warp<kDtFP8, false>(vec, unroll);
}
const void* seg_lane_f32(bool comp, int vec, int unroll) {
    return comp ? pick_seg_lane<kDtF32, true>(vec, unroll) : pick_seg_lane<kDtF32, false>(vec, unroll);
}
const void* seg_lane_i32(bool comp, int vec, int unroll) {
    (void)comp;  // integer sums are exact
    return pick_seg_lane<kDtI32, false>(vec, unroll);
}
const void* seg_lane_bf16(bool comp, int vec, int unroll) {
    return comp ? pick_seg_lane<kDtBF16, true>(vec, unroll) : pick_seg_lane<kDtBF16, false>(vec, unroll);
}
const void* seg_lane_fp8(bool comp, int vec, int unroll) {
    return comp ? pick_seg_lane<kDtFP8, true>(vec, unroll) : pick_seg_lane<kDtFP8, false>(vec, unroll);
}
}  // namespace sr
