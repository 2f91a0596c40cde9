// Argument block and kernel selection of the segmented sum, shared by the
// host planner (sr_segmented.cu) and the kernels (sr_segmented_kernels.cuh).
#pragma once
#include <cstdint>

#include "sr_kparams.h"

namespace sr {

constexpr int kErrBadOffsets = 4;  // the checked entry found offsets it may not read with
constexpr int kErrQueueFull = 8;   // adaptive form: chunk queue overflow (never by construction)

// Adaptive form: the chunk queue in the segmented workspace, after the
// flat split's tickets (which must stay zero between launches).
constexpr int64_t kAdaptQueueCap = 196608;       // chunk descriptors
constexpr int64_t kAdaptChunkBytes = 64 << 10;   // smallest chunk (bytes of input)

// Kernel argument block of the segmented sum (sr_segmented_kernels.cuh).
struct SegParams {
    const unsigned char* x;
    const int64_t* offsets;     // nseg + 1 entries, non-decreasing
    int64_t nseg;
    void* out;                  // nseg results
    unsigned char* carry_first; // W slots of 16 bytes (W = warps of the grid)
    unsigned char* carry_last;  // W slots of 16 bytes
    int64_t* last_seg;          // W entries: owned spanning segment or -1
    unsigned int* cnt;          // W self-resetting tickets (last-block form)
    int* err;
    float scale;
    int stage;
    int fp64;
    int stages;                 // TMA form: ring stages per warp
    uint64_t limit_ns;          // TMA form: bound of every mbarrier wait
    const int* bad;             // checked entry: nonzero = offsets invalid, read nothing (else NULL)
};

// The adaptive form's chunk queue (see sr_segmented_kernels.cuh), a second
// kernel parameter of that form only: the other segmented kernels keep their
// argument block as it is (with these fields in it the flat split's code
// generation changed and it ran 7 % slower).
struct SegQueue {
    unsigned int* ctr;          // [0] chunks queued, [1] next chunk to take, [2] warps done; zero between launches
    long long* desc;            // 2 per chunk: segment, (chunk index << 32) | chunks of the segment
    unsigned char* part;        // 16-byte partial per chunk
    unsigned int* tick;         // per segment, at its first chunk: chunks finished
    int64_t cap;                // chunk capacity
};

// Per-dtype segmented kernel selection, one function per kernel family and
// dtype (each in its own translation unit): the LDG form (which also returns
// the two-kernel form's second kernel), the dense variant, the TMA form.
const void* seg_ldg_f32(bool comp, int vec, int unroll, const void** fin);
const void* seg_dense_f32(bool comp, int vec, int unroll);
const void* seg_tma_f32(bool comp, int vec, int unroll);
const void* seg_ldg_i32(bool comp, int vec, int unroll, const void** fin);
const void* seg_dense_i32(bool comp, int vec, int unroll);
const void* seg_tma_i32(bool comp, int vec, int unroll);
const void* seg_ldg_bf16(bool comp, int vec, int unroll, const void** fin);
const void* seg_dense_bf16(bool comp, int vec, int unroll);
const void* seg_tma_bf16(bool comp, int vec, int unroll);
const void* seg_ldg_fp8(bool comp, int vec, int unroll, const void** fin);
const void* seg_dense_fp8(bool comp, int vec, int unroll);
const void* seg_tma_fp8(bool comp, int vec, int unroll);
// The warp-per-segment form, every dtype in one translation unit.
const void* seg_warp_f32(bool comp, int vec, int unroll);
const void* seg_warp_i32(bool comp, int vec, int unroll);
const void* seg_warp_bf16(bool comp, int vec, int unroll);
const void* seg_warp_fp8(bool comp, int vec, int unroll);
// The adaptive form (mixed layouts, one cooperative launch), same unit.
const void* seg_adapt_f32(bool comp, int vec, int unroll);
const void* seg_adapt_i32(bool comp, int vec, int unroll);
const void* seg_adapt_bf16(bool comp, int vec, int unroll);
const void* seg_adapt_fp8(bool comp, int vec, int unroll);
// The lane-per-segment form, in the same translation unit.
const void* seg_lane_f32(bool comp, int vec, int unroll);
const void* seg_lane_i32(bool comp, int vec, int unroll);
const void* seg_lane_bf16(bool comp, int vec, int unroll);
const void* seg_lane_fp8(bool comp, int vec, int unroll);

}  // namespace sr
