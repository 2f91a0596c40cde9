// Kernel argument block of the single-array reduction (host and device).
#pragma once
#include <cstdint>

namespace sr {

// Bits of the device error word.
constexpr int kErrTimeout = 1;         // a bounded wait expired
constexpr int kErrNotCooperative = 2;  // grid.sync kernel launched non-cooperatively

struct KParams {
    const unsigned char* x;   // input base (element-aligned)
    int64_t n;                // elements
    int64_t head;             // scalar elements before the aligned vector body
    int64_t nvec;             // vectors in the body (vec bytes each)
    int64_t tail_begin;       // first element after the body
    int64_t ntail;            // scalar elements after the body
    void* out;                // result (int64 / float / double)
    unsigned char* partials;  // unit partial slots (16 bytes each)
    unsigned int* ticket;     // last-block-done counter (self-resetting)
    int* err;                 // device error word
    float scale;              // applied once to the final float result
    int stage;                // grid stage (sr_stage)
    int fp64;                 // combine unit partials in binary64
    int fp64_auto;            // compensated partials: binary64 combine only when needed
    int units;                // number of units (= grid / cluster)
    int log2c;                // cluster size = 1 << log2c
    int tile_bytes;           // bulk path: bytes per stage
    int stages;               // bulk path: ring depth
    int64_t body_bytes;       // bulk path: nvec * 16
    int64_t ntiles;           // bulk path: ceil(body_bytes / tile_bytes)
    uint64_t limit_ns;        // bound on every device-side wait
};

struct KernelSet {
    const void* main = nullptr;   // thread..grid stages
    const void* final = nullptr;  // second kernel of the two-kernel form
};

// Per-dtype kernel selection (one translation unit per dtype).
bool kernels_f32(bool comp, bool fp64, bool bulk, int vec, int unroll, KernelSet* k);
bool kernels_i32(bool comp, bool fp64, bool bulk, int vec, int unroll, KernelSet* k);
bool kernels_bf16(bool comp, bool fp64, bool bulk, int vec, int unroll, KernelSet* k);
bool kernels_fp8(bool comp, bool fp64, bool bulk, int vec, int unroll, KernelSet* k);

}  // namespace sr
