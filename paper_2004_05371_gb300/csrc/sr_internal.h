// Host-side declarations shared by the C-ABI layer and the kernel
// translation units.  Not part of the public interface (see include/sr.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/sr.h"

namespace sr {

// Workspace owned by the library, one per (device, stream) pair.
//   tickets[32]  : self-resetting arrival counters (last-block-done)
//   err          : device-side error word (bounded waits that expired, ...)
//   partials     : kMaxUnits slots of 16 bytes (one unit partial each)
//   seg          : segmented-reduction carries
constexpr int kMaxUnits = 65536;
constexpr size_t kSlotBytes = 16;
constexpr size_t kSegBytes = 8u << 20;  // also holds the adaptive form's chunk queue (sr_segparams.h)
// Segmented carries: tickets (4 B), last_seg (8 B), carry_first and
// carry_last (16 B each) per warp: 44 B x 65536 warps = 2.75 MiB <= kSegBytes.
constexpr int64_t kSegMaxWarps = 65536;
constexpr size_t kHeaderBytes = 256;

struct Workspace {
    unsigned char* base = nullptr;
    unsigned int* tickets = nullptr;
    int* err = nullptr;
    unsigned char* partials = nullptr;
    unsigned char* seg = nullptr;
    int* check = nullptr;  // result of the checked segmented entry's offsets check (header byte 160)
};

struct DeviceInfo {
    int dev = 0;
    int sms = 0;
    int max_threads_per_sm = 0;
    int max_blocks_per_sm = 0;
    int smem_per_block_optin = 0;
    int smem_per_sm = 0;
    int l2_bytes = 0;
    int cc_major = 0, cc_minor = 0;
    int clock_khz = 0;
};

// A fully resolved single-array launch.
struct Plan {
    int dtype = 0, elem = 4;
    int stage = 0, log2c = 0, cluster = 1;
    bool comp = false, fp64 = false, fp64_auto = false, bulk = false;
    int block = 0, grid = 0, units = 0;
    int vec = 16, unroll = 4;
    int tile = 0, stages = 0;
    size_t smem = 0;
    float scale = 1.f;
    // geometry of the input (filled by plan_geometry)
    int64_t n = 0, head = 0, nvec = 0, tail_begin = 0, ntail = 0;
    int64_t body_bytes = 0, ntiles = 0;
};

// A resolved segmented launch.
struct SegPlan {
    int dtype = 0;
    int64_t nseg = 0;
    int stage = 0;
    bool comp = false, fp64 = false, dense = false, bulk = false, warp = false, lane = false, adapt = false;
    int vec = 16, unroll = 4, block = 256, grid = 0;
    int stages = 0;
    size_t smem = 0;  // dynamic shared memory of the TMA form
    int64_t warps = 0;
    float scale = 1.f;
    const void* main = nullptr;
    const void* fin = nullptr;
};

// C-ABI layer services
int status_from_cuda(cudaError_t e);           // records the error, returns SR_ERR_CUDA
const DeviceInfo* current_device(int* status);  // cached per device
int get_workspace(cudaStream_t s, Workspace* ws);
void release_workspace(cudaStream_t s);  // frees the workspace of (current device, s)
void release_host_pipe(cudaStream_t s);  // frees the host-entry staging of (current device, s)
uint64_t spin_limit_ns();

// Cached per-function launch facts (one query per function and shape).
int prepare_function(const void* fn, size_t dyn_smem, bool nonportable_cluster);
int blocks_per_sm(const DeviceInfo& d, const void* fn, int block, size_t dyn_smem, int* out);
int active_clusters(const DeviceInfo& d, const void* fn, const cudaLaunchConfig_t* lc, int* out);

inline int elem_size(int dtype) { return dtype == SR_BF16 ? 2 : (dtype == SR_FP8E4M3 ? 1 : 4); }

// Zeroes `bytes` (a multiple of 4, 4-byte aligned) at device address p with a
// small kernel launched with programmatic stream serialisation, ordered after
// the stream's previous work (sr_reduce.cu).  Used where the atomic finish
// needs a zeroed output: a memset node costs several microseconds more.
int launch_zero(void* p, size_t bytes, cudaStream_t s);

// Configuration and persisted selection state (sr_persist.cu)
// The identity a device's persisted entries are keyed by: "<SMs> <driver
// version> <name>" (cached per device ordinal).
int device_identity(int dev, std::string* id);
// The autotuner fallback's memo, shared by every selected entry point.
int tune_lookup(int dev, int64_t n, int dtype, int64_t nseg, double mean, double sd, double mx, sr_config* cfg,
                bool* found);
int tune_insert(int dev, int64_t n, int dtype, int64_t nseg, double mean, double sd, double mx,
                const sr_config& cfg);
// The variant SR_VARIANT names (SR_AUTO when unset); SR_ERR_ARG when it does not parse.
int env_variant(int* variant);
// A trained selector as stored in its text file.
struct SelectorFile {
    std::string ident;  // device_identity() of the GPU it was trained on
    int din = 0, dh = 0, dout = 0;
    float mu[SR_SELECTOR_FEATURES] = {}, sd[SR_SELECTOR_FEATURES] = {};
    std::vector<sr_config> cands;
    std::vector<float> params;
};
int read_selector_file(const char* path, SelectorFile* f);  // SR_ERR_ARG: unreadable or malformed
int write_selector_file(const char* path, const SelectorFile& f);

// Single-array reduction (sr_reduce.cu)
int reduce_validate(const void* x, int64_t n, int dtype, const void* out, const sr_config& cfg);
int reduce_plan(const void* x, int64_t n, int dtype, const sr_config& cfg, const DeviceInfo& d, Plan* p);
int reduce_launch(const void* x, void* out, const Plan& p, const DeviceInfo& d, const Workspace& ws,
                  cudaStream_t s, bool skip_final = false);
// Second kernel of the two-kernel form over `units` partial slots of ws.
int reduce_launch_final(const Plan& p, int units, void* out, const Workspace& ws, cudaStream_t s);

// Segmented sum (sr_segmented.cu)
int seg_validate(const void* x, const int64_t* offsets, int64_t nseg, int dtype, const void* out,
                 const sr_config& cfg);
int seg_plan(int64_t nseg, int dtype, const sr_config& cfg, const DeviceInfo& d, SegPlan* p);
// Validates offsets (non-decreasing, offsets[0] >= 0, offsets[nseg] <= n_elems)
// on the device into ws.check and the error word; the next seg_launch with
// check = true then reads nothing when they fail.
int seg_check(const int64_t* offsets, int64_t nseg, int64_t n_elems, const Workspace& ws, cudaStream_t s);
int seg_launch(const void* x, const int64_t* offsets, void* out, const SegPlan& p, const Workspace& ws,
               cudaStream_t s, bool check = false);

}  // namespace sr
