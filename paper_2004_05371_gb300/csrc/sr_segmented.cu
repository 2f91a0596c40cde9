// Segmented sum: validation, launch planning and launch (C ABI in sr_api.cu).
#include <algorithm>
#include <cstring>

#include "sr_device.cuh"
#include "sr_internal.h"
#include "sr_kparams.h"
#include "sr_segparams.h"

namespace sr {

namespace {

// Checked entry: every offset must be >= its predecessor (offsets[0] >= 0)
// and offsets[nseg] <= n_elems; a violation sets *bad (zeroed just before on
// the same stream) and the stream's error word.
__global__ void __launch_bounds__(256) seg_check_kernel(const int64_t* offsets, int64_t nseg, int64_t n_elems,
                                                        int* bad, int* err) {
    grid_dependency_wait();
    allow_dependents();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= nseg; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = offsets[i];
        const bool ok = (i == 0 ? a >= 0 : a >= offsets[i - 1]) && (i < nseg || a <= n_elems);
        if (!ok) {
            atomicOr(bad, 1);
            atomicOr(err, kErrBadOffsets);
        }
    }
}
constexpr int kKnownSegFlags =
    SR_STAGE_MASK | SR_F_KAHAN | SR_F_FP64_COMBINE | SR_F_DENSE_SEGMENTS | SR_F_BULK | SR_F_WARP_SEGMENTS |
    SR_F_LANE_SEGMENTS | SR_F_ADAPTIVE_SEGMENTS;
// the load-path / form flags, at most one of which a segmented call may set
constexpr int kSegFormFlags =
    SR_F_DENSE_SEGMENTS | SR_F_BULK | SR_F_WARP_SEGMENTS | SR_F_LANE_SEGMENTS | SR_F_ADAPTIVE_SEGMENTS;
constexpr int64_t kSegBulkMin = 32768;  // segments from which the default shape is the TMA form

const void* seg_adapt_kernel(int dtype, bool comp, int vec, int unroll) {
    switch (dtype) {
    case SR_F32: return seg_adapt_f32(comp, vec, unroll);
    case SR_I32: return seg_adapt_i32(comp, vec, unroll);
    case SR_BF16: return seg_adapt_bf16(comp, vec, unroll);
    case SR_FP8E4M3: return seg_adapt_fp8(comp, vec, unroll);
    default: return nullptr;
    }
}

bool seg_kernels(int dtype, bool comp, int vec, int unroll, bool dense, bool bulk, bool warp, bool lane,
                 const void** main, const void** fin) {
    const void* (*ldg)(bool, int, int, const void**) = nullptr;
    const void* (*den)(bool, int, int) = nullptr;
    const void* (*tma)(bool, int, int) = nullptr;
    const void* (*wrp)(bool, int, int) = nullptr;
    const void* (*lan)(bool, int, int) = nullptr;
    switch (dtype) {
    case SR_F32: ldg = seg_ldg_f32; den = seg_dense_f32; tma = seg_tma_f32; wrp = seg_warp_f32; lan = seg_lane_f32; break;
    case SR_I32: ldg = seg_ldg_i32; den = seg_dense_i32; tma = seg_tma_i32; wrp = seg_warp_i32; lan = seg_lane_i32; break;
    case SR_BF16:
        ldg = seg_ldg_bf16; den = seg_dense_bf16; tma = seg_tma_bf16; wrp = seg_warp_bf16; lan = seg_lane_bf16;
        break;
    case SR_FP8E4M3:
        ldg = seg_ldg_fp8; den = seg_dense_fp8; tma = seg_tma_fp8; wrp = seg_warp_fp8; lan = seg_lane_fp8;
        break;
    default: return false;
    }
    if (warp || lane) {  // one kernel, nothing to finish
        *fin = nullptr;
        *main = (dense || bulk || (warp && lane)) ? nullptr : (warp ? wrp(comp, vec, unroll) : lan(comp, vec, unroll));
        return *main != nullptr;
    }
    const void* plain = ldg(comp, vec, unroll, fin);  // also sets the second kernel
    if (bulk) *main = dense ? nullptr : tma(comp, vec, unroll);
    else *main = dense ? den(comp, vec, unroll) : plain;
    return *main != nullptr;
}
}  // namespace

int seg_validate(const void* x, const int64_t* offsets, int64_t nseg, int dtype, const void* out,
                 const sr_config& c) {
    if (dtype < SR_F32 || dtype > SR_FP8E4M3) return SR_ERR_DTYPE;
    if (nseg < 0) return SR_ERR_ARG;
    if (nseg > 0 && (x == nullptr || offsets == nullptr || out == nullptr)) return SR_ERR_ARG;
    if (x && reinterpret_cast<uintptr_t>(x) % elem_size(dtype)) return SR_ERR_ARG;
    if (offsets && reinterpret_cast<uintptr_t>(offsets) % 8) return SR_ERR_ARG;
    const bool fp64 = (c.variant & SR_F_FP64_COMBINE) && dtype != SR_I32;
    if (out && reinterpret_cast<uintptr_t>(out) % ((dtype == SR_I32 || fp64) ? 8 : 4)) return SR_ERR_ARG;
    if (c.variant & ~kKnownSegFlags)
        return (c.variant & (SR_CLUSTER_MASK | SR_F_FP64_AUTO)) ? SR_ERR_UNSUPPORTED : SR_ERR_ARG;
    const int forms = c.variant & kSegFormFlags;
    if (forms & (forms - 1)) return SR_ERR_UNSUPPORTED;  // two forms at once
    if ((c.variant & SR_F_BULK) && (c.unroll == 1)) return SR_ERR_ARG;  // chunks of 2, 4 or 8 rows
    if (c.stages != 0 && (c.stages < 2 || c.stages > 8)) return SR_ERR_ARG;
    const int stage = c.variant & SR_STAGE_MASK;
    if (stage > SR_SINGLE_CLUSTER) return SR_ERR_ARG;
    if (stage == SR_SINGLE_CLUSTER) return SR_ERR_UNSUPPORTED;
    if (c.block_threads != 0 && (c.block_threads < 32 || c.block_threads > 512 || c.block_threads % 32))
        return SR_ERR_ARG;
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 32) return SR_ERR_ARG;
    if (c.grid < 0) return SR_ERR_ARG;
    if (c.vec_bytes != 0 && c.vec_bytes != 16 && c.vec_bytes != 32) return SR_ERR_ARG;
    if (c.unroll != 0 && c.unroll != 1 && c.unroll != 2 && c.unroll != 4 && c.unroll != 8) return SR_ERR_ARG;
    if (!(c.scale == c.scale) || c.scale < 0.f) return SR_ERR_ARG;
    const int block = c.block_threads ? c.block_threads : 256;
    if ((int64_t)c.grid * (block / 32) > kSegMaxWarps) return SR_ERR_ARG;
    return SR_OK;
}

int seg_plan(int64_t nseg, int dtype, const sr_config& c, const DeviceInfo& d, SegPlan* out) {
    SegPlan p;
    p.dtype = dtype;
    p.nseg = nseg;
    p.comp = (c.variant & SR_F_KAHAN) && dtype != SR_I32;
    p.fp64 = (c.variant & SR_F_FP64_COMBINE) && dtype != SR_I32;
    p.stage = c.variant & SR_STAGE_MASK;
    // SR_AUTO: last-block-done; for int32 the atomic finish (int64 sums are
    // exact in any order, so it stays deterministic, and it is 2-3 % faster:
    // no ticket, no second read of the carries)
    if (p.stage == SR_AUTO) p.stage = dtype == SR_I32 ? SR_ATOMIC : SR_LAST_BLOCK;
    // defaults from autotuner sweeps of 10,000 lognormal segments (~2^28 FP32):
    // 32-byte vectors, 8 rows in flight per warp, 256-thread CTAs
    p.vec = c.vec_bytes ? c.vec_bytes : 32;
    p.unroll = c.unroll ? c.unroll : 8;
    p.block = c.block_threads ? c.block_threads : 256;
    p.scale = (dtype == SR_FP8E4M3 && c.scale != 0.f) ? c.scale : 1.f;
    p.dense = (c.variant & SR_F_DENSE_SEGMENTS) != 0;
    p.warp = (c.variant & SR_F_WARP_SEGMENTS) != 0;
    p.lane = (c.variant & SR_F_LANE_SEGMENTS) != 0;
    if (p.lane) {  // 16-byte vectors, 4 per step
        p.vec = c.vec_bytes ? c.vec_bytes : 16;
        p.unroll = c.unroll ? c.unroll : 4;
    }
    if (p.warp) {  // 16-byte vectors, 2 per lane and segment (64 registers: 32 warps per SM)
        p.vec = c.vec_bytes ? c.vec_bytes : 16;
        p.unroll = c.unroll ? c.unroll : 2;
    }
    p.adapt = (c.variant & SR_F_ADAPTIVE_SEGMENTS) != 0;
    if (p.adapt) {
        // one cooperative launch of the resident number of 256-thread CTAs;
        // phase 1 at the warp form's shape (16-byte vectors, 2 per lane)
        if ((c.vec_bytes && c.vec_bytes != 16) || (c.unroll && c.unroll != 2) ||
            (c.block_threads && c.block_threads != 256))
            return SR_ERR_UNSUPPORTED;
        p.vec = 16;
        p.unroll = 2;
        p.block = 256;
        p.main = seg_adapt_kernel(dtype, p.comp, p.vec, p.unroll);
        p.fin = nullptr;
        if (!p.main) return SR_ERR_UNSUPPORTED;
        int st = prepare_function(p.main, 0, false);
        if (st != SR_OK) return st;
        int resident = 0;
        st = blocks_per_sm(d, p.main, p.block, 0, &resident);
        if (st != SR_OK) return st;
        if (resident < 1) return SR_ERR_LAUNCH;
        int64_t grid = c.grid ? c.grid : (int64_t)resident * d.sms;
        if (grid > (int64_t)resident * d.sms) return SR_ERR_LAUNCH;  // could not be co-resident
        p.grid = (int)std::max<int64_t>(1, grid);
        p.warps = (int64_t)p.grid * (p.block / 32);
        *out = p;
        return SR_OK;
    }
    if (p.dense) {  // the dense kernel runs at most 4 rows in flight; 512-thread CTAs by default
        if (p.unroll > 4) p.unroll = 4;
        if (!c.block_threads) p.block = 512;
    }
    // Without an explicit shape, many segments (kSegBulkMin or more) take the TMA
    // form: measured 1.02-1.41x the LDG default from 100,000 to 16M segments of
    // ~2^28 elements, 1 % behind it at 10,000.
    const bool shape_given = c.vec_bytes || c.unroll || c.block_threads || c.stages;
    p.bulk = (c.variant & SR_F_BULK) != 0 || (!shape_given && !p.dense && !p.warp && !p.lane && nseg >= kSegBulkMin);
    if (p.bulk) {  // per-warp ring: stages x (unroll rows of 32 vectors) + one mbarrier per stage
        if (!c.unroll) p.unroll = 4;
        p.stages = c.stages ? c.stages : 2;
        p.smem = (size_t)(p.block / 32) * p.stages * ((size_t)p.unroll * 32 * p.vec + 8);
        if (p.smem > (size_t)d.smem_per_block_optin) return SR_ERR_LAUNCH;
    }
    if (!seg_kernels(dtype, p.comp, p.vec, p.unroll, p.dense, p.bulk, p.warp, p.lane, &p.main, &p.fin))
        return SR_ERR_UNSUPPORTED;
    int st = prepare_function(p.main, p.smem, false);
    if (st != SR_OK) return st;
    int resident = 0;
    st = blocks_per_sm(d, p.main, p.block, p.smem, &resident);
    if (st != SR_OK) return st;
    if (resident < 1) return SR_ERR_LAUNCH;
    int per_sm = c.ctas_per_sm ? std::min(c.ctas_per_sm, resident) : resident;
    int64_t grid = c.grid ? c.grid : (int64_t)d.sms * per_sm;
    grid = std::min<int64_t>(grid, kSegMaxWarps / (p.block / 32));
    if (p.stage == SR_GRID_SYNC && !p.warp && !p.lane && grid > (int64_t)resident * d.sms) {
        if (c.grid) return SR_ERR_LAUNCH;  // cannot be co-resident: never launched
        grid = (int64_t)resident * d.sms;
    }
    p.grid = (int)std::max<int64_t>(1, grid);
    p.warps = (int64_t)p.grid * (p.block / 32);
    *out = p;
    return SR_OK;
}

int seg_check(const int64_t* offsets, int64_t nseg, int64_t n_elems, const Workspace& ws, cudaStream_t s) {
    int st = launch_zero(ws.check, sizeof(int), s);
    if (st != SR_OK) return st;
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc;
    std::memset(&lc, 0, sizeof lc);
    lc.gridDim = dim3((unsigned)std::min<int64_t>((nseg + 256) / 256, 1024));
    lc.blockDim = dim3(256);
    lc.stream = s;
    lc.attrs = pdl;
    lc.numAttrs = 1;
    int* bad = ws.check;
    int* err = ws.err;
    void* args[] = {const_cast<int64_t**>(&offsets), &nseg, &n_elems, &bad, &err};
    cudaError_t e = cudaLaunchKernelExC(&lc, (const void*)seg_check_kernel, args);
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

int seg_launch(const void* x, const int64_t* offsets, void* out, const SegPlan& p, const Workspace& ws,
               cudaStream_t s, bool check) {
    SegParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.x = static_cast<const unsigned char*>(x);
    kp.offsets = offsets;
    kp.nseg = p.nseg;
    kp.out = out;
    kp.cnt = reinterpret_cast<unsigned int*>(ws.seg);
    kp.last_seg = reinterpret_cast<int64_t*>(ws.seg + (size_t)kSegMaxWarps * 4);
    kp.carry_first = ws.seg + (size_t)kSegMaxWarps * 12;
    kp.carry_last = ws.seg + (size_t)kSegMaxWarps * 28;
    kp.err = ws.err;
    kp.scale = p.scale;
    kp.stages = p.stages;
    kp.limit_ns = spin_limit_ns();
    kp.bad = check ? ws.check : nullptr;
    kp.stage = p.stage;
    kp.fp64 = p.fp64 ? 1 : 0;
    cudaError_t e;
    if (p.adapt) {
        // the chunk queue: counters at the head of the tickets (the last warp
        // of each launch resets them to zero), arrays after the tickets
        SegQueue kq;
        kq.ctr = reinterpret_cast<unsigned int*>(ws.seg);
        unsigned char* q = ws.seg + (size_t)kSegMaxWarps * 4;
        kq.desc = reinterpret_cast<long long*>(q);
        kq.part = q + (size_t)kAdaptQueueCap * 16;
        kq.tick = reinterpret_cast<unsigned int*>(q + (size_t)kAdaptQueueCap * 32);
        kq.cap = kAdaptQueueCap;
        void* aargs[] = {&kp, &kq};
        e = cudaLaunchCooperativeKernel(p.main, dim3(p.grid), dim3(p.block), aargs, 0, s);
        return e == cudaSuccess ? SR_OK : status_from_cuda(e);
    }
    if (p.stage == SR_ATOMIC && !p.warp && !p.lane) {
        const size_t ob = (p.dtype == SR_I32 || p.fp64) ? 8 : 4;
        const int zs = launch_zero(out, ob * (size_t)p.nseg, s);
        if (zs != SR_OK) return zs;
    }
    void* args[] = {&kp};
    // programmatic stream serialisation, as for the single-array kernels: a
    // kernel may be scheduled while its predecessor drains and waits for it
    // in grid_dependency_wait() before touching global memory
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc;
    std::memset(&lc, 0, sizeof lc);
    lc.stream = s;
    lc.attrs = pdl;
    lc.numAttrs = 1;
    if (p.stage == SR_GRID_SYNC && !p.warp && !p.lane) {
        e = cudaLaunchCooperativeKernel(p.main, dim3(p.grid), dim3(p.block), args, p.smem, s);
    } else {
        lc.gridDim = dim3(p.grid);
        lc.blockDim = dim3(p.block);
        lc.dynamicSmemBytes = p.smem;
        e = cudaLaunchKernelExC(&lc, p.main, args);
        lc.dynamicSmemBytes = 0;
    }
    if (e != cudaSuccess) return status_from_cuda(e);
    if (p.stage == SR_TWO_KERNEL && !p.warp && !p.lane) {
        int64_t wn = p.warps;
        int pv = p.vec / elem_size(p.dtype);
        void* fargs[] = {&kp, &wn, &pv};
        lc.gridDim = dim3((unsigned)((p.warps * 32 + 255) / 256));
        lc.blockDim = dim3(256);
        e = cudaLaunchKernelExC(&lc, p.fin, fargs);
        if (e != cudaSuccess) return status_from_cuda(e);
    }
    return SR_OK;
}

}  // namespace sr
