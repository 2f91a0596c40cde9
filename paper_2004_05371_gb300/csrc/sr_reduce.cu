// Single-array reduction: argument validation, launch planning and launch.
#include <algorithm>
#include <cstring>

#include "sr_device.cuh"
#include "sr_internal.h"
#include "sr_kparams.h"

namespace sr {

namespace {

// The output of an atomic finish starts at zero: this kernel writes it.  It
// waits for the stream's previous kernel like every kernel of the library,
// and lets the reduction kernel after it be scheduled at once.
__global__ void __launch_bounds__(256) zero_words_kernel(uint32_t* p, int64_t nwords) {
    grid_dependency_wait();
    allow_dependents();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0u;
}


constexpr int kKnownFlags = SR_STAGE_MASK | SR_CLUSTER_MASK | SR_F_KAHAN | SR_F_FP64_COMBINE | SR_F_BULK |
                            SR_F_HOST_DIRECT | SR_F_FP64_AUTO;
// SR_AUTO's launch shapes, from graph-timed size sweeps and autotuner sweeps
// on a GB300 (device time per call in a CUDA graph, FP32):
//   <= 32 KiB : one CTA, one 16 B x 2 batch per thread, no grid stage
//               (1.26 us at 4 KiB, 1.40 at 16 KiB)
//   <= 1 MiB  : a cluster of up to 16 CTAs of at least 256 threads, one
//               batch per thread, DSMEM merge, no grid stage (1.74 us at
//               64 KiB, 1.96 at 256 KiB, 2.47 at 1 MiB with four loads)
//   <= 64 MiB : two-kernel form, grid sized by the work, 32 B loads (2.9 us at
//               4 MiB, 3.5 at 16 MiB, 6.4 at 64 MiB with the input in L2)
//   larger    : per dtype, below: the two-kernel form with 16 B loads up to
//               512 MiB, then last-block-done on the TMA ring (HBM-bound)
// Every launch carries the programmatic-stream-serialisation attribute, so
// the second kernel of the two-kernel form, and the next call's kernel, are
// scheduled while their predecessor drains.
struct AutoShape {
    int stage, block, vec, unroll;
    bool bulk;
    int tile, stages;
};
constexpr int64_t kAutoClusterBytes = 1 << 20;
constexpr int64_t kAutoTwoKernelBytes = 64 << 20;
constexpr int64_t kAutoLdgBytes = 512 << 20;

// Above 64 MiB, per dtype, from warm (input streaming from HBM) and cold (L2
// full of another kernel's dirty lines) sweeps.  Up to 512 MiB the
// two-kernel form with 16-byte loads and one to four steps in flight per
// thread; beyond, the TMA ring, as fast as the best LDG shape when streaming
// and 5-13 % faster when L2 holds dirty lines.  The plain FP32 and FP8 rings
// are 64 KiB tiles with eight consumer warps (16 chunks per lane per tile,
// one block of the blocked thread stage): FP32 1 GiB 148.5 us warm / 164.6
// cold, FP8 1 GiB 149.5 / 169.0 (the FP8 LDG form: 161.1 / 167.7).
AutoShape auto_large_shape(int dtype, bool comp, int64_t bytes, bool allow_bulk) {
    const bool ldg = bytes <= kAutoLdgBytes || !allow_bulk;
    if (comp) {
        if (dtype == SR_F32)
            return ldg ? AutoShape{SR_TWO_KERNEL, 1024, 16, 1, false, 0, 0}
                       : AutoShape{SR_LAST_BLOCK, 544, 16, 4, true, 32 << 10, 4};
        if (dtype == SR_BF16)  // packed TwoSum: two loads in flight keep pace up to 1 GiB
            return ldg || bytes <= ((int64_t)1 << 30) ? AutoShape{SR_TWO_KERNEL, 1024, 16, 2, false, 0, 0}
                                                      : AutoShape{SR_LAST_BLOCK, 544, 16, 4, true, 64 << 10, 3};
        // FP8: a vector's 16 values sum exactly, one TwoSum per vector
        return ldg ? AutoShape{SR_TWO_KERNEL, 1024, 16, 1, false, 0, 0}
                   : AutoShape{SR_LAST_BLOCK, 544, 16, 1, true, 64 << 10, 3};
    }
    if (dtype == SR_BF16)
        return ldg ? AutoShape{SR_TWO_KERNEL, 512, 16, 2, false, 0, 0}
                   : AutoShape{SR_LAST_BLOCK, 544, 16, 1, true, 64 << 10, 2};
    if (dtype == SR_FP8E4M3)  // a vector's 16 values sum exactly: one addition per vector
        return ldg ? AutoShape{SR_TWO_KERNEL, 512, 16, 4, false, 0, 0}
                   : AutoShape{SR_LAST_BLOCK, 288, 16, 1, true, 64 << 10, 3};
    if (dtype == SR_F32)  // blocked thread stage: one block of 16 chunks per lane per 64 KiB tile
        return ldg ? AutoShape{SR_TWO_KERNEL, 512, 16, 1, false, 0, 0}
                   : AutoShape{SR_LAST_BLOCK, 288, 16, 1, true, 64 << 10, 2};
    return ldg ? AutoShape{SR_TWO_KERNEL, 512, 16, 1, false, 0, 0}  // int32
               : AutoShape{SR_LAST_BLOCK, 160, 16, 1, true, 32 << 10, 4};
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

bool kernels_for(const Plan& p, KernelSet* k) {
    switch (p.dtype) {
    case SR_F32: return kernels_f32(p.comp, p.fp64, p.bulk, p.vec, p.unroll, k);
    case SR_I32: return kernels_i32(p.comp, p.fp64, p.bulk, p.vec, p.unroll, k);
    case SR_BF16: return kernels_bf16(p.comp, p.fp64, p.bulk, p.vec, p.unroll, k);
    case SR_FP8E4M3: return kernels_fp8(p.comp, p.fp64, p.bulk, p.vec, p.unroll, k);
    default: return false;
    }
}

}  // namespace

int reduce_validate(const void* x, int64_t n, int dtype, const void* out, const sr_config& c) {
    if (dtype < SR_F32 || dtype > SR_FP8E4M3) return SR_ERR_DTYPE;
    if (n < 0 || out == nullptr || (n > 0 && x == nullptr)) return SR_ERR_ARG;
    const int es = elem_size(dtype);
    if (x != nullptr && (reinterpret_cast<uintptr_t>(x) % es) != 0) return SR_ERR_ARG;
    const bool fp64 = (c.variant & SR_F_FP64_COMBINE) && dtype != SR_I32;
    const size_t out_align = (dtype == SR_I32 || fp64) ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(out) % out_align) return SR_ERR_ARG;
    if (c.variant & ~kKnownFlags) return SR_ERR_ARG;
    const int stage = c.variant & SR_STAGE_MASK;
    const int log2c = (c.variant & SR_CLUSTER_MASK) >> SR_CLUSTER_SHIFT;
    if (stage > SR_SINGLE_CLUSTER || log2c > 4) return SR_ERR_ARG;
    if (c.block_threads != 0 && (c.block_threads < 32 || c.block_threads > 1024 || c.block_threads % 32))
        return SR_ERR_ARG;
    if ((c.variant & SR_F_BULK) && c.block_threads != 0 && c.block_threads < 64) return SR_ERR_ARG;
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 32) return SR_ERR_ARG;
    if (c.grid < 0 || c.grid > kMaxUnits) return SR_ERR_ARG;
    if (c.vec_bytes != 0 && c.vec_bytes != 16 && c.vec_bytes != 32) return SR_ERR_ARG;
    if (c.unroll != 0 && c.unroll != 1 && c.unroll != 2 && c.unroll != 4 && c.unroll != 8) return SR_ERR_ARG;
    if (c.tile_bytes != 0 && (c.tile_bytes < 1024 || c.tile_bytes % 1024 || c.tile_bytes > (224 << 10)))
        return SR_ERR_ARG;
    if (c.stages != 0 && (c.stages < 2 || c.stages > 8)) return SR_ERR_ARG;
    if (!(c.scale == c.scale) || c.scale < 0.f) return SR_ERR_ARG;  // NaN or negative
    if (stage == SR_GRID_SYNC && log2c > 0) return SR_ERR_UNSUPPORTED;
    return SR_OK;
}

int reduce_plan(const void* x, int64_t n, int dtype, const sr_config& c, const DeviceInfo& d, Plan* out) {
    Plan p;
    p.dtype = dtype;
    p.elem = elem_size(dtype);
    p.n = n;
    p.comp = (c.variant & (SR_F_KAHAN | SR_F_FP64_AUTO)) && dtype != SR_I32;
    p.fp64 = (c.variant & SR_F_FP64_COMBINE) && dtype != SR_I32;
    p.fp64_auto = (c.variant & SR_F_FP64_AUTO) && dtype != SR_I32 && !p.fp64;
    p.bulk = (c.variant & SR_F_BULK) != 0;
    p.scale = (dtype == SR_FP8E4M3 && c.scale != 0.f) ? c.scale : 1.f;
    p.stage = c.variant & SR_STAGE_MASK;
    p.log2c = (c.variant & SR_CLUSTER_MASK) >> SR_CLUSTER_SHIFT;

    int def_block = 512, def_vec = 16, def_unroll = 4, def_tile = 32 << 10, def_stages = 6;
    if (p.stage == SR_AUTO) {
        const int64_t bytes = n * p.elem;
        const bool chosen_cluster = p.log2c != 0;
        if (bytes <= kAutoClusterBytes) {
            // one 16 B x 2 batch (32 bytes) per thread: one CTA of up to 1024
            // threads, then a cluster of up to 16 CTAs of at least 256
            // threads, then four loads per thread (warm / cold graph sweeps
            // of every shape, 2^10..2^18 FP32)
            p.stage = SR_SINGLE_CLUSTER;
            def_vec = 16;
            def_unroll = 2;
            const int64_t threads = std::max<int64_t>(32, cdiv(bytes, 32));
            int log2c = 0;
            if (threads > 1024) {
                while (log2c < 4 && ((int64_t)256 << (log2c + 1)) <= threads) ++log2c;
            }
            if (chosen_cluster) log2c = p.log2c;
            else p.log2c = log2c;
            int64_t per_cta = cdiv(threads, (int64_t)1 << log2c);
            if (per_cta > 1024) {
                def_unroll = 4;
                per_cta = cdiv(per_cta, 2);
            }
            def_block = (int)std::min<int64_t>(1024, cdiv(per_cta, 32) * 32);
        } else if (bytes <= kAutoTwoKernelBytes) {
            p.stage = SR_TWO_KERNEL;
            if (!p.comp) {
                // 256-bit loads: inputs of this size are often still in L2,
                // where wider requests double the throughput (FP8, whose
                // decode sets the pace, keeps two in flight); below 4 MiB
                // 16 KiB per CTA, so the work-sized grid spans every SM: 256
                // threads x 32 B x 2, or for BF16 / FP8 (twice the threads to
                // decode) 512 x 16 B x 2 (2 MiB: 2.6-2.8 us against 3.1-3.4
                // with 512 x 32 B x 2)
                def_vec = 32;
                def_unroll = bytes >= (16 << 20) && dtype != SR_FP8E4M3 ? 8 : 2;
                if (bytes < (4 << 20)) {
                    const bool narrow = dtype == SR_BF16 || dtype == SR_FP8E4M3;
                    def_block = narrow ? 512 : 256;
                    def_vec = narrow ? 16 : 32;
                }
                if (dtype == SR_I32) {
                    // int64 sums are exact in any order, so the one-kernel
                    // atomic finish stays deterministic: 256 x 32 B x 4 (x 8
                    // from 32 MiB), 5-15 % ahead of the two-kernel form from
                    // 4 MiB (4 MiB 2.85 / 4.19 us warm / cold against 3.25 /
                    // 4.53); below 4 MiB the two-kernel form, 256 x 16 B x 4 (16 KiB
                    // per CTA: 2 MiB 2.65 us against 2.98 with 32-byte loads)
                    def_block = 256;
                    def_unroll = bytes >= (32 << 20) ? 8 : 4;
                    if (bytes >= (4 << 20)) p.stage = SR_ATOMIC;
                    else def_vec = 16;
                }
            } else {
                // compensated: 256-bit loads as well; 256 x 2 per thread below
                // 8 MiB (the work-sized grid then spans more SMs), 1024 x 4 up
                // to 32 MiB, 1024 x 8 (FP8 x 4) above (warm + cold graph sweeps
                // at 2, 16 and 64 MiB per dtype: 16-byte loads were 10-45 %
                // behind warm, e.g. 64 MiB FP32 15.5 us against 8.6)
                def_vec = 32;
                if (bytes < (8 << 20)) {
                    def_block = 256;
                    def_unroll = 2;
                } else {
                    def_block = 1024;
                    def_unroll = bytes < (32 << 20) ? 4 : (dtype == SR_FP8E4M3 ? 4 : 8);
                }
            }
        } else {
            p.stage = SR_LAST_BLOCK;
            if (!p.bulk && !chosen_cluster) {
                // explicit vector width or unroll ask for the LDG path
                const AutoShape a = auto_large_shape(dtype, p.comp, bytes, !c.vec_bytes && !c.unroll);
                p.stage = a.stage;
                p.bulk = a.bulk;
                def_block = a.block;
                def_vec = a.vec;
                def_unroll = a.unroll;
                if (a.bulk) {
                    def_tile = a.tile;
                    def_stages = a.stages;
                }
            }
        }
    }
    p.cluster = 1 << p.log2c;

    p.vec = p.bulk ? 16 : (c.vec_bytes ? c.vec_bytes : def_vec);
    p.unroll = c.unroll ? c.unroll : def_unroll;
    p.block = c.block_threads ? c.block_threads : (p.bulk ? (def_block == 512 ? 288 : def_block) : def_block);

    // geometry: scalar head up to the vector alignment, vector body, scalar tail
    const int64_t per_vec = p.vec / p.elem;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(x);
    const int64_t mis = (int64_t)(addr % (uintptr_t)p.vec);
    p.head = mis ? std::min<int64_t>(n, (p.vec - mis) / p.elem) : 0;
    p.nvec = (n - p.head) / per_vec;
    p.tail_begin = p.head + p.nvec * per_vec;
    p.ntail = n - p.tail_begin;

    int ctas_per_sm;
    int64_t work_ctas;
    if (p.bulk) {
        p.tile = c.tile_bytes ? c.tile_bytes : def_tile;
        p.stages = c.stages ? c.stages : def_stages;
        p.smem = (size_t)p.stages * p.tile + 16 * (size_t)p.stages;
        if (p.smem > (size_t)d.smem_per_block_optin) return SR_ERR_LAUNCH;
        p.body_bytes = p.nvec * 16;
        p.ntiles = cdiv(p.body_bytes, p.tile);
        const int fit = std::max(1, (int)(d.smem_per_sm / (p.smem + 2048)));
        ctas_per_sm = c.ctas_per_sm ? c.ctas_per_sm : std::min(fit, d.max_threads_per_sm / p.block);
        work_ctas = std::max<int64_t>(p.ntiles, 1);
        // the scalar head/tail are spread over consumer threads of all CTAs
    } else {
        ctas_per_sm = c.ctas_per_sm ? c.ctas_per_sm : std::max(1, d.max_threads_per_sm / p.block);
        work_ctas = std::max<int64_t>(1, cdiv(p.nvec, (int64_t)p.block * p.unroll));
    }
    if (!c.ctas_per_sm) {
        // default: as many CTAs per SM as are resident at once (registers and
        // shared memory of this kernel), so the grid is exactly one wave
        KernelSet ks;
        if (!kernels_for(p, &ks)) return SR_ERR_UNSUPPORTED;
        int st = prepare_function(ks.main, p.smem, p.cluster > 8);
        if (st != SR_OK) return st;
        int resident = 0;
        st = blocks_per_sm(d, ks.main, p.block, p.smem, &resident);
        if (st != SR_OK) return st;
        if (resident < 1) return SR_ERR_LAUNCH;
        ctas_per_sm = std::min(ctas_per_sm, resident);
    }
    ctas_per_sm = std::max(1, std::min(ctas_per_sm, d.max_blocks_per_sm));

    int64_t grid;
    if (p.stage == SR_SINGLE_CLUSTER) {
        grid = p.cluster;
    } else if (c.grid) {
        grid = c.grid;
    } else {
        grid = std::min<int64_t>((int64_t)d.sms * ctas_per_sm, work_ctas);
    }
    grid = cdiv(grid, p.cluster) * p.cluster;
    if (grid / p.cluster > kMaxUnits) return SR_ERR_ARG;

    if (p.stage == SR_GRID_SYNC) {
        // A grid.sync() grid must be co-resident: size the default grid to
        // what the occupancy calculator allows; reject an explicit grid that
        // does not fit (Section VIII-B: partial-grid synchronisation deadlocks).
        KernelSet ks;
        if (!kernels_for(p, &ks)) return SR_ERR_UNSUPPORTED;
        int st = prepare_function(ks.main, p.smem, false);
        if (st != SR_OK) return st;
        int per_sm = 0;
        st = blocks_per_sm(d, ks.main, p.block, p.smem, &per_sm);
        if (st != SR_OK) return st;
        const int64_t cap = (int64_t)per_sm * d.sms;
        if (!c.grid) grid = std::min(grid, cap);
        if (grid > cap || grid < 1) return SR_ERR_LAUNCH;
    }
    p.grid = (int)grid;
    p.units = p.grid / p.cluster;
    *out = p;
    return SR_OK;
}

int reduce_launch(const void* x, void* out, const Plan& p, const DeviceInfo& d, const Workspace& ws,
                  cudaStream_t s, bool skip_final) {
    KernelSet ks;
    if (!kernels_for(p, &ks)) return SR_ERR_UNSUPPORTED;

    KParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.x = static_cast<const unsigned char*>(x);
    kp.n = p.n;
    kp.head = p.head;
    kp.nvec = p.nvec;
    kp.tail_begin = p.tail_begin;
    kp.ntail = p.ntail;
    kp.out = out;
    kp.partials = ws.partials;
    kp.ticket = ws.tickets;
    kp.err = ws.err;
    kp.scale = p.scale;
    kp.stage = p.stage;
    kp.fp64 = p.fp64 ? 1 : 0;
    kp.fp64_auto = p.fp64_auto ? 1 : 0;
    kp.units = p.units;
    kp.log2c = p.log2c;
    kp.tile_bytes = p.tile;
    kp.stages = p.stages;
    kp.body_bytes = p.body_bytes;
    kp.ntiles = p.ntiles;
    kp.limit_ns = spin_limit_ns();

    cudaError_t e;
    int st = prepare_function(ks.main, p.smem, p.cluster > 8);
    if (st != SR_OK) return st;

    if (p.stage == SR_ATOMIC) {
        const size_t ob = (p.dtype == SR_I32 || p.fp64) ? 8 : 4;
        st = launch_zero(out, ob, s);
        if (st != SR_OK) return st;
    }

    void* args[] = {&kp};
    if (p.stage == SR_GRID_SYNC) {
        // Every CTA of a grid.sync() kernel must be resident at once: check
        // before launching rather than ever starting a grid that could wait
        // forever (Section VIII-B: partial-grid synchronisation deadlocks).
        int per_sm = 0;
        st = blocks_per_sm(d, ks.main, p.block, p.smem, &per_sm);
        if (st != SR_OK) return st;
        if ((int64_t)per_sm * d.sms < p.grid) return SR_ERR_LAUNCH;
        e = cudaLaunchCooperativeKernel(ks.main, dim3(p.grid), dim3(p.block), args, p.smem, s);
        if (e != cudaSuccess) return status_from_cuda(e);
        return SR_OK;
    }

    // Both kernels are launched with programmatic stream serialisation: each
    // may be scheduled while its predecessor in the stream runs, and waits in
    // grid_dependency_wait() for that predecessor's completion before it
    // touches global memory.
    cudaLaunchConfig_t lc;
    std::memset(&lc, 0, sizeof lc);
    lc.gridDim = dim3(p.grid);
    lc.blockDim = dim3(p.block);
    lc.dynamicSmemBytes = p.smem;
    lc.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    if (p.cluster > 1) {
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = p.cluster;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        cudaLaunchConfig_t q = lc;  // the occupancy query sees the cluster shape alone
        q.attrs = attr + 1;
        q.numAttrs = 1;
        int nclusters = 0;
        st = active_clusters(d, ks.main, &q, &nclusters);
        if (st != SR_OK) return st;
        if (nclusters < 1) return SR_ERR_LAUNCH;
        lc.numAttrs = 2;
    }
    e = cudaLaunchKernelExC(&lc, ks.main, args);
    if (e != cudaSuccess) return status_from_cuda(e);

    if (p.stage == SR_TWO_KERNEL && !skip_final) {
        // The implicit barrier (Section III-B-2): kernel 2 reads the partials
        // only after kernel 1 has completed — grid_dependency_wait() at its top.
        const int threads = std::min(1024, std::max(32, ((p.units + 31) / 32) * 32));
        std::memset(&lc, 0, sizeof lc);
        lc.gridDim = dim3(1);
        lc.blockDim = dim3(threads);
        lc.stream = s;
        lc.attrs = attr;
        lc.numAttrs = 1;
        e = cudaLaunchKernelExC(&lc, ks.final, args);
        if (e != cudaSuccess) return status_from_cuda(e);
    }
    return SR_OK;
}

int launch_zero(void* p, size_t bytes, cudaStream_t s) {
    const int64_t nwords = (int64_t)(bytes / 4);
    if (nwords == 0) return SR_OK;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc;
    std::memset(&lc, 0, sizeof lc);
    lc.gridDim = dim3((unsigned)std::min<int64_t>(cdiv(nwords, 256), 1024));
    lc.blockDim = dim3(256);
    lc.stream = s;
    lc.attrs = attr;
    lc.numAttrs = 1;
    uint32_t* w = static_cast<uint32_t*>(p);
    void* args[] = {&w, const_cast<int64_t*>(&nwords)};
    cudaError_t e = cudaLaunchKernelExC(&lc, (const void*)zero_words_kernel, args);
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

int reduce_launch_final(const Plan& p, int units, void* out, const Workspace& ws, cudaStream_t s) {
    KernelSet ks;
    if (!kernels_for(p, &ks)) return SR_ERR_UNSUPPORTED;
    KParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.out = out;
    kp.partials = ws.partials;
    kp.scale = p.scale;
    kp.fp64 = p.fp64 ? 1 : 0;
    kp.fp64_auto = p.fp64_auto ? 1 : 0;
    kp.units = units;
    void* args[] = {&kp};
    const int threads = std::min(1024, std::max(32, ((units + 31) / 32) * 32));
    cudaError_t e = cudaLaunchKernel(ks.final, dim3(1), dim3(threads), args, 0, s);
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

}  // namespace sr
