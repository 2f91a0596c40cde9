// C ABI of the library (declared in include/sr.h): argument checks, device
// facts, the per-(device, stream) workspace, and dispatch to the kernels.
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "sr_internal.h"
#include "sr_kparams.h"
#include "sr_segparams.h"

namespace sr {

namespace {

thread_local int g_last_cuda_error = 0;

std::mutex g_mu;
std::map<int, DeviceInfo> g_devices;
std::map<std::pair<int, cudaStream_t>, Workspace> g_workspaces;
// Per function: the largest dynamic shared memory size set so far, and
// whether non-portable cluster sizes were enabled.  The attribute is one
// maximum per function, so it only ever grows.
std::map<const void*, std::pair<size_t, bool>> g_prepared;
std::map<std::tuple<int, const void*, int, size_t>, int> g_blocks_per_sm;
std::map<std::tuple<int, const void*, int, int, size_t>, int> g_clusters;

uint64_t g_spin_limit_ns = 0;

}  // namespace

int status_from_cuda(cudaError_t e) {
    g_last_cuda_error = (int)e;
    cudaGetLastError();  // clear the sticky-free error so later calls start clean
    return SR_ERR_CUDA;
}

uint64_t spin_limit_ns() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_spin_limit_ns == 0) {
        const char* s = std::getenv("SR_SPIN_LIMIT_NS");
        g_spin_limit_ns = (s && *s) ? std::strtoull(s, nullptr, 10) : 2000000000ull;  // 2 s
        if (g_spin_limit_ns == 0) g_spin_limit_ns = 1;
    }
    return g_spin_limit_ns;
}

const DeviceInfo* current_device(int* status) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *status = status_from_cuda(e);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_devices.find(dev);
    if (it != g_devices.end()) {
        *status = SR_OK;
        return &it->second;
    }
    DeviceInfo d;
    d.dev = dev;
    struct {
        int* dst;
        cudaDeviceAttr a;
    } q[] = {
        {&d.sms, cudaDevAttrMultiProcessorCount},
        {&d.max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor},
        {&d.max_blocks_per_sm, cudaDevAttrMaxBlocksPerMultiprocessor},
        {&d.smem_per_block_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin},
        {&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor},
        {&d.l2_bytes, cudaDevAttrL2CacheSize},
        {&d.cc_major, cudaDevAttrComputeCapabilityMajor},
        {&d.cc_minor, cudaDevAttrComputeCapabilityMinor},
        {&d.clock_khz, cudaDevAttrClockRate},
    };
    for (auto& qq : q) {
        e = cudaDeviceGetAttribute(qq.dst, qq.a, dev);
        if (e != cudaSuccess) {
            *status = status_from_cuda(e);
            return nullptr;
        }
    }
    *status = SR_OK;
    return &(g_devices[dev] = d);
}

int get_workspace(cudaStream_t s, Workspace* ws) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return status_from_cuda(e);
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(dev, s);
    auto it = g_workspaces.find(key);
    if (it != g_workspaces.end()) {
        *ws = it->second;
        return SR_OK;
    }
    const size_t bytes = kHeaderBytes + (size_t)kMaxUnits * kSlotBytes + kSegBytes;
    void* base = nullptr;
    e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) return status_from_cuda(e);
    e = cudaMemset(base, 0, bytes);  // tickets and the error word start at zero
    if (e != cudaSuccess) {
        cudaFree(base);
        return status_from_cuda(e);
    }
    Workspace w;
    w.base = static_cast<unsigned char*>(base);
    w.tickets = reinterpret_cast<unsigned int*>(w.base);
    w.err = reinterpret_cast<int*>(w.base + 32 * sizeof(unsigned int));  // after 32 tickets
    w.partials = w.base + kHeaderBytes;
    w.seg = w.partials + (size_t)kMaxUnits * kSlotBytes;
    w.check = reinterpret_cast<int*>(w.base + 160);
    g_workspaces[key] = w;
    *ws = w;
    return SR_OK;
}

void release_workspace(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_workspaces.find(std::make_pair(dev, s));
    if (it == g_workspaces.end()) return;
    cudaFree(it->second.base);
    g_workspaces.erase(it);
}

int prepare_function(const void* fn, size_t dyn_smem, bool nonportable) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto& st = g_prepared[fn];
    cudaError_t e;
    if (dyn_smem > 48 * 1024 && dyn_smem > st.first) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
        if (e != cudaSuccess) return status_from_cuda(e);
        st.first = dyn_smem;
    }
    if (nonportable && !st.second) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return status_from_cuda(e);
        st.second = true;
    }
    return SR_OK;
}

int blocks_per_sm(const DeviceInfo& d, const void* fn, int block, size_t dyn_smem, int* out) {
    auto key = std::make_tuple(d.dev, fn, block, dyn_smem);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_blocks_per_sm.find(key);
        if (it != g_blocks_per_sm.end()) {
            *out = it->second;
            return SR_OK;
        }
    }
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, block, dyn_smem);
    if (e != cudaSuccess) return status_from_cuda(e);
    std::lock_guard<std::mutex> lk(g_mu);
    g_blocks_per_sm[key] = v;
    *out = v;
    return SR_OK;
}

int active_clusters(const DeviceInfo& d, const void* fn, const cudaLaunchConfig_t* lc, int* out) {
    int cluster = 1;
    for (unsigned i = 0; i < lc->numAttrs; ++i)
        if (lc->attrs[i].id == cudaLaunchAttributeClusterDimension) cluster = (int)lc->attrs[i].val.clusterDim.x;
    auto key = std::make_tuple(d.dev, fn, cluster, (int)lc->blockDim.x, lc->dynamicSmemBytes);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_clusters.find(key);
        if (it != g_clusters.end()) {
            *out = it->second;
            return SR_OK;
        }
    }
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&v, fn, lc);
    if (e != cudaSuccess) return status_from_cuda(e);
    std::lock_guard<std::mutex> lk(g_mu);
    g_clusters[key] = v;
    *out = v;
    return SR_OK;
}

}  // namespace sr

using namespace sr;

namespace {
sr_config default_config(int variant) {
    sr_config c;
    std::memset(&c, 0, sizeof c);
    c.variant = variant;
    return c;
}

// The configuration of a single-array sum: the caller's, or — cfg == NULL,
// the library's choice — SR_AUTO unless SR_VARIANT names a variant.
int library_choice(const sr_config* cfg, sr_config* c) {
    if (cfg) {
        *c = *cfg;
        return SR_OK;
    }
    int v = SR_AUTO;
    const int st = env_variant(&v);
    if (st != SR_OK) return st;
    *c = default_config(v);
    return SR_OK;
}
}  // namespace

extern "C" {

int sr_reduce_sum_ex(const void* x, int64_t n, int dtype, void* out, const sr_config* cfg, sr_stream_t stream) {
    sr_config c;
    int st = library_choice(cfg, &c);
    if (st != SR_OK) return st;
    st = reduce_validate(x, n, dtype, out, c);
    if (st != SR_OK) return st;
    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    Plan p;
    st = reduce_plan(x, n, dtype, c, *d, &p);
    if (st != SR_OK) return st;
    Workspace ws;
    st = get_workspace((cudaStream_t)stream, &ws);
    if (st != SR_OK) return st;
    return reduce_launch(x, out, p, *d, ws, (cudaStream_t)stream);
}

int sr_reduce_sum(const void* x, int64_t n, int dtype, void* out, int variant, sr_stream_t stream) {
    if (variant == SR_AUTO) return sr_reduce_sum_ex(x, n, dtype, out, nullptr, stream);
    const sr_config c = default_config(variant);
    return sr_reduce_sum_ex(x, n, dtype, out, &c, stream);
}

int sr_reduce_sum_segmented_ex(const void* x, const int64_t* offsets, int64_t nseg, int dtype, void* out,
                               const sr_config* cfg, sr_stream_t stream) {
    const sr_config c = cfg ? *cfg : default_config(SR_AUTO);
    int st = seg_validate(x, offsets, nseg, dtype, out, c);
    if (st != SR_OK) return st;
    if (nseg == 0) return SR_OK;
    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    SegPlan p;
    st = seg_plan(nseg, dtype, c, *d, &p);
    if (st != SR_OK) return st;
    Workspace ws;
    st = get_workspace((cudaStream_t)stream, &ws);
    if (st != SR_OK) return st;
    return seg_launch(x, offsets, out, p, ws, (cudaStream_t)stream);
}

int sr_reduce_sum_segmented_checked(const void* x, int64_t n_elems, const int64_t* offsets, int64_t nseg,
                                    int dtype, void* out, const sr_config* cfg, sr_stream_t stream) {
    const sr_config c = cfg ? *cfg : default_config(SR_AUTO);
    if (n_elems < 0 || (n_elems > 0 && x == nullptr)) return SR_ERR_ARG;
    int st = seg_validate(x ? x : offsets, offsets, nseg, dtype, out, c);
    if (st != SR_OK) return st;
    if (nseg == 0) return SR_OK;
    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    SegPlan p;
    st = seg_plan(nseg, dtype, c, *d, &p);
    if (st != SR_OK) return st;
    Workspace ws;
    st = get_workspace((cudaStream_t)stream, &ws);
    if (st != SR_OK) return st;
    st = seg_check(offsets, nseg, n_elems, ws, (cudaStream_t)stream);
    if (st != SR_OK) return st;
    return seg_launch(x ? x : offsets, offsets, out, p, ws, (cudaStream_t)stream, /*check=*/true);
}

int sr_reduce_sum_segmented(const void* x, const int64_t* offsets, int64_t nseg, int dtype, void* out,
                            sr_stream_t stream) {
    return sr_reduce_sum_segmented_ex(x, offsets, nseg, dtype, out, nullptr, stream);
}

int sr_plan_segmented(int64_t nseg, int dtype, const sr_config* cfg, sr_config* resolved) {
    if (!resolved) return SR_ERR_ARG;
    const sr_config c = cfg ? *cfg : default_config(SR_AUTO);
    const void* fake = reinterpret_cast<const void*>(uintptr_t(1) << 20);
    int st = seg_validate(fake, reinterpret_cast<const int64_t*>(fake), nseg, dtype, fake, c);
    if (st != SR_OK) return st;
    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    SegPlan p;
    st = seg_plan(nseg, dtype, c, *d, &p);
    if (st != SR_OK) return st;
    sr_config r = c;
    r.variant = (c.variant & ~(SR_STAGE_MASK | SR_F_BULK)) | p.stage | (p.bulk ? SR_F_BULK : 0);
    r.block_threads = p.block;
    r.grid = p.grid;
    r.vec_bytes = p.vec;
    r.unroll = p.unroll;
    r.stages = p.bulk ? p.stages : 0;
    r.scale = p.scale;
    *resolved = r;
    return SR_OK;
}

struct sr_graph_s {
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

int sr_graph_capture_segmented(const void* x, const int64_t* offsets, int64_t nseg, int dtype, void* out,
                               const sr_config* cfg, sr_graph* g) {
    if (!g) return SR_ERR_ARG;
    *g = nullptr;
    const sr_config c = cfg ? *cfg : default_config(SR_AUTO);
    int st = seg_validate(x, offsets, nseg, dtype, out, c);
    if (st != SR_OK) return st;
    if (nseg == 0) return SR_ERR_ARG;
    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    SegPlan p;
    st = seg_plan(nseg, dtype, c, *d, &p);
    if (st != SR_OK) return st;
    sr_graph h = new sr_graph_s;
    cudaError_t e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete h;
        return status_from_cuda(e);
    }
    Workspace ws;
    st = get_workspace(h->capture_stream, &ws);  // allocated before capture begins
    if (st == SR_OK) {
        e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = status_from_cuda(e);
    }
    if (st == SR_OK) {
        int lst = seg_launch(x, offsets, out, p, ws, h->capture_stream);
        e = cudaStreamEndCapture(h->capture_stream, &h->graph);
        st = lst != SR_OK ? lst : (e != cudaSuccess ? status_from_cuda(e) : SR_OK);
    }
    if (st == SR_OK) {
        e = cudaGraphInstantiate(&h->exec, h->graph, 0);
        if (e != cudaSuccess) st = status_from_cuda(e);
    }
    if (st != SR_OK) {
        sr_graph_destroy(h);
        return st;
    }
    *g = h;
    return SR_OK;
}

int sr_graph_launch(sr_graph g, sr_stream_t stream) {
    if (!g || !g->exec) return SR_ERR_ARG;
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

int sr_graph_destroy(sr_graph g) {
    if (!g) return SR_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->capture_stream) {
        release_workspace(g->capture_stream);
        cudaStreamDestroy(g->capture_stream);
    }
    delete g;
    return SR_OK;
}

int sr_plan(int64_t n, int dtype, const sr_config* cfg, sr_config* resolved) {
    if (!resolved) return SR_ERR_ARG;
    sr_config c;
    int st0 = library_choice(cfg, &c);
    if (st0 != SR_OK) return st0;
    // A 256-byte-aligned stand-in address: plans assume an aligned array.
    const void* fake = reinterpret_cast<const void*>(uintptr_t(1) << 20);
    int st = reduce_validate(fake, n, dtype, fake, c);
    if (st != SR_OK) return st;
    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    Plan p;
    st = reduce_plan(fake, n, dtype, c, *d, &p);
    if (st != SR_OK) return st;
    sr_config r = c;
    r.variant = (c.variant & ~(SR_STAGE_MASK | SR_CLUSTER_MASK | SR_F_BULK)) | p.stage | SR_CLUSTER(p.log2c) |
                (p.bulk ? SR_F_BULK : 0) | (p.comp ? SR_F_KAHAN : 0);
    r.block_threads = p.block;
    r.grid = p.grid;
    r.vec_bytes = p.vec;
    r.unroll = p.unroll;
    r.tile_bytes = p.tile;
    r.stages = p.stages;
    r.scale = p.scale;
    *resolved = r;
    return SR_OK;
}

int sr_stream_status(sr_stream_t stream) {
    Workspace ws;
    int st = get_workspace((cudaStream_t)stream, &ws);
    if (st != SR_OK) return st;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    int err = 0;
    e = cudaMemcpy(&err, ws.err, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return status_from_cuda(e);
    if (err) {
        // A kernel that gave up may have left tickets half-counted (a segmented
        // warp that stopped never arrives): start the stream's next call clean.
        e = cudaMemset(ws.err, 0, sizeof err);
        if (e == cudaSuccess) e = cudaMemset(ws.tickets, 0, 32 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(ws.seg, 0, (size_t)kSegMaxWarps * sizeof(unsigned int));
        if (e != cudaSuccess) return status_from_cuda(e);
    }
    if (err & kErrTimeout) return SR_ERR_TIMEOUT;
    if (err & kErrBadOffsets) return SR_ERR_ARG;
    if (err & kErrQueueFull) return SR_ERR_LAUNCH;
    if (err) return SR_ERR_LAUNCH;
    return SR_OK;
}

int sr_stream_release(sr_stream_t stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    release_workspace((cudaStream_t)stream);
    release_host_pipe((cudaStream_t)stream);
    return SR_OK;
}

const char* sr_status_string(int s) {
    switch (s) {
    case SR_OK: return "SR_OK";
    case SR_ERR_ARG: return "SR_ERR_ARG: invalid argument";
    case SR_ERR_DTYPE: return "SR_ERR_DTYPE: unsupported dtype";
    case SR_ERR_LAUNCH: return "SR_ERR_LAUNCH: launch shape cannot run";
    case SR_ERR_CUDA: return "SR_ERR_CUDA: CUDA runtime error";
    case SR_ERR_TIMEOUT: return "SR_ERR_TIMEOUT: a bounded device wait expired";
    case SR_ERR_UNSUPPORTED: return "SR_ERR_UNSUPPORTED: unsupported option combination";
    default: return "unknown status";
    }
}

int sr_last_cuda_error(void) { return g_last_cuda_error; }

const char* sr_version(void) { return "sr 0.1 (sm_103a)"; }

}  // extern "C"
