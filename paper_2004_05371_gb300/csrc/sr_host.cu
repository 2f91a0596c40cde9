// sr_reduce_sum_host: the sum of an array in HOST memory, result to host.
//
// The input streams to the device in chunks through two staging buffers, on
// two copy streams (both copy engines), while the caller's stream reduces the
// chunk that already arrived: each chunk's units write their partials into
// their own range of the workspace slots (the first kernel of the two-kernel
// form), one final kernel reduces all slots in order, and the scalar is copied
// back.  Copy of chunk k+1 overlaps the reduction of chunk k.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "sr_internal.h"

namespace sr {
namespace {

constexpr size_t kChunkBytes = 64u << 20;

struct HostPipe {
    unsigned char* stage[2] = {nullptr, nullptr};
    cudaStream_t copy[2] = {nullptr, nullptr};
    cudaEvent_t copied[2] = {nullptr, nullptr};
    cudaEvent_t consumed[2] = {nullptr, nullptr};
    size_t chunk = 0;
};

std::mutex g_hp_mu;
std::map<std::pair<int, cudaStream_t>, HostPipe> g_pipes;

int get_pipe(cudaStream_t s, size_t chunk, HostPipe** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return status_from_cuda(e);
    std::lock_guard<std::mutex> lk(g_hp_mu);
    HostPipe& p = g_pipes[std::make_pair(dev, s)];
    if (p.chunk < chunk) {
        for (int b = 0; b < 2; ++b) {
            if (p.stage[b]) cudaFree(p.stage[b]);
            p.stage[b] = nullptr;
        }
        for (int b = 0; b < 2; ++b) {
            e = cudaMalloc(&p.stage[b], chunk);
            if (e != cudaSuccess) {
                p.chunk = 0;
                return status_from_cuda(e);
            }
        }
        p.chunk = chunk;
    }
    for (int b = 0; b < 2; ++b) {
        if (!p.copy[b]) {
            e = cudaStreamCreateWithFlags(&p.copy[b], cudaStreamNonBlocking);
            if (e != cudaSuccess) return status_from_cuda(e);
        }
        if (!p.copied[b]) {
            e = cudaEventCreateWithFlags(&p.copied[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.consumed[b], cudaEventDisableTiming);
            if (e != cudaSuccess) return status_from_cuda(e);
        }
    }
    *out = &p;
    return SR_OK;
}

}  // namespace

void release_host_pipe(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_hp_mu);
    auto it = g_pipes.find(std::make_pair(dev, s));
    if (it == g_pipes.end()) return;
    HostPipe& p = it->second;
    for (int b = 0; b < 2; ++b) {
        if (p.copy[b]) cudaStreamSynchronize(p.copy[b]);
        if (p.stage[b]) cudaFree(p.stage[b]);
        if (p.copy[b]) cudaStreamDestroy(p.copy[b]);
        if (p.copied[b]) cudaEventDestroy(p.copied[b]);
        if (p.consumed[b]) cudaEventDestroy(p.consumed[b]);
    }
    g_pipes.erase(it);
}

}  // namespace sr

using namespace sr;

namespace {

// The reduction reads the host array in place (no staging copies).
int host_direct(const void* host_x, int64_t n, int dtype, void* host_out, sr_config c, sr_stream_t stream) {
    const int stage = c.variant & SR_STAGE_MASK;
    if ((stage != SR_AUTO && stage != SR_LAST_BLOCK) || (c.variant & SR_F_BULK)) return SR_ERR_UNSUPPORTED;
    c.variant = (c.variant & ~(SR_STAGE_MASK | SR_F_HOST_DIRECT)) | SR_LAST_BLOCK;
    const void* fake_out = reinterpret_cast<const void*>(uintptr_t(1) << 20);
    int st = reduce_validate(host_x, n, dtype, fake_out, c);
    if (st != SR_OK) return st;
    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    const void* dx = host_x;
    if (n > 0) {
        cudaPointerAttributes a;
        cudaError_t e = cudaPointerGetAttributes(&a, host_x);
        if (e != cudaSuccess) return status_from_cuda(e);
        if (a.type == cudaMemoryTypeHost) {
            void* mapped = nullptr;
            e = cudaHostGetDevicePointer(&mapped, const_cast<void*>(host_x), 0);
            if (e != cudaSuccess) return status_from_cuda(e);
            dx = mapped;
        } else if (a.type == cudaMemoryTypeUnregistered) {
            int pageable = 0;
            e = cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, d->dev);
            if (e != cudaSuccess) return status_from_cuda(e);
            if (!pageable) return SR_ERR_UNSUPPORTED;
        } else {
            return SR_ERR_ARG;  // device or managed memory: use sr_reduce_sum_ex
        }
    }
    Plan p;
    cudaStream_t s = (cudaStream_t)stream;
    st = reduce_plan(dx, n, dtype, c, *d, &p);
    if (st != SR_OK) return st;
    Workspace ws;
    st = get_workspace(s, &ws);
    if (st != SR_OK) return st;
    unsigned char* dev_out = ws.base + 192;
    st = reduce_launch(dx, dev_out, p, *d, ws, s);
    if (st != SR_OK) return st;
    const size_t out_bytes = (dtype == SR_I32 || p.fp64) ? 8 : 4;
    cudaError_t e = cudaMemcpyAsync(host_out, dev_out, out_bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

}  // namespace

extern "C" int sr_reduce_sum_host(const void* host_x, int64_t n, int dtype, void* host_out, const sr_config* cfg,
                                  sr_stream_t stream) {
    sr_config c;
    std::memset(&c, 0, sizeof c);
    if (cfg) c = *cfg;
    if (host_out == nullptr) return SR_ERR_ARG;
    if (c.variant & SR_F_HOST_DIRECT) return host_direct(host_x, n, dtype, host_out, c, stream);
    const int stage = c.variant & SR_STAGE_MASK;
    if (stage != SR_AUTO && stage != SR_TWO_KERNEL) return SR_ERR_UNSUPPORTED;
    if (c.variant & SR_F_BULK) return SR_ERR_UNSUPPORTED;
    c.variant = (c.variant & ~SR_STAGE_MASK) | SR_TWO_KERNEL;
    // validate with a device-style stand-in for out (the host result is copied)
    const void* fake_out = reinterpret_cast<const void*>(uintptr_t(1) << 20);
    int st = reduce_validate(host_x, n, dtype, fake_out, c);
    if (st != SR_OK) return st;
    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws;
    st = get_workspace(s, &ws);
    if (st != SR_OK) return st;
    const int es = elem_size(dtype);
    const size_t bytes = (size_t)n * es;
    size_t chunk = kChunkBytes;
    // at most kMaxUnits partial slots in total: bigger chunks for huge inputs
    const int64_t max_chunks = kMaxUnits / (8 * d->sms);
    if ((int64_t)((bytes + chunk - 1) / chunk) > max_chunks) {
        chunk = (bytes + max_chunks - 1) / max_chunks;
        chunk = (chunk + (1u << 20) - 1) & ~((size_t)(1u << 20) - 1);
    }
    HostPipe* hp = nullptr;
    st = get_pipe(s, chunk, &hp);
    if (st != SR_OK) return st;

    const bool fp64 = (c.variant & SR_F_FP64_COMBINE) && dtype != SR_I32;
    const size_t out_bytes = (dtype == SR_I32 || fp64) ? 8 : 4;
    unsigned char* dev_out = ws.base + 192;  // result slot in the workspace header
    int slot = 0;
    Plan last;
    bool have_plan = false;
    const unsigned char* hx = static_cast<const unsigned char*>(host_x);
    const size_t per_chunk = chunk / es;  // elements per chunk (chunk is a multiple of 16 B)
    for (size_t k = 0, off = 0; off < bytes || k == 0; ++k, off += chunk) {
        const int b = (int)(k & 1);
        const size_t len = std::min(chunk, bytes - off);
        const int64_t nk = (int64_t)(len / es);
        cudaError_t e;
        if (k >= 2) {
            e = cudaStreamWaitEvent(hp->copy[b], hp->consumed[b], 0);
            if (e != cudaSuccess) return status_from_cuda(e);
        }
        if (len) {
            e = cudaMemcpyAsync(hp->stage[b], hx + off, len, cudaMemcpyHostToDevice, hp->copy[b]);
            if (e != cudaSuccess) return status_from_cuda(e);
        }
        e = cudaEventRecord(hp->copied[b], hp->copy[b]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, hp->copied[b], 0);
        if (e != cudaSuccess) return status_from_cuda(e);
        Plan p;
        st = reduce_plan(hp->stage[b], nk, dtype, c, *d, &p);
        if (st != SR_OK) return st;
        if (slot + p.units > kMaxUnits) return SR_ERR_ARG;
        Workspace wk = ws;
        wk.partials = ws.partials + (size_t)slot * kSlotBytes;
        st = reduce_launch(hp->stage[b], dev_out, p, *d, wk, s, /*skip_final=*/true);
        if (st != SR_OK) return st;
        slot += p.units;
        last = p;
        have_plan = true;
        e = cudaEventRecord(hp->consumed[b], s);
        if (e != cudaSuccess) return status_from_cuda(e);
        (void)per_chunk;
        if (len == 0) break;
    }
    if (!have_plan) return SR_ERR_ARG;
    st = reduce_launch_final(last, slot, dev_out, ws, s);
    if (st != SR_OK) return st;
    cudaError_t e = cudaMemcpyAsync(host_out, dev_out, out_bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}
