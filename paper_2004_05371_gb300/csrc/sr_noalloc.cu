// sr_reduce_sum_noalloc: the last-block-done sum without any device
// allocation, for callers that cannot call cudaMalloc (see include/sr.h).
//
// The scratch the last-block-done grid stage needs (one 16-byte partial slot
// per unit, the arrival ticket, an error word) lives in a file-scope
// __device__ array of fixed size instead of the per-stream workspace.  Every
// GPU that loads this library holds the array until the process exits.
#include <cstring>
#include <map>
#include <mutex>

#include "sr_internal.h"
#include "sr_kparams.h"

namespace sr {
namespace {

constexpr int kNoAllocMaxUnits = 4096;
constexpr size_t kNoAllocHeader = 256;  // ticket (bytes 0-3), error word (bytes 128-131)
constexpr size_t kNoAllocBytes = kNoAllocHeader + (size_t)kNoAllocMaxUnits * kSlotBytes;  // 64 KiB + 256 B

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_na_mu;
std::map<int, unsigned char*> g_na_addr;  // device -> device address of g_noalloc_scratch

// In host code `g_noalloc_scratch` names a host-side shadow, not device
// memory: the kernel must be given the address the runtime reports for the
// current device.  Looked up once per device, with that device current.
int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return status_from_cuda(e);
    std::lock_guard<std::mutex> lk(g_na_mu);
    auto it = g_na_addr.find(dev);
    if (it != g_na_addr.end()) {
        *out = it->second;
        return SR_OK;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return status_from_cuda(e);
    g_na_addr[dev] = static_cast<unsigned char*>(p);
    *out = static_cast<unsigned char*>(p);
    return SR_OK;
}

}  // namespace
}  // namespace sr

using namespace sr;

extern "C" int sr_reduce_sum_noalloc(const void* x, int64_t n, int dtype, void* out, const sr_config* cfg,
                                     sr_stream_t stream) {
    sr_config c;
    std::memset(&c, 0, sizeof c);
    if (cfg) c = *cfg;
    const int stage = c.variant & SR_STAGE_MASK;
    if (stage != SR_AUTO && stage != SR_LAST_BLOCK) return SR_ERR_UNSUPPORTED;
    if (c.variant & SR_F_BULK) return SR_ERR_UNSUPPORTED;
    c.variant = (c.variant & ~SR_STAGE_MASK) | SR_LAST_BLOCK;
    int st = reduce_validate(x, n, dtype, out, c);
    if (st != SR_OK) return st;
    const int log2c = (c.variant & SR_CLUSTER_MASK) >> SR_CLUSTER_SHIFT;
    if ((int64_t)c.grid > ((int64_t)kNoAllocMaxUnits << log2c)) return SR_ERR_ARG;  // too many units

    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    Plan p;
    st = reduce_plan(x, n, dtype, c, *d, &p);
    if (st != SR_OK) return st;
    if (p.units > kNoAllocMaxUnits) return SR_ERR_ARG;

    unsigned char* base = nullptr;
    st = scratch_address(&base);
    if (st != SR_OK) return st;
    Workspace ws;
    ws.base = base;
    ws.tickets = reinterpret_cast<unsigned int*>(base);
    // The load path here has no bounded wait and the finish is last-block-done
    // (never grid.sync), so no kernel of this call writes the error word; it
    // points into the array only so that the kernel parameters stay valid.
    ws.err = reinterpret_cast<int*>(base + 128);
    ws.partials = base + kNoAllocHeader;
    ws.seg = nullptr;
    // The array keeps the previous call's contents: start the ticket at zero.
    cudaError_t e = cudaMemsetAsync(ws.tickets, 0, sizeof(unsigned int), (cudaStream_t)stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    return reduce_launch(x, out, p, *d, ws, (cudaStream_t)stream);
}
