// Self-test of the bounded-wait failure path: a kernel waits on an mbarrier
// that nothing ever completes; the wait gives up after `limit_ns` of
// %globaltimer time, the kernel records the timeout in the stream
// workspace's error word and returns, and the host reads it with
// sr_stream_status — the GPU context stays usable.
#include "sr_device.cuh"
#include "sr_internal.h"
#include "sr_kparams.h"

namespace sr {
namespace {

__global__ void never_completed_wait_kernel(int* err, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);  // one arrival expected; none will come
        mbar_fence_init();
    }
    __syncthreads();
    if (!mbar_wait_bounded(b, 0, limit_ns)) {
        if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
    }
}

}  // namespace
}  // namespace sr

using namespace sr;

extern "C" int sr_selftest_bounded_wait(uint64_t limit_ns, sr_stream_t stream) {
    if (limit_ns == 0 || limit_ns > 10000000000ull) return SR_ERR_ARG;  // (0, 10 s]
    Workspace ws;
    int st = get_workspace((cudaStream_t)stream, &ws);
    if (st != SR_OK) return st;
    never_completed_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(ws.err, limit_ns);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}
