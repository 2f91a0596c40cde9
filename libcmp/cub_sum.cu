// Library comparison point for the benchmark suites — not part of libsr and
// never on its path: CUB's DeviceReduce over the same inputs the library
// reduces (FP32 -> FP32; int32 -> int64, exact).  Temporary storage is
// reserved up front by cmp_prepare so that calls allocate nothing and can be
// captured in CUDA graphs.
#include <cstdint>

#include <cub/device/device_reduce.cuh>
#include <cuda/std/functional>

namespace {
void* g_tmp = nullptr;
size_t g_tmp_bytes = 0;

size_t need_f32(int64_t n) {
    size_t b = 0;
    cub::DeviceReduce::Sum(nullptr, b, static_cast<const float*>(nullptr), static_cast<float*>(nullptr), n);
    return b;
}

size_t need_i32(int64_t n) {
    size_t b = 0;
    cub::DeviceReduce::Reduce(nullptr, b, static_cast<const int*>(nullptr), static_cast<long long*>(nullptr), n,
                              cuda::std::plus<long long>{}, 0LL);
    return b;
}
}  // namespace

extern "C" {

// Reserves temporary storage for inputs of up to max_n elements of either
// type.  Returns a cudaError_t value (0 = success).
int cmp_prepare(int64_t max_n) {
    if (max_n < 1) return (int)cudaErrorInvalidValue;
    size_t need = need_f32(max_n);
    size_t ni = need_i32(max_n);
    if (ni > need) need = ni;
    if (need <= g_tmp_bytes) return 0;
    if (g_tmp) cudaFree(g_tmp);
    g_tmp = nullptr;
    g_tmp_bytes = 0;
    cudaError_t e = cudaMalloc(&g_tmp, need);
    if (e == cudaSuccess) g_tmp_bytes = need;
    return (int)e;
}

// out[0] = sum of x[0..n) (device pointers), stream-ordered.  n must not
// exceed the cmp_prepare size.
int cmp_cub_sum_f32(const float* x, int64_t n, float* out, cudaStream_t stream) {
    size_t b = need_f32(n);
    if (b > g_tmp_bytes) return (int)cudaErrorInvalidValue;
    return (int)cub::DeviceReduce::Sum(g_tmp, b, x, out, n, stream);
}

int cmp_cub_sum_i32(const int* x, int64_t n, long long* out, cudaStream_t stream) {
    size_t b = need_i32(n);
    if (b > g_tmp_bytes) return (int)cudaErrorInvalidValue;
    return (int)cub::DeviceReduce::Reduce(g_tmp, b, x, out, n, cuda::std::plus<long long>{}, 0LL, stream);
}

}  // extern "C"
