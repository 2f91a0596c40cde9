// Barrier-latency micro-benchmark (paper Section V and Section IX):
//   warp / coalesced / shuffle / block / cluster / grid synchronisation, each
//   repeated r times back to back inside one kernel;
//   - intra-SM cost by Wong's method (Section IX-C): clock64() before and
//     after the r repetitions, averaged;
//   - inter-SM cost by the paper's CPU-clock differential method (Section
//     IX-D, Eq. 7): kernel total latency L_k measured with a host clock around
//     launch + synchronise for two repeat counts r1 > r2, T = (L1 - L2)/(r1 - r2),
//     with its standard deviation from Eq. 8 over N runs of each;
//   - the implicit kernel-boundary barrier by kernel fusion (Section IX-B,
//     Eq. 6): i launches of j wait units against j launches of i wait units
//     (each unit a nanosleep of 1 us), O = (L_ij - L_ji)/(i - j);
//   - a dependent FP32 add chain as the methods' self-check (Section IX-D);
//   - the warp-level reductions of Table V: 32 FP64 values summed by one warp
//     serially, by shared-memory trees under each warp synchronisation, and by
//     shuffle trees; the result is checked against the exact sum.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "sr_internal.h"

namespace cg = cooperative_groups;

namespace sr {
namespace {

struct BarParams {
    int64_t iters;
    int group;
    long long* t;             // per warp: start, end clock64
    unsigned long long* gt;   // block 0 thread 0: globaltimer start, end; clock start, end
    float* sink;
    unsigned int* bad;        // SR_LEVEL_WARP_REDUCE: reductions that missed the exact sum
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int LEVEL>
__global__ void __launch_bounds__(1024) bar_kernel(const BarParams p) {
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    float v = (float)lane;
    unsigned long long g0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) g0 = gtimer();
    __syncthreads();
    const long long c0 = clock64();
    if constexpr (LEVEL == SR_LEVEL_WARP) {
        // tile of `group` lanes: the lanes of one tile synchronise together
        const int g = p.group;
        const unsigned tile = (g == 32) ? 0xffffffffu : (((1u << g) - 1u) << ((lane / g) * g));
#pragma unroll 16
        for (int64_t i = 0; i < p.iters; ++i) __syncwarp(tile);
    } else if constexpr (LEVEL == SR_LEVEL_COALESCED) {
        if (lane < p.group) {  // only `group` lanes are active: a coalesced group of that size
            cg::coalesced_group cgp = cg::coalesced_threads();
#pragma unroll 16
            for (int64_t i = 0; i < p.iters; ++i) cgp.sync();
        }
    } else if constexpr (LEVEL == SR_LEVEL_SHUFFLE) {
#pragma unroll 16
        for (int64_t i = 0; i < p.iters; ++i) v = __shfl_xor_sync(0xffffffffu, v, 1);
    } else if constexpr (LEVEL == SR_LEVEL_BLOCK) {
#pragma unroll 16
        for (int64_t i = 0; i < p.iters; ++i) __syncthreads();
    } else if constexpr (LEVEL == SR_LEVEL_CLUSTER) {
        cg::cluster_group cl = cg::this_cluster();
#pragma unroll 8
        for (int64_t i = 0; i < p.iters; ++i) cl.sync();
    } else if constexpr (LEVEL == SR_LEVEL_GRID) {
        cg::grid_group g = cg::this_grid();
        if (g.is_valid()) {
            for (int64_t i = 0; i < p.iters; ++i) g.sync();
        }
    } else if constexpr (LEVEL == SR_LEVEL_FADD) {
        float q = v + 1.0f;  // Wong's dependent chain: p = p + q; q = p + q
#pragma unroll 16
        for (int64_t i = 0; i < p.iters; ++i) {
            v = __fadd_rn(v, q);
            q = __fadd_rn(v, q);
        }
        v = q;
    }
    const long long c1 = clock64();
    if (lane == 0) {
        p.t[2 * gw] = c0;
        p.t[2 * gw + 1] = c1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.gt[0] = g0;
        p.gt[1] = gtimer();
        p.gt[2] = (unsigned long long)c0;
        p.gt[3] = (unsigned long long)c1;
    }
    if (v == -12345.f) p.sink[0] = v;  // keeps the shuffle / add chains alive
}

// Table V: every warp sums its lanes' values x = lane + 1 (exact sum 528 in
// any order, all partial sums small integers) `iters` times by method M, in
// FP64 as the paper does or in binary32 (T = float).  The next
// repetition's input depends on this one's result (x0 + 0 unless the result is
// NaN), so repetitions run one after another, and two shared-memory buffers
// alternate so that a repetition's stores never overwrite values that a
// lagging lane of the previous one still reads.
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

template <int M, class T>
__global__ void __launch_bounds__(1024) warp_reduce_kernel(const BarParams p) {
    __shared__ T sh[2][32][32];  // [buffer][warp of the CTA][lane]
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const T x0 = (T)(lane + 1);
    cg::thread_block_tile<32> tile = cg::tiled_partition<32>(cg::this_thread_block());
    cg::coalesced_group co = cg::coalesced_threads();
    T s = 0;
    unsigned int bad = 0;
    unsigned long long g0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) g0 = gtimer();
    __syncthreads();
    const long long c0 = clock64();
    for (int64_t i = 0; i < p.iters; ++i) {
        const T x = x0 + ((s != s) ? (T)1 : (T)0);
        T* b = sh[i & 1][wib];
        if constexpr (M == SR_WR_SERIAL) {
            b[lane] = x;
            __syncwarp();
            if (lane == 0) {
                T a = 0;
#pragma unroll
                for (int k = 0; k < 32; ++k) a = add_rn(a, b[k]);
                s = a;
            }
        } else if constexpr (M == SR_WR_NOSYNC) {
            b[lane] = x;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1)
                if (lane < off) b[lane] = add_rn(b[lane], b[lane + off]);
            s = b[0];
        } else if constexpr (M == SR_WR_VOLATILE_TILE) {
            volatile T* v = b;
            v[lane] = x;
            tile.sync();
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                if (lane < off) v[lane] = add_rn(v[lane], v[lane + off]);
                tile.sync();
            }
            s = v[0];
        } else if constexpr (M == SR_WR_TILE || M == SR_WR_COALESCED) {
            b[lane] = x;
            if constexpr (M == SR_WR_TILE) tile.sync(); else co.sync();
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                if (lane < off) b[lane] = add_rn(b[lane], b[lane + off]);
                if constexpr (M == SR_WR_TILE) tile.sync(); else co.sync();
            }
            s = b[0];
        } else if constexpr (M == SR_WR_TILE_SHUFFLE) {
            s = x;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) s = add_rn(s, tile.shfl_down(s, off));
        } else {
            s = x;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) s = add_rn(s, co.shfl_down(s, off));
        }
        if (lane == 0) bad += (s != (T)528) ? 1u : 0u;
    }
    const long long c1 = clock64();
    if (lane == 0) {
        p.t[2 * gw] = c0;
        p.t[2 * gw + 1] = c1;
        if (bad) atomicAdd(p.bad, bad);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.gt[0] = g0;
        p.gt[1] = gtimer();
        p.gt[2] = (unsigned long long)c0;
        p.gt[3] = (unsigned long long)c1;
    }
}

// One wait unit = a 1 us nanosleep (the paper's null-kernel filler).
__global__ void sleep_kernel(int units) {
    for (int u = 0; u < units; ++u) __nanosleep(1000);
}

const void* bar_fn(int level) {
    switch (level) {
    case SR_LEVEL_WARP: return (const void*)bar_kernel<SR_LEVEL_WARP>;
    case SR_LEVEL_COALESCED: return (const void*)bar_kernel<SR_LEVEL_COALESCED>;
    case SR_LEVEL_BLOCK: return (const void*)bar_kernel<SR_LEVEL_BLOCK>;
    case SR_LEVEL_CLUSTER: return (const void*)bar_kernel<SR_LEVEL_CLUSTER>;
    case SR_LEVEL_GRID: return (const void*)bar_kernel<SR_LEVEL_GRID>;
    case SR_LEVEL_SHUFFLE: return (const void*)bar_kernel<SR_LEVEL_SHUFFLE>;
    case SR_LEVEL_FADD: return (const void*)bar_kernel<SR_LEVEL_FADD>;
    default: return nullptr;
    }
}

template <class T> const void* warp_reduce_fn_t(int m) {
    switch (m) {
    case SR_WR_SERIAL: return (const void*)warp_reduce_kernel<SR_WR_SERIAL, T>;
    case SR_WR_NOSYNC: return (const void*)warp_reduce_kernel<SR_WR_NOSYNC, T>;
    case SR_WR_VOLATILE_TILE: return (const void*)warp_reduce_kernel<SR_WR_VOLATILE_TILE, T>;
    case SR_WR_TILE: return (const void*)warp_reduce_kernel<SR_WR_TILE, T>;
    case SR_WR_COALESCED: return (const void*)warp_reduce_kernel<SR_WR_COALESCED, T>;
    case SR_WR_TILE_SHUFFLE: return (const void*)warp_reduce_kernel<SR_WR_TILE_SHUFFLE, T>;
    case SR_WR_COALESCED_SHUFFLE: return (const void*)warp_reduce_kernel<SR_WR_COALESCED_SHUFFLE, T>;
    default: return nullptr;
    }
}

const void* warp_reduce_fn(int method) {
    return (method & SR_WR_FP32) ? warp_reduce_fn_t<float>(method & ~SR_WR_FP32)
                                 : warp_reduce_fn_t<double>(method);
}

thread_local sr_barrier_result g_last;

double now_ns() {
    return (double)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Bench {
    cudaStream_t s = nullptr;
    long long* t = nullptr;
    unsigned long long* gt = nullptr;
    float* sink = nullptr;
    unsigned int* bad = nullptr;
    ~Bench() {
        if (t) cudaFree(t);
        if (gt) cudaFree(gt);
        if (sink) cudaFree(sink);
        if (bad) cudaFree(bad);
        if (s) cudaStreamDestroy(s);
    }
};

int launch_bar(const Bench& b, const sr_barrier_config& c, const void* fn, int64_t iters) {
    BarParams p;
    p.iters = iters;
    p.group = c.group;
    p.t = b.t;
    p.gt = b.gt;
    p.sink = b.sink;
    p.bad = b.bad;
    void* args[] = {&p};
    cudaError_t e;
    if (c.level == SR_LEVEL_GRID) {
        e = cudaLaunchCooperativeKernel(fn, dim3(c.blocks), dim3(c.threads), args, 0, b.s);
    } else {
        cudaLaunchConfig_t lc;
        std::memset(&lc, 0, sizeof lc);
        lc.gridDim = dim3(c.blocks);
        lc.blockDim = dim3(c.threads);
        lc.stream = b.s;
        cudaLaunchAttribute a[1];
        if (c.level == SR_LEVEL_CLUSTER) {
            a[0].id = cudaLaunchAttributeClusterDimension;
            a[0].val.clusterDim.x = c.cluster;
            a[0].val.clusterDim.y = 1;
            a[0].val.clusterDim.z = 1;
            lc.attrs = a;
            lc.numAttrs = 1;
        }
        e = cudaLaunchKernelExC(&lc, fn, args);
    }
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

// Kernel total latency (host clock around launch + synchronise), ns.
int timed_run(const Bench& b, const sr_barrier_config& c, const void* fn, int64_t iters, double* ns) {
    const double t0 = now_ns();
    int st = launch_bar(b, c, fn, iters);
    if (st != SR_OK) return st;
    cudaError_t e = cudaStreamSynchronize(b.s);
    if (e != cudaSuccess) return status_from_cuda(e);
    *ns = now_ns() - t0;
    return SR_OK;
}

void mean_sd(const std::vector<double>& v, double* m, double* sd) {
    double a = 0;
    for (double x : v) a += x;
    a /= v.size();
    double q = 0;
    for (double x : v) q += (x - a) * (x - a);
    *m = a;
    *sd = v.size() > 1 ? std::sqrt(q / (v.size() - 1)) : 0.0;
}

// One launch of the wait-unit kernel by launch function `kind` (Table I).
cudaError_t launch_sleep(const sr_barrier_config& c, int units, cudaStream_t s) {
    void* args[] = {&units};
    if (c.method == SR_LAUNCH_COOPERATIVE)
        return cudaLaunchCooperativeKernel((const void*)sleep_kernel, dim3(c.blocks), dim3(32), args, 0, s);
    if (c.method == SR_LAUNCH_CLUSTER) {
        cudaLaunchConfig_t lc;
        std::memset(&lc, 0, sizeof lc);
        lc.gridDim = dim3(c.blocks);
        lc.blockDim = dim3(32);
        lc.stream = s;
        cudaLaunchAttribute a[1];
        a[0].id = cudaLaunchAttributeClusterDimension;
        a[0].val.clusterDim.x = c.cluster;
        a[0].val.clusterDim.y = 1;
        a[0].val.clusterDim.z = 1;
        lc.attrs = a;
        lc.numAttrs = 1;
        return cudaLaunchKernelExC(&lc, (const void*)sleep_kernel, args);
    }
    return cudaLaunchKernel((const void*)sleep_kernel, dim3(c.blocks), dim3(32), args, 0, s);
}

int kernel_level(const sr_barrier_config& c, sr_barrier_result* r) {
    // Eq. 6 with i = 20 launches of j = 5 units against 5 launches of 20 units,
    // and the null-kernel total latency of Fig. "Sample code to micro-benchmark
    // implicit barriers": ((t3 - t2) - (t2 - t1)) / (5 - 1).
    Bench b;
    cudaError_t e = cudaStreamCreateWithFlags(&b.s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return status_from_cuda(e);
    const int i = 20, j = 5;
    auto run = [&](int launches, int units, double* ns) -> int {
        const double t0 = now_ns();
        for (int k = 0; k < launches; ++k) {
            cudaError_t ee = launch_sleep(c, units, b.s);
            if (ee != cudaSuccess) return status_from_cuda(ee);
        }
        cudaError_t ee = cudaStreamSynchronize(b.s);
        if (ee != cudaSuccess) return status_from_cuda(ee);
        *ns = now_ns() - t0;
        return SR_OK;
    };
    double w;
    for (int k = 0; k < 3; ++k) {  // warm-up launches, not reported (Section IV)
        int st = run(1, 1, &w);
        if (st != SR_OK) return st;
    }
    std::vector<double> O, null_total;
    for (int rep = 0; rep < c.reps; ++rep) {
        double lij, lji, t1, t5;
        int st = run(i, j, &lij);
        if (st == SR_OK) st = run(j, i, &lji);
        if (st == SR_OK) st = run(1, 0, &t1);
        if (st == SR_OK) st = run(5, 0, &t5);
        if (st != SR_OK) return st;
        O.push_back((lij - lji) / (i - j));
        null_total.push_back((t5 - t1) / (5 - 1));
    }
    double m, sd;
    mean_sd(O, &m, &sd);
    r->ns_per_sync = m;
    r->ns_sigma = sd;
    mean_sd(null_total, &m, &sd);
    r->null_kernel_total_ns = m;
    r->cycles_per_sync = NAN;
    r->syncs_per_cycle_per_sm = NAN;
    r->clock_mhz = NAN;
    r->blocks = c.blocks;
    r->threads = 32;
    r->correct = -1;
    return SR_OK;
}

}  // namespace
}  // namespace sr

using namespace sr;

extern "C" {

int sr_barrier_bench_ex(const sr_barrier_config* cfg, sr_barrier_result* out) {
    if (!cfg || !out) return SR_ERR_ARG;
    sr_barrier_config c = *cfg;
    if (c.level < SR_LEVEL_WARP || c.level > SR_LEVEL_WARP_REDUCE) return SR_ERR_ARG;
    if (c.level == SR_LEVEL_WARP_REDUCE) {
        const int m = c.method & ~SR_WR_FP32;
        if (c.method < 0 || m < SR_WR_SERIAL || m > SR_WR_COALESCED_SHUFFLE) return SR_ERR_ARG;
    } else if (c.level == SR_LEVEL_KERNEL) {
        if (c.method < SR_LAUNCH_TRADITIONAL || c.method > SR_LAUNCH_CLUSTER) return SR_ERR_ARG;
    } else if (c.method != 0) {
        return SR_ERR_ARG;
    }
    if (c.iters == 0) c.iters = 100000;
    if (c.reps == 0) c.reps = 10;
    if (c.iters < 10 || c.iters > (int64_t)1 << 32 || c.reps < 2 || c.reps > 1000) return SR_ERR_ARG;
    const bool warp_level = c.level == SR_LEVEL_WARP || c.level == SR_LEVEL_COALESCED ||
                            c.level == SR_LEVEL_SHUFFLE || c.level == SR_LEVEL_FADD ||
                            c.level == SR_LEVEL_WARP_REDUCE;
    if (c.threads == 0) c.threads = warp_level ? 32 : (c.level == SR_LEVEL_GRID ? 256 : 1024);
    if (c.threads < 32 || c.threads > 1024 || c.threads % 32) return SR_ERR_ARG;
    if (c.group == 0) c.group = 32;
    if (c.group < 1 || c.group > 32) return SR_ERR_ARG;
    if (c.level == SR_LEVEL_WARP && (c.group & (c.group - 1))) return SR_ERR_ARG;  // tiles are powers of 2
    const bool cluster_launch = c.level == SR_LEVEL_CLUSTER ||
                                (c.level == SR_LEVEL_KERNEL && c.method == SR_LAUNCH_CLUSTER);
    if (c.cluster == 0) c.cluster = cluster_launch ? 2 : 1;
    if (c.cluster < 1 || c.cluster > 16 || (c.cluster & (c.cluster - 1))) return SR_ERR_ARG;
    if (!cluster_launch && c.cluster != 1) return SR_ERR_ARG;
    if (c.blocks < 0 || (cluster_launch && c.blocks % c.cluster)) return SR_ERR_ARG;

    std::memset(out, 0, sizeof *out);
    int st = SR_OK;
    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    if (c.blocks == 0) c.blocks = c.level == SR_LEVEL_GRID ? d->sms : (cluster_launch ? c.cluster : 1);

    if (c.level == SR_LEVEL_KERNEL) {
        // never start a cooperative grid that cannot be co-resident, nor a
        // cluster shape the device cannot schedule
        const void* sfn = (const void*)sleep_kernel;
        st = prepare_function(sfn, 0, c.cluster > 8);
        if (st != SR_OK) return st;
        if (c.method == SR_LAUNCH_COOPERATIVE) {
            int per_sm = 0;
            st = blocks_per_sm(*d, sfn, 32, 0, &per_sm);
            if (st != SR_OK) return st;
            if ((int64_t)per_sm * d->sms < c.blocks) return SR_ERR_LAUNCH;
        } else if (c.method == SR_LAUNCH_CLUSTER) {
            cudaLaunchConfig_t lc;
            std::memset(&lc, 0, sizeof lc);
            lc.gridDim = dim3(c.blocks);
            lc.blockDim = dim3(32);
            cudaLaunchAttribute a[1];
            a[0].id = cudaLaunchAttributeClusterDimension;
            a[0].val.clusterDim.x = c.cluster;
            a[0].val.clusterDim.y = 1;
            a[0].val.clusterDim.z = 1;
            lc.attrs = a;
            lc.numAttrs = 1;
            int nc = 0;
            st = active_clusters(*d, sfn, &lc, &nc);
            if (st != SR_OK) return st;
            if (nc < 1) return SR_ERR_LAUNCH;
        }
        st = kernel_level(c, out);
        if (st == SR_OK) g_last = *out;
        return st;
    }
    const void* fn = c.level == SR_LEVEL_WARP_REDUCE ? warp_reduce_fn(c.method) : bar_fn(c.level);
    st = prepare_function(fn, 0, c.cluster > 8);
    if (st != SR_OK) return st;
    if (c.level == SR_LEVEL_GRID) {
        int per_sm = 0;
        st = blocks_per_sm(*d, fn, c.threads, 0, &per_sm);
        if (st != SR_OK) return st;
        if ((int64_t)per_sm * d->sms < c.blocks) return SR_ERR_LAUNCH;  // never start a grid that cannot meet
    }
    if (c.level == SR_LEVEL_CLUSTER) {
        cudaLaunchConfig_t lc;
        std::memset(&lc, 0, sizeof lc);
        lc.gridDim = dim3(c.blocks);
        lc.blockDim = dim3(c.threads);
        cudaLaunchAttribute a[1];
        a[0].id = cudaLaunchAttributeClusterDimension;
        a[0].val.clusterDim.x = c.cluster;
        a[0].val.clusterDim.y = 1;
        a[0].val.clusterDim.z = 1;
        lc.attrs = a;
        lc.numAttrs = 1;
        int nc = 0;
        st = active_clusters(*d, fn, &lc, &nc);
        if (st != SR_OK) return st;
        if (nc < 1) return SR_ERR_LAUNCH;
    }

    Bench b;
    cudaError_t e = cudaStreamCreateWithFlags(&b.s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return status_from_cuda(e);
    const int64_t nwarps = (int64_t)c.blocks * (c.threads / 32);
    if ((e = cudaMalloc(&b.t, sizeof(long long) * 2 * nwarps)) != cudaSuccess) return status_from_cuda(e);
    if ((e = cudaMalloc(&b.gt, sizeof(unsigned long long) * 4)) != cudaSuccess) return status_from_cuda(e);
    if ((e = cudaMalloc(&b.sink, sizeof(float))) != cudaSuccess) return status_from_cuda(e);
    if ((e = cudaMalloc(&b.bad, sizeof(unsigned int))) != cudaSuccess) return status_from_cuda(e);

    double w;
    for (int k = 0; k < 2; ++k) {  // warm-up (Section IV: the first launch is not reported)
        st = timed_run(b, c, fn, 10, &w);
        if (st != SR_OK) return st;
    }
    // Wong's method: clock64 around r1 repetitions, from the last of N runs.
    const int64_t r1 = c.iters, r2 = std::max<int64_t>(1, c.iters / 10);
    std::vector<double> L1, L2;
    for (int rep = 0; rep < c.reps; ++rep) {
        double a, bb;
        st = timed_run(b, c, fn, r1, &a);
        if (st == SR_OK) st = timed_run(b, c, fn, r2, &bb);
        if (st != SR_OK) return st;
        L1.push_back(a);
        L2.push_back(bb);
    }
    if ((e = cudaMemsetAsync(b.bad, 0, sizeof(unsigned int), b.s)) != cudaSuccess) return status_from_cuda(e);
    st = timed_run(b, c, fn, r1, &w);
    if (st != SR_OK) return st;
    unsigned int nbad = 0;
    if ((e = cudaMemcpy(&nbad, b.bad, sizeof nbad, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return status_from_cuda(e);
    std::vector<long long> t(2 * nwarps);
    unsigned long long gt[4];
    if ((e = cudaMemcpy(t.data(), b.t, sizeof(long long) * 2 * nwarps, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return status_from_cuda(e);
    if ((e = cudaMemcpy(gt, b.gt, sizeof gt, cudaMemcpyDeviceToHost)) != cudaSuccess) return status_from_cuda(e);

    // Latency: the slowest measuring warp's cycles per repetition.  Throughput:
    // warp-level syncs completed per SM per cycle (a block / cluster / grid
    // sync counts once per participating warp, Table II's per-warp view).
    long long worst = 1;
    for (int64_t wdx = 0; wdx < nwarps; ++wdx) worst = std::max(worst, t[2 * wdx + 1] - t[2 * wdx]);
    const int64_t measured = nwarps;
    const int sms_used = std::min<int64_t>(c.blocks, d->sms);
    out->cycles_per_sync = (double)worst / (double)r1;
    out->syncs_per_cycle_per_sm = (double)measured * (double)r1 / (double)worst / (double)sms_used;
    const double dns = (double)(gt[1] - gt[0]);
    const double dcyc = (double)((long long)gt[3] - (long long)gt[2]);
    out->clock_mhz = dns > 0 ? dcyc / dns * 1e3 : NAN;
    // Eq. 7 and Eq. 8 on the host-clock kernel total latencies
    double m1, s1, m2, s2;
    mean_sd(L1, &m1, &s1);
    mean_sd(L2, &m2, &s2);
    out->ns_per_sync = (m1 - m2) / (double)(r1 - r2);
    out->ns_sigma = std::sqrt(s1 * s1 + s2 * s2) / (double)(r1 - r2);
    out->null_kernel_total_ns = NAN;
    out->blocks = c.blocks;
    out->threads = c.threads;
    out->correct = c.level == SR_LEVEL_WARP_REDUCE ? (nbad == 0 ? 1 : 0) : -1;
    g_last = *out;
    return SR_OK;
}

int sr_barrier_bench(int level, int64_t iters) {
    sr_barrier_config c;
    std::memset(&c, 0, sizeof c);
    c.level = level;
    c.iters = iters;
    sr_barrier_result r;
    return sr_barrier_bench_ex(&c, &r);
}

int sr_barrier_bench_last(sr_barrier_result* out) {
    if (!out) return SR_ERR_ARG;
    *out = g_last;
    return SR_OK;
}

int sr_differential_latency(const double* L1, int64_t n1, const double* L2, int64_t n2, int64_t r1, int64_t r2,
                            double* t, double* sigma) {
    if (!L1 || !L2 || !t || !sigma || n1 < 2 || n2 < 2 || r1 == r2) return SR_ERR_ARG;
    std::vector<double> a(L1, L1 + n1), b(L2, L2 + n2);
    double m1, s1, m2, s2;
    mean_sd(a, &m1, &s1);
    mean_sd(b, &m2, &s2);
    *t = (m1 - m2) / (double)(r1 - r2);
    *sigma = std::sqrt(s1 * s1 + s2 * s2) / std::fabs((double)(r1 - r2));
    return SR_OK;
}

}  // extern "C"
