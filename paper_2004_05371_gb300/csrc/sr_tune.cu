// Autotuner and analytic selector.
//
// Candidates: grid stage x grid size x vector width (x unroll for the full
// sweep).  sr_autotune times each candidate on the caller's data with CUDA
// events; sr_select_analytic predicts each candidate's time with the paper's
// performance model (Section VII-A: Little's law, Eq. 1, and the cost
// comparison of Eq. 2 with Eq. 3's T_more = T + T_sync) and returns the
// cheapest.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sr_internal.h"

namespace sr {
namespace {

// Grid sizes of the candidate set, as CTAs of 256 threads: one cluster-sized
// group of 8 CTAs, then 1, 2, 4, 8 CTAs per SM (8 x 256 = 2048 threads/SM,
// full occupancy).  The per-SM levels are filled in per device.
constexpr int kGridLevels = 5;
constexpr int kStages[4] = {SR_TWO_KERNEL, SR_ATOMIC, SR_LAST_BLOCK, SR_GRID_SYNC};
constexpr int kVecs[2] = {16, 32};
constexpr int kUnrolls[4] = {1, 2, 4, 8};

int grid_for_level(int level, int sms) {
    switch (level) {
    case 0: return 8;
    case 1: return sms;
    case 2: return 2 * sms;
    case 3: return 4 * sms;
    default: return 8 * sms;
    }
}

}  // namespace
}  // namespace sr

using namespace sr;

extern "C" {

int sr_candidates(int full, int sms, sr_config* out, int cap) {
    if (sms <= 0 || cap < 0 || (cap > 0 && !out)) return -SR_ERR_ARG;
    const int nu = full ? 4 : 1;
    const int total = 4 * kGridLevels * 2 * nu;
    if (!out) return total;
    int k = 0;
    for (int si = 0; si < 4; ++si)
        for (int g = 0; g < kGridLevels; ++g)
            for (int vi = 0; vi < 2; ++vi)
                for (int ui = 0; ui < nu; ++ui) {
                    if (k >= cap) return -SR_ERR_ARG;
                    sr_config c;
                    std::memset(&c, 0, sizeof c);
                    c.variant = kStages[si];
                    c.block_threads = 256;
                    c.grid = grid_for_level(g, sms);
                    c.vec_bytes = kVecs[vi];
                    c.unroll = full ? kUnrolls[ui] : 4;
                    out[k++] = c;
                }
    return k;
}

int sr_autotune(const void* x, int64_t n, const int64_t* offsets, int64_t nseg, int dtype, void* out,
                const sr_config* cands, int ncand, int reps, float* us, sr_stream_t stream) {
    if (!cands || ncand <= 0 || !us || reps < 1 || reps > 10000) return SR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return status_from_cuda(e);
    }
    int result = SR_OK;
    for (int i = 0; i < ncand && result == SR_OK; ++i) {
        auto call = [&]() -> int {
            return offsets ? sr_reduce_sum_segmented_ex(x, offsets, nseg, dtype, out, &cands[i], stream)
                           : sr_reduce_sum_ex(x, n, dtype, out, &cands[i], stream);
        };
        int st = call();  // warm-up; also rejects candidates that cannot run here
        if (st == SR_ERR_LAUNCH || st == SR_ERR_UNSUPPORTED || st == SR_ERR_ARG) {
            us[i] = INFINITY;
            continue;
        }
        if (st != SR_OK) {
            result = st;
            break;
        }
        cudaEventRecord(a, s);
        for (int r = 0; r < reps && st == SR_OK; ++r) st = call();
        cudaEventRecord(b, s);
        if (st != SR_OK) {
            result = st;
            break;
        }
        e = cudaEventSynchronize(b);
        if (e != cudaSuccess) {
            result = status_from_cuda(e);
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        us[i] = ms * 1000.f / (float)reps;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return result;
}

// Selector features of one call (host only): log2 n, one-hot dtype (4),
// log2 nseg, log2(1 + mean), log2(1 + std), log2(1 + max) of the segment
// lengths (a single array is one segment of length n).
int sr_selector_features(int64_t n, int dtype, int64_t nseg, double len_mean, double len_std, double len_max,
                         float* out) {
    if (!out || n < 0 || nseg < 1 || dtype < SR_F32 || dtype > SR_FP8E4M3 || len_mean < 0 || len_std < 0 ||
        len_max < 0)
        return SR_ERR_ARG;
    out[0] = (float)std::log2((double)std::max<int64_t>(n, 1));
    for (int k = 0; k < 4; ++k) out[1 + k] = (k == dtype) ? 1.f : 0.f;
    out[5] = (float)std::log2((double)nseg);
    out[6] = (float)std::log2(1.0 + len_mean);
    out[7] = (float)std::log2(1.0 + len_std);
    out[8] = (float)std::log2(1.0 + len_max);
    return SR_OK;
}

// A candidate the planner rejects on the current device (a grid.sync() grid
// that cannot be co-resident, Section VIII-B; a shape the kernels do not
// cover) can never run, so the model never chooses it.  With no device
// visible the planner cannot answer and every candidate stays eligible.
static bool rejected_by_planner(const sr_config& c, int64_t n, int dtype, int64_t nseg) {
    sr_config r;
    const int st = nseg > 1 ? sr_plan_segmented(nseg, dtype, &c, &r) : sr_plan(n, dtype, &c, &r);
    return st == SR_ERR_LAUNCH || st == SR_ERR_UNSUPPORTED || st == SR_ERR_ARG;
}

// Performance-model selector (host only: it launches nothing).
int sr_select_analytic(const sr_model_params* mp, int64_t n, int dtype, int64_t nseg, const sr_config* cands,
                       int ncand, float* predicted_us) {
    if (!mp || !cands || ncand <= 0 || n < 0 || nseg < 1 || dtype < SR_F32 || dtype > SR_FP8E4M3) return -SR_ERR_ARG;
    const double N = (double)n * elem_size(dtype);  // bytes
    int best = -1;
    double best_t = INFINITY;
    for (int i = 0; i < ncand; ++i) {
        const sr_config& c = cands[i];
        if (rejected_by_planner(c, n, dtype, nseg)) {
            if (predicted_us) predicted_us[i] = INFINITY;
            continue;
        }
        const int stage = c.variant & SR_STAGE_MASK;
        const double warps = (double)(c.grid > 0 ? c.grid : mp->sms) * (c.block_threads > 0 ? c.block_threads : 256) / 32.0;
        const double per_warp_bytes = 32.0 * (c.vec_bytes > 0 ? c.vec_bytes : 16) * (c.unroll > 0 ? c.unroll : 4);
        // Eq. 1: concurrency C = T * Thr.  The bytes a configuration keeps in
        // flight bound its throughput: Thr = min(peak, in-flight / T).
        const double thr = std::min(mp->hbm_bytes_per_ns, warps * per_warp_bytes / mp->mem_latency_ns);
        const double C = mp->mem_latency_ns * thr;
        double t_sync = mp->last_block_ns;
        if (stage == SR_TWO_KERNEL) t_sync = mp->launch_ns;  // the implicit barrier costs a launch
        else if (stage == SR_GRID_SYNC) t_sync = mp->grid_sync_ns;
        else if (stage == SR_ATOMIC) t_sync = mp->atomic_ns;
        // Eq. 2 / Eq. 3: T_more + max(0, N - C) / Thr with T_more = T + T_sync;
        // partial-result traffic grows with the number of CTAs.
        double t = mp->launch_ns + mp->mem_latency_ns + t_sync + std::max(0.0, N - C) / thr +
                   mp->per_cta_ns * (c.grid > 0 ? c.grid : mp->sms) / std::max(1, mp->sms);
        if (nseg > 1) t += mp->per_segment_ns * (double)nseg / std::max(1.0, warps);
        if (predicted_us) predicted_us[i] = (float)(t / 1e3);
        if (t < best_t) {
            best_t = t;
            best = i;
        }
    }
    return best >= 0 ? best : -SR_ERR_LAUNCH;
}

}  // extern "C"
