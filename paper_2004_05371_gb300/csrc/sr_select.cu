// Per-call launch selection: a trained MLP (served by its inference kernel)
// or, without one, exhaustive autotuning on the call's own data — both
// memoised per call shape, so a shape pays the choice once.  Selectors are
// saved to and loaded from text files; SR_MODEL_FILE names one that calls
// made without a selector use instead of the autotuner.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "sr_internal.h"

namespace sr {
namespace {

using ShapeKey = std::tuple<int, int64_t, int, int64_t, int64_t, int64_t, int64_t>;  // dev, n, dtype, nseg, stats

ShapeKey make_key(int dev, int64_t n, int dtype, int64_t nseg, double mean, double sd, double mx) {
    // segment statistics enter at 1/16-octave resolution
    auto q = [](double v) { return (int64_t)std::llround(16.0 * std::log2(1.0 + v)); };
    return ShapeKey(dev, n, dtype, nseg, q(mean), q(sd), q(mx));
}

int current_dev(int* dev) {
    cudaError_t e = cudaGetDevice(dev);
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

}  // namespace
}  // namespace sr

namespace {
// Per device: the selector SR_MODEL_FILE names, loaded at its first use
// (status, selector); kept until the process exits.
std::mutex g_env_sel_mu;
std::map<int, std::pair<int, sr_selector>> g_env_sel;

// The selector of a call made without one: SR_MODEL_FILE's when the
// variable is set (its load status otherwise), else none (the autotuner).
int env_selector(sr_selector* s) {
    *s = nullptr;
    const char* path = std::getenv("SR_MODEL_FILE");
    if (!path || !*path) return SR_OK;
    int dev = 0;
    int st = sr::current_dev(&dev);
    if (st != SR_OK) return st;
    std::lock_guard<std::mutex> lk(g_env_sel_mu);
    auto it = g_env_sel.find(dev);
    if (it == g_env_sel.end()) {
        sr_selector sel = nullptr;
        const int ls = sr_selector_load(path, &sel);
        it = g_env_sel.emplace(dev, std::make_pair(ls, sel)).first;
    }
    *s = it->second.second;
    return it->second.first;
}
}  // namespace

using namespace sr;

struct sr_selector_s {
    sr_mlp mlp = nullptr;
    bool owns_mlp = false;  // made by sr_selector_load
    float mu[SR_SELECTOR_FEATURES];
    float sd[SR_SELECTOR_FEATURES];
    std::vector<sr_config> cands;
    float* d_x = nullptr;  // device feature row
    int* d_cls = nullptr;  // device class
    std::mutex mu_memo;
    std::map<ShapeKey, int> memo;
};

extern "C" {

int sr_selector_create(sr_mlp mlp, const float* mu, const float* sd, const sr_config* cands, int ncand,
                       sr_selector* out) {
    if (!mlp || !mu || !sd || !cands || ncand < 2 || !out) return SR_ERR_ARG;
    *out = nullptr;
    int din = 0, dh = 0, dout = 0;
    if (sr_mlp_dims(mlp, &din, &dh, &dout) != SR_OK || din != SR_SELECTOR_FEATURES || dout != ncand)
        return SR_ERR_ARG;
    sr_selector s = new sr_selector_s;
    s->mlp = mlp;
    for (int i = 0; i < SR_SELECTOR_FEATURES; ++i) {
        s->mu[i] = mu[i];
        s->sd[i] = sd[i] > 0.f ? sd[i] : 1.f;
    }
    s->cands.assign(cands, cands + ncand);
    cudaError_t e = cudaMalloc(&s->d_x, sizeof(float) * SR_SELECTOR_FEATURES);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_cls, sizeof(int));
    if (e != cudaSuccess) {
        sr_selector_destroy(s);
        return status_from_cuda(e);
    }
    *out = s;
    return SR_OK;
}

int sr_selector_destroy(sr_selector s) {
    if (!s) return SR_OK;
    cudaFree(s->d_x);
    cudaFree(s->d_cls);
    if (s->owns_mlp) sr_mlp_destroy(s->mlp);  // otherwise the MLP stays owned by the caller
    delete s;
    return SR_OK;
}

int sr_selector_save(sr_selector s, const char* path) {
    if (!s || !path || !*path) return SR_ERR_ARG;
    int dev = 0;
    int st = current_dev(&dev);
    if (st != SR_OK) return st;
    SelectorFile f;
    st = device_identity(dev, &f.ident);
    if (st != SR_OK) return st;
    st = sr_mlp_dims(s->mlp, &f.din, &f.dh, &f.dout);
    if (st != SR_OK) return st;
    std::memcpy(f.mu, s->mu, sizeof f.mu);
    std::memcpy(f.sd, s->sd, sizeof f.sd);
    f.cands = s->cands;
    f.params.resize((size_t)sr_mlp_param_count(s->mlp));
    st = sr_mlp_get_params(s->mlp, f.params.data(), (int64_t)f.params.size());
    if (st != SR_OK) return st;
    return write_selector_file(path, f);
}

int sr_selector_load(const char* path, sr_selector* out) {
    if (!out) return SR_ERR_ARG;
    *out = nullptr;
    SelectorFile f;
    int st = read_selector_file(path, &f);  // the whole file parses before any device call
    if (st != SR_OK) return st;
    int dev = 0;
    st = current_dev(&dev);
    if (st != SR_OK) return st;
    std::string id;
    st = device_identity(dev, &id);
    if (st != SR_OK) return st;
    if (id != f.ident) return SR_ERR_UNSUPPORTED;  // trained on another GPU model or driver
    sr_mlp m = nullptr;
    st = sr_mlp_create(f.din, f.dh, f.dout, &m);
    if (st != SR_OK) return st;
    if (sr_mlp_param_count(m) != (int64_t)f.params.size()) st = SR_ERR_ARG;
    if (st == SR_OK) st = sr_mlp_set_params(m, f.params.data(), (int64_t)f.params.size());
    sr_selector s = nullptr;
    if (st == SR_OK) st = sr_selector_create(m, f.mu, f.sd, f.cands.data(), (int)f.cands.size(), &s);
    if (st != SR_OK) {
        sr_mlp_destroy(m);
        return st;
    }
    s->owns_mlp = true;
    *out = s;
    return SR_OK;
}

int sr_selector_choose(sr_selector s, int64_t n, int dtype, int64_t nseg, double len_mean, double len_std,
                       double len_max, sr_config* out, sr_stream_t stream) {
    if (!s || !out) return SR_ERR_ARG;
    int dev = 0;
    int st = current_dev(&dev);
    if (st != SR_OK) return st;
    const ShapeKey key = make_key(dev, n, dtype, nseg, len_mean, len_std, len_max);
    {
        std::lock_guard<std::mutex> lk(s->mu_memo);
        auto it = s->memo.find(key);
        if (it != s->memo.end()) {
            *out = s->cands[it->second];
            return SR_OK;
        }
    }
    float f[SR_SELECTOR_FEATURES];
    st = sr_selector_features(n, dtype, nseg, len_mean, len_std, len_max, f);
    if (st != SR_OK) return st;
    for (int i = 0; i < SR_SELECTOR_FEATURES; ++i) f[i] = (f[i] - s->mu[i]) / s->sd[i];
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(s->d_x, f, sizeof f, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return status_from_cuda(e);
    st = sr_mlp_predict(s->mlp, s->d_x, 1, s->d_cls, nullptr, stream);  // the inference kernel
    if (st != SR_OK) return st;
    int cls = 0;
    e = cudaMemcpyAsync(&cls, s->d_cls, sizeof cls, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return status_from_cuda(e);
    if (cls < 0 || cls >= (int)s->cands.size()) return SR_ERR_ARG;  // model trained for another candidate set
    {
        std::lock_guard<std::mutex> lk(s->mu_memo);
        s->memo[key] = cls;
    }
    *out = s->cands[cls];
    return SR_OK;
}

// Fallback: exhaustive autotuning over the 40 candidates on this call's data.
static int tuned_config(const void* x, int64_t n, const int64_t* offsets, int64_t nseg, int dtype, void* out,
                        double mean, double sd, double mx, sr_config* cfg, sr_stream_t stream) {
    int dev = 0;
    int st = current_dev(&dev);
    if (st != SR_OK) return st;
    bool found = false;
    st = tune_lookup(dev, n, dtype, nseg, mean, sd, mx, cfg, &found);
    if (st != SR_OK || found) return st;
    const DeviceInfo* d = current_device(&st);
    if (!d) return st;
    const int nc = sr_candidates(0, d->sms, nullptr, 0);
    std::vector<sr_config> c(nc);
    if (sr_candidates(0, d->sms, c.data(), nc) != nc) return SR_ERR_ARG;
    std::vector<float> us(nc);
    st = sr_autotune(x, n, offsets, nseg, dtype, out, c.data(), nc, 2, us.data(), stream);
    if (st != SR_OK) return st;
    int best = 0;
    for (int i = 1; i < nc; ++i)
        if (us[i] < us[best]) best = i;
    if (!std::isfinite(us[best])) return SR_ERR_LAUNCH;
    *cfg = c[best];
    return tune_insert(dev, n, dtype, nseg, mean, sd, mx, c[best]);
}

int sr_reduce_sum_selected(sr_selector s, const void* x, int64_t n, int dtype, void* out, sr_stream_t stream) {
    if (n < 0) return SR_ERR_ARG;
    sr_config c;
    const double dn = (double)n;
    int st = s ? SR_OK : env_selector(&s);
    if (st != SR_OK) return st;
    st = s ? sr_selector_choose(s, n, dtype, 1, dn, 0.0, dn, &c, stream)
           : tuned_config(x, n, nullptr, 1, dtype, out, dn, 0.0, dn, &c, stream);
    if (st != SR_OK) return st;
    return sr_reduce_sum_ex(x, n, dtype, out, &c, stream);
}

int sr_reduce_sum_segmented_selected(sr_selector s, const void* x, const int64_t* offsets, int64_t nseg, int dtype,
                                     void* out, double len_mean, double len_std, double len_max,
                                     sr_stream_t stream) {
    if (nseg < 1) return nseg == 0 ? SR_OK : SR_ERR_ARG;
    const int64_t n = (int64_t)std::llround(len_mean * (double)nseg);
    sr_config c;
    int st = s ? SR_OK : env_selector(&s);
    if (st != SR_OK) return st;
    st = s ? sr_selector_choose(s, n, dtype, nseg, len_mean, len_std, len_max, &c, stream)
           : tuned_config(x, n, offsets, nseg, dtype, out, len_mean, len_std, len_max, &c, stream);
    if (st != SR_OK) return st;
    const sr::DeviceInfo* d = sr::current_device(&st);
    if (!d) return st;
    const int form = sr_segmented_layout_flags(d->sms, dtype, nseg, len_mean, len_std, len_max);
    if (form < 0) return -form;
    if (form == SR_F_WARP_SEGMENTS || form == SR_F_LANE_SEGMENTS) {  // the form's own shape; no grid stage
        c.variant = (c.variant & ~(SR_F_BULK | SR_F_DENSE_SEGMENTS)) | form;
        c.vec_bytes = c.unroll = c.block_threads = c.stages = c.grid = c.ctas_per_sm = 0;
        // the lane form with 32-byte vectors from 128 bytes per segment (measured: 16M x 16
        // FP32 185 us with 16 B against 196; 4M x 64 226 against 179; 1M x 268 208 against 196)
        if (form == SR_F_LANE_SEGMENTS && len_mean * (double)sr::elem_size(dtype) >= 128.0) c.vec_bytes = 32;
    } else {
        c.variant |= form;
    }
    return sr_reduce_sum_segmented_ex(x, offsets, nseg, dtype, out, &c, stream);
}

// Measured at ~2^28 FP32 elements (U[-1,1]) against every form:
//  - 16M segments of 16 elements: one thread per segment (SR_F_LANE_SEGMENTS)
//    184 us, the dense kernel 711, one warp per segment 206;
//  - 4M of 64: thread 179 us (32-byte vectors), warp 229, dense 610;
//  - 1M of 268: thread 196 us (32-byte vectors), warp 211, the best
//    flat-split form 328;
//  - 4M lognormal of median 40 (empty ones included): warp 284 us (its
//    short segments summed by single lanes), thread 991, flat split 973;
//  - 10^4-10^5 lognormal segments: the flat split (LDG below 32,768
//    segments, the TMA ring above); the whole-segment forms are 13-500x
//    slower there, one warp or thread holding a segment of millions.
// The dense kernel (a warp-wide pass over rows with many segment ends) is
// 1.4-5.5x the plain kernel on uniformly short segments of fewer segments.
// The rule keeps each form inside the range it was measured in: the thread
// form for 2^19 or more uniform segments of at most 1 KiB with none above 4x
// the mean; the dense kernel up to 128 bytes (uniform); the warp
// form for 2^19 or more segments none of which exceeds twice a warp's even
// share of the elements (32 resident warps per SM, its occupancy at its
// default shape); the dense kernel up to 512 bytes (uniform); else the
// plain form.
int sr_segmented_layout_flags(int sms, int dtype, int64_t nseg, double len_mean, double len_std, double len_max) {
    if (dtype < SR_F32 || dtype > SR_FP8E4M3) return -SR_ERR_DTYPE;
    if (sms < 1 || nseg < 0 || !(len_mean >= 0.0) || !(len_std >= 0.0) || len_max != len_max) return -SR_ERR_ARG;
    const double bytes = len_mean * (double)sr::elem_size(dtype);
    const bool uniform = len_std <= 0.5 * len_mean;
    const bool many = nseg >= (int64_t)1 << 19;
    const double longest = len_max > 0.0 ? len_max : len_mean + 4.0 * len_std;
    if (many && bytes <= 1024.0 && uniform && longest <= 4.0 * len_mean) return SR_F_LANE_SEGMENTS;
    if (bytes <= 128.0 && uniform) return SR_F_DENSE_SEGMENTS;
    const double share = len_mean * (double)nseg / (32.0 * (double)sms);
    if (many && longest <= 2.0 * share) return SR_F_WARP_SEGMENTS;
    if (bytes <= 512.0 && uniform) return SR_F_DENSE_SEGMENTS;
    return 0;
}

}  // extern "C"
