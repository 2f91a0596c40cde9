// Configuration and persisted launch-selection state (host only).
//  - SR_VARIANT: the variant of single-array sums whose caller leaves the
//    choice to the library (sr_reduce_sum with SR_AUTO; sr_reduce_sum_ex and
//    sr_plan with cfg == NULL).
//  - The autotuner fallback's memo of the selected entry points, saved to and
//    loaded from a versioned text file (sr_tune_save / sr_tune_load); with
//    SR_TUNE_FILE set it is read from that file at first use and the file is
//    rewritten after every new entry.
// Entries are keyed by the device's identity (name, SM count, driver
// version): a table made on one GPU model and driver is carried along in the
// file but never applied on another.
#include <unistd.h>

#include <atomic>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "sr_internal.h"

namespace sr {
namespace {

constexpr const char* kTuneMagic = "sr-tune";
constexpr int kTuneVersion = 1;

std::mutex g_mu;
std::map<int, std::string> g_dev_ident;  // device ordinal -> identity
std::vector<std::string> g_idents;       // interned identities (tags index this)

// (identity tag, n, dtype, nseg, quantised mean, std, max)
using TuneKey = std::tuple<int, int64_t, int, int64_t, int64_t, int64_t, int64_t>;
std::map<TuneKey, sr_config> g_tuned;

bool g_env_tune_done = false;
bool g_env_tune_save = false;
std::string g_env_tune_path;

bool g_env_variant_done = false;
int g_env_variant_status = SR_OK;
bool g_env_variant_set = false;
int g_env_variant = SR_AUTO;

int intern(const std::string& id) {
    for (size_t i = 0; i < g_idents.size(); ++i)
        if (g_idents[i] == id) return (int)i;
    g_idents.push_back(id);
    return (int)g_idents.size() - 1;
}

// Segment statistics enter the key at 1/16-octave resolution.
int64_t quantise(double v) { return (int64_t)std::llround(16.0 * std::log2(1.0 + v)); }

// Whole non-negative decimal integer (no sign, no trailing characters).
bool parse_i64(const std::string& s, int64_t* v) {
    if (s.empty() || s.size() > 19) return false;
    int64_t r = 0;
    for (char ch : s) {
        if (ch < '0' || ch > '9') return false;
        r = r * 10 + (ch - '0');
    }
    *v = r;
    return true;
}

bool parse_int(const std::string& s, int* v) {
    // a decimal int that may be negative (quantised statistics are >= 0, config fields too)
    if (s.empty()) return false;
    const bool neg = s[0] == '-';
    int64_t r = 0;
    if (!parse_i64(neg ? s.substr(1) : s, &r) || r > 0x7fffffff) return false;
    *v = (int)(neg ? -r : r);
    return true;
}

bool parse_float(const std::string& s, float* v) {
    if (s.empty()) return false;
    char* end = nullptr;
    errno = 0;
    const float r = std::strtof(s.c_str(), &end);
    if (end != s.c_str() + s.size() || errno == ERANGE || !(r == r)) return false;
    *v = r;
    return true;
}

std::vector<std::string> split_ws(const std::string& line) {
    std::vector<std::string> f;
    std::istringstream is(line);
    std::string t;
    while (is >> t) f.push_back(t);
    return f;
}

// "device <sms> <driver> <name...>" -> identity "<sms> <driver> <name>"
bool parse_device_line(const std::string& line, std::string* id) {
    std::vector<std::string> f = split_ws(line);
    int64_t sms = 0, drv = 0;
    if (f.size() < 4 || f[0] != "device" || !parse_i64(f[1], &sms) || !parse_i64(f[2], &drv) || sms < 1)
        return false;
    std::string name = f[3];
    for (size_t i = 4; i < f.size(); ++i) name += " " + f[i];
    *id = f[1] + " " + f[2] + " " + name;
    return true;
}

void format_config(std::ostringstream& os, const sr_config& c) {
    char sc[32];
    std::snprintf(sc, sizeof sc, "%.9g", (double)c.scale);
    os << c.variant << ' ' << c.block_threads << ' ' << c.ctas_per_sm << ' ' << c.grid << ' ' << c.vec_bytes << ' '
       << c.unroll << ' ' << c.tile_bytes << ' ' << c.stages << ' ' << sc;
}

bool parse_config(const std::vector<std::string>& f, size_t at, sr_config* c) {
    if (f.size() != at + 9) return false;
    std::memset(c, 0, sizeof *c);
    int* ints[8] = {&c->variant, &c->block_threads, &c->ctas_per_sm, &c->grid,
                    &c->vec_bytes, &c->unroll,        &c->tile_bytes,  &c->stages};
    for (int i = 0; i < 8; ++i)
        if (!parse_int(f[at + i], ints[i]) || *ints[i] < 0) return false;
    return parse_float(f[at + 8], &c->scale);
}

// Writes `text` to `path` through a temporary file in the same directory and
// a rename, so a reader never sees a partly written file.
std::atomic<unsigned long long> g_tmp_seq{0};

int write_atomically(const std::string& path, const std::string& text) {
    // process id and a per-process sequence number: concurrent writers, in
    // this process or another, never share a temporary file
    const std::string tmp = path + ".tmp." + std::to_string((long long)getpid()) + "." +
                            std::to_string(g_tmp_seq.fetch_add(1));
    FILE* fp = std::fopen(tmp.c_str(), "wb");
    if (!fp) return SR_ERR_ARG;
    const bool ok = std::fwrite(text.data(), 1, text.size(), fp) == text.size();
    const bool closed = std::fclose(fp) == 0;
    if (!ok || !closed || std::rename(tmp.c_str(), path.c_str()) != 0) {
        std::remove(tmp.c_str());
        return SR_ERR_ARG;
    }
    return SR_OK;
}

int read_file(const char* path, std::string* text) {
    if (!path || !*path) return SR_ERR_ARG;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return SR_ERR_ARG;
    std::string s;
    char buf[1 << 14];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof buf, fp)) > 0) s.append(buf, k);
    const bool err = std::ferror(fp) != 0;
    std::fclose(fp);
    if (err) return SR_ERR_ARG;
    *text = std::move(s);
    return SR_OK;
}

// Parses a whole tuning table; nothing is merged unless every line parses.
int parse_tune(const std::string& text, std::vector<std::pair<std::string, std::pair<TuneKey, sr_config>>>* out) {
    std::istringstream is(text);
    std::string line;
    bool header = false;
    std::string id;
    while (std::getline(is, line)) {
        if (!line.empty() && line.back() == '\r') line.pop_back();
        std::vector<std::string> f = split_ws(line);
        if (f.empty() || f[0][0] == '#') continue;
        if (!header) {
            int64_t v = 0;
            if (f.size() != 2 || f[0] != kTuneMagic || !parse_i64(f[1], &v) || v != kTuneVersion) return SR_ERR_ARG;
            header = true;
            continue;
        }
        if (f[0] == "device") {
            if (!parse_device_line(line, &id)) return SR_ERR_ARG;
            continue;
        }
        // e <n> <dtype> <nseg> <q_mean> <q_std> <q_max> <config: 9 fields>
        int64_t n = 0, nseg = 0, qm = 0, qs = 0, qx = 0;
        int dtype = 0;
        sr_config c;
        if (id.empty() || f[0] != "e" || f.size() != 16 || !parse_i64(f[1], &n) || !parse_int(f[2], &dtype) ||
            dtype < SR_F32 || dtype > SR_FP8E4M3 || !parse_i64(f[3], &nseg) || nseg < 1 || !parse_i64(f[4], &qm) ||
            !parse_i64(f[5], &qs) || !parse_i64(f[6], &qx) || !parse_config(f, 7, &c))
            return SR_ERR_ARG;
        out->push_back({id, {TuneKey(-1, n, dtype, nseg, qm, qs, qx), c}});
    }
    return header ? SR_OK : SR_ERR_ARG;
}

std::string format_tune_locked() {
    std::ostringstream os;
    os << kTuneMagic << ' ' << kTuneVersion << '\n'
       << "# device <SMs> <driver version> <name>\n"
       << "# e <n> <dtype> <segments> <16*log2(1+mean)> <16*log2(1+std)> <16*log2(1+max)> <variant> "
          "<block_threads> <ctas_per_sm> <grid> <vec_bytes> <unroll> <tile_bytes> <stages> <scale>\n";
    for (size_t tag = 0; tag < g_idents.size(); ++tag) {
        bool any = false;
        for (const auto& kv : g_tuned) {
            if (std::get<0>(kv.first) != (int)tag) continue;
            if (!any) os << "device " << g_idents[tag] << '\n';
            any = true;
            const TuneKey& k = kv.first;
            os << "e " << std::get<1>(k) << ' ' << std::get<2>(k) << ' ' << std::get<3>(k) << ' ' << std::get<4>(k)
               << ' ' << std::get<5>(k) << ' ' << std::get<6>(k) << ' ';
            format_config(os, kv.second);
            os << '\n';
        }
    }
    return os.str();
}

int load_tune_locked(const char* path, int64_t* entries) {
    std::string text;
    int st = read_file(path, &text);
    if (st != SR_OK) return st;
    std::vector<std::pair<std::string, std::pair<TuneKey, sr_config>>> parsed;
    st = parse_tune(text, &parsed);
    if (st != SR_OK) return st;
    for (auto& e : parsed) {
        TuneKey k = e.second.first;
        std::get<0>(k) = intern(e.first);
        g_tuned[k] = e.second.second;
    }
    if (entries) *entries = (int64_t)parsed.size();
    return SR_OK;
}

// First use of the memo: read SR_TUNE_FILE.  A missing file is created at the
// first new entry; a file that does not parse is neither used nor rewritten.
void env_tune_locked() {
    if (g_env_tune_done) return;
    g_env_tune_done = true;
    const char* p = std::getenv("SR_TUNE_FILE");
    if (!p || !*p) return;
    g_env_tune_path = p;
    FILE* fp = std::fopen(p, "rb");
    if (!fp) {
        g_env_tune_save = errno == ENOENT;
        return;
    }
    std::fclose(fp);
    g_env_tune_save = load_tune_locked(p, nullptr) == SR_OK;
}

}  // namespace

int device_identity(int dev, std::string* id) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_dev_ident.find(dev);
        if (it != g_dev_ident.end()) {
            *id = it->second;
            return SR_OK;
        }
    }
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, dev);
    int drv = 0;
    if (e == cudaSuccess) e = cudaDriverGetVersion(&drv);
    if (e != cudaSuccess) return status_from_cuda(e);
    std::string name = prop.name;
    for (char& ch : name)
        if (ch == '\n' || ch == '\r' || ch == '\t') ch = ' ';
    std::vector<std::string> words = split_ws(name);
    std::string norm;
    for (const auto& w : words) norm += (norm.empty() ? "" : " ") + w;
    if (norm.empty()) norm = "unnamed";
    const std::string s = std::to_string(prop.multiProcessorCount) + " " + std::to_string(drv) + " " + norm;
    std::lock_guard<std::mutex> lk(g_mu);
    g_dev_ident[dev] = s;
    *id = s;
    return SR_OK;
}

int tune_lookup(int dev, int64_t n, int dtype, int64_t nseg, double mean, double sd, double mx, sr_config* cfg,
                bool* found) {
    *found = false;
    std::string id;
    int st = device_identity(dev, &id);
    if (st != SR_OK) return st;
    std::lock_guard<std::mutex> lk(g_mu);
    env_tune_locked();
    const TuneKey k(intern(id), n, dtype, nseg, quantise(mean), quantise(sd), quantise(mx));
    auto it = g_tuned.find(k);
    if (it != g_tuned.end()) {
        *cfg = it->second;
        *found = true;
    }
    return SR_OK;
}

int tune_insert(int dev, int64_t n, int dtype, int64_t nseg, double mean, double sd, double mx,
                const sr_config& cfg) {
    std::string id;
    int st = device_identity(dev, &id);
    if (st != SR_OK) return st;
    std::lock_guard<std::mutex> lk(g_mu);
    env_tune_locked();
    g_tuned[TuneKey(intern(id), n, dtype, nseg, quantise(mean), quantise(sd), quantise(mx))] = cfg;
    // Persisting is best effort: the call that tuned still runs with its choice.
    if (g_env_tune_save) write_atomically(g_env_tune_path, format_tune_locked());
    return SR_OK;
}

namespace {
constexpr const char* kSelectorMagic = "sr-selector";
constexpr int kSelectorVersion = 1;
}  // namespace

int write_selector_file(const char* path, const SelectorFile& f) {
    if (!path || !*path) return SR_ERR_ARG;
    std::ostringstream os;
    char b[32];
    auto num = [&](float v) {
        std::snprintf(b, sizeof b, "%.9g", (double)v);  // nine digits: every binary32 value round-trips
        return std::string(b);
    };
    os << kSelectorMagic << ' ' << kSelectorVersion << '\n'
       << "device " << f.ident << '\n'
       << "dims " << f.din << ' ' << f.dh << ' ' << f.dout << '\n'
       << "mu";
    for (float v : f.mu) os << ' ' << num(v);
    os << "\nsd";
    for (float v : f.sd) os << ' ' << num(v);
    os << "\ncands " << f.cands.size() << '\n';
    for (const sr_config& c : f.cands) {
        os << "c ";
        format_config(os, c);
        os << '\n';
    }
    os << "params " << f.params.size() << '\n';
    for (size_t i = 0; i < f.params.size(); ++i) os << num(f.params[i]) << ((i % 8 == 7) ? '\n' : ' ');
    os << '\n';
    return write_atomically(path, os.str());
}

int read_selector_file(const char* path, SelectorFile* out) {
    std::string text;
    int st = read_file(path, &text);
    if (st != SR_OK) return st;
    std::istringstream is(text);
    std::string line;
    auto next = [&](std::vector<std::string>* f) {
        while (std::getline(is, line)) {
            if (!line.empty() && line.back() == '\r') line.pop_back();
            *f = split_ws(line);
            if (!f->empty() && (*f)[0][0] != '#') return true;
        }
        return false;
    };
    SelectorFile r;
    std::vector<std::string> f;
    int64_t v = 0;
    if (!next(&f) || f.size() != 2 || f[0] != kSelectorMagic || !parse_i64(f[1], &v) || v != kSelectorVersion)
        return SR_ERR_ARG;
    if (!next(&f) || !parse_device_line(line, &r.ident)) return SR_ERR_ARG;
    if (!next(&f) || f.size() != 4 || f[0] != "dims" || !parse_int(f[1], &r.din) || !parse_int(f[2], &r.dh) ||
        !parse_int(f[3], &r.dout) || r.din != SR_SELECTOR_FEATURES || r.dh < 1 || r.dout < 2)
        return SR_ERR_ARG;
    for (int which = 0; which < 2; ++which) {
        float* dst = which == 0 ? r.mu : r.sd;
        if (!next(&f) || (int)f.size() != 1 + SR_SELECTOR_FEATURES || f[0] != (which == 0 ? "mu" : "sd"))
            return SR_ERR_ARG;
        for (int i = 0; i < SR_SELECTOR_FEATURES; ++i)
            if (!parse_float(f[1 + i], &dst[i])) return SR_ERR_ARG;
    }
    if (!next(&f) || f.size() != 2 || f[0] != "cands" || !parse_i64(f[1], &v) || v != r.dout) return SR_ERR_ARG;
    r.cands.resize((size_t)r.dout);
    for (auto& c : r.cands)
        if (!next(&f) || f[0] != "c" || !parse_config(f, 1, &c)) return SR_ERR_ARG;
    if (!next(&f) || f.size() != 2 || f[0] != "params" || !parse_i64(f[1], &v) || v < 1 || v > (int64_t)1 << 26)
        return SR_ERR_ARG;
    r.params.reserve((size_t)v);
    while ((int64_t)r.params.size() < v && next(&f)) {
        for (const auto& t : f) {
            float p = 0.f;
            if ((int64_t)r.params.size() == v || !parse_float(t, &p)) return SR_ERR_ARG;
            r.params.push_back(p);
        }
    }
    if ((int64_t)r.params.size() != v || next(&f)) return SR_ERR_ARG;  // short, or trailing lines
    *out = std::move(r);
    return SR_OK;
}

int env_variant(int* variant) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_env_variant_done) {
        g_env_variant_done = true;
        const char* s = std::getenv("SR_VARIANT");
        if (s && *s) {
            g_env_variant_set = true;
            g_env_variant_status = sr_parse_variant(s, &g_env_variant);
        }
    }
    if (g_env_variant_status != SR_OK) return g_env_variant_status;
    *variant = g_env_variant_set ? g_env_variant : SR_AUTO;
    return SR_OK;
}

}  // namespace sr

using namespace sr;

extern "C" {

int sr_parse_variant(const char* text, int* variant) {
    if (!text || !variant) return SR_ERR_ARG;
    std::string s(text);
    while (!s.empty() && (s.back() == ' ' || s.back() == '\n' || s.back() == '\t')) s.pop_back();
    size_t b = 0;
    while (b < s.size() && (s[b] == ' ' || s[b] == '\t')) ++b;
    s = s.substr(b);
    if (s.empty()) return SR_ERR_ARG;
    if (s[0] >= '0' && s[0] <= '9') {  // a number: decimal or 0x-prefixed hexadecimal
        char* end = nullptr;
        errno = 0;
        const long v = std::strtol(s.c_str(), &end, 0);
        if (end != s.c_str() + s.size() || errno == ERANGE || v < 0 || v > 0x7fffffff) return SR_ERR_ARG;
        *variant = (int)v;
        return SR_OK;
    }
    // names joined by '+': one grid stage at most, then flags and one cluster size
    static const struct {
        const char* name;
        int bits;
        int kind;  // 0 stage, 1 flag, 2 cluster
    } names[] = {
        {"auto", SR_AUTO, 0},           {"two_kernel", SR_TWO_KERNEL, 0}, {"atomic", SR_ATOMIC, 0},
        {"last_block", SR_LAST_BLOCK, 0}, {"grid_sync", SR_GRID_SYNC, 0},   {"single_cluster", SR_SINGLE_CLUSTER, 0},
        {"kahan", SR_F_KAHAN, 1},        {"fp64_combine", SR_F_FP64_COMBINE, 1},
        {"fp64_auto", SR_F_FP64_AUTO, 1}, {"bulk", SR_F_BULK, 1},
        {"cluster2", SR_CLUSTER(1), 2},   {"cluster4", SR_CLUSTER(2), 2},   {"cluster8", SR_CLUSTER(3), 2},
        {"cluster16", SR_CLUSTER(4), 2},
    };
    int v = 0;
    bool stage = false, cluster = false;
    size_t at = 0;
    while (true) {
        const size_t plus = s.find('+', at);
        const std::string tok = s.substr(at, plus == std::string::npos ? std::string::npos : plus - at);
        bool found = false;
        for (const auto& e : names) {
            if (tok != e.name) continue;
            found = true;
            if (e.kind == 0) {
                if (stage) return SR_ERR_ARG;
                stage = true;
            } else if (e.kind == 2) {
                if (cluster) return SR_ERR_ARG;
                cluster = true;
            } else if (v & e.bits) {
                return SR_ERR_ARG;
            }
            v |= e.bits;
        }
        if (!found) return SR_ERR_ARG;
        if (plus == std::string::npos) break;
        at = plus + 1;
    }
    *variant = v;
    return SR_OK;
}

int sr_tune_save(const char* path) {
    if (!path || !*path) return SR_ERR_ARG;
    std::string text;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        env_tune_locked();
        text = format_tune_locked();
    }
    return write_atomically(path, text);
}

int sr_tune_load(const char* path, int64_t* entries) {
    std::lock_guard<std::mutex> lk(g_mu);
    env_tune_locked();
    return load_tune_locked(path, entries);
}

int64_t sr_tune_size(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    env_tune_locked();
    return (int64_t)g_tuned.size();
}

int sr_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    env_tune_locked();
    g_tuned.clear();
    return SR_OK;
}

}  // extern "C"
