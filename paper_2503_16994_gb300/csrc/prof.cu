// Kernel launch accounting: every launch is counted per kernel kind with its
// algorithmic bytes (each operand touched once); when timing is enabled a
// pair of CUDA events brackets each launch on its own stream and the elapsed
// times are summed when the statistics are read.
#include <algorithm>
#include <array>
#include <string>
#include <tuple>
#include <vector>
#include <cstdio>
#include <cstring>
#include <map>

#include "lqcd_impl.h"

namespace lqcd {

namespace {
struct Stat {
    long long launches = 0;
    double ms = 0.0, bytes = 0.0, timed_bytes = 0.0;
    long long timed = 0;
};
struct Pending {
    std::string name;
    cudaEvent_t a, b;
    double bytes;
};
std::mutex g_mu;
std::map<std::string, Stat> g_stats;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
bool g_timing = false;

cudaEvent_t get_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    LQCD_CUDA(cudaEventCreate(&e));
    return e;
}

void drain_locked()
{
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Stat &s = g_stats[p.name];
            s.ms += ms;
            s.timed += 1;
            s.timed_bytes += p.bytes;
        }
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
}
}  // namespace

ProfScope::ProfScope(const char *name_, double bytes_, cudaStream_t st_) : name(name_), bytes(bytes_), st(st_)
{
    std::lock_guard<std::mutex> lk(g_mu);
    Stat &s = g_stats[name];
    s.launches += 1;
    s.bytes += bytes;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (g_timing && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
        a = get_event();
        b = get_event();
        LQCD_CUDA(cudaEventRecord(a, st));
        timed = true;
    }
}

ProfScope::~ProfScope()
{
    if (!timed) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cudaEventRecord(b, st) == cudaSuccess) {
        g_pending.push_back({name, a, b, bytes});
        if (g_pending.size() > 100000) drain_locked();
    }
}

namespace {
std::mutex g_tune_mu;
std::string g_tune;  // JSON objects, comma separated
struct Decision {
    std::string prec;
    int mode, vh, nrhs, nr, gpb, minb, swz;
};
std::vector<Decision> g_decisions;  // made or imported in this process, in order
// imported shapes: (format, mode, sites per parity, nrhs) -> (nr, gpb, minb, swz)
std::map<std::tuple<std::string, int, int, int>, std::array<int, 4>> g_imported;

// a shape the launcher accepts for its storage format (the candidates of the tuner)
bool shape_valid(const std::string &prec, int mode, int vh, int nrhs, int nr, int gpb, int minb, int swz)
{
    if ((mode != 0 && mode != 1) || vh <= 0 || nrhs < 1 || gpb < 1 || gpb > 12) return false;
    if (minb != 1 && minb != 3 && minb != 4 && minb != 6) return false;
    if (swz != 1 && swz != 8 && swz != 32) return false;
    const bool tile = nr == 20 || nr == 21;
    if (prec == "f64") return nr == 1 && (minb == 1 || minb == 6);
    const bool common = (nr >= 0 && nr <= 3) || nr == -2 || nr == -4 || nr == -8;
    if (prec == "f32") return common;
    if (prec == "f16") return common || nr == 12 || nr == 13 || (tile && gpb <= 6);
    return false;
}
}  // namespace

bool tune_imported(const char *prec, int mode, int vh, int nrhs, int shape[4])
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_imported.find(std::make_tuple(std::string(prec), mode, vh, nrhs));
    if (it == g_imported.end()) return false;
    for (int k = 0; k < 4; ++k) shape[k] = it->second[k];
    return true;
}

void tune_record(const char *prec, int mode, int vh, int nrhs, int nr, int gpb, int minb, int swz, float ms)
{
    static const char *modes[] = {"hopclov", "selfclov", "self", "clovsum", "resid"};
    // shape code nr: 1-3 scalar (nr RHS per thread), 0 paired, -2/-4/-8
    // prefetching (loads of that many directions ahead), 12/13 paired with
    // 2/3 directions staged in shared memory, 20/21 tile kernel (links and
    // clover shared by the block, gpb = pairs per block; spinor words staged
    // 1 or 2 directions ahead)
    const bool tile = nr == 20 || nr == 21;
    const char *variant = tile ? "paired_tile"
                               : (nr >= 12 ? "paired_staged" : (nr == 0 ? "paired" : (nr < 0 ? "prefetch" : "scalar")));
    const int per_thread = nr >= 12 || nr == 0 ? 2 : (nr < 0 ? 1 : nr);
    const int ahead = tile ? nr - 19 : (nr >= 12 ? nr - 10 : (nr < 0 ? -nr : 0));
    const int block = tile ? 32 * gpb : kBlock;
    char buf[480];
    std::snprintf(buf, sizeof buf,
                  "{\"kernel\": \"hop_%s_%s\", \"sites\": %d, \"nrhs\": %d, \"variant\": \"%s\", "
                  "\"rhs_per_thread\": %d, \"directions_ahead\": %d, "
                  "\"rhs_groups_per_block\": %d, \"min_blocks_per_sm\": %d, \"tiles_per_supertile\": %d, "
                  "\"block\": %d, \"us\": %.2f, \"source\": \"%s\"}",
                  prec, modes[mode], vh, nrhs, variant, per_thread, ahead, gpb, minb, swz, block,
                  ms >= 0.f ? ms * 1e3 : 0.0, ms >= 0.f ? "timed" : "imported");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune.empty()) g_tune += ", ";
    g_tune += buf;
    g_decisions.push_back(Decision{prec, mode, vh, nrhs, nr, gpb, minb, swz});
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_profile_reset(int enable_timing)
{
    try {
        std::lock_guard<std::mutex> lk(g_mu);
        drain_locked();
        g_stats.clear();
        g_timing = enable_timing != 0;
        return LQCD_OK;
    } catch (const Error &e) {
        return fail(e.code, e.msg);
    }
}

int lqcd_tune_report(char *buf, size_t len)
{
    if (!buf || len == 0) return fail(LQCD_EINVAL, "null buffer");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::string j = "[" + g_tune + "]";
    std::strncpy(buf, j.c_str(), len - 1);
    buf[len - 1] = 0;
    return j.size() < len ? LQCD_OK : LQCD_EINVAL;
}

int lqcd_tune_export(char *buf, size_t len)
{
    if (!buf || len == 0) return fail(LQCD_EINVAL, "null buffer");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::string t = "lqcd-tune 1\n";
    char line[160];
    for (const Decision &d : g_decisions) {
        std::snprintf(line, sizeof line, "%s %d %d %d %d %d %d %d\n", d.prec.c_str(), d.mode, d.vh, d.nrhs, d.nr,
                      d.gpb, d.minb, d.swz);
        t += line;
    }
    std::strncpy(buf, t.c_str(), len - 1);
    buf[len - 1] = 0;
    return t.size() < len ? LQCD_OK : fail(LQCD_EINVAL, "buffer too small");
}

int lqcd_tune_import(const char *text)
{
    if (!text) return fail(LQCD_EINVAL, "null text");
    std::vector<std::pair<std::tuple<std::string, int, int, int>, std::array<int, 4>>> rows;
    const char *p = text;
    int lineno = 0;
    while (*p) {
        const char *e = std::strchr(p, '\n');
        std::string line = e ? std::string(p, e - p) : std::string(p);
        p = e ? e + 1 : p + line.size();
        ++lineno;
        if (line.find_first_not_of(" \t\r") == std::string::npos) continue;
        if (lineno == 1) {
            if (line.rfind("lqcd-tune 1", 0) != 0) return fail(LQCD_EINVAL, "tune import: header 'lqcd-tune 1' expected");
            continue;
        }
        char prec[8] = {0};
        int v[7];
        char extra = 0;
        const int n = std::sscanf(line.c_str(), "%7s %d %d %d %d %d %d %d %c", prec, &v[0], &v[1], &v[2], &v[3], &v[4],
                                  &v[5], &v[6], &extra);
        if (n != 8 || !shape_valid(prec, v[0], v[1], v[2], v[3], v[4], v[5], v[6]))
            return fail(LQCD_EINVAL, "tune import: invalid line " + std::to_string(lineno));
        rows.push_back({std::make_tuple(std::string(prec), v[0], v[1], v[2]), std::array<int, 4>{v[3], v[4], v[5], v[6]}});
    }
    if (lineno == 0) return fail(LQCD_EINVAL, "tune import: empty text");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &r : rows) g_imported[r.first] = r.second;
    return LQCD_OK;
}

int lqcd_profile_read(lqcd_kernel_stat *out, int max, int *count)
{
    if (!count || (max > 0 && !out)) return fail(LQCD_EINVAL, "null argument");
    try {
        std::lock_guard<std::mutex> lk(g_mu);
        drain_locked();
        int n = 0;
        for (auto &kv : g_stats) {
            if (n < max) {
                lqcd_kernel_stat &o = out[n];
                std::memset(&o, 0, sizeof o);
                std::strncpy(o.name, kv.first.c_str(), sizeof(o.name) - 1);
                o.launches = kv.second.launches;
                o.bytes = kv.second.bytes;
                o.timed_launches = kv.second.timed;
                o.timed_ms = kv.second.ms;
                o.timed_bytes = kv.second.timed_bytes;
            }
            ++n;
        }
        *count = n;
        return LQCD_OK;
    } catch (const Error &e) {
        return fail(e.code, e.msg);
    }
}

}  // extern "C"
