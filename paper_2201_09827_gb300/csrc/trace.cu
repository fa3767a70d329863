// Kernel launch counter and optional phase timing shared by all translation units.
//
// Timing records a pair of CUDA events on the launching stream around each phase without
// synchronising; elapsed times are resolved and summed per phase name when the report is
// requested (or when the event pool fills up).
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gir_internal.cuh"
#include "trace.cuh"

namespace gir {

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(); }

namespace {
struct Slot {
    const char* name;
    cudaEvent_t a, b;
};
struct Agg {
    const char* name;
    double ms;
    long long cnt;
};
struct TraceState {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<Slot> slots;
    std::vector<Agg> agg;
    size_t used = 0;
    int open = 0;   // phases begun and not yet ended (slots may not be recycled meanwhile)
    void resolve() {
        if (slots.empty()) return;
        cudaDeviceSynchronize();
        for (auto& s : slots) {
            float t = 0.0f;
            if (!s.name || !s.b) continue;  // a phase that was begun but not ended
            if (cudaEventElapsedTime(&t, s.a, s.b) != cudaSuccess) {
                cudaGetLastError();  // do not leave the failure as the runtime's last error
                continue;
            }
            bool found = false;
            for (auto& g : agg)
                if (std::strcmp(g.name, s.name) == 0) {
                    g.ms += t;
                    g.cnt += 1;
                    found = true;
                    break;
                }
            if (!found) agg.push_back({s.name, (double)t, 1});
        }
        slots.clear();
        used = 0;
    }
    cudaEvent_t next() {
        if (used >= pool.size()) {
            if (pool.size() >= 16384 && open == 0) resolve();
            if (used >= pool.size()) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                pool.push_back(e);
            }
        }
        return pool[used++];
    }
};
TraceState g_trace;
std::mutex g_trace_mu;   // the batch runs solves on several host threads
}  // namespace

bool trace_on() { return g_trace.on; }

// Phase names to time (empty: all). Phases outside the selection record no events, so a run can
// time a few kernels without the event records between every launch.
static std::vector<std::string> g_select;

int trace_begin(cudaStream_t s, const char* name) {
    if (!g_trace.on) return -1;
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (!g_select.empty()) {
        if (!name) return -1;   // a phase named only at its end (diagnostic detail)
        bool hit = false;
        for (const auto& n : g_select)
            if (n == name) { hit = true; break; }
        if (!hit) return -1;
    }
    cudaEvent_t a = g_trace.next();
    cudaEventRecord(a, s);
    g_trace.slots.push_back({nullptr, a, nullptr});
    ++g_trace.open;
    return (int)g_trace.slots.size() - 1;
}

void trace_end(int slot, const char* name, cudaStream_t s) {
    if (!g_trace.on) return;
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (slot < 0 || slot >= (int)g_trace.slots.size()) return;
    cudaEvent_t b = g_trace.next();
    cudaEventRecord(b, s);
    g_trace.slots[slot].name = name;
    g_trace.slots[slot].b = b;
    if (g_trace.open > 0) --g_trace.open;
}

void trace_add(const char* name, double ms, long long cnt) {
    if (!g_trace.on) return;
    std::lock_guard<std::mutex> lk(g_trace_mu);
    for (auto& g : g_trace.agg)
        if (std::strcmp(g.name, name) == 0) {
            g.ms += ms;
            g.cnt += cnt;
            return;
        }
    g_trace.agg.push_back({name, ms, cnt});
}

static int env_flag(const char* name) {
    const char* e = getenv(name);
    return (e && e[0] == '1') ? 1 : 0;
}

bool trace_detail() {
    static const int v = env_flag("GIR_TRACE_DETAIL");
    return g_trace.on && v == 1;
}

}  // namespace gir

extern "C" {

void gir_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(gir::g_trace_mu);
    gir::g_trace.open = 0;
    gir::g_trace.resolve();
    gir::g_trace.agg.clear();
    gir::g_trace.on = on != 0;
}

int gir_trace_report(char* buf, int buflen) {
    std::lock_guard<std::mutex> lk(gir::g_trace_mu);
    gir::g_trace.resolve();
    std::string out;
    char line[256];
    for (auto& g : gir::g_trace.agg) {
        snprintf(line, sizeof(line), "%s\t%.6f\t%lld\n", g.name, g.ms, g.cnt);
        out += line;
    }
    if (buf && buflen > 0) {
        int n = (int)out.size() < buflen - 1 ? (int)out.size() : buflen - 1;
        memcpy(buf, out.data(), n);
        buf[n] = 0;
        gir::g_trace.agg.clear();  // a size query (buf == NULL) keeps the totals
    }
    return (int)out.size();
}

void gir_trace_select(const char* names) {
    std::lock_guard<std::mutex> lk(gir::g_trace_mu);
    gir::g_select.clear();
    if (!names) return;
    std::string cur;
    for (const char* p = names;; ++p) {
        if (*p == ',' || *p == 0) {
            if (!cur.empty()) gir::g_select.push_back(cur);
            cur.clear();
            if (*p == 0) break;
        } else {
            cur += *p;
        }
    }
}

unsigned long long gir_launch_count(void) { return gir::g_launches.load(); }

}  // extern "C"
