// trace.cu -- optional per-kernel timing: a CUDA event pair recorded on the launching
// stream around each traced launch, accumulated per kernel name (mode 1), or launch counts
// alone with no events and no extra work (mode 2). Off by default; when off a trace scope
// costs one relaxed atomic load.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pcms_internal.cuh"
#include "trace.cuh"

namespace pcms {

namespace {

struct Pending {
    std::string name;
    cudaEvent_t a, b;
};
struct Stat {
    int64_t launches = 0;
    double total_ms = 0.0;
};

std::atomic<int> g_on{0};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
std::map<std::string, Stat> g_stats;

cudaEvent_t get_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void drain_locked() {
    for (Pending& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Stat& s = g_stats[p.name];
            s.launches += 1;
            s.total_ms += ms;
        } else {
            cudaGetLastError();
        }
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace

bool trace_on() { return g_on.load(std::memory_order_relaxed) != 0; }
bool trace_timing() { return g_on.load(std::memory_order_relaxed) == 1; }

TraceScope::TraceScope(const char* name, cudaStream_t s) : name_(name), s_(s) {
    const int mode = g_on.load(std::memory_order_relaxed);
    if (!mode || !name) return;   // a null name: not recorded
    std::lock_guard<std::mutex> lk(g_mu);
    if (mode == 2) {
        g_stats[name_].launches += 1;
        return;
    }
    a_ = get_event();
    if (a_) cudaEventRecord(a_, s_);
}

TraceScope::~TraceScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = get_event();
    if (!b) {
        g_free.push_back(a_);
        return;
    }
    cudaEventRecord(b, s_);
    g_pending.push_back(Pending{name_, a_, b});
}

void trace_count(const char* name, int64_t n) {
    if (!trace_on()) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_stats[std::string("count:") + name].launches += n;
}

void trace_enable(int mode) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    if (mode) g_stats.clear();
    g_on.store(mode == 2 ? 2 : (mode ? 1 : 0));
}

int trace_count() {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    return (int)g_stats.size();
}

int trace_get(int i, char* name, int name_len, int64_t* launches, double* total_ms) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    if (i < 0 || i >= (int)g_stats.size()) return 0;
    auto it = g_stats.begin();
    std::advance(it, i);
    if (name && name_len > 0) {
        std::strncpy(name, it->first.c_str(), (size_t)name_len - 1);
        name[name_len - 1] = 0;
    }
    if (launches) *launches = it->second.launches;
    if (total_ms) *total_ms = it->second.total_ms;
    return 1;
}

}  // namespace pcms
