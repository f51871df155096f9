// Per-kernel device timing: when enabled, every launch made by the library is
// bracketed by two CUDA events recorded on the stream it is launched on; the
// elapsed times are summed per kernel name when the profile is collected.
#include "bem_internal.cuh"

#include <atomic>
#include <cstdio>
#include <cstring>
#include <iterator>
#include <map>
#include <mutex>

namespace bem {

namespace {

struct Live {
    const char* name;
    cudaEvent_t a, b;
};

std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Live> g_live;
std::vector<cudaEvent_t> g_pool;
std::map<std::string, std::pair<double, int64_t>> g_acc;
std::vector<std::string> g_select;  // name prefixes to time (empty: every kernel)

bool selected_locked(const char* name) {
    if (g_select.empty()) return true;
    for (const auto& p : g_select)
        if (std::strncmp(name, p.c_str(), p.size()) == 0) return true;
    return false;
}

cudaEvent_t take_event() {
    cudaEvent_t e = nullptr;
    if (!g_pool.empty()) {
        e = g_pool.back();
        g_pool.pop_back();
    } else {
        cudaEventCreate(&e);
    }
    return e;
}

// fold finished records into the totals (caller holds the lock)
void drain_locked() {
    for (auto& L : g_live) {
        float ms = 0.f;
        if (cudaEventSynchronize(L.b) == cudaSuccess && cudaEventElapsedTime(&ms, L.a, L.b) == cudaSuccess) {
            auto& acc = g_acc[L.name];
            acc.first += ms;
            acc.second += 1;
        }
        g_pool.push_back(L.a);
        g_pool.push_back(L.b);
    }
    g_live.clear();
}

}  // namespace

int prof_begin(const char* name, cudaStream_t s) {
    if (!g_on.load(std::memory_order_relaxed)) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!selected_locked(name)) return -1;
    if (g_live.size() >= 65536) drain_locked();  // bound the number of pending events
    Live L{name, take_event(), take_event()};
    cudaEventRecord(L.a, s);
    g_live.push_back(L);
    return (int)g_live.size() - 1;
}

bool prof_times_every_kernel() {
    if (!g_on.load(std::memory_order_relaxed)) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    return g_select.empty();
}

void prof_end(int slot, cudaStream_t s) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot < (int)g_live.size()) cudaEventRecord(g_live[slot].b, s);
}

}  // namespace bem

using namespace bem;

extern "C" {

void bem_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!on) drain_locked();
    g_on.store(on != 0);
}

void bem_profile_select(const char* prefixes) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_select.clear();
    if (!prefixes) return;
    std::string all(prefixes);
    size_t pos = 0;
    while (pos <= all.size()) {
        const size_t c = all.find(',', pos);
        const std::string item = all.substr(pos, c == std::string::npos ? std::string::npos : c - pos);
        if (!item.empty()) g_select.push_back(item);
        if (c == std::string::npos) break;
        pos = c + 1;
    }
}

void bem_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    g_acc.clear();
}

bem_status bem_profile_get(int index, char* name, int name_len, double* total_ms, int64_t* launches) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    BEM_REQUIRE(index >= 0 && index < (int)g_acc.size(), "profile index out of range");
    auto it = g_acc.begin();
    std::advance(it, index);
    if (name && name_len > 0) {
        std::snprintf(name, (size_t)name_len, "%s", it->first.c_str());
    }
    if (total_ms) *total_ms = it->second.first;
    if (launches) *launches = it->second.second;
    return BEM_OK;
}

int bem_profile_count(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    return (int)g_acc.size();
}

}  // extern "C"
