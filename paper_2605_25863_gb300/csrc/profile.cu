// profile.cu -- event-based launch timing and launch counting (see profile.h).
#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/linac.h"
#include "profile.h"

namespace linac {

namespace {
struct Rec {
    int cls;
    cudaEvent_t a, b;
};
std::mutex g_pmu;
std::atomic<int> g_enabled{0};
std::atomic<long long> g_launches{0};
std::vector<Rec> g_pending;
std::vector<cudaEvent_t> g_pool;
Rec g_open[64];            // one open bracket per class (launches of a class never nest)
double g_ms[PROF_NCLASSES];
long long g_count[PROF_NCLASSES];
const char* g_names[PROF_NCLASSES] = {"init", "panel", "gather_f", "gather_w", "inverse", "trsm", "move",
                                      "update_plain", "update_limb", "limb_split", "finish", "batched",
                                      "solve_pack", "solve_extract", "validate", "pattern", "matmul",
                                      "load_matrix", "derived", "u64_panel", "u64_update",
                                      "update_crt", "crt_split", "host_copy", "lup", "update_hybrid"};

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return e;
}

void drain_locked() {
    for (Rec& r : g_pending) {
        if (r.a && r.b && cudaEventSynchronize(r.b) == cudaSuccess) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                g_ms[r.cls] += ms;
                g_count[r.cls] += 1;
            }
        }
        (void)cudaGetLastError();
        if (r.a) g_pool.push_back(r.a);
        if (r.b) g_pool.push_back(r.b);
    }
    g_pending.clear();
}
}  // namespace

const char* prof_name(int cls) { return cls >= 0 && cls < PROF_NCLASSES ? g_names[cls] : "?"; }

void prof_begin(cudaStream_t s, int cls) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_pmu);
    if (g_pending.size() > 100000) drain_locked();
    cudaEvent_t a = take_event();
    if (a) cudaEventRecord(a, s);
    g_open[cls] = Rec{cls, a, nullptr};
}

void prof_end(cudaStream_t s, int cls) {
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_pmu);
    Rec r = g_open[cls];
    if (!r.a) return;
    r.b = take_event();
    if (r.b) cudaEventRecord(r.b, s);
    g_pending.push_back(r);
    g_open[cls].a = nullptr;
}

}  // namespace linac

using namespace linac;

extern "C" {

void linac_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_pmu);
    g_enabled.store(on ? 1 : 0);
}

void linac_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_pmu);
    drain_locked();
    for (int i = 0; i < PROF_NCLASSES; ++i) {
        g_ms[i] = 0.0;
        g_count[i] = 0;
    }
}

int linac_profile_read(linac_profile_entry* out, int max_entries) {
    std::lock_guard<std::mutex> lk(g_pmu);
    drain_locked();
    int n = 0;
    for (int i = 0; i < PROF_NCLASSES && n < max_entries; ++i) {
        if (!g_count[i]) continue;
        out[n].name = g_names[i];
        out[n].launches = g_count[i];
        out[n].total_ms = g_ms[i];
        ++n;
    }
    return n;
}

long long linac_launch_count(void) { return g_launches.load(); }

}  // extern "C"
