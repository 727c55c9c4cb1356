// isax_profile.cu - launch counting and optional per-kernel timing with CUDA
// events recorded on the launching stream (tracing for benchmarks and tests).
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "isax_common.cuh"

namespace isax {

namespace {
struct Record {
    const char* name;
    cudaEvent_t e0, e1;
};
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_mode{0};  // 0 off, 1 every kernel, 2 build kernels only
std::mutex g_mu;
std::vector<Record> g_records;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

KernelScope::KernelScope(const char* name, cudaStream_t st) : name_(name), st_(st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    const int mode = g_mode.load(std::memory_order_relaxed);
    // query kernels are named q_*; mode 2 leaves them untimed
    if (mode == 1 || (mode == 2 && name[0] != 'q')) {
        std::lock_guard<std::mutex> lk(g_mu);
        e0_ = take_event();
        e1_ = take_event();
        if (e0_ && e1_) cudaEventRecord(static_cast<cudaEvent_t>(e0_), st_);
    }
}

KernelScope::~KernelScope() {
    if (!e0_ || !e1_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(static_cast<cudaEvent_t>(e1_), st_);
    g_records.push_back({name_, static_cast<cudaEvent_t>(e0_), static_cast<cudaEvent_t>(e1_)});
}

bool profiling_on() { return g_mode.load(std::memory_order_relaxed) == 1; }

void count_launches(int kernels) { g_launches.fetch_add((unsigned long long)kernels, std::memory_order_relaxed); }

}  // namespace isax

using namespace isax;

extern "C" {

isax_status isax_profile(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (enable) {
        for (auto& r : g_records) {
            g_pool.push_back(r.e0);
            g_pool.push_back(r.e1);
        }
        g_records.clear();
        // create the events now, so no event is created while launches are timed
        while (g_pool.size() < 16384) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) break;
            g_pool.push_back(e);
        }
    }
    g_mode.store(enable == 1 ? 1 : enable == 2 ? 2 : 0);
    return ISAX_OK;
}

int32_t isax_profile_report(isax_kernel_time* out, int32_t max) {
    std::lock_guard<std::mutex> lk(g_mu);
    std::map<std::string, std::pair<int64_t, double>> agg;
    for (auto& r : g_records) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.e1) != cudaSuccess) continue;
        if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) continue;
        auto& a = agg[r.name];
        a.first += 1;
        a.second += ms;
    }
    int32_t i = 0;
    for (auto& kv : agg) {
        if (out && i < max) {
            memset(&out[i], 0, sizeof out[i]);
            strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = kv.second.first;
            out[i].total_ms = kv.second.second;
        }
        ++i;
    }
    return i;
}

uint64_t isax_launch_count(void) { return g_launches.load(); }

}  // extern "C"
