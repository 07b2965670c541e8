// Self-check flag shared by the kernels that index through offset tables, and
// the DGELL_DEBUG_SYNC switch (synchronise after every checked launch and
// report the launch by name).
#include <cstdlib>
#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace dg {
namespace {
__device__ int g_check_flag_dev;
std::mutex g_mu;
int* g_flag_addr[64] = {};
}  // namespace

int* device_check_flag() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_flag_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_check_flag_dev) == cudaSuccess) {
            g_flag_addr[dev] = static_cast<int*>(p);
            cudaMemset(p, 0, sizeof(int));
        }
    }
    return g_flag_addr[dev];
}

namespace {
std::mutex g_plan_mu;
std::unordered_map<unsigned long long, int> g_plans;
}  // namespace

int plan_cache_get(unsigned long long key) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(key);
    return it == g_plans.end() ? -1 : it->second;
}

void plan_cache_put(unsigned long long key, int plan) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans.emplace(key, plan);
}

bool debug_sync() {
    static const bool v = [] {   // read once (thread-safe static initialisation)
        const char* e = std::getenv("DGELL_DEBUG_SYNC");
        return e && e[0] == '1';
    }();
    return v;
}

}  // namespace dg
