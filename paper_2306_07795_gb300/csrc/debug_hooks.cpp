// debug_hooks.cpp -- host-side fault injection (include/bmmc_debug.h).
#include <atomic>

#include "bmmc_debug.h"
#include "debug_hooks.hpp"

namespace {
std::atomic<int> g_fail_allocs{0};
std::atomic<int> g_fail_launches{0};

bool take(std::atomic<int> &counter)
{
    int n = counter.load(std::memory_order_relaxed);
    while (n > 0)
        if (counter.compare_exchange_weak(n, n - 1, std::memory_order_relaxed)) return true;
    return false;
}
}  // namespace

namespace bmmc {
bool debug_fail_alloc() { return take(g_fail_allocs); }
bool debug_fail_launch() { return take(g_fail_launches); }
}  // namespace bmmc

extern "C" {

void bmmc_debug_fail_allocs(int count) { g_fail_allocs.store(count > 0 ? count : 0); }

void bmmc_debug_fail_launches(int count) { g_fail_launches.store(count > 0 ? count : 0); }

}  // extern "C"
