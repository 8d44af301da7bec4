// plan_internal.hpp -- the plan object behind the opaque bmmc_plan handle:
// the validated matrix (Sec. 3), its one or two tiled passes (Sec. 5.1, 5.2)
// and each pass's launch tables (Sec. 4.1-4.3).
#pragma once
#include <stdint.h>

#include <mutex>

#include "f2.hpp"
#include "pass_desc.h"
#include "plan.hpp"

struct bmmc_plan_s {
    int n = 0;
    int e_log = 0;
    uint64_t c = 0;
    bmmc::f2::Mat a;
    bmmc::PlanOptions opt;
    int npass = 0;
    bmmc::f2::Mat t[2];
    uint64_t tc[2] = {0, 0};
    bmmc::PassDesc desc[2];
    bmmc::PassInfo info[2];
    // Workspace owned by the plan for bmmc_execute (two-pass plans only).
    std::mutex ws_mu;
    void *ws = nullptr;
    int ws_device = -1;

    uint64_t bytes() const { return (1ull << n) << e_log; }
};
