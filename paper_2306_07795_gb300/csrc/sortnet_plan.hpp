// sortnet_plan.hpp -- the fused sorting-network plan behind bmmc_sort_plan.
#pragma once
#include <stdint.h>

#include <vector>

#include "f2.hpp"
#include "pass_desc.h"
#include "plan.hpp"
#include "sort_desc.h"

struct bmmc_sort_plan_s {
    int n = 0;       // keys per row: 2^n
    int b = 0;       // rows: 2^b
    int N = 0;       // n + b
    int e_log = 0;   // key bytes = 2^e_log (4 or 8)
    int key = 0;     // bmmc_key_type
    int block_bits = 0;  // slot bits of a fused pass's thread block
    bool small = false;  // the whole network in one thread block
    bmmc::SortSmallDesc sdesc;
    std::vector<bmmc::PassDesc> pass;  // fused passes, in order
    std::vector<bmmc::SortDesc> ce;    // their comparator tables
    std::vector<bmmc::f2::Mat> layout; // layout after each pass (for checks)
    int stages = 0;  // comparator stages of the network
};

namespace bmmc {
namespace sortnet {

// Build the plan (host only).  Returns 0 or a negative bmmc status.
int plan_sort(bmmc_sort_plan_s *p, int n, int b, int key, int block_log2, int compare_code);

// Run the plan's tables on the host, exactly as the kernels index them:
// in and out hold 2^N keys.  Returns 0.
int emulate(const bmmc_sort_plan_s *p, const void *in, void *out);

}  // namespace sortnet
}  // namespace bmmc
