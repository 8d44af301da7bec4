// plan_internal.hpp -- the plan object behind the opaque bmmc_plan handle:
// the validated matrix (Sec. 3), its one or two tiled passes (Sec. 5.1, 5.2)
// and each pass's launch tables (Sec. 4.1-4.3).
#pragma once
#include <stdint.h>

#include <mutex>

#include "bmmc.h"
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
    // Passes whose tables are derived.  Every plan handed out by the public
    // API has all of them; the request server derives the second pass of a
    // two-pass plan after launching the first (plan_create_first_pass).
    int derived = 0;
    // Workspace owned by the plan for bmmc_execute (two-pass plans only).
    std::mutex ws_mu;
    void *ws = nullptr;
    int ws_device = -1;

    uint64_t bytes() const { return (1ull << n) << e_log; }
};

namespace bmmc {

// As bmmc_plan_create_ex, deriving the launch tables of the first pass only;
// plan_derive_rest derives the others.  Until then the plan may only be used
// by plan_launch_pass for its derived passes, and every public entry point
// that runs, inspects or batches it returns BMMC_ERR_INVALID.
int plan_create_first_pass(bmmc_plan *out, int n, const uint64_t *rows, uint64_t c,
                           size_t elem_bytes, const bmmc_plan_options *opts);
// Derive the tables of the passes not derived yet.  BMMC_OK or the planner's
// status for that pass.
int plan_derive_rest(bmmc_plan p);
// Launch pass `pass` alone, in -> out (the first pass reads the input and
// writes the workspace, the second the reverse).  Asynchronous on s.
int plan_launch_pass(bmmc_plan p, int pass, const void *in, void *out,
                     bmmc_stream_t s);

}  // namespace bmmc
