// debug_hooks.hpp -- queries of the fault-injection counters of
// include/bmmc_debug.h.  Each call consumes one injected failure if any.
#pragma once

namespace bmmc {
bool debug_fail_alloc();   // the next device allocation must report OOM
bool debug_fail_launch();  // the next launch must report a launch failure
}  // namespace bmmc
