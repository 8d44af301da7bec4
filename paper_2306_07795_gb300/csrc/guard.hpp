// guard.hpp -- keep C++ exceptions from crossing the C ABI.
//
// The entry points of include/*.h are extern "C": an exception escaping one
// would be undefined behaviour in a C caller.  Those that allocate through
// the standard library (plans, batches, the server) run their body through
// guarded(), which turns std::bad_alloc into BMMC_ERR_OOM and anything else
// into BMMC_ERR_INVALID.
#pragma once
#include <new>

#include "bmmc.h"

namespace bmmc {

template <typename F>
int guarded(F &&body) noexcept
{
    try {
        return body();
    } catch (const std::bad_alloc &) {
        return BMMC_ERR_OOM;
    } catch (...) {
        return BMMC_ERR_INVALID;
    }
}

}  // namespace bmmc
