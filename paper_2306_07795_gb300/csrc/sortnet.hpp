// sortnet.hpp -- the sorting network of Sec. 6.1 unrolled into stages (host).
#pragma once
#include <vector>

#include "f2.hpp"

namespace bmmc {
namespace sortnet {

// The n (n + 1) / 2 stages of sort n: stage s is "permute by stages[s], then
// order the pairs (2j, 2j + 1)"; the network ends with final_perm.
void schedule(int n, std::vector<f2::Mat> *stages, f2::Mat *final_perm);

}  // namespace sortnet
}  // namespace bmmc
