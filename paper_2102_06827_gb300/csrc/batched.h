// Batched triples-like contractions: one persistent launch over many small, uneven blocks.
#pragma once
#include <string>

#include "plan.hpp"

namespace comet {
std::string describe_batched(const Plan &p);
}  // namespace comet
