// Batched triples-like contractions: one persistent launch over many small, uneven blocks of
// the same two-operand expression.
#pragma once
#include <string>

#include "plan.hpp"

namespace comet {

// One block, as the kernel reads it (in the longest-first order of the plan).
struct BlockDesc {
    Radix ma, nb, k;             // M: (A strides, output strides); N: (B strides, output
                                 // strides); K: (A strides, B strides)
    uint32_t M, N, K;
    uint32_t index;              // the block's position in the caller's tables
    int64_t a_elems, b_elems;
    int64_t a_parts, b_parts;    // split path: workspace offsets of the operands' bfloat16 planes,
                                 // [3][rows][kpad] each (rows = M for A, N for B)
    uint32_t kpad;               // K rounded up to a multiple of 32
    uint32_t pad;
};

constexpr int kBatchedCfgF64 = 4;     // tile configurations of the FP64 path
constexpr int kBatchedCfgSplit = 3;   // tile configurations of the split path

struct BatchedParams {
    const BlockDesc *desc;       // n_blocks descriptors, longest first
    const uint32_t *prefix;      // n_blocks + 1 tile prefix sums for the launched configuration
    uint32_t n_blocks, total_tiles;
    const void *const *inputs;   // 2 per block (caller's order)
    int swap;                    // 1: the M operand is the block's second input
    int mode;                    // 0 reduce, 1 store
    void *result;
    uint32_t key;
    unsigned int *counter;       // work counter (zeroed by the launch sequence)
    const int *exps;             // split path: scale exponents of the M and N operands, 2 per block
    double alpha;
    char *ws;                    // workspace base (the split planes live at desc offsets)
};

std::string describe_batched(const Plan &p);

}  // namespace comet
