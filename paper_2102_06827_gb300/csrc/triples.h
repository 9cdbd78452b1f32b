// The fused triples accumulation (comet_plan_triples / comet_triples_energy): kernel geometry,
// the kernel's argument block, and the host functions that plan it.  Shared by the kernel
// (k_triples.cu), the host planner (triples_plan.cpp) and the CPU replay of the kernel's index
// arithmetic (tests/triples_check.cpp).
#pragma once
#include <stdint.h>

#include <string>

#include "../../include/comet.h"
#include "plan.hpp"

namespace comet {

namespace tri {
constexpr int TS = 4;          // tile edge per label
constexpr int NT = 256;        // threads: 4^4 fixed-label combinations
constexpr int KC = 32;         // summed-label values staged per pass (FP32; 16 for FP64)
constexpr int R = TS * TS * TS;   // operand tile rows (three T labels)
constexpr int RP = R + 4;         // row pitch: 16-byte aligned rows, shifted banks
constexpr int CHUNK = 16;      // items taken per counter increment
constexpr int PK_TRIPLES_ID = 9;

// FP32 kernel: a CTA of 64 threads per 4^6 tile.  Thread t holds the 2^6 elements whose tile
// coordinate along T label j is 2 h_j + l_j, h_j = bit j of t, l_j = 0 or 1 (64 accumulators);
// an operand's staged tile row r holds the entry with coordinate 2 (bit 3 + i of r) + (bit i
// of r) along the operand's i-th T label in T order, so that a thread's 8 entries of a summed
// index are one 32-byte run.
// Each step stages the operand holding T label 0 (P) and the other one (B), [KC32][RP32] each.
constexpr int NT32 = 64;
constexpr int KC32 = 16;       // summed-label values staged per pass
constexpr int ROW32 = 64;      // entries per staged row (4^3)
constexpr int RP32 = ROW32;    // row pitch (a warp's staging writes are 32 consecutive entries)
constexpr int CTAS32 = 8;      // resident CTAs per SM the FP32 kernel is built for

struct TermDev {
    double alpha;
    int8_t x_q[4], y_q[4];     // T label position per operand dimension, -1 = summed label
    int8_t x_col[4], y_col[4]; // extent-table column per operand dimension
    int8_t x_dig[4], y_dig[4]; // tile-row digit per dimension (owned labels first), -1 = summed
    int8_t x_rank[4], y_rank[4];   // per operand dimension: rank of its T label among the
                                   // operand's three in T order, -1 = summed (FP32 kernel)
    int8_t d_col;
    int8_t amode;              // alpha: 0 = 1, 1 = -1, 2 = any other value (integer tests per step:
                               // the FP64 pipe is slow on this part)
    int8_t xmask;              // bit j set: T label j is on X (FP32 kernel)
    int8_t pad[5];
};

struct Args {
    int n_terms, n_labels, n_blocks;
    int8_t t_col[6], own[2], fixed[4];
    float own_sign[2], fixed_sign[4];
    float sign[6];             // sign of each T label's eps in D
    TermDev term[16];
    const int32_t *ext;        // n_blocks x n_labels
    const int64_t *prefix;     // n_blocks + 1
    const void *const *ops;    // n_blocks x n_terms x 2
    const void *const *eps;    // n_blocks x 6
    double *energies;
    unsigned long long *counter;
    int64_t total;
};
}  // namespace tri

// the whole triples plan (host only): terms, owned pair, block table, prefix sums, workspace
comet_status_t plan_triples(const char *const *terms, int n_terms, const char *const *names, int n_labels,
                            int n_blocks, const int64_t *extents, const int *signs, comet_dtype_t dtype, Plan *P,
                            std::string *err);

// the kernel's argument block from a plan (every field but the device pointers and the total)
void triples_args(const Plan &P, tri::Args *a);

}  // namespace comet
