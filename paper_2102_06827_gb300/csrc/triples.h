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

// FP32 tensor-core path (k_triples_tc.cu).  A work item is a pair-tile of T: 8 values along T
// label 0 and 4 along each other label.  For each term the operand holding label 0 gives 128
// rows (8 x 4 x 4), the other one 64 (4 x 4 x 4); a pre-pass writes every operand as tile-
// blocked split-BF16 planes (rows of 32 summed indices, 64 bytes, [tile][chunk][plane][row]),
// and one 128 x 64 tcgen05 MMA tile per term and chunk accumulates the six products in tensor
// memory; sixteen warps (four per lane quadrant) drain each term into the pair-tile in shared
// memory, which then gives the energy.
namespace tc {
constexpr int WA = 8;              // pair-tile extent along T label 0
constexpr int KCH = 32;            // summed indices per plane row
constexpr int ROWB = 64;           // bytes per plane row
constexpr int WROWS = 128;         // rows of the operand holding label 0 (8 x 4 x 4)
constexpr int NROWS = 64;          // rows of the other operand (4 x 4 x 4)
constexpr int BOX = 64;            // rows per TMA box
constexpr int WPLANE = WROWS * ROWB, NPLANE = NROWS * ROWB;
constexpr int SLOT = 3 * (WPLANE + NPLANE);   // one (term, chunk): three planes of both operands
constexpr int RING = 4;
constexpr int NACC = 4;            // tensor-memory accumulators (64 columns each)
constexpr int DRAIN_WARPS = 16;    // four per tensor-memory lane quadrant, 16 columns each
constexpr int THREADS = 64 + 32 * DRAIN_WARPS;
constexpr uint32_t TMEM_COLS = NACC * NROWS;
constexpr int TSZ = 10912;         // the pair-tile in shared memory (floats)
// element strides of the pair-tile per T label: every label but 0 has a stride = 8 mod 32, so
// the 32 rows a warp drains (8 along label 0 x 4 along one more label) hit 32 different banks
constexpr int tstride(int q) {
    return q == 0 ? 1 : q == 1 ? 8 : q == 2 ? 40 : q == 3 ? 168 : q == 4 ? 680 : 2728;
}
constexpr int64_t MAX_BATCH_ROWS = int64_t(1) << 27;   // plane rows per batch (8 GB)
constexpr int SMEM = 1024 + RING * SLOT + 512;   // dynamic; the pair-tile is a static array
}  // namespace tc

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
    int *status;               // debug builds: device status word for an operand access out of range
};

// One term of one block on the tensor-core path: the plane rows of its two operand tiles for a
// pair-tile with tile coordinates c[6] are row0[w] + sum_q coef[w][q] c[q] (w = 0: the operand
// holding T label 0, 128 rows per tile; w = 1: the other one, 64), then + (chunk * 3 + plane) *
// rows per tile.
struct TcRec {
    int32_t row0[2];
    int32_t coef[2][6];
    int32_t nch;               // chunks of 32 summed indices
    int32_t ed;                // extent of the summed label
};
static_assert(sizeof(TcRec) == 64, "records are read as four 16-byte words");

// the tensor-core path's launch arguments (one batch of blocks)
struct TcArgs {
    const int64_t *prefix;     // pair-tiles before each block; n_blocks + 1
    const int32_t *row0;       // n_blocks x n_terms x 2: first plane row of each operand in its batch
    const TcRec *rec;          // n_blocks x n_terms
    char *planes;              // the batch's plane rows
    int b0, b1;                // the batch's blocks
    int64_t item0, n_items;    // its pair-tiles
    int *status;               // device status word (a wait that ran out records COMET_ERR_TIMEOUT)
    int64_t timeout_ns;        // limit of every wait
    int debug_flags;           // bit 0: one ring slot's loads withheld (fault injection, host side)
    int64_t planes_bytes;      // debug builds: size of the batch's plane region
};
}  // namespace tri

// the whole triples plan (host only): terms, owned pair, block table, prefix sums, workspace
comet_status_t plan_triples(const char *const *terms, int n_terms, const char *const *names, int n_labels,
                            int n_blocks, const int64_t *extents, const int *signs, comet_dtype_t dtype, Plan *P,
                            std::string *err);

// the kernel's argument block from a plan (every field but the device pointers and the total)
void triples_args(const Plan &P, tri::Args *a);

// the FP32 tensor-core layout of a plan: pair-tile prefix, batches, plane rows of every operand
// (no batches when some block's planes exceed one batch: the FMA kernel then runs the plan)
void plan_triples_tc(Plan *P);

// plane rows of one operand of a block: tiles x chunks x 3 planes x rows per tile
// (q: T label per operand dimension, -1 = the summed label)
int64_t tc_operand_rows(const int *q, const int64_t *ext_t, int64_t ext_d);

}  // namespace comet
