// Batched triples-like contractions: one persistent launch over many small, uneven blocks of
// the same two-operand expression.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "plan.hpp"

namespace comet {

// One block, as the kernels read it (in the longest-first order of the plan).
struct BlockDesc {
    Radix ma, nb, k;             // M: (A strides, output strides); N: (B strides, output
                                 // strides); K: (A strides, B strides)
    uint32_t M, N, K;
    uint32_t index;              // the block's position in the caller's tables
    int64_t a_elems, b_elems;
    // split path: the operands' bfloat16 planes, in rows of 32 K values (64 bytes) counted from
    // the start of the plane region; operand X occupies ceil(K/32) chunks x 3 planes x x_pad
    // rows, [chunk][plane][row], rows beyond M (N) and K values beyond K zero
    int64_t a_row0, b_row0;
    uint32_t nk16;               // K in MMA steps of 16
    uint32_t m_pad, n_pad;       // M and N rounded up to a multiple of 256
    uint32_t pad[3];
};

// One work item of the tensor-core split kernel (block, strip of output columns), built on the
// host per tile configuration so that the kernel's roles read it with one 48-byte load.
struct ItemRec {
    uint32_t pos;                // the block's position in launch order (descriptor index)
    uint32_t index;              // the block's position in the caller's tables
    uint32_t n0;                 // first output column of the strip
    uint32_t mtiles;             // 128-row tiles of the block
    uint32_t nk16, M, N;
    uint32_t m_pad, n_pad;
    int32_t a_row0, b_row0;      // first plane row of each operand
    uint32_t pad;
};
static_assert(sizeof(ItemRec) == 48, "item records are read as three 16-byte words");

constexpr int kBatchedCfgF64 = 4;     // tile configurations of the FP64 path
constexpr int kBatchedCfgSplit = 2;   // tile configurations of the split path (strip widths)
constexpr int kBatchedPlaneRow = 64;  // bytes of one plane row (32 bfloat16 K values)

struct BatchedParams {
    const BlockDesc *desc;       // n_blocks descriptors, longest first
    const uint32_t *prefix;      // n_blocks + 1 work-item prefix sums for the launched configuration
    const ItemRec *items;        // split path: the launched configuration's work items
    uint32_t n_blocks, total_tiles;
    const void *const *inputs;   // 2 per block (caller's order)
    int swap;                    // 1: the M operand is the block's second input
    int mode;                    // 0 reduce, 1 store
    void *result;
    uint32_t key;
    unsigned int *counter;       // work counter (zeroed by the launch sequence)
    const int *exps;             // split path: scale exponents of the M and N operands, 2 per block
    double alpha;
    char *ws;                    // workspace base
    char *planes;                // split path: start of the plane region
    int64_t planes_bytes;        // split path: its size (debug builds check the pre-pass writes)
    int *status;                 // device status word (a wait that ran out records COMET_ERR_TIMEOUT)
    int64_t timeout_ns;          // limit of every wait of the tensor-core kernel
    int debug_flags;             // bit 0: one operand load withheld (fault injection, host side)
};

// tile configurations: rows x columns of a work item's tiles (the split path's rows are the
// tcgen05 M; its columns are the strip width of a work item)
struct TileCfg { int bm, bn; };
inline TileCfg batched_cfg(bool split, int c) {
    static const TileCfg f64[kBatchedCfgF64] = {{64, 64}, {64, 32}, {32, 64}, {32, 32}};
    static const TileCfg spl[kBatchedCfgSplit] = {{128, 256}, {128, 128}};
    return split ? spl[c] : f64[c];
}
inline int n_cfg(const Plan &P) { return P.opts.precision == COMET_PREC_SPLIT_BF16 ? kBatchedCfgSplit : kBatchedCfgF64; }
inline TileCfg cfg_of(const Plan &P, int c) { return batched_cfg(P.opts.precision == COMET_PREC_SPLIT_BF16, c); }

// workspace layout: [counter 256 B][exps 8*n][prefix n_cfg*(n+1)*4][descs n*sizeof(BlockDesc)]
// [split path: item records of every configuration][split path: the plane rows of every
// block's operands]
struct BLayout {
    size_t exps, prefix, desc, items, parts, total;
};

inline BLayout layout_of(int n_blocks, int ncfg, size_t item_bytes, size_t parts_bytes) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    BLayout L;
    L.exps = 256;
    L.prefix = al(L.exps + 8 * (size_t)n_blocks);
    L.desc = al(L.prefix + 4 * (size_t)ncfg * (n_blocks + 1));
    L.items = al(L.desc + sizeof(BlockDesc) * (size_t)n_blocks);
    L.parts = al(L.items + item_bytes);
    L.total = al(L.parts + parts_bytes);
    return L;
}

// geometry of the tensor-core batched kernel (k_batched_tc.cu), shared with its CPU replay
namespace btc {
constexpr int BM = 128;                               // tile rows (tcgen05 M, tensor-memory lanes)
constexpr int ROW = kBatchedPlaneRow;                 // 64 bytes: 32 bf16 K values (one chunk)
constexpr int BOX_ROWS = 128;
constexpr int BOX_BYTES = BOX_ROWS * ROW;             // 8 KB: one plane of one 128-row chunk tile
constexpr int SLOT_BYTES = 3 * BOX_BYTES;             // 24 KB: three planes
constexpr int RING = 5;                               // ring slots
constexpr int MAX_RES_NK = 2;                         // K <= 32 (one chunk, at most two MMA steps):
                                                      // the strip's B tile stays resident
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t SW64 = 4;                          // descriptor swizzle code: 64-byte swizzle
constexpr uint32_t SBO = 8 * ROW;                     // 8-row core-matrix groups, 512 bytes apart

template <int BN>
struct Cfg {
    static constexpr int STRIP_BYTES = 3 * BN * ROW;                  // 48 KB at BN = 256
    static constexpr int BARS = 2 * RING + 4 + 2 * 4 + 1;
    static constexpr int SMEM = 1024 + 2 * STRIP_BYTES + RING * SLOT_BYTES + BN * 4 + BN * 8 +
                                (int)((sizeof(Radix) + 15) / 16 * 16) + BARS * 8 + 16;
};
}  // namespace btc

std::string describe_batched(const Plan &p);
std::string batched_signature(const Plan &p);
int tune_cache_lookup(const std::string &sig);          // -1 if the class has no entry
void tune_cache_record(const std::string &sig, int cfg);

// the whole batched plan (host only): descriptors, prefix sums, plane layout, workspace size
comet_status_t build_batched_plan(const char *expr, int n_blocks, const char *const *label_names, int n_labels,
                                  const int64_t *extents, const comet_dtype_t *dtypes, int n_dtypes,
                                  const comet_plan_opts_t *opts, int tile_hint, Plan *out, std::string *err);

// split path on the tensor cores (k_batched_tc.cu): per-block operand pre-split into planes,
// then the persistent tcgen05 kernel; strip = columns per work item (256 or 128), dual = every
// tile keeps the exact hh products in an accumulator of their own (some block has K > 32)
cudaError_t launch_batched_presplit(const BatchedParams &bp, int n_blocks, bool f64_in, cudaStream_t s);
cudaError_t launch_batched_tc(const BatchedParams &bp, int64_t plane_rows, int strip, bool dual, bool f64_in,
                              cudaStream_t s);

}  // namespace comet
