// Host-side planner: parsing (Fig. 2b grammar), label classification (Section 2), operand
// ordering (Section 6 "Multi-Operand Expression") and TTGT form choice (Section 6 "TTGT",
// "Optimal permutation for TTGT").  No device work happens here.
#pragma once
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/comet.h"
#include "params.h"

namespace comet {

struct ParsedTensor {
    std::string name;
    std::vector<std::string> labels;
};

struct ParsedExpr {
    ParsedTensor out;
    std::vector<ParsedTensor> ins;
    int op = 0;                  // 0 "=", 1 "+=", 2 "-="
    double alpha = 1.0;
    bool has_sum = false;
    std::vector<std::string> sum_labels;
};

comet_status_t parse_expr(const char *s, ParsedExpr *e, std::string *err);

enum KernelKind { KK_GEMM_F64 = 0, KK_GEMM_SPLIT = 1, KK_COPY = 2, KK_GEMM_EMU = 3, KK_GEMV = 4, KK_REDUCE = 5 };

// One TTGT form of a binary step: which input provides the M (row) group, and the order of
// the labels inside M, N and K (first = fastest in the merged index).
struct Form {
    int swap = 0;                // 0: the step's first input is the M operand
    std::vector<int> M, N, K;
    std::vector<int> Bt;         // batch labels: on both inputs and the result (not merged)
    double cost = 0;             // modelled seconds
    double pre_bytes = 0;        // bytes moved by explicit pre-passes
    double eff_store = 1, eff_a = 1, eff_b = 1;
};

enum SlotKind { SLOT_INPUT = 0, SLOT_INTER = 1, SLOT_OUTPUT = 2 };

struct Slot {
    int kind = SLOT_INPUT;
    int index = 0;               // input position for SLOT_INPUT
    std::vector<int> labels;     // column-major label order of this tensor (each label once)
    int64_t elems = 1;           // elements the operation touches (product of label extents)
    size_t ws_off = 0;           // SLOT_INTER: byte offset in the workspace
    // inputs and the output: element strides by label id and the offset of the first element
    // touched.  A plain tensor is dense column-major (offset 0, storage = elems); a view (a
    // dimension sliced by lo:step, or a label written twice, i.e. a diagonal) has the strides
    // of its stored tensor times the steps, summed over the dimensions that share a label.
    bool view = false;
    std::map<int, int64_t> strides;
    int64_t offset = 0;
    int64_t storage = 1;         // elements of the stored tensor (declared extents)
    Radix vradix;                // view inputs: every label, smallest stride first (abs-max)
};

struct Step {
    int a = -1, b = -1, c = -1;  // slots (b = -1 for a copy)
    int kernel = KK_GEMM_F64;
    Form form;
    int n_forms = 1;
    int form_index = 0;
    double flops = 0;
    bool final_step = false;
    // split path workspace for the bf16 parts: [3][rows][kpad]
    size_t ws_parts_a = 0, ws_parts_b = 0;
    size_t ws_scales = 0;        // two 8-byte words: max |A|, max |B| of the step's operands
    int64_t kpad = 0;
    uint32_t ksplit = 1;         // split GEMM: K slices per output tile
    size_t ws_ksplit = 0;        // workspace offset of the slices' FP32 partials
    size_t ksplit_bytes = 0;     // their size (K slices of every tile, or of a partial last wave)
    uint32_t tail_tiles = 0, tail_slices = 1;   // whole-K split GEMM on 152 SMs: the partial last
                                                // wave's tiles and their K slices (1 = no tail split)
    // precomputed parameter blocks (pointers filled at launch)
    GemmParams gemm;             // for both GEMM kernels (offsets in elements)
    XposeParams pre_a, pre_b;    // split pre-passes (A then B operand)
    XposeParams copy;            // KK_COPY
    GemvParams gemv;             // KK_GEMV (one operand has no free label)
    bool gemv_vec_is_a = true;   // the vector is the GEMM's A (M) operand, else its B operand
    size_t ws_partial = 0;       // KK_GEMV: workspace offset of the chunk partial sums
    // batch labels of the step: the kernels run once per batch index, with the operands' and
    // the result's base offsets (elements) of that index; extents and the three stride sets
    std::vector<int64_t> bt_ext, bt_sa, bt_sb, bt_sc;
    int64_t n_batch = 1;
    int pre_a_vec = 1, pre_b_vec = 1, pre_a_vout = 1, pre_b_vout = 1;
    int copy_vec_in = 1, copy_vec_out = 1;
};

// Host-buffer pipeline of a one-step split or emulated-FP64 plan (comet_contract_host): the
// larger operand X crosses in slices along the last (slowest) label L of its GEMM row group, the
// other operand W in slices along the last label of its own row group.  Each slice lands compact
// (its own column-major layout with the label shortened), gets its own scale word and planes,
// and is pre-passed when its copy is in; GEMM block (i, j) = W slice i x X slice j (the step's
// GEMM with both row groups shortened, writing through the full result strides) runs once both
// are in.  Copies alternate W_0, X_0, W_1, X_1, ...; blocks run in the order their inputs
// arrive; results go back block by block when the result's layout makes a block a 3-D box,
// else column by column after a column's last block.
struct HostPipe {
    bool ok = false;
    int side = 1;                // 1: X is the N operand (GEMM B), 0: the M operand (GEMM A)
    int x_in = 1, w_in = 0;      // input positions of X and W
    int label = -1;              // L
    int64_t ext = 0;             // extent of L
    int n_chunks = 0;            // X slices
    std::vector<int64_t> xb;     // X slice boundaries along L (n_chunks + 1)
    int64_t x_inner = 1, x_outer = 1;  // X elements below L (its stride), and the count above it
    int64_t c_inner = 1, c_outer = 1;  // the same for the result
    int64_t rows_inner = 1;      // GEMM rows of X's group per unit of L
    std::vector<XposeParams> pre;      // pre-pass of each X slice
    std::vector<int> pre_vec, pre_vout;
    int w_label = -1;
    int64_t w_ext = 1;
    int w_n = 1;
    std::vector<int64_t> wb;     // W slice boundaries along its label (w_n + 1)
    int64_t w_inner = 1, w_outer = 1, wc_inner = 1, w_rows_inner = 1;
    std::vector<XposeParams> w_pre;
    std::vector<int> w_pre_vec, w_pre_vout;
    std::vector<int> copies;     // copy order: j >= 0 X slice j, -1 - i W slice i
    std::vector<int> blocks;     // GEMM order: i * n_chunks + j
    bool blockwise = false;      // results go back block by block
    double model_s[2] = {0, 0};  // modelled seconds: unpipelined, pipelined
};

// Fused triples accumulation (comet_plan_triples): T_b = sum_p alpha_p X_bp * Y_bp over terms
// that each contract one label between two 4-index operands into the same six-index T, and
// E_b = sum T_b^2 / D_b.  Label maps per term; extents per block.
struct TriTerm {
    double alpha = 1.0;
    int x_q[4] = {0, 0, 0, 0}, y_q[4] = {0, 0, 0, 0};   // per operand dimension: T label position, -1 = summed
    int x_col[4] = {0, 0, 0, 0}, y_col[4] = {0, 0, 0, 0};   // extent-table column of each dimension's label
    int d_col = 0;                                       // extent-table column of the summed label
};
struct TriplesPlan {
    int n_terms = 0, n_labels = 0, n_blocks = 0;
    std::vector<TriTerm> terms;
    int t_col[6] = {0, 0, 0, 0, 0, 0};   // extent-table column of each T label
    int signs[6] = {1, 1, 1, 1, 1, 1};   // sign of each T label's eps in D
    int own[2] = {0, 1};                 // T labels a thread holds 4 x 4 of (the other four are fixed)
    std::vector<int32_t> ext;            // n_blocks x n_labels
    std::vector<int64_t> prefix;         // tiles (4 per label) before each block; n_blocks + 1
    size_t ws_ext = 0, ws_prefix = 0, ws_counter = 0;
    // FP32 plans, tensor-core path: pair-tiles (8 along T label 0, 4 along the others), blocks in
    // batches whose split operand planes fit the workspace
    std::vector<int64_t> tc_prefix;      // pair-tiles before each block; n_blocks + 1
    std::vector<int32_t> tc_row0;        // n_blocks x n_terms x 2: first plane row of each operand in its batch
    std::vector<int32_t> tc_rec;         // n_blocks x n_terms records of 16 words (tri::TcRec)
    std::vector<int64_t> tc_rows;        // plane rows of each block (all its operands)
    std::vector<int> tc_batch;           // first block of each batch, then n_blocks
    int64_t tc_max_rows = 0;             // plane rows of the largest batch
    size_t ws_tc_row0 = 0, ws_tc_prefix = 0, ws_tc_rec = 0, ws_tc_planes = 0;
};

struct Plan {
    std::string expr;
    ParsedExpr parsed;
    std::vector<std::string> label_names;
    std::vector<int64_t> extent;
    int n_in = 0;
    comet_dtype_t dtype = COMET_F64;
    comet_plan_opts_t opts;
    double alpha = 1.0;          // expression alpha times opts.alpha
    int op = 0;
    std::vector<Slot> slots;
    std::vector<Step> steps;
    size_t workspace = 0;
    double flops = 0, flops_natural = 0;
    std::string tree;            // parenthesised order, e.g. "((A*B)*C)"
    // batched plans
    bool batched = false;
    int n_blocks = 0;
    std::vector<int64_t> block_extents;   // n_blocks x n_labels
    int tile_cfg = 0;
    size_t batched_ws = 0;
    size_t batched_parts = 0;             // split path: bytes of the pre-split operand planes
    std::vector<uint8_t> batched_table;   // host image of the prefix sums and the descriptors
    std::vector<std::vector<uint32_t>> batched_prefix;   // per tile configuration
    std::vector<double> block_flops;
    bool batched_ak = false, batched_bk = false, batched_swap = false;
    bool batched_dual = false;            // split path: some block has K > 32 (hh kept apart)
    int64_t batched_plane_rows = 0;       // split path: rows of 16 bf16 in the plane region
    size_t batched_item_bytes = 0;        // split path: item records of every configuration
    std::vector<size_t> batched_item_off; // split path: byte offset of each configuration's records
    HostPipe pipe;                        // comet_contract_host slicing (one-step plans)
    bool triples = false;                 // comet_plan_triples
    TriplesPlan tri;
};

size_t dtype_size(comet_dtype_t t);

comet_status_t build_plan(const char *expr, const comet_extent_t *extents, int n_extents,
                          const comet_view_t *views, int n_views, const comet_dtype_t *dtypes,
                          int n_dtypes, const comet_plan_opts_t *opts, Plan *plan, std::string *err);

std::string describe_plan(const Plan &p);
std::string describe_triples(const Plan &p);

// GEMM parameters of one binary step for given extents: lm / ln = labels of the M and N
// operands, lc = labels of the output (all column-major), f = the TTGT form.
void gemm_params_for(const std::vector<int64_t> &extent, const std::vector<int> &lm,
                     const std::vector<int> &ln, const std::vector<int> &lc, const Form &f,
                     GemmParams *g);

// Transpose engine set-up for a permutation of a dense column-major tensor with arbitrary
// output strides.  in_strides/out_strides in elements; returns the vector widths usable for
// loads and stores (1, 2 or 4 elements of elem_bytes).  in_off / out_off: element offsets of
// the first element from 16-byte aligned bases (16-byte accesses need them aligned too).
void setup_xpose(int rank, const int64_t *ext, const int64_t *in_strides,
                 const int64_t *out_strides, int elem_bytes, XposeParams *p,
                 int *vec_in, int *vec_out, double *eff, int64_t in_off = 0, int64_t out_off = 0);

}  // namespace comet
