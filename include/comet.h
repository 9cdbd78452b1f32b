/*
 * comet.h — C ABI of the GB300 tensor-contraction library.
 *
 * The library evaluates dense tensor contractions written in index (Einstein) notation, the
 * operation of the COMET paper (Section 2, "Tensor Contractions"; the operation grammar of
 * Fig. 2b), by the transpose-transpose-GEMM-transpose (TTGT) reformulation of Section 2 and
 * Section 6 ("TTGT", "Optimal permutation for TTGT"), with the multi-operand ordering of
 * Section 6 ("Multi-Operand Expression") and the transpose of Section 6 ("Transpose
 * optimization").  All device work runs in the library's own sm_103a kernels.
 *
 * Conventions shared by every entry point
 *   Layout     Every tensor is dense and column-major in the label order written in the
 *              expression: the first label has stride 1.  (A tensor declared with labels
 *              [k,a,c,i] and extents (64,192,192,64) has element (k,a,c,i) at linear
 *              position k + 64*(a + 192*(c + 192*i)).)
 *   Ownership  The caller owns every device buffer and the stream.  A plan owns host memory
 *              only.  Scratch space ("workspace") is allocated by the caller, sized by
 *              comet_plan_workspace().  No entry point allocates device memory.
 *   Pointers   Device pointers must be 16-byte aligned (COMET_ERR_ALIGN otherwise).
 *   Streams    `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *              Work is enqueued asynchronously; nothing synchronises the host except
 *              comet_sync_status() and comet_contract_host().
 *   Errors     Every call returns a status code; nothing aborts the process, throws across
 *              the ABI or traps on the device.  A kernel whose internal wait runs out of time
 *              records COMET_ERR_TIMEOUT in a device status word and returns; the code
 *              surfaces at the next comet_sync_status().  In a library built with COMET_DEBUG
 *              (libcomet_debug.so) the transpose, GEMM and gemv kernels also test every global
 *              access against the buffers of their launch, skip any access outside them and
 *              record COMET_ERR_BOUNDS the same way.
 *   Threads    Plans are immutable after comet_plan() and may be used from several host
 *              threads at once.
 */
#ifndef COMET_H
#define COMET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct comet_plan_s *comet_plan_t;

typedef enum {
    COMET_OK = 0,
    COMET_ERR_PARSE = 1,        /* expression does not follow the grammar */
    COMET_ERR_LABEL = 2,        /* label without extent, or output label not on the right */
    COMET_ERR_SHAPE = 3,        /* non-positive or inconsistent extent, size overflow */
    COMET_ERR_DTYPE = 4,        /* unknown dtype or operands of different dtypes */
    COMET_ERR_UNSUPPORTED = 5,  /* valid expression outside what the kernels implement */
    COMET_ERR_ALIGN = 6,        /* device pointer not 16-byte aligned */
    COMET_ERR_NULL = 7,         /* required pointer is NULL */
    COMET_ERR_WORKSPACE = 8,    /* workspace missing or smaller than the plan needs */
    COMET_ERR_CUDA = 9,         /* a CUDA runtime call failed (no device, launch error...) */
    COMET_ERR_TIMEOUT = 10,     /* a device-side wait ran out of time (see comet_sync_status) */
    COMET_ERR_INTERNAL = 11,
    COMET_ERR_ARG = 12,         /* an argument is out of range */
    COMET_ERR_BOUNDS = 13       /* builds with COMET_DEBUG only: a kernel access outside the buffer
                                   it belongs to was skipped (see comet_sync_status) */
} comet_status_t;

typedef enum { COMET_F32 = 0, COMET_F64 = 1 } comet_dtype_t;

typedef enum {
    /* FP64 arithmetic: FP64 tensor-core MMA (mma.sync f64) with FP64 accumulation.  For
       FP32-stored operands the values are widened exactly and the result rounded once. */
    COMET_PREC_NATIVE = 0,
    /* Split precision: each operand is scaled by 2^-e (e = exponent of its largest magnitude)
       and every element split into three bfloat16 fixed-point parts, x * 2^-e rounded to
       nearest on the grids 2^-6, 2^-14 and 2^-22; six of the nine part products (hh, hm, mh,
       hl, lh, mm) run on the tensor cores with FP32 accumulation, the hh products in chunks of
       up to 1024 K values that sum exactly.  Target: normwise relative error <= 1e-6 against
       FP64 (measured 3.4e-7 on the o=64 v=192 workload). */
    COMET_PREC_SPLIT_BF16 = 1,
    /* FP64 emulated on the BF16 tensor cores (FP64 storage only, else COMET_ERR_DTYPE): each
       operand is scaled by 2^-e and written as six integer-valued bfloat16 slices on the grids
       2^-6, 2^-14, ..., 2^-46 (residual below 2^-47 of its largest magnitude); the 21 slice
       products of weight <= 5 run on the tensor cores in chunks of 192 K values whose sums of
       weight <= 4 are exact, and are folded into one 64-bit integer per output element, scaled
       and rounded once to FP64.  Merged contraction length K <= 98304.  Target: normwise relative
       error <= 1e-12 against FP64 (an extension of the split form; the paper has no reduced
       precision). */
    COMET_PREC_EMU_F64 = 2
} comet_precision_t;

typedef enum {
    COMET_ORDER_PLANNED = 0,    /* Section 6: fewest operations, ties broken deterministically */
    COMET_ORDER_NATURAL = 1     /* left to right, the baseline of Table 1 */
} comet_order_t;

typedef struct {
    const char *label;          /* label name as written in the expression */
    int64_t extent;             /* > 0 */
} comet_extent_t;

typedef struct {
    comet_precision_t precision;
    comet_order_t order;
    double alpha;               /* extra scale, multiplied into the expression's own alpha */
    size_t workspace_cap;       /* 0 = unlimited; intermediates above it are refused */
    int form;                   /* -1 = planner's choice; k >= 0 = k-th enumerated TTGT form
                                   of every binary step (for the permutation ablation) */
    int64_t kc;                 /* split path: K elements per FP32 accumulation chunk before
                                   the chunk is added into the compensated sum (0 = whole K) */
    int64_t timeout_ms;         /* device-side wait limit; 0 = default (2000 ms) */
    int debug_flags;            /* bit 0: withhold one operand load in the split GEMM so that
                                   its wait runs out (fault-injection test); bit 3, builds with
                                   COMET_DEBUG only: the first thread of a copy step aims its
                                   stores outside the output, so that the range check skips them
                                   and reports COMET_ERR_BOUNDS (test of the check); others
                                   reserved */
    int ksplit;                 /* split path: K slices per output tile; 0 = planner's choice
                                   (more slices when a GEMM has fewer tiles than the GPU has
                                   SMs; their FP32 partials are summed by a second kernel),
                                   1 = off, k > 1 = k slices */
    int host_slices;            /* comet_contract_host on a one-step split or emulated plan:
                                   slices of the larger operand that are copied in, multiplied
                                   and copied back in a pipeline; 0 = planner's choice, 1 = off
                                   (copy all inputs, contract, copy back), s > 1 = s slices */
    int host_slices_w;          /* the same pipeline (unless host_slices is 1): slices of the
                                   smaller operand (0 = planner's choice, 1 = whole, s > 1 = s) */
} comet_plan_opts_t;

/* Fills *opts with the defaults: NATIVE precision, planned order, alpha 1, no cap, planner's
 * form, kc 0, default timeout, no debug flags, planner's K slicing and host slices. */
void comet_plan_opts_default(comet_plan_opts_t *opts);

/*
 * comet_plan — parse, classify and plan a contraction (Section 2; Section 5 ops ta.tc,
 * ta.mult, ta.set; Section 6 TTGT, permutation choice and multi-operand order).
 *
 *   expr       "C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]".  Accepted forms (Fig. 2b):
 *              lhs "=", "+=" or "-=" rhs; rhs is an optional numeric alpha followed by one
 *              or more labelled tensors joined by "*"; an optional "sum_{k,c}" after the
 *              assignment names the summed labels and is checked.  Labels may be written in
 *              [] or ().  The summed labels are those on the right that are not on the left.
 *   extents    n_extents (label, extent) pairs covering every label of the expression.
 *   dtypes     n_dtypes entries: one per right-hand operand, then the output.  All equal.
 *   opts       NULL = defaults.
 *   out_plan   receives the plan; release it with comet_plan_destroy().
 *
 * Supported: one operand (scaled copy / transpose, ta.copy) and two or more operands joined
 * in a binary tree of ta.tc steps.  A label on both operands of a step and on its result is a
 * batch label (the step's GEMM runs once per batch index); a label on one operand only, and
 * not on the result, is summed inside that operand by a reduction step before the tree.
 * A label written twice inside one tensor takes its diagonal.  No device work, no GPU needed.
 */
comet_status_t comet_plan(const char *expr, const comet_extent_t *extents, int n_extents,
                          const comet_dtype_t *dtypes, int n_dtypes,
                          const comet_plan_opts_t *opts, comet_plan_t *out_plan);

/*
 * comet_view_t — one dimension of a stored tensor taken as a slice (Section 4: a label whose
 * range differs from the one the tensor was declared with makes a view, and the operation
 * works on that slice).  The operation reads or writes the indices lo, lo + step, ...,
 * lo + (n - 1) step of a dimension that the stored tensor declares with `declared` indices,
 * n being the extent of the dimension's label in the expression.
 */
typedef struct {
    int operand;                /* 0 .. n_in-1: right-hand operands in expression order;
                                   n_in: the left-hand tensor */
    int dim;                    /* position of the dimension in that tensor's labels as written */
    int64_t declared;           /* extent of the dimension in the stored tensor */
    int64_t lo;                 /* first index taken, >= 0 */
    int64_t step;               /* increment, >= 1; lo + (n - 1) step < declared */
} comet_view_t;

/*
 * comet_plan_views — comet_plan() on views of stored tensors.  The pointers later passed to
 * comet_contract() are the stored (declared) tensors, dense column-major; the plan touches only
 * the view's elements (an output view leaves the rest of the stored tensor unchanged).  Each
 * (operand, dim) pair may appear once; dimensions not listed are whole.  A label written twice
 * inside one tensor (a diagonal, e.g. "t[] = A[i,i]") is accepted by comet_plan() as well: both
 * dimensions take the label's indices.  Views need views' element counts below 2^31 per tensor;
 * batched plans take no views or diagonals.  Errors: COMET_ERR_ARG (operand or dim out of
 * range, a pair given twice), COMET_ERR_SHAPE (declared < 1, lo < 0, step < 1, or the range
 * past the declared extent), then as comet_plan().
 */
comet_status_t comet_plan_views(const char *expr, const comet_extent_t *extents, int n_extents,
                                const comet_view_t *views, int n_views, const comet_dtype_t *dtypes,
                                int n_dtypes, const comet_plan_opts_t *opts, comet_plan_t *out_plan);

/*
 * comet_plan_triples — fused accumulation of permuted contributions into six-index blocks and
 * their energies (the CCSD(T) pattern of Section 3: a 6-D output from two 4-D inputs, with
 * several permuted terms per block):
 *     T_b = sum_p alpha_p * X_bp * Y_bp             (term p: the contraction terms[p])
 *     E_b = sum over the elements of T_b of T_b^2 / D_b,
 *     D_b[l_1..l_6] = sum_q signs[q] * eps_bq[l_q]  (l_q: the q-th label of T)
 * T never goes to memory. COMET_F32 plans run on the tensor cores: a pre-pass writes every
 * operand as three bfloat16 parts (x = h + m + l, residual at most 2^-24 |x|) into the workspace,
 * blocks taken in batches whose parts fit it (at most 2^27 rows of 64 bytes, 8 GB; the
 * environment variable COMET_TRIPLES_BATCH_ROWS lowers the cap); each CTA forms, per tile of
 * 8 x 4^5 values of T_b and term, the six-product split sum in tensor memory, adds it into the
 * tile in shared memory and reduces the tile's energy. A plan with a block whose parts exceed
 * one batch, and COMET_F64 plans, run on the FMA pipes with 4^6 tiles held in registers.
 *   terms        n_terms (1..16) expressions with the same left-hand side T[l_1,...,l_6] (six
 *                distinct labels) and two four-label operands that share exactly one label (the
 *                summed one) and hold three labels of T each, e.g.
 *                "T[a,b,c,i,j,k] = -1.0 * X[d,c,b,i] * Y[a,d,j,k]"
 *   label_names  n_labels (<= 16) names covering every label of the terms
 *   extents      n_blocks x n_labels extents >= 1 (row b: block b, columns as label_names)
 *   signs        six entries, +1 or -1, in T's label order
 *   dtype        COMET_F32 (T from the six split products accumulated in FP32, each T^2 / D
 *                and sums of 16 of them in FP32) or COMET_F64; the block energies are summed
 *                in FP64
 * Errors: COMET_ERR_PARSE / COMET_ERR_LABEL / COMET_ERR_UNSUPPORTED for terms outside this form,
 * COMET_ERR_SHAPE for extents below 1 or a block of 2^31 tiles or more, COMET_ERR_ARG otherwise.
 * comet_plan_workspace() gives the device bytes of the block table (and, for COMET_F32, of the
 * split parts of the largest batch).
 */
comet_status_t comet_plan_triples(const char *const *terms, int n_terms, const char *const *label_names,
                                  int n_labels, int n_blocks, const int64_t *extents, const int *signs,
                                  comet_dtype_t dtype, comet_plan_t *out_plan);

/* comet_triples_prepare — uploads the block table into the workspace (once per workspace). */
comet_status_t comet_triples_prepare(comet_plan_t plan, void *workspace, void *stream);

/*
 * comet_triples_energy — evaluates a triples plan (asynchronous on `stream`; graph-capturable
 * after comet_triples_prepare).
 *   operands   device array of n_blocks * n_terms * 2 device pointers, block-major: X then Y of
 *              term 0, then of term 1, ...; each operand dense column-major in its term's label
 *              order with the block's extents; 16-byte alignment not required
 *   eps        device array of n_blocks * 6 device pointers to the eps vectors (dtype of the plan),
 *              in T's label order
 *   energies   device array of n_blocks doubles, overwritten
 *   workspace  the prepared workspace
 * A device wait of the tensor-core path that runs out (2 s, or COMET_WAIT_TIMEOUT_MS) records
 * COMET_ERR_TIMEOUT for comet_sync_status().
 */
comet_status_t comet_triples_energy(comet_plan_t plan, const void *operands, const void *eps,
                                    double *energies, void *workspace, void *stream);

/*
 * comet_adjoint_expr — the expression of the gradient of a contraction with respect to one
 * operand.  For out = alpha * prod_t X_t (every label in exactly two tensors), the gradient of
 * <G, out> with respect to X_p is alpha * (G contracted with every X_t, t != p) written onto
 * X_p's labels: itself a contraction, planned and run like any other (so a multi-operand
 * adjoint gets its own operand order, which recomputes the intermediates it needs).
 *   expr       a "=" expression accepted by comet_plan
 *   operand    0-based position of X_p on the right-hand side
 *   buf, len   receives "dX[...] = alpha * _G[...] * Y[...] * ..." with the gradient operand
 *              named _G first and the other operands in their original order
 * COMET_ERR_UNSUPPORTED for "+=" / "-=" expressions; COMET_ERR_ARG if buf is too small or
 * operand is out of range.
 */
comet_status_t comet_adjoint_expr(const char *expr, int operand, char *buf, size_t len);

/* Bytes of device workspace comet_contract() needs for this plan (may be 0). */
comet_status_t comet_plan_workspace(comet_plan_t plan, size_t *bytes);

/* Algorithmic flop count of the planned evaluation: sum over binary steps of
 * 2 * product of the extents of all labels of the step. */
comet_status_t comet_plan_flops(comet_plan_t plan, double *flops);

/* Flop count the natural left-to-right order would need (the Table 1 baseline). */
comet_status_t comet_plan_flops_natural(comet_plan_t plan, double *flops);

/* Human-readable JSON description of the plan: steps, operand order, the M/N/K label groups
 * and their order, the chosen form among those enumerated, costs; for a pure permutation step
 * the transpose engine's vector widths in elements (a negative vec_out: copy mode) and tile.
 * Writes at most len bytes including the terminating NUL; COMET_ERR_ARG if it does not fit. */
comet_status_t comet_plan_describe(comet_plan_t plan, char *buf, size_t len);

/*
 * comet_contract — evaluate the plan on device buffers (asynchronous on `stream`).
 *   inputs     one device pointer per right-hand operand, in expression order.
 *   output     device pointer to the left-hand tensor; read as well when the operator is
 *              "+=" or "-=".
 *   workspace  device scratch of at least comet_plan_workspace() bytes (may be NULL if 0).
 * Output and inputs must not overlap.  Launch errors return COMET_ERR_CUDA.
 */
comet_status_t comet_contract(comet_plan_t plan, const void *const *inputs, void *output,
                              void *workspace, void *stream);

/*
 * comet_contract_noalloc — comet_contract() for callers that cannot allocate device memory.
 * (The paper has no counterpart: this exists for library users, not for the method.)
 *
 * Some callers cannot call cudaMalloc or any allocator at the point where they contract: code
 * running under a strict memory budget that was fixed at start-up, plug-ins inside a host
 * application that owns every allocation, or callers with no allocator handle at hand.  This
 * entry point takes the plan's scratch space (the split path's bfloat16 planes and scale words,
 * the intermediates of multi-operand plans) from one array that lives inside the library
 * instead of from a caller buffer.  The caller still passes the inputs and the output.
 *
 *   limit      COMET_NOALLOC_MAX_BYTES of scratch; a plan whose comet_plan_workspace() is
 *              larger is refused with COMET_ERR_WORKSPACE (nothing is launched).
 *   memory     the array is a static device variable: every GPU that loads the library holds
 *              these bytes until the process exits, whether or not this entry point is used.
 *   set-up     the first call on each device looks up the array's device address (with that
 *              device current); make that first call before any stream capture begins.
 *   sharing    every call uses the same array, and the array keeps whatever the last call left
 *              in it (the path clears what it needs cleared).  Calls whose GPU work overlaps,
 *              e.g. on two streams without ordering between them, race on the array.
 *   reset      the looked-up address belongs to the device's current context: after
 *              cudaDeviceReset() (or any teardown of the primary context) the library's device
 *              state, this address included, is stale; reload the library before further calls.
 * Returns the codes of comet_contract().  Allocates no device memory: no cudaMalloc and no
 * allocator call on any path.  Host-side bookkeeping is not covered by that promise: a refusal
 * builds its error message, and with the kernel profiler on (comet_profile_enable) the call
 * creates CUDA timing events like every other entry point.
 */
#define COMET_NOALLOC_MAX_BYTES (32u << 20)
comet_status_t comet_contract_noalloc(comet_plan_t plan, const void *const *inputs, void *output,
                                      void *stream);

/*
 * comet_contract_host — the same evaluation from host buffers: copies every input from host
 * to the caller's device buffers, runs the plan and copies the output back, then synchronises
 * `stream`.  host_* may be pageable or pinned host memory; dev_* are caller-owned device
 * buffers of the operands' sizes (16-byte aligned; for views, the stored tensors' sizes).  For
 * "+=" / "-=" and for an output view the host output is copied to the device as well.  Returns the first error, including a device status word set by a
 * kernel (as comet_sync_status()).
 *
 * Pipeline: for a one-step split or emulated-FP64 plan whose description lists "host_pipe"
 * (comet_plan_opts_t.host_slices), and with every host buffer pinned, the larger operand is
 * copied in slices along the last label of its GEMM row group and each slice is multiplied
 * while the next one is copied in and the previous result slice is copied out (two extra
 * streams of the call, joined into `stream` before it returns).  The result equals that of
 * comet_contract() up to the operand scales of the split, which are taken per slice.  After
 * the call that operand's device buffer holds its slices one after another, each in its own
 * compact column-major layout; the device output holds the result.  Otherwise every copy and
 * kernel runs in order on `stream`.
 */
comet_status_t comet_contract_host(comet_plan_t plan, const void *const *host_inputs,
                                   void *host_output, void *const *dev_inputs, void *dev_output,
                                   void *workspace, void *stream);

/*
 * comet_contract_host_n — n_calls independent evaluations of the same plan from host buffers to
 * host buffers (the contraction of Section 2 each time), through one set of device buffers,
 * then synchronises `stream`.  comet_contract_host() is this call with n_calls = 1.
 *
 *   host_inputs   n_calls x n_in host pointers, call-major: call t's input i is
 *                 host_inputs[t * n_in + i].  The same host buffer may serve several calls.
 *   host_outputs  n_calls host pointers; call t's result lands in host_outputs[t] (for "+=" /
 *                 "-=" it is read as well).  Calls that share an output buffer write it in call
 *                 order, so the buffer ends with the last of them.
 *   dev_inputs, dev_output, workspace   as for comet_contract_host(), shared by every call; the
 *                 device output holds the last call's result afterwards.
 * Pipeline: with the slice pipeline (see comet_contract_host()), the copies of call t + 1 run
 * while call t computes: a slice's copy into its device buffer waits only for call t's
 * pre-pass of that slice, and each GEMM block of call t + 1 waits only for call t's copy-out
 * of the same result region, so that in steady state the host link is hidden behind the GEMMs.
 * Every call's result is the one comet_contract_host() gives for its inputs, bit for bit.
 * Otherwise the calls run one after another on `stream`.
 * Returns COMET_ERR_ARG for n_calls < 1, COMET_ERR_NULL for a missing pointer, else the codes
 * of comet_contract_host(); the host buffers stay in use until the call returns.
 */
comet_status_t comet_contract_host_n(comet_plan_t plan, int n_calls, const void *const *host_inputs,
                                     void *const *host_outputs, void *const *dev_inputs, void *dev_output,
                                     void *workspace, void *stream);

/*
 * comet_transpose — pure permutation of a dense tensor (Section 6, "Transpose optimization";
 * the ta.copy of Section 5 with alpha = 1).  Elements are moved as raw 4- or 8-byte words,
 * so the result is bit-exact (NaN payloads, -0.0, subnormals survive).
 *   rank       1 .. 8
 *   extents    input extents, column-major (extents[0] has stride 1)
 *   perm       output dimension d is input dimension perm[d]: out.extent[d] =
 *              extents[perm[d]] and out[j_0..j_{r-1}] = in[i] with i[perm[d]] = j_d
 *   in, out    device buffers of prod(extents) elements; must not overlap
 */
comet_status_t comet_transpose(int rank, const int64_t *extents, const int *perm,
                               comet_dtype_t dtype, const void *in, void *out, void *stream);

/*
 * comet_fill — every element of a dense device buffer set to one value (the ta.fill operation
 * of the paper's tensor-algebra dialect, Section 5).
 *   out    device buffer of n elements of dtype (16-byte aligned, else COMET_ERR_ALIGN)
 *   value  rounded once to dtype
 * Asynchronous on stream; n = 0 does nothing.
 */
comet_status_t comet_fill(void *out, int64_t n, double value, comet_dtype_t dtype, void *stream);

/*
 * Batched triples-like blocks: many small contractions of the same expression with uneven
 * extents, all run by one persistent launch (the 6-D triples output of the CCSD(T) remark in
 * Section 2 is the model: T[a,b,c,i,j,k] = sum_d A[d,a,b,i] * B[c,d,j,k] per block).
 *
 * comet_plan_batched — expr must be a two-operand "=" contraction.  label_names lists the
 *   n_labels labels; extents is an n_blocks x n_labels row-major table (block b, label l at
 *   extents[b*n_labels + l]).  dtypes as in comet_plan.  tile_hint: -1 = the tile
 *   configuration the autotuner recorded for this problem class in this process (else the
 *   default), k >= 0 = the k-th configuration.  No device work.
 */
comet_status_t comet_plan_batched(const char *expr, int n_blocks, const char *const *label_names,
                                  int n_labels, const int64_t *extents,
                                  const comet_dtype_t *dtypes, int n_dtypes,
                                  const comet_plan_opts_t *opts, int tile_hint,
                                  comet_plan_t *out_plan);

/* Number of tile configurations comet_plan_batched() accepts as tile_hint (for the precision
 * of `plan`; NULL = the FP64 path). */
int comet_batched_num_tiles(comet_plan_t plan);

/* Selects tile configuration cfg for a batched plan. */
comet_status_t comet_batched_set_tile(comet_plan_t plan, int cfg);

/*
 * comet_batched_prepare — copies the plan's per-block descriptors (label groups, strides,
 * divisors, the longest-first block order and the tile prefix sums) into `workspace`
 * (comet_plan_workspace() bytes) and synchronises the stream.  Call once per workspace,
 * before any stream capture; comet_contract_batched() then only reads it.
 */
comet_status_t comet_batched_prepare(comet_plan_t plan, void *workspace, void *stream);

/*
 * comet_contract_batched — run every block in one persistent launch (capturable in a CUDA
 * graph once comet_batched_prepare() has run on `workspace`).
 *   block_inputs   device array of n_blocks * 2 device pointers (block-major: A_b, B_b),
 *                  each a dense column-major operand of that block's extents.
 *   mode 0 (reduce): `result` is a device array of 2*n_blocks doubles; block b gets
 *                  s_b = sum T*W and q_b = sum T^2 over its output T.  The weight of an
 *                  element is W = h(weight_key, b, oA) * h(~weight_key, b, oB), where the
 *                  element's column-major linear index in T is oA + oB, oA the part that the
 *                  labels of the expression's first operand contribute and oB that of the
 *                  second operand's labels, and h(k, b, x) = (fmix32(k ^ fmix32(b *
 *                  0x9E3779B9 + x)) >> 8) * 2^-23 - 1 (MurmurHash3 finalizer, 32-bit
 *                  wraparound).  T is never stored.
 *   mode 1 (store):  `result` is a device array of n_blocks device pointers; block b's output
 *                  is written there in full (blocks whose pointer is NULL are skipped).
 *   The launch resets its own work counter and, in mode 0, zeroes `result` first.
 *   Split precision runs on the tcgen05 tensor cores (blocks of K <= 1024); its waits are
 *   bounded by opts.timeout_ms (COMET_ERR_TIMEOUT at comet_sync_status() when one runs out).
 */
comet_status_t comet_contract_batched(comet_plan_t plan, const void *const *block_inputs,
                                      int mode, void *result, uint32_t weight_key,
                                      void *workspace, void *stream);

/*
 * comet_batched_autotune — times every tile configuration on the first sample_blocks blocks
 * of the longest-first order (0 = all) in reduce mode, writes each configuration's time to
 * ms_per_cfg (n_cfg entries, may be NULL), selects the fastest for `plan`, and records it for
 * later comet_plan_batched(tile_hint = -1) calls of the same problem class in this process
 * (and in the file named by the environment variable COMET_AUTOTUNE_CACHE, if set).
 * Needs a prepared workspace; synchronises the stream; not capturable.
 */
comet_status_t comet_batched_autotune(comet_plan_t plan, const void *const *block_inputs, void *result,
                                      void *workspace, int sample_blocks, void *stream,
                                      double *ms_per_cfg, int n_cfg, int *best);

/*
 * Kernel timing (tracing).  While enabled, every kernel launch the library makes is bracketed
 * by a pair of CUDA events recorded on the launching stream (not allowed during stream
 * capture).  comet_profile_read() synchronises on the recorded events and returns, per kernel
 * kind, the number of launches and their summed device time, then clears the record.
 *   kind names: "transpose", "scale_copy", "split_prepass", "gemm_split_bf16", "gemm_f64",
 *               "batched_f64", "batched_split" (the tcgen05 kernel), "batched_prepass" (its
 *               abs-max and split passes), "gemm_emu_bf16x6", "gemv", "triples_energy"
 */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} comet_kernel_stat_t;

comet_status_t comet_profile_enable(int on);
comet_status_t comet_profile_read(comet_kernel_stat_t *stats, int max_stats, int *n_stats);

/*
 * comet_probe_fp64 — FP64 throughput probe, the measured denominator of the FP64 rooflines
 * (a measurement utility; the paper has no counterpart).  Launches one kernel on `stream` that
 * keeps the FP64 pipe busy with independent dependency chains and no memory traffic; the caller
 * times it (CUDA events on the same stream) and divides *flops by the elapsed time.
 *   kind   0 DFMA (FP64 FMA pipe), 1 f64 tensor-core MMA m8n8k4, 2 m16n8k4, 3 m16n8k16
 *   iters  loop trips per thread, 1 .. 2^24 (the launch's duration grows linearly with it)
 *   flops  host out: the FP64 flops the launch performs (an FMA counts 2)
 *   sink   device buffer of at least 8 bytes (caller-owned; written only under a condition
 *          that never holds, so that the arithmetic cannot be dropped by the compiler)
 * Errors: COMET_ERR_NULL, COMET_ERR_ARG (kind or iters out of range), COMET_ERR_CUDA (launch).
 */
comet_status_t comet_probe_fp64(int kind, int iters, double *flops, void *sink, void *stream);

/* Synchronises `stream`, then reads and clears the device status word: COMET_OK, or
 * COMET_ERR_TIMEOUT if a kernel's wait ran out, COMET_ERR_BOUNDS (debug builds only) if a
 * kernel skipped an access outside its buffers, or COMET_ERR_CUDA if the stream reported an
 * error. */
comet_status_t comet_sync_status(void *stream);

void comet_plan_destroy(comet_plan_t plan);

const char *comet_status_string(comet_status_t status);

/* Detail of the last error returned to the calling host thread (empty if none). */
const char *comet_last_error_message(void);

/* Library version string ("... debug ..." for the COMET_DEBUG build). */
const char *comet_version(void);

#ifdef __cplusplus
}
#endif

#endif /* COMET_H */
