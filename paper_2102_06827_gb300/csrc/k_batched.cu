// Batched triples-like contractions in one persistent launch: plan, workspace, launch
// sequence, autotuner, and the FP64 kernel.
//
// Many small contractions of one two-operand expression with uneven extents (the model is the
// 6-D triples output of the CCSD(T) remark in Section 2: T[a,b,c,i,j,k] = sum_d A[d,a,b,i] *
// B[c,d,j,k] per block).  Every block is a GEMM over its merged label groups (the TTGT view of
// Section 2, with the permutations folded into the index arithmetic).  Work items are (block,
// strip of output columns) pairs numbered through prefix sums of the blocks' strip counts,
// blocks in longest-first order, so uneven blocks balance across the SMs.
//
// Two arithmetic paths:
//   FP64   f64 tensor-core MMA (mma.sync m8n8k4; every f64 MMA shape of sm_103a runs at the
//          same rate), FP64 accumulation; persistent CTAs take items from an atomic counter
//   split  the fixed-point three-way bfloat16 split of each operand, then the tcgen05 kernel
//          of k_batched_tc.cu (TMA tiles, tensor-memory accumulators)
// The output T of a block is either consumed in the epilogue (reduce mode: s_b = sum T*W and
// q_b = sum T^2 with the separable hashed weight of triples_weight.cuh) or stored (store mode).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <numeric>
#include <sstream>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/comet.h"
#include "batched.h"
#include "launch.h"
#include "params.h"
#include "split.cuh"
#include "triples_weight.cuh"

static_assert(sizeof(comet::BlockDesc) % 16 == 0, "descriptors are copied as 16-byte words");

struct comet_plan_s {
    comet::Plan p;
};

namespace comet {

int prof_begin(int kind, cudaStream_t s);
void prof_end(int idx, cudaStream_t s);
enum { PK_BATCHED_F64_ID = 5, PK_BATCHED_SPLIT_ID = 6, PK_BATCHED_PREPASS_ID = 10 };
void set_error_message(const std::string &s);

// ---- device helpers ----------------------------------------------------------------------------
__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

constexpr int BT = 128;      // threads per CTA (2 x 2 warps)
constexpr int KCH = 32;      // K chunk staged in shared memory

// Takes the next work item; returns false when none is left.  Thread 0 takes it, everyone
// reads it after the barrier.
__device__ __forceinline__ bool next_item(const BatchedParams &P, uint32_t &item, uint32_t &pos,
                                          uint32_t *s_item, uint32_t *s_pos) {
    if (threadIdx.x == 0) {
        uint32_t it = atomicAdd(P.counter, 1u);
        uint32_t lo = 0;
        if (it < P.total_tiles) {
            uint32_t hi = P.n_blocks;   // prefix[lo] <= it < prefix[hi]
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (P.prefix[mid] <= it) lo = mid; else hi = mid;
            }
        }
        *s_item = it;
        *s_pos = lo;
    }
    __syncthreads();
    item = *s_item;
    pos = *s_pos;
    return item < P.total_tiles;
}

__device__ __forceinline__ void copy_desc(const BlockDesc *src, BlockDesc *dst) {
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(BlockDesc) / 16); i += BT) d[i] = s[i];
}

// CTA-wide sum of two doubles; thread 0 adds them to result[2*idx], result[2*idx+1]
__device__ __forceinline__ void reduce_add(double s, double q, double *red, double *result, uint32_t idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        q += __shfl_down_sync(0xffffffffu, q, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[2 * w] = s; red[2 * w + 1] = q; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ss = 0, qq = 0;
        for (int i = 0; i < BT / 32; ++i) { ss += red[2 * i]; qq += red[2 * i + 1]; }
        atomicAdd(result + 2 * idx, ss);
        atomicAdd(result + 2 * idx + 1, qq);
    }
}

// A work item is one N-strip of one block: BN output columns and every M tile of them.  When
// the contracted extent fits one chunk (K <= KCH, the triples case), the strip's B operand is
// loaded (and split) once and reused by every M tile; s and q accumulate over the strip, so
// one pair of atomic additions closes it.

// ---- FP64 path -------------------------------------------------------------------------------
template <int BM, int BN, bool AK, bool BKC, typename TIn>
__global__ void __launch_bounds__(BT) batched_f64_kernel(const BatchedParams P) {
    constexpr int MI = BM / 16, NJ = BN / 16;   // 8-row / 8-column MMA tiles per warp
    __shared__ double As[KCH][BM + 4];
    __shared__ double Bs[KCH][BN + 4];
    __shared__ int64_t a_row[BM], o_row[BM], b_col[BN], o_col[BN], a_k[KCH], b_k[KCH];
    __shared__ float w_row[BM], w_col[BN];   // weight factors of the tile's rows and the strip's columns
    __shared__ __align__(16) BlockDesc sd;
    __shared__ double red[2 * BT / 32];
    __shared__ uint32_t s_item, s_pos;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, wm = warp & 1, wn = warp >> 1;
    uint32_t item, pos;
    while (next_item(P, item, pos, &s_item, &s_pos)) {
        copy_desc(P.desc + pos, &sd);
        __syncthreads();
        const uint32_t M = sd.M, N = sd.N, K = sd.K, idx = sd.index;
        const uint32_t mtiles = (M + BM - 1) / BM;
        const uint32_t n0 = (item - P.prefix[pos]) * BN;
        const bool bres = K <= (uint32_t)KCH;
        const uint32_t hb = idx * 0x9E3779B9u, key_m = P.swap ? ~P.key : P.key, key_n = ~key_m;
        for (int i = t; i < BN; i += BT) {
            int64_t o0 = 0, o1 = 0;
            if (n0 + i < N) radix_offsets(sd.nb, n0 + i, o0, o1);
            b_col[i] = o0; o_col[i] = o1;
            w_col[i] = tri_factor(key_n, hb, (uint32_t)o1);
        }
        if (t < KCH) {
            int64_t o0 = 0, o1 = 0;
            if ((uint32_t)t < K) radix_offsets(sd.k, t, o0, o1);
            a_k[t] = o0; b_k[t] = o1;
        }
        const TIn *A = reinterpret_cast<const TIn *>(P.inputs[2 * idx + P.swap]);
        const TIn *B = reinterpret_cast<const TIn *>(P.inputs[2 * idx + 1 - P.swap]);
        auto load_b = [&](uint32_t k0) {
            for (int e = t; e < BN * KCH; e += BT) {
                int n, k;
                if (BKC) { k = e % KCH; n = e / KCH; } else { n = e % BN; k = e / BN; }
                Bs[k][n] = (n0 + n < N && k0 + k < K &&
                            dbg_ok(dbg_range(B, sd.b_elems * (int64_t)sizeof(TIn)), B + b_col[n] + b_k[k],
                                   (int)sizeof(TIn), P.status))
                               ? (double)B[b_col[n] + b_k[k]] : 0.0;
            }
        };
        __syncthreads();
        if (bres) load_b(0);
        double s = 0.0, q = 0.0;
        TIn *out = P.mode == 1 ? reinterpret_cast<TIn *const *>(P.result)[idx] : nullptr;
        for (uint32_t mt = 0; mt < mtiles; ++mt) {
            const uint32_t m0 = mt * BM;
            __syncthreads();
            for (int i = t; i < BM; i += BT) {
                int64_t o0 = 0, o1 = 0;
                if (m0 + i < M) radix_offsets(sd.ma, m0 + i, o0, o1);
                a_row[i] = o0; o_row[i] = o1;
                w_row[i] = tri_factor(key_m, hb, (uint32_t)o1);
            }
            __syncthreads();
            double acc[MI][NJ][2];
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
            for (uint32_t k0 = 0; k0 < K; k0 += KCH) {
                if (!bres) {
                    __syncthreads();
                    if (t < KCH) {
                        int64_t o0 = 0, o1 = 0;
                        if (k0 + t < K) radix_offsets(sd.k, k0 + t, o0, o1);
                        a_k[t] = o0; b_k[t] = o1;
                    }
                    __syncthreads();
                    load_b(k0);
                }
                for (int e = t; e < BM * KCH; e += BT) {
                    int m, k;
                    if (AK) { k = e % KCH; m = e / KCH; } else { m = e % BM; k = e / BM; }
                    As[k][m] = (m0 + m < M && k0 + k < K &&
                                dbg_ok(dbg_range(A, sd.a_elems * (int64_t)sizeof(TIn)), A + a_row[m] + a_k[k],
                                       (int)sizeof(TIn), P.status))
                                   ? (double)A[a_row[m] + a_k[k]] : 0.0;
                }
                __syncthreads();
                const int kmax = (int)min((uint32_t)KCH, K - k0);
#pragma unroll
                for (int k4 = 0; k4 < KCH / 4; ++k4) {
                    if (k4 * 4 >= kmax) break;
                    const int kk = k4 * 4 + (lane & 3);
                    double af[MI], bf[NJ];
#pragma unroll
                    for (int i = 0; i < MI; ++i) af[i] = As[kk][wm * (BM / 2) + i * 8 + (lane >> 2)];
#pragma unroll
                    for (int j = 0; j < NJ; ++j) bf[j] = Bs[kk][wn * (BN / 2) + j * 8 + (lane >> 2)];
#pragma unroll
                    for (int i = 0; i < MI; ++i)
#pragma unroll
                        for (int j = 0; j < NJ; ++j) dmma(acc[i][j], af[i], bf[j]);
                }
            }
#pragma unroll
            for (int i = 0; i < MI; ++i) {
                const int ml = wm * (BM / 2) + i * 8 + (lane >> 2);
#pragma unroll
                for (int j = 0; j < NJ; ++j)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int nl = wn * (BN / 2) + j * 8 + (lane & 3) * 2 + h;
                        if (m0 + ml < M && n0 + nl < N) {
                            const double T = P.alpha * acc[i][j][h];
                            if (P.mode == 0) {
                                s += T * ((double)w_row[ml] * (double)w_col[nl]);
                                q += T * T;
                            } else if (out && dbg_ok(dbg_range(out, (int64_t)M * N * (int64_t)sizeof(TIn)),
                                                     out + o_row[ml] + o_col[nl], (int)sizeof(TIn), P.status)) {
                                out[o_row[ml] + o_col[nl]] = (TIn)T;
                            }
                        }
                    }
            }
        }
        if (P.mode == 0) reduce_add(s, q, red, reinterpret_cast<double *>(P.result), idx);
        __syncthreads();
    }
}

// per-block operand scale exponents (split path): CTA c reduces operand c%2 of block c/2.
// The largest magnitude is taken on the bit patterns with the sign bit cleared (for finite
// values the unsigned integer order is the order of magnitudes), so the reduction is exact
// and runs on the integer pipe for both input precisions.
template <typename TIn>
__global__ void __launch_bounds__(256) batched_absmax_kernel(const BatchedParams P) {
    using U = typename std::conditional<sizeof(TIn) == 4, uint32_t, unsigned long long>::type;
    constexpr U MAG = sizeof(TIn) == 4 ? (U)0x7FFFFFFFu : (U)0x7FFFFFFFFFFFFFFFull;
    __shared__ U red[8];
    const BlockDesc &d = P.desc[blockIdx.x >> 1];
    const int op = blockIdx.x & 1;
    const int64_t n = op ? d.b_elems : d.a_elems;
    const U *x = reinterpret_cast<const U *>(P.inputs[2 * d.index + (op ^ P.swap)]);
    U m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    int64_t i = threadIdx.x;
    for (; i + 3 * 256 < n; i += 4 * 256) {
        m0 = max(m0, x[i] & MAG);
        m1 = max(m1, x[i + 256] & MAG);
        m2 = max(m2, x[i + 512] & MAG);
        m3 = max(m3, x[i + 768] & MAG);
    }
    for (; i < n; i += 256) m0 = max(m0, x[i] & MAG);
    U m = max(max(m0, m1), max(m2, m3));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, (U)__shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        U mm = 0;
        for (int w = 0; w < 8; ++w) mm = max(mm, red[w]);
        // exponent e with max |x| in [2^e, 2^(e+1)); 0 for an all-zero or non-finite operand
        int e = 0;
        if constexpr (sizeof(TIn) == 4) {
            const float v = __uint_as_float((uint32_t)mm);
            if (v > 0.0f && !isinf(v) && !isnan(v)) { frexpf(v, &e); e -= 1; }
        } else {
            const double v = __longlong_as_double((long long)mm);
            if (v > 0.0 && !isinf(v) && !isnan(v)) { frexp(v, &e); e -= 1; }
        }
        const_cast<int *>(P.exps)[2 * d.index + op] = e;
    }
}

// ---- host side ---------------------------------------------------------------------------------
static cudaError_t launch_batched_f64(const Plan &P, int cfg, const BatchedParams &bp, cudaStream_t s, int ctas) {
    const bool f32 = P.dtype == COMET_F32;
    const bool ak = P.batched_ak, bk = P.batched_bk;
#define CM_F64(BMv, BNv, T)                                                                         \
    do {                                                                                            \
        if (ak && bk) batched_f64_kernel<BMv, BNv, true, true, T><<<ctas, BT, 0, s>>>(bp);         \
        else if (ak) batched_f64_kernel<BMv, BNv, true, false, T><<<ctas, BT, 0, s>>>(bp);         \
        else if (bk) batched_f64_kernel<BMv, BNv, false, true, T><<<ctas, BT, 0, s>>>(bp);         \
        else batched_f64_kernel<BMv, BNv, false, false, T><<<ctas, BT, 0, s>>>(bp);                \
    } while (0)
    if (f32) {
        switch (cfg) { case 0: CM_F64(64, 64, float); break; case 1: CM_F64(64, 32, float); break;
                       case 2: CM_F64(32, 64, float); break; default: CM_F64(32, 32, float); }
    } else {
        switch (cfg) { case 0: CM_F64(64, 64, double); break; case 1: CM_F64(64, 32, double); break;
                       case 2: CM_F64(32, 64, double); break; default: CM_F64(32, 32, double); }
    }
#undef CM_F64
    return cudaGetLastError();
}

static int resident_ctas() {
    static int n = 0;
    if (!n) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        n = std::max(1, sms) * 4;   // four 128-thread CTAs per SM
    }
    return n;
}

// the launch sequence of one batched contraction (on a prepared workspace)
static comet_status_t run_batched(const Plan &P, const void *const *block_inputs, int mode, void *result,
                                  uint32_t key, void *ws, cudaStream_t s, int cfg, int sample_blocks) {
    const BLayout L = layout_of(P.n_blocks, n_cfg(P), P.batched_item_bytes, P.batched_parts);
    char *w = static_cast<char *>(ws);
    BatchedParams bp;
    bp.desc = reinterpret_cast<const BlockDesc *>(w + L.desc);
    bp.prefix = reinterpret_cast<const uint32_t *>(w + L.prefix) + (size_t)cfg * (P.n_blocks + 1);
    bp.n_blocks = (uint32_t)P.n_blocks;
    const std::vector<uint32_t> &pre = P.batched_prefix[cfg];
    const int nb = sample_blocks > 0 ? std::min(sample_blocks, P.n_blocks) : P.n_blocks;
    bp.total_tiles = pre[nb];
    bp.inputs = block_inputs;
    bp.swap = P.batched_swap ? 1 : 0;
    bp.mode = mode;
    bp.result = result;
    bp.key = key;
    bp.counter = reinterpret_cast<unsigned int *>(w);
    bp.exps = reinterpret_cast<const int *>(w + L.exps);
    bp.alpha = P.alpha;
    bp.ws = w;
    bp.planes = w + L.parts;
    bp.planes_bytes = P.batched_plane_rows * (int64_t)kBatchedPlaneRow;
    bp.items = P.batched_item_off.empty() ? nullptr
                                          : reinterpret_cast<const ItemRec *>(w + L.items + P.batched_item_off[cfg]);
    bp.status = device_status_word();
    bp.timeout_ns = (P.opts.timeout_ms > 0 ? P.opts.timeout_ms : 2000) * 1000000ll;
    bp.debug_flags = P.opts.debug_flags;
    if (!bp.status) return COMET_ERR_CUDA;
    cudaError_t e = cudaMemsetAsync(w, 0, 16, s);
    if (e == cudaSuccess && mode == 0) e = cudaMemsetAsync(result, 0, 16 * (size_t)P.n_blocks, s);
    if (e != cudaSuccess) return COMET_ERR_CUDA;
    if (P.opts.precision == COMET_PREC_SPLIT_BF16) {
        int h = prof_begin(PK_BATCHED_PREPASS_ID, s);
        if (P.dtype == COMET_F32) batched_absmax_kernel<float><<<2 * nb, 256, 0, s>>>(bp);
        else batched_absmax_kernel<double><<<2 * nb, 256, 0, s>>>(bp);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_batched_presplit(bp, nb, P.dtype == COMET_F64, s);
        prof_end(h, s);
        if (e == cudaSuccess) {
            h = prof_begin(PK_BATCHED_SPLIT_ID, s);
            e = launch_batched_tc(bp, P.batched_plane_rows, cfg_of(P, cfg).bn, P.batched_dual, P.dtype == COMET_F64, s);
            prof_end(h, s);
        }
    } else {
        int h = prof_begin(PK_BATCHED_F64_ID, s);
        const int ctas = (int)std::max<uint32_t>(1, std::min<uint32_t>(bp.total_tiles, (uint32_t)resident_ctas()));
        e = launch_batched_f64(P, cfg, bp, s, ctas);
        prof_end(h, s);
    }
    if (e != cudaSuccess) {
        set_error_message(std::string("batched kernel: ") + cudaGetErrorString(e));
        return COMET_ERR_CUDA;
    }
    return COMET_OK;
}

}  // namespace comet

using namespace comet;

extern "C" {

comet_status_t comet_plan_batched(const char *expr, int n_blocks, const char *const *label_names, int n_labels,
                                  const int64_t *extents, const comet_dtype_t *dtypes, int n_dtypes,
                                  const comet_plan_opts_t *opts, int tile_hint, comet_plan_t *out_plan) {
    if (!out_plan) return COMET_ERR_NULL;
    *out_plan = nullptr;
    comet_plan_s *h = new (std::nothrow) comet_plan_s;
    if (!h) return COMET_ERR_INTERNAL;
    std::string err;
    comet_status_t st;
    try {
        st = build_batched_plan(expr, n_blocks, label_names, n_labels, extents, dtypes, n_dtypes, opts, tile_hint,
                                &h->p, &err);
    } catch (...) {
        st = COMET_ERR_INTERNAL;
    }
    if (st != COMET_OK) {
        set_error_message(err);
        delete h;
        return st;
    }
    *out_plan = h;
    return COMET_OK;
}

int comet_batched_num_tiles(comet_plan_t plan) {
    if (plan && plan->p.opts.precision == COMET_PREC_SPLIT_BF16) return kBatchedCfgSplit;
    return kBatchedCfgF64;
}

comet_status_t comet_batched_set_tile(comet_plan_t plan, int cfg) {
    if (!plan) return COMET_ERR_NULL;
    if (!plan->p.batched || cfg < 0 || cfg >= n_cfg(plan->p)) return COMET_ERR_ARG;
    plan->p.tile_cfg = cfg;
    return COMET_OK;
}

comet_status_t comet_batched_prepare(comet_plan_t plan, void *workspace, void *stream) {
    if (!plan || !workspace) return COMET_ERR_NULL;
    const Plan &P = plan->p;
    if (!P.batched) return COMET_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) & 15u) != 0) return COMET_ERR_ALIGN;
    const BLayout L = layout_of(P.n_blocks, n_cfg(P), P.batched_item_bytes, P.batched_parts);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(static_cast<char *>(workspace) + L.prefix, P.batched_table.data(),
                                    P.batched_table.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error_message(std::string("batched prepare: ") + cudaGetErrorString(e));
        return COMET_ERR_CUDA;
    }
    return COMET_OK;
}

comet_status_t comet_contract_batched(comet_plan_t plan, const void *const *block_inputs, int mode, void *result,
                                      uint32_t weight_key, void *workspace, void *stream) {
    if (!plan || !block_inputs || !result || !workspace) return COMET_ERR_NULL;
    const Plan &P = plan->p;
    if (!P.batched) return COMET_ERR_ARG;
    if (mode != 0 && mode != 1) return COMET_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) & 15u) != 0) return COMET_ERR_ALIGN;
    return run_batched(P, block_inputs, mode, result, weight_key, workspace, static_cast<cudaStream_t>(stream),
                       P.tile_cfg, 0);
}

comet_status_t comet_batched_autotune(comet_plan_t plan, const void *const *block_inputs, void *result,
                                      void *workspace, int sample_blocks, void *stream, double *ms_per_cfg,
                                      int n_cfg_out, int *best) {
    if (!plan || !block_inputs || !result || !workspace) return COMET_ERR_NULL;
    Plan &P = plan->p;
    if (!P.batched) return COMET_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ncfg = n_cfg(P);
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return COMET_ERR_CUDA;
    int win = 0;
    double best_ms = 1e300;
    comet_status_t st = COMET_OK;
    for (int c = 0; c < ncfg && st == COMET_OK; ++c) {
        st = run_batched(P, block_inputs, 0, result, 1u, workspace, s, c, sample_blocks);   // warm-up
        if (st != COMET_OK) break;
        cudaEventRecord(a, s);
        st = run_batched(P, block_inputs, 0, result, 1u, workspace, s, c, sample_blocks);
        cudaEventRecord(b, s);
        if (st != COMET_OK || cudaEventSynchronize(b) != cudaSuccess) { st = COMET_ERR_CUDA; break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (ms_per_cfg && c < n_cfg_out) ms_per_cfg[c] = ms;
        if (ms < best_ms) { best_ms = ms; win = c; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != COMET_OK) return st;
    P.tile_cfg = win;
    if (best) *best = win;
    tune_cache_record(batched_signature(P), win);
    return COMET_OK;
}

}  // extern "C"
