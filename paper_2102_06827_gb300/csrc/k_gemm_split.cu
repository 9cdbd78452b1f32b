// Split-BF16 contraction kernel on the tcgen05 tensor cores.
//
// The GEMM of the TTGT reformulation (Section 2, C_p[i,k] = A_p[i,j] * B_p[j,k]; Section 6
// "GEMM optimizations" for the blocking of C into tiles and of K into panels) with FP32
// operands carried as three bfloat16 parts x = hi + mid + lo (written by the split pre-pass in
// [plane][row][K] order, K contiguous).  Per K step the six products hh, hm, mh, hl, lh, mm
// are accumulated in FP32 in tensor memory; the three smallest (ml, lm, ll, below 2^-24 of
// the leading term) are dropped.
//
// GB300 form (one persistent CTA per SM, 192 threads):
//   warp 0      TMA producer: one 3-D tensor load per operand and stage brings all three
//               planes of a 128 x 32 (A) and 256 x 32 (B) K-panel, 64-byte swizzled
//   warp 1      allocates 512 tensor-memory columns; lane 0 issues tcgen05.mma
//               (M=128, N=256, K=16) and tcgen05.commit
//   warps 2..5  epilogue: tcgen05.ld of the 128 x 256 FP32 accumulator, alpha/beta, store
//               through the output's strides (the output permutation of TTGT folded into
//               the store addresses)
//   3-stage shared-memory ring (72 KB per stage); two accumulator buffers in tensor memory
//   so the epilogue of one tile overlaps the main loop of the next.
// Every wait is bounded (deadline on %globaltimer); on expiry the CTA records
// COMET_ERR_TIMEOUT in the status word, drains its own copies in flight, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "launch.h"
#include "params.h"
#include "sm100.cuh"

namespace comet {

namespace split {
constexpr int BM = 128, BN = 256, BK = 32, STAGES = 3;
constexpr int A_PLANE = BM * BK * 2;            // 8 KB
constexpr int B_PLANE = BN * BK * 2;            // 16 KB
constexpr int A_STAGE = 3 * A_PLANE;            // 24 KB
constexpr int B_STAGE = 3 * B_PLANE;            // 48 KB
constexpr int STAGE_BYTES = A_STAGE + B_STAGE;  // 72 KB
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 512;             // two 256-column accumulators
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + BN * 8 /*c_col*/ + 256;
constexpr uint32_t SW64 = 4;                    // descriptor swizzle code: 64-byte swizzle
constexpr uint32_t SBO = 8 * BK * 2;            // 8 rows of 64 bytes
}  // namespace split

struct SplitArgs {
    uint32_t m_tiles, n_tiles, nkb;
    int debug_flags;
    int out_f64;
};

template <typename TOut>
__global__ void __launch_bounds__(split::THREADS, 1)
    gemm_split_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const GemmParams p, const SplitArgs x) {
    using namespace split;
    using namespace sm100;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + (((raw + 1023) & ~1023u) - raw);
    uint8_t *stage_base = smem;
    int64_t *c_col = reinterpret_cast<int64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES + BN * 8);
    uint64_t *full = bars, *empty = bars + STAGES, *tfull = bars + 2 * STAGES,
             *tempty = bars + 2 * STAGES + 2, *mma_done = bars + 2 * STAGES + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t tmo = (uint64_t)p.timeout_ns;
    const uint32_t n_tiles_total = x.m_tiles * x.n_tiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 4); }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        fence_barrier_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(p.status, (int)COMET_ERR_TIMEOUT);
    };
    // tile t -> (m tile, n tile): bands of 16 m-tiles, n-major inside a band, for L2 reuse
    auto tile_coords = [&](uint32_t t, uint32_t &mt, uint32_t &nt) {
        const uint32_t G = 16;
        uint32_t band = t / (G * x.n_tiles);
        uint32_t base = band * G;
        uint32_t g = min(G, x.m_tiles - base);
        uint32_t r = t - band * G * x.n_tiles;
        mt = base + r % g;
        nt = r / g;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            uint32_t it = 0;
            bool ok = true;
            bool injected = false;
            for (uint32_t t = blockIdx.x; t < n_tiles_total && ok; t += gridDim.x) {
                uint32_t mt, nt;
                tile_coords(t, mt, nt);
                for (uint32_t kb = 0; kb < x.nkb; ++kb, ++it) {
                    const uint32_t s = it % STAGES, round = it / STAGES;
                    if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1, tmo, abort_flag)) {
                        fail(); ok = false; break;
                    }
                    mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                    if ((x.debug_flags & 1) && !injected && blockIdx.x == 0) {
                        injected = true;   // fault injection: this stage's loads are withheld
                        continue;
                    }
                    uint8_t *sa = stage_base + s * STAGE_BYTES;
                    tma_load_3d(&tmA, &full[s], sa, kb * BK, mt * BM, 0);
                    tma_load_3d(&tmB, &full[s], sa + A_STAGE, kb * BK, nt * BN, 0);
                }
            }
            // drain: wait for every load still in flight (at most one per stage)
            uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0;
            for (uint32_t j = first; j < it; ++j) {
                const uint32_t s = j % STAGES, round = j / STAGES;
                mbar_wait(&full[s], round & 1, tmo, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
            uint32_t it = 0, lt = 0;
            bool ok = true;
            for (uint32_t t = blockIdx.x; t < n_tiles_total && ok; t += gridDim.x, ++lt) {
                const uint32_t buf = lt & 1, use = lt >> 1;
                if (use > 0 && !mbar_wait(&tempty[buf], (use - 1) & 1, tmo, abort_flag)) {
                    fail(); ok = false; break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + buf * BN;
                for (uint32_t kb = 0; kb < x.nkb; ++kb, ++it) {
                    const uint32_t s = it % STAGES, round = it / STAGES;
                    if (!mbar_wait(&full[s], round & 1, tmo, abort_flag)) { fail(); ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(stage_base + s * STAGE_BYTES);
                    const uint32_t sb = sa + A_STAGE;
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
                        uint64_t ah = smem_desc(sa + 0 * A_PLANE + ks * 32, 16, SBO, SW64);
                        uint64_t am = smem_desc(sa + 1 * A_PLANE + ks * 32, 16, SBO, SW64);
                        uint64_t al = smem_desc(sa + 2 * A_PLANE + ks * 32, 16, SBO, SW64);
                        uint64_t bh = smem_desc(sb + 0 * B_PLANE + ks * 32, 16, SBO, SW64);
                        uint64_t bm = smem_desc(sb + 1 * B_PLANE + ks * 32, 16, SBO, SW64);
                        uint64_t bl = smem_desc(sb + 2 * B_PLANE + ks * 32, 16, SBO, SW64);
                        const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;
                        // small products first, the leading hh term last
                        mma_bf16(d_tmem, am, bm, idesc, first);
                        mma_bf16(d_tmem, al, bh, idesc, 1);
                        mma_bf16(d_tmem, ah, bl, idesc, 1);
                        mma_bf16(d_tmem, am, bh, idesc, 1);
                        mma_bf16(d_tmem, ah, bm, idesc, 1);
                        mma_bf16(d_tmem, ah, bh, idesc, 1);
                    }
                    mma_commit(&empty[s]);   // frees the stage once these MMAs have read it
                }
                if (!ok) break;
                mma_commit(&tfull[buf]);
            }
            // make sure no MMA is still writing tensor memory before it is freed
            mma_commit(mma_done);
            mbar_wait(mma_done, 0, tmo, nullptr);
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int quad = warp & 3;                 // tensor-memory lanes 32*quad .. 32*quad+31
        const int et = threadIdx.x - 64;           // 0..127
        uint32_t lt = 0;
        bool dead = false;   // once set, the warp keeps pace with the barriers but does no work
        TOut *C = reinterpret_cast<TOut *>(p.C);
        for (uint32_t t = blockIdx.x; t < n_tiles_total; t += gridDim.x, ++lt) {
            uint32_t mt, nt;
            tile_coords(t, mt, nt);
            const uint32_t buf = lt & 1, use = lt >> 1;
            // column offsets of this tile in C (all four epilogue warps always meet here)
            named_bar_sync(1, 128);
            for (int j = et; j < BN; j += 128) {
                int64_t o0 = 0, o1 = 0;
                if (nt * BN + j < p.N) radix_offsets(p.nb, nt * BN + j, o0, o1);
                c_col[j] = o1;
            }
            named_bar_sync(1, 128);
            if (dead) continue;
            const uint32_t m = mt * BM + quad * 32 + lane;
            int64_t r0 = 0, c_row = 0;
            if (m < p.M) radix_offsets(p.ma, m, r0, c_row);
            bool ok = mbar_wait(&tfull[buf], use & 1, tmo, abort_flag);
            ok = __all_sync(0xffffffffu, ok);   // warp-uniform before the .sync.aligned loads
            if (!ok) { if (lane == 0) fail(); dead = true; continue; }
            tc_fence_after();
            const uint32_t taddr = tmem_base + buf * BN + ((uint32_t)(quad * 32) << 16);
            const uint32_t n_valid = min((uint32_t)BN, p.N - nt * BN);
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t r[32];
                tmem_ld32(taddr + c * 32, r);
                tmem_ld_wait();
                if (m < p.M) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const uint32_t n = c * 32 + j;
                        if (n < n_valid) {
                            TOut *dst = C + c_row + c_col[n];
                            double v = p.alpha * (double)__uint_as_float(r[j]);
                            if (p.beta != 0.0) v += p.beta * (double)*dst;
                            *dst = (TOut)v;
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}

// ---- host side --------------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

// 3-D map over [3 planes][rows][K] bf16 with rows of kpad elements; box = K 32 x rows box_rows x 3
static bool make_map(CUtensorMap *m, const void *base, uint64_t rows, uint64_t K, uint64_t kpad,
                     uint32_t box_rows) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[3] = {K, rows, 3};
    cuuint64_t strides[2] = {kpad * 2, rows * kpad * 2};
    cuuint32_t box[3] = {(cuuint32_t)split::BK, box_rows, 3};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

cudaError_t launch_gemm_split(const GemmParams &p, const void *parts_a, const void *parts_b,
                              int64_t kpad, int out_bytes, int debug_flags, cudaStream_t s,
                              int max_ctas) {
    using namespace split;
    if (p.M == 0 || p.N == 0) return cudaSuccess;
    CUtensorMap ta, tb;
    if (!make_map(&ta, parts_a, p.M, p.K, (uint64_t)kpad, BM)) return cudaErrorInvalidValue;
    if (!make_map(&tb, parts_b, p.N, p.K, (uint64_t)kpad, BN)) return cudaErrorInvalidValue;
    SplitArgs x;
    x.m_tiles = (p.M + BM - 1) / BM;
    x.n_tiles = (p.N + BN - 1) / BN;
    x.nkb = (p.K + BK - 1) / BK;
    x.debug_flags = debug_flags;
    x.out_f64 = out_bytes == 8;
    uint32_t tiles = x.m_tiles * x.n_tiles;
    int ctas = sm_count();
    if (max_ctas > 0 && max_ctas < ctas) ctas = max_ctas;
    if ((uint32_t)ctas > tiles) ctas = (int)tiles;
    static bool attr_set[2] = {false, false};
    if (out_bytes == 8) {
        if (!attr_set[1]) {
            cudaFuncSetAttribute(gemm_split_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
            attr_set[1] = true;
        }
        gemm_split_kernel<double><<<ctas, THREADS, SMEM_BYTES, s>>>(ta, tb, p, x);
    } else {
        if (!attr_set[0]) {
            cudaFuncSetAttribute(gemm_split_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
            attr_set[0] = true;
        }
        gemm_split_kernel<float><<<ctas, THREADS, SMEM_BYTES, s>>>(ta, tb, p, x);
    }
    return cudaGetLastError();
}

}  // namespace comet
