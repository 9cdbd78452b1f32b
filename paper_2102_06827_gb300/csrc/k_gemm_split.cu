// Split-BF16 contraction kernel on the tcgen05 tensor cores.
//
// The GEMM of the TTGT reformulation (Section 2, C_p[i,k] = A_p[i,j] * B_p[j,k]; Section 6
// "GEMM optimizations" for the blocking of C into tiles and of K into panels) with FP32 (or
// FP64) operands carried as three bfloat16 fixed-point parts x * 2^-e = hi + mid + lo (written
// by the split pre-pass in [plane][row][K] order, K contiguous; see split3 in k_xpose.cu).
//
// Numerics.  The tensor core's FP32 accumulation truncates, so a long K would pile up a
// one-sided error.  The fixed-point split makes every hh product an integer multiple of 2^-12
// no larger than 2^2 in magnitude, so a chunk of up to 1024 K values of hh sums EXACTLY in
// the FP32 accumulator P0.  The five correction products (hm, mh, hl, lh, mm; 2^-7 and below
// of the result) go to a second accumulator P1, whose rounding is 2^-7 smaller.  After every
// chunk the epilogue warps add P0 and P1 into FP32 register sums (round to nearest); the
// products ml, lm, ll (2^-22 and below) are dropped.  At the end of a tile the sum is scaled
// by alpha * 2^(eA + eB) and stored.
//
// GB300 form (one persistent CTA per SM, 320 threads):
//   warp 0      TMA producer: one 3-D tensor load per operand and stage brings all three
//               planes of a 128 x 32 (A) and 256 x 32 (B) K-panel, 64-byte swizzled
//   warp 1      allocates 512 tensor-memory columns (P0 = columns 0..255, P1 = 256..511);
//               lane 0 issues tcgen05.mma (M=128, N=256, K=16) and tcgen05.commit
//   warps 2..9  epilogue: each owns one tensor-memory lane quadrant and one half of the
//               columns; drains P0/P1 after every chunk into 128 register sums per thread,
//               and at the end of the tile stores through the output's strides (the output
//               permutation of TTGT folded into the store addresses)
//   3-stage shared-memory ring (72 KB per stage).
// Every wait is bounded (%globaltimer); on expiry the CTA records COMET_ERR_TIMEOUT in the
// status word, drains its own copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>

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
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;             // P0 (256 columns) and P1 (256 columns)
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + BN * 8 /*c_col*/ + 256;
constexpr uint32_t SW64 = 4;                    // descriptor swizzle code: 64-byte swizzle
constexpr uint32_t SBO = 8 * BK * 2;            // 8 rows of 64 bytes
constexpr int MAX_KC = 1024;                    // exactness limit of the hh chunk
}  // namespace split

struct SplitArgs {
    uint32_t m_tiles, n_tiles, nkb;
    uint32_t tile0, ntiles;      // the launch's output tiles: tile0 .. tile0 + ntiles - 1
    uint32_t items;              // work items: ntiles x ksplit
    uint32_t kc_blocks;          // K blocks (of BK) per exact chunk
    uint32_t ksplit;             // K slices (1 = whole K per tile; > 1: FP32 partials to `partial`)
    uint32_t kslice_blocks;      // K blocks per slice
    float *partial;              // ksplit x ntiles tiles of BM x BN partial sums (scaled by
                                 // 2^(eA+eB)), [slice][tile][column][row], row fastest
    DbgRange dbg_p;              // debug builds: the partial sums' buffer
    int debug_flags;
    const void *scale_a;         // bits of max |A|, max |B| (input precision)
    const void *scale_b;
};

template <typename T>
__device__ __forceinline__ int exp_of_max(const void *bits) {
    if constexpr (sizeof(T) == 4) {
        const float m = __uint_as_float(*reinterpret_cast<const unsigned int *>(bits));
        if (!(m > 0.0f) || isinf(m)) return 0;
        int e;
        frexpf(m, &e);
        return e - 1;
    } else {
        const double m = __longlong_as_double(*reinterpret_cast<const long long *>(bits));
        if (!(m > 0.0) || isinf(m)) return 0;
        int e;
        frexp(m, &e);
        return e - 1;
    }
}

// output tile -> (m tile, n tile): bands of 16 m-tiles, n-major inside a band, for L2 reuse
__device__ __forceinline__ void split_tile_coords(uint32_t tile, uint32_t m_tiles, uint32_t n_tiles, uint32_t &mt,
                                                  uint32_t &nt) {
    const uint32_t G = 16;
    const uint32_t band = tile / (G * n_tiles);
    const uint32_t base = band * G;
    const uint32_t g = min(G, m_tiles - base);
    const uint32_t r = tile - band * G * n_tiles;
    mt = base + r % g;
    nt = r / g;
}

template <typename TOut, bool KSPLIT>
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
             *tempty = bars + 2 * STAGES + 1, *mma_done = bars + 2 * STAGES + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t tmo = (uint64_t)p.timeout_ns;
    const uint32_t n_tiles_total = x.items;
    // work item t: K slice t / ntiles of output tile tile0 + t % ntiles
    auto kslice = [&](uint32_t t, uint32_t &kb0, uint32_t &kb1) -> uint32_t {
        if constexpr (!KSPLIT) {
            kb0 = 0;
            kb1 = x.nkb;
            return 0;
        } else {
            const uint32_t ks = t / x.ntiles;
            kb0 = ks * x.kslice_blocks;
            kb1 = min(x.nkb, kb0 + x.kslice_blocks);
            return ks;
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(tfull, 1);
        mbar_init(tempty, EPI_WARPS);
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
    // work item t -> (m tile, n tile) of its output tile
    auto tile_coords = [&](uint32_t t, uint32_t &mt, uint32_t &nt) {
        if constexpr (KSPLIT) t %= x.ntiles;
        split_tile_coords(x.tile0 + t, x.m_tiles, x.n_tiles, mt, nt);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            uint32_t it = 0;
            bool ok = true;
            bool injected = false;
            for (uint32_t t = blockIdx.x; t < n_tiles_total && ok; t += gridDim.x) {
                uint32_t mt, nt, kb0, kb1;
                tile_coords(t, mt, nt);
                kslice(t, kb0, kb1);
                for (uint32_t kb = kb0; kb < kb1; ++kb, ++it) {
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
            const uint32_t p0 = tmem_base, p1 = tmem_base + BN;
            uint32_t it = 0, chunk = 0;
            bool ok = true;
            for (uint32_t t = blockIdx.x; t < n_tiles_total && ok; t += gridDim.x) {
                uint32_t kb0, kb1;
                kslice(t, kb0, kb1);
                for (uint32_t kb = kb0; kb < kb1; ++kb, ++it) {
                    const uint32_t kin = (KSPLIT ? kb - kb0 : kb) % x.kc_blocks;
                    if (kin == 0) {
                        // the epilogue must have drained the previous chunk
                        if (chunk > 0 && !mbar_wait(tempty, (chunk - 1) & 1, tmo, abort_flag)) {
                            fail(); ok = false; break;
                        }
                        tc_fence_after();
                    }
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
                        const uint32_t acc = (kin == 0 && ks == 0) ? 0u : 1u;
                        mma_bf16(p1, am, bm, idesc, acc);    // corrections, smallest first
                        mma_bf16(p1, al, bh, idesc, 1);
                        mma_bf16(p1, ah, bl, idesc, 1);
                        mma_bf16(p1, am, bh, idesc, 1);
                        mma_bf16(p1, ah, bm, idesc, 1);
                        mma_bf16(p0, ah, bh, idesc, acc);    // the exact leading product
                    }
                    mma_commit(&empty[s]);   // frees the stage once these MMAs have read it
                    if (kin == x.kc_blocks - 1 || kb == kb1 - 1) {
                        mma_commit(tfull);   // chunk complete: P0 and P1 ready to drain
                        ++chunk;
                    }
                }
            }
            // make sure no MMA is still writing tensor memory before it is freed
            mma_commit(mma_done);
            mbar_wait(mma_done, 0, tmo, nullptr);
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        const int quad = warp & 3;                  // tensor-memory lanes 32*quad .. 32*quad+31
        const int half = (warp - 2) >> 2;           // columns 128*half .. 128*half+127
        const int et = threadIdx.x - 64;            // 0..255
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        const int e_sum = exp_of_max<TOut>(x.scale_a) + exp_of_max<TOut>(x.scale_b);
        const double scale = ldexp(p.alpha, e_sum);
        uint32_t chunk = 0;
        bool dead = false;   // once set, the warp keeps pace with the barriers but does no work
        TOut *C = reinterpret_cast<TOut *>(p.C);
        for (uint32_t t = blockIdx.x; t < n_tiles_total; t += gridDim.x) {
            uint32_t mt, nt, kb0, kb1;
            tile_coords(t, mt, nt);
            const uint32_t ks = kslice(t, kb0, kb1);
            const uint32_t nchunks = (kb1 - kb0 + x.kc_blocks - 1) / x.kc_blocks;
            // column offsets of this tile in C (all eight epilogue warps always meet here)
            named_bar_sync(1, 32 * EPI_WARPS);
            {
                int64_t o0 = 0, o1 = 0;
                if (nt * BN + et < p.N) radix_offsets(p.nb, nt * BN + et, o0, o1);
                c_col[et] = o1;
            }
            named_bar_sync(1, 32 * EPI_WARPS);
            float S[128];
#pragma unroll
            for (int j = 0; j < 128; ++j) S[j] = 0.0f;
            for (uint32_t ch = 0; ch < nchunks; ++ch, ++chunk) {
                if (dead) continue;
                bool ok = mbar_wait(tfull, chunk & 1, tmo, abort_flag);
                ok = __all_sync(0xffffffffu, ok);   // warp-uniform before the .sync.aligned loads
                if (!ok) { if (lane == 0) fail(); dead = true; continue; }
                tc_fence_after();
                // 16 columns at a time keeps the 128 sums plus the loaded values within the
                // 168 registers a thread has when three warps share a sub-partition
#pragma unroll
                for (int c8 = 0; c8 < 8; ++c8) {
                    uint32_t r[16];
                    tmem_ld16(tmem_base + lane_base + half * 128 + c8 * 16, r);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) S[c8 * 16 + j] += __uint_as_float(r[j]);
                    tmem_ld16(tmem_base + BN + lane_base + half * 128 + c8 * 16, r);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) S[c8 * 16 + j] += __uint_as_float(r[j]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty);
            }
            if (dead) continue;
            const uint32_t m = mt * BM + quad * 32 + lane;
            if constexpr (KSPLIT) {   // K slice partial: scaled sums to the tile's slot, row fastest (coalesced)
                if (m < p.M) {
                    const uint32_t n_valid = min((uint32_t)BN, p.N - nt * BN);
                    const int n_here = (int)min(128u, n_valid > (uint32_t)(half * 128) ? n_valid - half * 128 : 0u);
                    const float sc = (float)ldexp(1.0, e_sum);
                    float *P = x.partial + ((size_t)(ks * x.ntiles + t % x.ntiles) * BN + half * 128) * BM +
                               (quad * 32 + lane);
#pragma unroll
                    for (int j = 0; j < 128; ++j)
                        if (j < n_here && dbg_ok(x.dbg_p, P + (size_t)j * BM, 4, p.status)) P[(size_t)j * BM] = sc * S[j];
                }
                continue;
            }
            if (m < p.M) {
                int64_t r0 = 0, c_row = 0;
                radix_offsets(p.ma, m, r0, c_row);
                const uint32_t n_valid = min((uint32_t)BN, p.N - nt * BN);
                TOut *row = C + c_row;
                const int64_t *cc = c_col + half * 128;
                const int n_here = (int)min(128u, n_valid > (uint32_t)(half * 128) ? n_valid - half * 128 : 0u);
                if (p.beta == 0.0) {
                    const TOut sc = (TOut)scale;
#pragma unroll
                    for (int j = 0; j < 128; ++j)
                        if (j < n_here && dbg_ok(p.dbg_c, row + cc[j], (int)sizeof(TOut), p.status))
                            row[cc[j]] = sc * (TOut)S[j];
                } else {
#pragma unroll
                    for (int j = 0; j < 128; ++j)
                        if (j < n_here && dbg_ok(p.dbg_c, row + cc[j], (int)sizeof(TOut), p.status)) {
                            TOut *dst = row + cc[j];
                            *dst = (TOut)(scale * (double)S[j] + p.beta * (double)*dst);
                        }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}

// K-slice partials -> C for the launch's tiles: C[m, n] = alpha * sum_ks P[ks][tile][n][m]
// (+ beta C), through C's strides; one thread per element of a tile
template <typename TOut>
__global__ void __launch_bounds__(256) split_reduce_kernel(const GemmParams p, const SplitArgs x) {
    using namespace split;
    const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= (uint64_t)x.ntiles * BM * BN) return;
    const uint32_t jt = (uint32_t)(i / (BM * BN)), e = (uint32_t)(i - (uint64_t)jt * (BM * BN));
    const uint32_t nl = e / BM, ml = e - nl * BM;
    uint32_t mt, nt;
    split_tile_coords(x.tile0 + jt, x.m_tiles, x.n_tiles, mt, nt);
    const uint32_t m = mt * BM + ml, n = nt * BN + nl;
    if (m >= p.M || n >= p.N) return;
    double s = 0.0;
    for (uint32_t k = 0; k < x.ksplit; ++k) {
        const float *q = x.partial + ((size_t)(k * x.ntiles + jt) * BN + nl) * BM + ml;
        if (dbg_ok(x.dbg_p, q, 4, p.status)) s += (double)*q;
    }
    int64_t a, cm, b, cn;
    radix_offsets(p.ma, m, a, cm);
    radix_offsets(p.nb, n, b, cn);
    TOut *c = reinterpret_cast<TOut *>(p.C) + cm + cn;
    if (!dbg_ok(p.dbg_c, c, (int)sizeof(TOut), p.status)) return;
    const double r = p.alpha * s;
    *c = (TOut)(p.beta != 0.0 ? r + p.beta * (double)*c : r);
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

// the shared-memory attribute is set once per kernel instantiation
template <typename TOut, bool KSPLIT>
static void launch_split_kernel(const CUtensorMap &ta, const CUtensorMap &tb, const GemmParams &p,
                                const SplitArgs &x, int ctas, cudaStream_t s) {
    static const bool attr = [] {
        cudaFuncSetAttribute(gemm_split_kernel<TOut, KSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             split::SMEM_BYTES);
        return true;
    }();
    (void)attr;
    gemm_split_kernel<TOut, KSPLIT><<<ctas, split::THREADS, split::SMEM_BYTES, s>>>(ta, tb, p, x);
}

// one launch over output tiles tile0 .. tile0 + ntiles - 1 in k K slices (k > 1: FP32 partials
// of every slice, then the reduce kernel)
static cudaError_t launch_range(const CUtensorMap &ta, const CUtensorMap &tb, const GemmParams &p, SplitArgs x,
                                uint32_t tile0, uint32_t ntiles, uint32_t k, int out_bytes, int max_ctas,
                                cudaStream_t s) {
    using namespace split;
    x.tile0 = tile0;
    x.ntiles = ntiles;
    x.kslice_blocks = (x.nkb + k - 1) / k;    // at least one K block per slice
    x.ksplit = (x.nkb + x.kslice_blocks - 1) / x.kslice_blocks;
    x.items = ntiles * x.ksplit;
    x.dbg_p = dbg_range(x.partial, x.ksplit > 1 ? (int64_t)x.ksplit * ntiles * BM * BN * 4 : 0);
    int ctas = sm_count();
    if (max_ctas > 0 && max_ctas < ctas) ctas = max_ctas;
    if ((uint32_t)ctas > x.items) ctas = (int)x.items;
    if (out_bytes == 8) {
        if (x.ksplit > 1) launch_split_kernel<double, true>(ta, tb, p, x, ctas, s);
        else launch_split_kernel<double, false>(ta, tb, p, x, ctas, s);
    } else {
        if (x.ksplit > 1) launch_split_kernel<float, true>(ta, tb, p, x, ctas, s);
        else launch_split_kernel<float, false>(ta, tb, p, x, ctas, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || x.ksplit == 1) return e;
    const uint64_t n = (uint64_t)ntiles * BM * BN;
    const uint32_t blocks = (uint32_t)((n + 255) / 256);
    if (out_bytes == 8) split_reduce_kernel<double><<<blocks, 256, 0, s>>>(p, x);
    else split_reduce_kernel<float><<<blocks, 256, 0, s>>>(p, x);
    return cudaGetLastError();
}

cudaError_t launch_gemm_split(const GemmParams &p, const void *parts_a, const void *parts_b,
                              int64_t kpad, const void *scale_a, const void *scale_b, int64_t kc,
                              int out_bytes, int debug_flags, cudaStream_t s, int max_ctas,
                              uint32_t ksplit, float *partial, int64_t partial_bytes) {
    using namespace split;
    if (p.M == 0 || p.N == 0) return cudaSuccess;
    CUtensorMap ta, tb;
    if (!make_map(&ta, parts_a, p.M, p.K, (uint64_t)kpad, BM)) return cudaErrorInvalidValue;
    if (!make_map(&tb, parts_b, p.N, p.K, (uint64_t)kpad, BN)) return cudaErrorInvalidValue;
    SplitArgs x;
    x.m_tiles = (p.M + BM - 1) / BM;
    x.n_tiles = (p.N + BN - 1) / BN;
    x.nkb = (p.K + BK - 1) / BK;
    if (kc <= 0 || kc > MAX_KC) kc = MAX_KC;
    x.kc_blocks = (uint32_t)((kc + BK - 1) / BK);
    if (x.kc_blocks * BK > (uint32_t)MAX_KC) x.kc_blocks = MAX_KC / BK;
    x.debug_flags = debug_flags;
    x.scale_a = scale_a;
    x.scale_b = scale_b;
    x.partial = partial;
    const uint32_t tiles = x.m_tiles * x.n_tiles;
    const int64_t tile_bytes = (int64_t)BM * BN * 4;
    if (ksplit > 1 && partial && (int64_t)ksplit * tiles * tile_bytes <= partial_bytes)   // every tile in K slices
        return launch_range(ta, tb, p, x, 0, tiles, ksplit, out_bytes, max_ctas, s);
    // whole-K tiles in full waves over the SMs, then a partial last wave in K slices (a
    // stream-K tail): its tiles' slices fill the SMs the wave would leave idle
    const uint32_t sms = (uint32_t)(max_ctas > 0 ? std::min(max_ctas, sm_count()) : sm_count());
    const uint32_t tail = tiles % sms;
    uint32_t tsplit = 1;
    if (tiles > sms && tail > 0 && 2 * tail <= sms) tsplit = std::min({4u, sms / tail, x.nkb});
    if (tsplit > 1 && partial && (int64_t)tsplit * tail * tile_bytes <= partial_bytes) {
        cudaError_t e = launch_range(ta, tb, p, x, 0, tiles - tail, 1, out_bytes, max_ctas, s);
        if (e != cudaSuccess) return e;
        return launch_range(ta, tb, p, x, tiles - tail, tail, tsplit, out_bytes, max_ctas, s);
    }
    return launch_range(ta, tb, p, x, 0, tiles, 1, out_bytes, max_ctas, s);
}

}  // namespace comet
