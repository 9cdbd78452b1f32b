// FP64-accurate contraction emulated on the BF16 tensor cores (tcgen05).
//
// The GEMM of the TTGT reformulation (Section 2) for FP64 operands, computed from six
// fixed-point bfloat16 slices per operand (an extension of the split form to FP64 accuracy;
// the paper itself has no reduced-precision arithmetic).  Each operand is scaled by 2^-e
// (e = exponent of its largest magnitude, so |x'| < 2) and written by the pre-pass as six
// integer-valued planes s_0..s_5 with x' = sum_k s_k 2^-(6+8k), |s_k| <= 128 (exact in bf16);
// what remains is below 2^-47.  A product of slices i and j is an integer of magnitude <= 2^14
// in units of 2^-(12+8w), w = i+j.
//
// The 21 slice products with w <= 5 run as ten tcgen05.mma per K step: for slice i of A, the B
// slices j = 0..5-i sit in consecutive 80-row planes of one shared-memory tile, so one MMA with
// N = 80 x (number of slices) lands A_i B_j in tensor-memory columns 80(i+j).. -- the
// accumulator of weight group w = i+j.  Groups 0..4 sum at most 5 products of <= 2^14 per K, so
// a chunk of 192 K values stays below 2^24 and is exact in the FP32 accumulator whatever its
// rounding; group 5 (2^-40 of the result) is inexact and rounded.  After every chunk the
// epilogue converts the groups to integers and folds them into one int64 per output element in
// units of 2^-44:  I += G0 2^32 + G1 2^24 + G2 2^16 + G3 2^8 + G4 + rint(G5 2^-8)  -- exact except
// the last term (G4 + rn(G5 2^-8) is formed exactly in FP32 first).  The result is
// alpha 2^(eA+eB-44) I, rounded once to FP64.
//
// GB300 form (one persistent CTA per SM, 320 threads), as the split kernel:
//   warp 0      TMA producer: one 3-D load per operand and stage brings all six planes of a
//               128 x 32 (A) and 80 x 32 (B) K-panel, 64-byte swizzled
//   warp 1      allocates 512 tensor-memory columns (six groups of 80); lane 0 issues the MMAs
//   warps 2..9  epilogue: lane quadrant x half of the 80 columns; int64 sums in registers
//   2-stage shared-memory ring (78 KB per stage).
// Every wait is bounded (%globaltimer); on expiry the CTA records COMET_ERR_TIMEOUT in the
// status word, drains its own copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "launch.h"
#include "params.h"
#include "sm100.cuh"

namespace comet {

namespace emu {
constexpr int S = 6;                            // slices per operand
constexpr int BM = 128, BG = 80, BK = 32, STAGES = 2;
constexpr int A_PLANE = BM * BK * 2;            // 8 KB
constexpr int B_PLANE = BG * BK * 2;            // 5 KB
constexpr int A_STAGE = S * A_PLANE;            // 48 KB
constexpr int B_STAGE = S * B_PLANE;            // 30 KB
constexpr int STAGE_BYTES = A_STAGE + B_STAGE;  // 78 KB
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int GROUPS = 6;                       // weight groups of the slice products
constexpr uint32_t TMEM_COLS = 512;             // groups at columns 80 w, w = 0..5
static_assert(GROUPS * BG <= (int)TMEM_COLS, "every weight group's accumulator in tensor memory");
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + BG * 8 /*c_col*/ + 256;
constexpr uint32_t SW64 = 4;
constexpr uint32_t SBO = 8 * BK * 2;
constexpr uint32_t KC_BLOCKS = 6;               // 192 K values per exact chunk
constexpr uint32_t MAX_K = 96 * 1024;           // keeps the int64 sums below 2^63
constexpr int HALF = BG / 2;                    // columns per epilogue thread
}  // namespace emu

struct EmuArgs {
    uint32_t m_tiles, n_tiles, nkb;
    int debug_flags;
    const void *scale_a;         // bits of max |A|, max |B| (FP64)
    const void *scale_b;
};

__device__ __forceinline__ int exp_of_max_f64(const void *bits) {
    const double m = __longlong_as_double(*reinterpret_cast<const long long *>(bits));
    if (!(m > 0.0) || isinf(m)) return 0;
    int e;
    frexp(m, &e);
    return e - 1;
}

__global__ void __launch_bounds__(emu::THREADS, 1)
    gemm_emu_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const GemmParams p, const EmuArgs x) {
    using namespace emu;
    using namespace sm100;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + (((raw + 1023) & ~1023u) - raw);
    uint8_t *stage_base = smem;
    int64_t *c_col = reinterpret_cast<int64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES + BG * 8);
    uint64_t *full = bars, *empty = bars + STAGES, *tfull = bars + 2 * STAGES,
             *tempty = bars + 2 * STAGES + 1, *mma_done = bars + 2 * STAGES + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t tmo = (uint64_t)p.timeout_ns;
    const uint32_t n_tiles_total = x.m_tiles * x.n_tiles;

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
                    tma_load_3d(&tmB, &full[s], sa + A_STAGE, kb * BK, nt * BG, 0);
                }
            }
            uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0;
            for (uint32_t j = first; j < it; ++j) {
                const uint32_t s = j % STAGES, round = j / STAGES;
                mbar_wait(&full[s], round & 1, tmo, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t id1 = idesc_bf16_f32(BM, BG), id2 = idesc_bf16_f32(BM, 2 * BG),
                               id3 = idesc_bf16_f32(BM, 3 * BG);
            auto G = [&](int w) { return tmem_base + (uint32_t)(w * BG); };
            uint32_t it = 0, chunk = 0;
            bool ok = true;
            for (uint32_t t = blockIdx.x; t < n_tiles_total && ok; t += gridDim.x) {
                for (uint32_t kb = 0; kb < x.nkb; ++kb, ++it) {
                    const uint32_t kin = kb % KC_BLOCKS;
                    if (kin == 0) {
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
                        auto a = [&](int i) { return smem_desc(sa + i * A_PLANE + ks * 32, 16, SBO, SW64); };
                        auto b = [&](int j) { return smem_desc(sb + j * B_PLANE + ks * 32, 16, SBO, SW64); };
                        const uint32_t acc = (kin == 0 && ks == 0) ? 0u : 1u;
                        // slice 0 of A against B slices 0..5 (groups 0..5): overwrites at a chunk start
                        mma_bf16(G(0), a(0), b(0), id3, acc);
                        mma_bf16(G(3), a(0), b(3), id3, acc);
                        mma_bf16(G(1), a(1), b(0), id3, 1);   // groups 1..3
                        mma_bf16(G(4), a(1), b(3), id2, 1);   // groups 4..5
                        mma_bf16(G(2), a(2), b(0), id3, 1);   // groups 2..4
                        mma_bf16(G(5), a(2), b(3), id1, 1);   // group 5
                        mma_bf16(G(3), a(3), b(0), id3, 1);   // groups 3..5
                        mma_bf16(G(4), a(4), b(0), id2, 1);   // groups 4..5
                        mma_bf16(G(5), a(5), b(0), id1, 1);   // group 5
                    }
                    mma_commit(&empty[s]);
                    if (kin == KC_BLOCKS - 1 || kb == x.nkb - 1) {
                        mma_commit(tfull);
                        ++chunk;
                    }
                }
            }
            mma_commit(mma_done);
            mbar_wait(mma_done, 0, tmo, nullptr);
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;           // columns HALF*half .. +HALF-1 of each group
        const int et = threadIdx.x - 64;            // 0..255
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        const int e_sum = exp_of_max_f64(x.scale_a) + exp_of_max_f64(x.scale_b);
        const double scale = ldexp(p.alpha, e_sum - 44);
        const uint32_t nchunks = (x.nkb + KC_BLOCKS - 1) / KC_BLOCKS;
        uint32_t chunk = 0;
        bool dead = false;
        double *C = reinterpret_cast<double *>(p.C);
        for (uint32_t t = blockIdx.x; t < n_tiles_total; t += gridDim.x) {
            uint32_t mt, nt;
            tile_coords(t, mt, nt);
            named_bar_sync(1, 32 * EPI_WARPS);
            if (et < BG) {
                int64_t o0 = 0, o1 = 0;
                if (nt * BG + et < p.N) radix_offsets(p.nb, nt * BG + et, o0, o1);
                c_col[et] = o1;
            }
            named_bar_sync(1, 32 * EPI_WARPS);
            long long I[HALF];
#pragma unroll
            for (int j = 0; j < HALF; ++j) I[j] = 0;
            for (uint32_t ch = 0; ch < nchunks; ++ch, ++chunk) {
                if (dead) continue;
                bool ok = mbar_wait(tfull, chunk & 1, tmo, abort_flag);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) { if (lane == 0) fail(); dead = true; continue; }
                tc_fence_after();
                // groups 0..3: exact integers, one conversion each, shifted into 2^-44 units
#pragma unroll 1
                for (int w = 0; w < 4; ++w) {
                    const int sh = 8 * (4 - w);
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        const int c0 = part == 0 ? 0 : 3, nc = part == 0 ? 3 : 2;
                        uint32_t r[24];
#pragma unroll
                        for (int c8 = 0; c8 < nc; ++c8)
                            tmem_ld8(tmem_base + lane_base + w * BG + half * HALF + (c0 + c8) * 8,
                                     *reinterpret_cast<uint32_t(*)[8]>(&r[c8 * 8]));
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < nc * 8; ++j)
                            I[c0 * 8 + j] += (long long)__float2int_rn(__uint_as_float(r[j])) * (1ll << sh);
                    }
                }
                // groups 4 and 5 merged exactly in FP32: G4 + rn(G5 2^-8) stays an integer below
                // 2^24 (rn by the 1.5 * 2^23 addition, valid below 2^22), then one conversion
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    const int c0 = part == 0 ? 0 : 3, nc = part == 0 ? 3 : 2;
                    uint32_t r4[24], r5[24];
#pragma unroll
                    for (int c8 = 0; c8 < nc; ++c8) {
                        tmem_ld8(tmem_base + lane_base + 4 * BG + half * HALF + (c0 + c8) * 8,
                                 *reinterpret_cast<uint32_t(*)[8]>(&r4[c8 * 8]));
                        tmem_ld8(tmem_base + lane_base + 5 * BG + half * HALF + (c0 + c8) * 8,
                                 *reinterpret_cast<uint32_t(*)[8]>(&r5[c8 * 8]));
                    }
                    tmem_ld_wait();
                    if (part == 1) {
                        // every group is in registers: the MMAs of the next chunk may start
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tempty);
                    }
                    const float magic = 12582912.0f;   // 1.5 * 2^23
#pragma unroll
                    for (int j = 0; j < nc * 8; ++j) {
                        const float g5 = __fsub_rn(__fadd_rn(__uint_as_float(r5[j]) * (1.0f / 256.0f), magic), magic);
                        I[c0 * 8 + j] += (long long)__float2int_rn(__fadd_rn(__uint_as_float(r4[j]), g5));
                    }
                }
            }
            if (dead) continue;
            const uint32_t m = mt * BM + quad * 32 + lane;
            if (m < p.M) {
                int64_t r0 = 0, c_row = 0;
                radix_offsets(p.ma, m, r0, c_row);
                const uint32_t n_valid = min((uint32_t)BG, p.N - nt * BG);
                double *row = C + c_row;
                const int64_t *cc = c_col + half * HALF;
                const int n_here = (int)min((uint32_t)HALF, n_valid > (uint32_t)(half * HALF) ? n_valid - half * HALF : 0u);
                if (p.beta == 0.0) {
#pragma unroll
                    for (int j = 0; j < HALF; ++j)
                        if (j < n_here && dbg_ok(p.dbg_c, row + cc[j], 8, p.status)) row[cc[j]] = scale * (double)I[j];
                } else {
#pragma unroll
                    for (int j = 0; j < HALF; ++j)
                        if (j < n_here && dbg_ok(p.dbg_c, row + cc[j], 8, p.status)) {
                            double *dst = row + cc[j];
                            *dst = scale * (double)I[j] + p.beta * *dst;
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

// ---- host side --------------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 get_encode_emu() {
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

// 3-D map over [6 planes][rows][K] bf16 with rows of kpad elements; box = K 32 x rows x 6
static bool make_map6(CUtensorMap *m, const void *base, uint64_t rows, uint64_t K, uint64_t kpad,
                      uint32_t box_rows) {
    auto enc = get_encode_emu();
    if (!enc) return false;
    cuuint64_t dims[3] = {K, rows, (cuuint64_t)emu::S};
    cuuint64_t strides[2] = {kpad * 2, rows * kpad * 2};
    cuuint32_t box[3] = {(cuuint32_t)emu::BK, box_rows, (cuuint32_t)emu::S};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static int sm_count_emu() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

cudaError_t launch_gemm_emu(const GemmParams &p, const void *parts_a, const void *parts_b, int64_t kpad,
                            const void *scale_a, const void *scale_b, int debug_flags, cudaStream_t s,
                            int max_ctas) {
    using namespace emu;
    if (p.M == 0 || p.N == 0) return cudaSuccess;
    if (p.K > MAX_K) return cudaErrorInvalidValue;
    CUtensorMap ta, tb;
    if (!make_map6(&ta, parts_a, p.M, p.K, (uint64_t)kpad, BM)) return cudaErrorInvalidValue;
    if (!make_map6(&tb, parts_b, p.N, p.K, (uint64_t)kpad, BG)) return cudaErrorInvalidValue;
    EmuArgs x;
    x.m_tiles = (p.M + BM - 1) / BM;
    x.n_tiles = (p.N + BG - 1) / BG;
    x.nkb = (p.K + BK - 1) / BK;
    x.debug_flags = debug_flags;
    x.scale_a = scale_a;
    x.scale_b = scale_b;
    const uint32_t tiles = x.m_tiles * x.n_tiles;
    int ctas = sm_count_emu();
    if (max_ctas > 0 && max_ctas < ctas) ctas = max_ctas;
    if ((uint32_t)ctas > tiles) ctas = (int)tiles;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(gemm_emu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        attr_set = true;
    }
    gemm_emu_kernel<<<ctas, THREADS, SMEM_BYTES, s>>>(ta, tb, p, x);
    return cudaGetLastError();
}

}  // namespace comet
