// Batched split-BF16 contractions on the tcgen05 tensor cores: one persistent launch over many
// small, uneven blocks of one two-operand expression (the 6-D triples outputs of the CCSD(T)
// remark in Section 2, T[a,b,c,i,j,k] = sum_d A[d,a,b,i] * B[c,d,j,k]; every block is the GEMM
// of its TTGT view with the permutations folded into the index arithmetic).
//
// Operands.  A pre-pass splits each block operand once into the fixed-point bfloat16 parts
// hi, mid, lo (split.cuh) and writes them in "plane rows" of 32 K values (64 bytes): operand X
// occupies ceil(K/32) chunks x 3 planes x rows_pad rows, [chunk][plane][row], zero beyond its
// rows and its K.  All blocks' planes form one array, so ONE two-dimensional tensor map serves
// every block: a 128-row box at row (block base + (chunk*3 + plane)*rows_pad + r0) is a 64-byte
// swizzled K-major operand tile of the MMA (two K steps of 16).  Zero padding rows make
// out-of-range outputs exactly zero, so the reduction needs no masks.
//
// Work items are (block, strip of BN output columns), blocks longest first, dealt to the
// persistent CTAs round robin.  A block with K <= 32 (one chunk) keeps its strip's B tile (all
// planes, BN rows) resident in shared memory while its M tiles stream through a ring; larger K
// streams the B chunks beside the A chunks.
//
// Roles (320 threads, one CTA per SM):
//   warp 0      TMA producer (one elected lane)
//   warp 1      tensor memory allocation; one lane issues tcgen05.mma (M=128, N=BN or 128,
//               K=16, bf16 in, FP32 accumulate) and tcgen05.commit
//   warps 2..9  epilogue: warp w owns tensor-memory lanes 32*(w%4).. (rows); the two warps of
//               a lane quadrant take alternate tiles (all columns), or split the columns when
//               there is one accumulator buffer; a tile drains while the MMA fills the next
//
// Numerics.  Six part products per K chunk (hh, hm, mh, hl, lh, mm; ml, lm, ll dropped, as
// in the large split GEMM).  Blocks of this plan with K <= 32 (at most two hh MMAs per tile)
// share one accumulator: the correction products are accumulated first and the hh products
// last, so the accumulator's truncating FP32 additions cost at most one unit in the last
// place of the running sum per hh MMA.  A plan with any K > 32 keeps the hh products in an
// accumulator of their own (P0, exact for K <= 1024) and the corrections in P1.
//
// Epilogue.  Reduce mode: per thread (one output row m) sum_n T[m,n] v[n] and sum_n T^2 with
// packed FP32x2 FMAs, v[n] the column factor of the weight (triples_weight.cuh) formed once per
// strip; the row factor u[m] multiplies the row's sum; per-tile sums are added with a
// compensated (two-sum) FP32 accumulation, per-item totals in FP64 with one atomic pair per
// warp.  Store mode: alpha 2^(eA+eB) T through the output's strides.
//
// Every wait is bounded (%globaltimer); on expiry the CTA records COMET_ERR_TIMEOUT in the
// status word, waits (bounded) for its own copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "../../include/comet.h"
#include "batched.h"
#include "params.h"
#include "sm100.cuh"
#include "split.cuh"
#include "triples_weight.cuh"

namespace comet {


namespace {

__device__ __forceinline__ uint64_t pack2(uint32_t lo, uint32_t hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float lo_f(uint64_t x) { return __uint_as_float((uint32_t)x); }
__device__ __forceinline__ float hi_f(uint64_t x) { return __uint_as_float((uint32_t)(x >> 32)); }

// sum += x with the rounding error of the addition collected in comp (Knuth's two-sum)
__device__ __forceinline__ void two_sum_add(float &sum, float &comp, float x) {
    const float t = sum + x;
    const float z = t - sum;
    comp += (sum - (t - z)) + (x - z);
    sum = t;
}

// one work item's record (three 16-byte loads through the read-only path)
__device__ __forceinline__ ItemRec load_item(const ItemRec *items, uint32_t it) {
    const uint4 *p = reinterpret_cast<const uint4 *>(items + it);
    const uint4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    ItemRec r;
    r.pos = a.x; r.index = a.y; r.n0 = a.z; r.mtiles = a.w;
    r.nk16 = b.x; r.M = b.y; r.N = b.z; r.m_pad = b.w;
    r.n_pad = c.x; r.a_row0 = (int32_t)c.y; r.b_row0 = (int32_t)c.z; r.pad = c.w;
    return r;
}

// K-major, 64-byte-swizzled operand tile at shared address `a` (rows 64 bytes apart; the
// second K step of a row starts 32 bytes in)
__device__ __forceinline__ uint64_t tile_desc(uint32_t a) {
    return sm100::smem_desc(a, 16, btc::SBO, btc::SW64);
}

}  // namespace

template <int BN, bool DUAL, typename TIn>
__global__ void __launch_bounds__(btc::THREADS, 1)
    batched_tc_kernel(const __grid_constant__ CUtensorMap map, const BatchedParams P) {
    using namespace btc;
    using namespace sm100;
    using C = Cfg<BN>;
    constexpr uint32_t BUF_COLS = DUAL ? 2 * BN : BN;   // P0 (and P1) of one tile
    constexpr uint32_t NBUF = TMEM_COLS / BUF_COLS;     // accumulator buffers in flight
    constexpr int HALVES = BN / BOX_ROWS;               // 128-row boxes per strip
    static_assert(NBUF >= 1 && NBUF <= 4, "tensor-memory buffers");
    // With an even number of buffers the two epilogue warps of a lane quadrant take alternate
    // tiles (each then meets only the phases of its own buffers, in order); with one buffer they
    // split every tile's columns instead (a warp may never wait two phases ahead on a barrier).
    constexpr bool ALT = NBUF % 2 == 0;
    constexpr int EW = ALT ? BN : BN / 2;              // columns one epilogue warp drains per tile

    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + (((raw + 1023) & ~1023u) - raw);
    uint8_t *strip = smem;                                          // 2 x STRIP_BYTES
    uint8_t *ring = smem + 2 * C::STRIP_BYTES;                      // RING x SLOT_BYTES
    float *vcol = reinterpret_cast<float *>(ring + RING * SLOT_BYTES);   // BN column factors
    int64_t *ocol = reinterpret_cast<int64_t *>(vcol + BN);              // BN column offsets
    Radix *s_ma = reinterpret_cast<Radix *>(ocol + BN);                  // the item's row digits
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(s_ma) + (sizeof(Radix) + 15) / 16 * 16);
    uint64_t *ring_full = bars, *ring_empty = bars + RING, *strip_full = bars + 2 * RING,
             *strip_empty = strip_full + 2, *acc_full = strip_empty + 2, *acc_empty = acc_full + 4,
             *mma_done = acc_empty + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t tmo = (uint64_t)P.timeout_ns;
    const uint32_t n_items = P.total_tiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RING; ++s) { mbar_init(&ring_full[s], 1); mbar_init(&ring_empty[s], 1); }
        for (int s = 0; s < 2; ++s) { mbar_init(&strip_full[s], 1); mbar_init(&strip_empty[s], 1); }
        for (int s = 0; s < 4; ++s) { mbar_init(&acc_full[s], 1); mbar_init(&acc_empty[s], ALT ? EPI_WARPS / 2 : EPI_WARPS); }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        fence_barrier_init();
        tma_prefetch_desc(&map);
    }
    if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(P.status, (int)COMET_ERR_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            uint32_t rit = 0, sit = 0;
            bool ok = true, injected = false;
            // one ring slot: three 128-row plane boxes of chunk kc, rows r0.. of an operand
            auto load_slot = [&](int64_t row0, uint32_t pad, uint32_t kc, uint32_t r0) -> bool {
                const uint32_t s = rit % RING, rnd = rit / RING;
                if (rnd > 0 && !mbar_wait(&ring_empty[s], (rnd - 1) & 1, tmo, abort_flag)) return false;
                mbar_arrive_expect_tx(&ring_full[s], SLOT_BYTES);
                ++rit;
                if ((P.debug_flags & 1) && !injected && blockIdx.x == 0) {
                    injected = true;   // fault injection: this slot's loads are withheld
                    return true;
                }
                uint8_t *dst = ring + s * SLOT_BYTES;
                for (uint32_t p = 0; p < 3; ++p)
                    tma_load_2d(&map, &ring_full[s], dst + p * BOX_BYTES, 0,
                                (int)(row0 + (int64_t)(kc * 3 + p) * pad + r0));
                return true;
            };
            ItemRec nxt;
            if (blockIdx.x < n_items) nxt = load_item(P.items, blockIdx.x);
            for (uint32_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                const ItemRec cur = nxt;
                if (it + gridDim.x < n_items) nxt = load_item(P.items, it + gridDim.x);   // one item ahead
                const uint32_t n0 = cur.n0, nk = cur.nk16, mtiles = cur.mtiles;
                const int64_t a0 = cur.a_row0, b0 = cur.b_row0;
                const uint32_t mp = cur.m_pad, np = cur.n_pad;
                const bool res = nk <= (uint32_t)MAX_RES_NK;
                if (res) {
                    const uint32_t sl = sit & 1, rnd = sit >> 1;
                    if (rnd > 0 && !mbar_wait(&strip_empty[sl], (rnd - 1) & 1, tmo, abort_flag)) {
                        fail(); ok = false; break;
                    }
                    mbar_arrive_expect_tx(&strip_full[sl], 3 * BN * ROW);
                    ++sit;
                    uint8_t *dst = strip + sl * C::STRIP_BYTES;
                    for (uint32_t p = 0; p < 3; ++p)
                        for (int h = 0; h < HALVES; ++h)
                            tma_load_2d(&map, &strip_full[sl], dst + (p * BN + h * BOX_ROWS) * ROW, 0,
                                        (int)(b0 + (int64_t)p * np + n0 + h * BOX_ROWS));
                }
                const uint32_t nkc = (nk + 1) / 2;   // chunks of 32 K values
                for (uint32_t mt = 0; mt < mtiles && ok; ++mt)
                    for (uint32_t kc = 0; kc < nkc && ok; ++kc) {
                        ok = load_slot(a0, mp, kc, mt * BM);
                        for (int h = 0; h < HALVES && ok && !res; ++h) ok = load_slot(b0, np, kc, n0 + h * BOX_ROWS);
                    }
                if (!ok) fail();
            }
            // drain: wait (bounded) for every load still in flight before the CTA may exit
            for (uint32_t j = rit > (uint32_t)RING ? rit - RING : 0; j < rit; ++j)
                mbar_wait(&ring_full[j % RING], (j / RING) & 1, tmo, nullptr);
            for (uint32_t j = sit > 2u ? sit - 2 : 0; j < sit; ++j) mbar_wait(&strip_full[j & 1], (j >> 1) & 1, tmo, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t idesc_full = idesc_bf16_f32(BM, BN);
            constexpr uint32_t idesc_half = idesc_bf16_f32(BM, BOX_ROWS);
            uint32_t rit = 0, sit = 0, tit = 0;
            bool ok = true;
            auto wait_slot = [&](uint32_t j) -> bool {
                return mbar_wait(&ring_full[j % RING], (j / RING) & 1, tmo, abort_flag);
            };
            ItemRec nxt;
            if (blockIdx.x < n_items) nxt = load_item(P.items, blockIdx.x);
            for (uint32_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                const ItemRec cur = nxt;
                if (it + gridDim.x < n_items) nxt = load_item(P.items, it + gridDim.x);   // one item ahead
                const uint32_t nk = cur.nk16, mtiles = cur.mtiles;
                const bool res = nk <= (uint32_t)MAX_RES_NK;
                uint32_t sl = 0;
                if (res) {
                    sl = sit & 1;
                    if (!mbar_wait(&strip_full[sl], (sit >> 1) & 1, tmo, abort_flag)) { fail(); ok = false; break; }
                    tc_fence_after();
                }
                const uint32_t sbase = smem_u32(strip + sl * C::STRIP_BYTES);
                for (uint32_t mt = 0; mt < mtiles && ok; ++mt) {
                    const uint32_t buf = tit % NBUF, rnd = tit / NBUF;
                    if (rnd > 0 && !mbar_wait(&acc_empty[buf], (rnd - 1) & 1, tmo, abort_flag)) {
                        fail(); ok = false; break;
                    }
                    tc_fence_after();
                    const uint32_t d0 = tmem_base + buf * BUF_COLS, d1 = DUAL ? d0 + BN : d0;
                    if (res) {
                        // one chunk: A in one ring slot, B resident in the strip; nk K steps of 16
                        if (!wait_slot(rit)) { fail(); ok = false; break; }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(ring + (rit % RING) * SLOT_BYTES);
                        uint64_t ad[MAX_RES_NK][3], bd[MAX_RES_NK][3];
#pragma unroll
                        for (int ks = 0; ks < MAX_RES_NK; ++ks)
#pragma unroll
                            for (int p = 0; p < 3; ++p) {
                                ad[ks][p] = tile_desc(sa + p * BOX_BYTES + ks * 32);
                                bd[ks][p] = tile_desc(sbase + p * BN * ROW + ks * 32);
                            }
                        // corrections of every K step first (smallest first), the hh products last
#pragma unroll
                        for (int ks = 0; ks < MAX_RES_NK; ++ks) {
                            if (ks >= (int)nk) break;
                            mma_bf16(d1, ad[ks][1], bd[ks][1], idesc_full, ks > 0 ? 1u : 0u);   // mm
                            mma_bf16(d1, ad[ks][2], bd[ks][0], idesc_full, 1);                 // lh
                            mma_bf16(d1, ad[ks][0], bd[ks][2], idesc_full, 1);                 // hl
                            mma_bf16(d1, ad[ks][1], bd[ks][0], idesc_full, 1);                 // mh
                            mma_bf16(d1, ad[ks][0], bd[ks][1], idesc_full, 1);                 // hm
                        }
#pragma unroll
                        for (int ks = 0; ks < MAX_RES_NK; ++ks) {
                            if (ks >= (int)nk) break;
                            mma_bf16(d0, ad[ks][0], bd[ks][0], idesc_full, (DUAL && ks == 0) ? 0u : 1u);   // hh
                        }
                        mma_commit(&ring_empty[rit % RING]);
                        rit += 1;
                    } else {
                        // K > 32 (dual accumulators): per chunk of 32, an A slot, then the B chunk's
                        // HALVES slots; the last chunk may hold a single K step
                        const uint32_t nkc = (nk + 1) / 2;
                        for (uint32_t kc = 0; kc < nkc && ok; ++kc) {
                            for (int q = 0; q <= HALVES && ok; ++q) ok = wait_slot(rit + q);
                            if (!ok) { fail(); break; }
                            tc_fence_after();
                            const uint32_t sa = smem_u32(ring + (rit % RING) * SLOT_BYTES);
                            const int ksteps = (int)min(2u, nk - 2 * kc);
                            for (int h = 0; h < HALVES; ++h) {
                                const uint32_t sb = smem_u32(ring + ((rit + 1 + h) % RING) * SLOT_BYTES);
                                const uint32_t e0 = d0 + h * BOX_ROWS, e1 = d1 + h * BOX_ROWS;
                                for (int ks = 0; ks < ksteps; ++ks) {
                                    const uint64_t a_h = tile_desc(sa + ks * 32), a_m = tile_desc(sa + BOX_BYTES + ks * 32),
                                                   a_l = tile_desc(sa + 2 * BOX_BYTES + ks * 32);
                                    const uint64_t b_h = tile_desc(sb + ks * 32), b_m = tile_desc(sb + BOX_BYTES + ks * 32),
                                                   b_l = tile_desc(sb + 2 * BOX_BYTES + ks * 32);
                                    const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                                    mma_bf16(e1, a_m, b_m, idesc_half, acc);
                                    mma_bf16(e1, a_l, b_h, idesc_half, 1);
                                    mma_bf16(e1, a_h, b_l, idesc_half, 1);
                                    mma_bf16(e1, a_m, b_h, idesc_half, 1);
                                    mma_bf16(e1, a_h, b_m, idesc_half, 1);
                                    mma_bf16(e0, a_h, b_h, idesc_half, acc);
                                }
                            }
                            for (int q = 0; q <= HALVES; ++q) mma_commit(&ring_empty[(rit + q) % RING]);
                            rit += 1 + HALVES;
                        }
                        if (!ok) break;
                    }
                    mma_commit(&acc_full[buf]);   // tile complete: the epilogue may drain it
                    ++tit;
                }
                if (!ok) break;
                if (res) {
                    mma_commit(&strip_empty[sl]);   // frees the strip once its MMAs have read it
                    ++sit;
                }
            }
            // no MMA may still write tensor memory when it is freed
            mma_commit(mma_done);
            mbar_wait(mma_done, 0, tmo, nullptr);
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        const int quad = warp & 3;                   // tensor-memory lanes 32*quad .. +31
        const uint32_t par = (uint32_t)(warp - 2) >> 2;   // ALT: the tile parity it drains; else its column half
        const int col0 = ALT ? 0 : (int)par * (BN / 2);
        const int et = threadIdx.x - 64;             // 0..255
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        const uint32_t key_m = P.swap ? ~P.key : P.key, key_n = ~key_m;
        uint32_t tit = 0;
        bool dead = false;   // once set, the warp keeps pace with the named barriers only
        ItemRec nxt;
        if (blockIdx.x < n_items) nxt = load_item(P.items, blockIdx.x);
        for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
            const ItemRec cur = nxt;
            if (it + gridDim.x < n_items) nxt = load_item(P.items, it + gridDim.x);   // one item ahead
            const BlockDesc *d = P.desc + cur.pos;
            const uint32_t M = cur.M, N = cur.N, idx = cur.index, mtiles = cur.mtiles, n0 = cur.n0;
            const uint32_t hb = idx * 0x9E3779B9u;
            const int e_sum = P.exps[2 * idx] + P.exps[2 * idx + 1];
            // the strip's column offsets and weight factors, and the block's row digits in shared
            // memory (all eight warps meet here)
            named_bar_sync(1, 32 * EPI_WARPS);
            for (int n = et; n < BN; n += 32 * EPI_WARPS) {
                int64_t o0 = 0, o1 = 0;
                const bool nv = n0 + n < N;
                if (nv) radix_offsets(d->nb, n0 + n, o0, o1);
                ocol[n] = o1;
                vcol[n] = nv ? tri_factor(key_n, hb, (uint32_t)o1) : 0.0f;
            }
            {
                constexpr int W = (int)(sizeof(Radix) / 8);
                const uint64_t *src = reinterpret_cast<const uint64_t *>(&d->ma);
                uint64_t *dst = reinterpret_cast<uint64_t *>(s_ma);
                if (et < W) dst[et] = __ldg(src + et);
            }
            named_bar_sync(1, 32 * EPI_WARPS);
            float S = 0.0f, cS = 0.0f, Q = 0.0f, cQ = 0.0f;
            TIn *out = P.mode == 1 ? reinterpret_cast<TIn *const *>(P.result)[idx] : nullptr;
            const double scale = ldexp(P.alpha, e_sum);
            for (uint32_t mt = 0; mt < mtiles; ++mt, ++tit) {
                const uint32_t buf = tit % NBUF, rnd = tit / NBUF;
                if (dead || (ALT && (tit & 1) != par)) continue;
                const uint32_t m = mt * BM + quad * 32 + lane;
                const bool mv = m < M;
                int64_t r0 = 0, orow = 0;
                if (mv) radix_offsets(*s_ma, m, r0, orow);   // while the tile's MMAs may still run
                bool ok = mbar_wait(&acc_full[buf], rnd & 1, tmo, abort_flag);
                ok = __all_sync(0xffffffffu, ok);   // warp-uniform before the .sync.aligned loads
                if (!ok) { if (lane == 0) fail(); dead = true; continue; }
                tc_fence_after();
                const uint32_t taddr = tmem_base + lane_base + buf * BUF_COLS + col0;
                if (P.mode == 0) {
                    // columns in batches (two or one 32-column loads per wait, P1 beside P0 when
                    // DUAL); two accumulator pairs per sum keep the FMA chains short
                    constexpr int CB = DUAL ? 32 : 64;
                    uint64_t ps0 = 0, ps1 = 0, pq0 = 0, pq1 = 0;   // two FP32 lanes each
#pragma unroll
                    for (int c = 0; c < EW; c += CB) {
                        uint32_t r[CB], r1[DUAL ? CB : 1];
#pragma unroll
                        for (int h = 0; h < CB; h += 32) {
                            tmem_ld32(taddr + c + h, *reinterpret_cast<uint32_t(*)[32]>(&r[h]));
                            if constexpr (DUAL) tmem_ld32(taddr + BN + c + h, *reinterpret_cast<uint32_t(*)[32]>(&r1[h]));
                        }
                        tmem_ld_wait();
                        if (c + CB >= EW) {   // every value of the tile is in registers
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&acc_empty[buf]);
                        }
                        const uint64_t *v2 = reinterpret_cast<const uint64_t *>(vcol + col0 + c);
#pragma unroll
                        for (int j = 0; j < CB; j += 4) {
                            uint64_t t0 = pack2(r[j], r[j + 1]), t1 = pack2(r[j + 2], r[j + 3]);
                            if constexpr (DUAL) {   // P0 + P1
                                t0 = add2(t0, pack2(r1[j], r1[j + 1]));
                                t1 = add2(t1, pack2(r1[j + 2], r1[j + 3]));
                            }
                            ps0 = fma2(t0, v2[j >> 1], ps0);
                            ps1 = fma2(t1, v2[(j >> 1) + 1], ps1);
                            pq0 = fma2(t0, t0, pq0);
                            pq1 = fma2(t1, t1, pq1);
                        }
                    }
                    if (mv) {
                        const uint64_t ps = add2(ps0, ps1), pq = add2(pq0, pq1);
                        two_sum_add(S, cS, (lo_f(ps) + hi_f(ps)) * tri_factor(key_m, hb, (uint32_t)orow));
                        two_sum_add(Q, cQ, lo_f(pq) + hi_f(pq));
                    }
                } else {
#pragma unroll 1
                    for (int c = 0; c < EW; c += 32) {
                        uint32_t r[32];
                        tmem_ld32(taddr + c, r);
                        if constexpr (DUAL) {
                            uint32_t r1[32];
                            tmem_ld32(taddr + BN + c, r1);
                            tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(r1[j]));
                        } else {
                            tmem_ld_wait();
                        }
                        if (c + 32 >= EW) {
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&acc_empty[buf]);
                        }
                        if (mv && out) {
                            TIn *row = out + orow;
                            const TIn sc = (TIn)scale;
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const int n = col0 + c + j;
                                if (n0 + n < N && dbg_ok(dbg_range(out, (int64_t)M * N * (int64_t)sizeof(TIn)),
                                                         row + ocol[n], (int)sizeof(TIn), P.status))
                                    row[ocol[n]] = sc * (TIn)__uint_as_float(r[j]);
                            }
                        }
                    }
                }
            }
            if (P.mode == 0 && !dead) {
                double s = (double)S + (double)cS, q = (double)Q + (double)cQ;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    s += __shfl_down_sync(0xffffffffu, s, o);
                    q += __shfl_down_sync(0xffffffffu, q, o);
                }
                if (lane == 0) {
                    double *res = reinterpret_cast<double *>(P.result);
                    atomicAdd(res + 2 * idx, s * scale);
                    atomicAdd(res + 2 * idx + 1, q * scale * scale);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}

// Split pre-pass: CTA c writes operand c%2 of block c/2 (launch order) as plane rows
// [chunk][plane][row] of 32 K values, rows to the operand's padded row count, scaled by the
// block's exponent; one thread per row, 64 bytes per plane row (coalesced across the warp).
template <typename TIn>
__global__ void __launch_bounds__(256) batched_presplit_tc_kernel(const BatchedParams P) {
    __shared__ int64_t k_off[1024];
    const BlockDesc &d = P.desc[blockIdx.x >> 1];
    const int op = blockIdx.x & 1;
    const Radix &rr = op ? d.nb : d.ma;
    const uint32_t rows = op ? d.N : d.M, pad = op ? d.n_pad : d.m_pad, K = d.K, nkc = (d.K + 31) / 32;
    const TIn *x = reinterpret_cast<const TIn *>(P.inputs[2 * d.index + (op ^ P.swap)]);
    const DbgRange xr = dbg_range(x, (op ? d.b_elems : d.a_elems) * (int64_t)sizeof(TIn));
    const DbgRange pr = dbg_range(P.planes, P.planes_bytes);
    const int e = P.exps[2 * d.index + op];
    uint4 *base = reinterpret_cast<uint4 *>(P.planes + (op ? d.b_row0 : d.a_row0) * kBatchedPlaneRow);
    for (uint32_t k = threadIdx.x; k < nkc * 32; k += 256) {
        int64_t o0 = 0, o1 = 0;
        if (k < K) radix_offsets(d.k, k, o0, o1);
        k_off[k] = op ? o1 : o0;
    }
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < pad; r += 256) {
        int64_t ro = 0, o1 = 0;
        const bool valid = r < rows;
        if (valid) radix_offsets(rr, r, ro, o1);
        for (uint32_t kc = 0; kc < nkc; ++kc) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {   // 16 K values (32 bytes) per plane at a time
                uint32_t w[3][8];
#pragma unroll
                for (int j = 0; j < 16; j += 2) {
                    __nv_bfloat16 h0, m0, l0, h1, m1, l1;
                    const uint32_t k = kc * 32 + half * 16 + j;
                    const TIn v0 = (valid && k < K && dbg_ok(xr, x + ro + k_off[k], (int)sizeof(TIn), P.status))
                                       ? x[ro + k_off[k]] : (TIn)0;
                    const TIn v1 = (valid && k + 1 < K && dbg_ok(xr, x + ro + k_off[k + 1], (int)sizeof(TIn), P.status))
                                       ? x[ro + k_off[k + 1]] : (TIn)0;
                    split3<TIn>(v0, e, h0, m0, l0);
                    split3<TIn>(v1, e, h1, m1, l1);
                    w[0][j >> 1] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                    w[1][j >> 1] = (uint32_t)__bfloat16_as_ushort(m0) | ((uint32_t)__bfloat16_as_ushort(m1) << 16);
                    w[2][j >> 1] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                }
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    uint4 *dst = base + ((size_t)(kc * 3 + p) * pad + r) * 4 + half * 2;
                    if (!dbg_ok(pr, dst, 32, P.status)) continue;
                    dst[0] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
                    dst[1] = make_uint4(w[p][4], w[p][5], w[p][6], w[p][7]);
                }
            }
        }
    }
}

// ---- host side --------------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

cudaError_t launch_batched_presplit(const BatchedParams &bp, int n_blocks, bool f64_in, cudaStream_t s) {
    if (n_blocks <= 0) return cudaSuccess;
    if (f64_in) batched_presplit_tc_kernel<double><<<2 * n_blocks, 256, 0, s>>>(bp);
    else batched_presplit_tc_kernel<float><<<2 * n_blocks, 256, 0, s>>>(bp);
    return cudaGetLastError();
}

template <int BN, bool DUAL, typename TIn>
static void launch_tc(const CUtensorMap &m, const BatchedParams &bp, int ctas, cudaStream_t s) {
    static const bool attr = [] {
        cudaFuncSetAttribute(batched_tc_kernel<BN, DUAL, TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             btc::Cfg<BN>::SMEM);
        return true;
    }();
    (void)attr;
    batched_tc_kernel<BN, DUAL, TIn><<<ctas, btc::THREADS, btc::Cfg<BN>::SMEM, s>>>(m, bp);
}

cudaError_t launch_batched_tc(const BatchedParams &bp, int64_t plane_rows, int strip, bool dual, bool f64_in,
                              cudaStream_t s) {
    if (bp.total_tiles == 0) return cudaSuccess;
    auto enc = encode_fn();
    if (!enc || plane_rows <= 0 || plane_rows >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
    // one map over every block's plane rows: 32 bf16 per row, 128-row boxes, 64-byte swizzle
    CUtensorMap m;
    cuuint64_t dims[2] = {32, (cuuint64_t)plane_rows};
    cuuint64_t strides[1] = {(cuuint64_t)kBatchedPlaneRow};
    cuuint32_t box[2] = {32, (cuuint32_t)btc::BOX_ROWS};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, bp.planes, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ctas = (int)std::min<uint32_t>(bp.total_tiles, (uint32_t)std::max(1, sms));
#define CM_TC(BNv, DUALv)                                                            \
    do {                                                                             \
        if (f64_in) launch_tc<BNv, DUALv, double>(m, bp, ctas, s);                   \
        else launch_tc<BNv, DUALv, float>(m, bp, ctas, s);                           \
    } while (0)
    if (strip == 256) {
        if (dual) CM_TC(256, true); else CM_TC(256, false);
    } else {
        if (dual) CM_TC(128, true); else CM_TC(128, false);
    }
#undef CM_TC
    return cudaGetLastError();
}

}  // namespace comet
