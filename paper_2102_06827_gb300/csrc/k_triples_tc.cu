// Fused triples accumulation and energy in FP32 on the tensor cores (comet_triples_energy for
// FP32 plans; the CCSD(T) pattern the paper's Section 3 cites, see k_triples.cu).
//
// Every term of a block's T is one contraction over a summed label d: T[.] += alpha X[d, three
// T labels] Y[d, the other three].  For a pair-tile of T (8 values along T label 0, 4 along the
// others: 8192 elements) and one term, that is a 128 x 64 x d matrix product: the operand
// holding label 0 gives the 128 rows (8 x 4 x 4), the other one the 64 columns (4 x 4 x 4).
// No accumulator layout serves two terms (their operands split the six labels differently),
// so each term's product is formed in tensor memory and then added into the pair-tile in
// shared memory through the term's own index map; after the last term the pair-tile gives its
// share of E_b = sum T^2 / D_b.
//
//   * pre-pass (triples_tc_split_kernel): every operand of the batch's blocks is written once
//     as split-BF16 planes (x = h + m + l, three bfloat16, residual at most 2^-24 |x|), in rows of
//     32 summed indices (64 bytes), tile-blocked: [tile][chunk][plane][row of the tile], rows
//     and summed indices outside the block zero;
//   * main kernel (triples_tc_kernel), persistent, one CTA per SM: a TMA warp loads, per work
//     item, term and chunk, the three planes of both operand tiles into a ring slot (one 2-D
//     tensor map over all plane rows, 64-row boxes, 64-byte swizzle); one thread issues the six
//     products (hh, hm, mh, hl, lh, mm; the dropped ml, lm, ll sum to at most 2^-23 relative) as tcgen05
//     MMAs of 128 x 64 x 16 into one of four tensor-memory accumulators; sixteen drain warps
//     (four per lane quadrant, 16 columns each) load the accumulator and add alpha times it into
//     the pair-tile, the first term storing (column offsets are constants of the term's label
//     split: one code path per split); then the energy of the pair-tile's elements inside the
//     block, one FP64 atomic per pair-tile.
// Every wait is bounded; a wait that runs out records COMET_ERR_TIMEOUT in the status word.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/comet.h"
#include "launch.h"
#include "sm100.cuh"
#include "triples.h"

namespace comet {

using namespace tri;

namespace {

// x = h + m + l with each part the bfloat16 nearest to what is left (8 significant bits each):
// |x - h| <= 2^-8 |x|, |x - h - m| <= 2^-16 |x|, and the residual after l is at most 2^-24 |x|
// (each subtraction is exact in FP32)
__device__ __forceinline__ void split_bf16x3(float x, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
    h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    l = __float2bfloat16_rn(r2);
}

// One operand of one term for one block: its three T labels in T order (rank 0..2), their
// element strides and extents, tile sizes (8 for label 0, else 4) and tile counts, the summed
// label's stride and extent.
struct OpGeo {
    int lab[3], st[3], ext[3], ts[3], nt[3];
    int sd, ed, nch, rpt;
    bool wide;   // holds T label 0 (its rank 0)
};

__device__ __forceinline__ OpGeo op_geo(const TermDev &tm, int side, const int32_t *ext_b) {
    const int8_t *q = side ? tm.y_q : tm.x_q, *col = side ? tm.y_col : tm.x_col, *rk = side ? tm.y_rank : tm.x_rank;
    OpGeo g;
    int st = 1;
    g.sd = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int e = ext_b[col[m]];
        if (q[m] < 0) {
            g.sd = st;
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i)
                if (rk[m] == i) { g.lab[i] = q[m]; g.st[i] = st; g.ext[i] = e; }
        }
        st *= e;
    }
    g.ed = ext_b[tm.d_col];
    g.nch = (g.ed + tc::KCH - 1) / tc::KCH;
    g.wide = g.lab[0] == 0;
    g.rpt = g.wide ? tc::WROWS : tc::NROWS;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        g.ts[i] = g.lab[i] == 0 ? tc::WA : TS;
        g.nt[i] = (g.ext[i] + g.ts[i] - 1) / g.ts[i];
    }
    return g;
}

// coordinates inside a tile of plane row r: label 0 (wide operand) 8 values, the others 4
__device__ __forceinline__ void row_coords(bool wide, int r, int &c0, int &c1, int &c2) {
    if (wide) { c0 = r & 7; c1 = (r >> 3) & 3; c2 = r >> 5; }
    else { c0 = r & 3; c1 = (r >> 2) & 3; c2 = r >> 4; }
}

// K-major, 64-byte-swizzled operand tile at shared address a (rows 64 bytes apart; the second
// MMA step of 16 summed indices starts 32 bytes in)
__device__ __forceinline__ uint64_t tile_desc(uint32_t a) { return sm100::smem_desc(a, 16, 8 * tc::ROWB, 4); }

// the work item's block and pair-tile coordinates (tile index per T label; label 0 in tiles of 8)
struct Item {
    int b;
    int tc[6];
};

// The items blockIdx.x, + gridDim.x, ... of one launch, walked in order: the block is found by a
// forward scan of the pair-tile prefix sums, and within a block the coordinates advance by
// mixed-radix addition of the stride (divisions only when the block changes).
struct ItemWalk {
    Item item;
    uint32_t local, count;     // the item's index within its block, the block's pair-tiles
    int rad[6], step[6];       // tile counts per label; the stride in that radix
    int64_t g;                 // the item's global index

    __device__ __forceinline__ void enter_block(const Args &a, const TcArgs &t, uint32_t stride) {
        const int32_t *ext_b = a.ext + (int64_t)item.b * a.n_labels;
        uint32_t rem = local, st = stride;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const uint32_t ts = q == 0 ? tc::WA : TS;
            const uint32_t n = ((uint32_t)ext_b[a.t_col[q]] + ts - 1) / ts;
            rad[q] = (int)n;
            const uint32_t qt = rem / n;
            item.tc[q] = (int)(rem - qt * n);
            rem = qt;
            const uint32_t qs = st / n;
            step[q] = (int)(st - qs * n);
            st = qs;
        }
        count = (uint32_t)(t.prefix[item.b + 1] - t.prefix[item.b]);
    }
    // position on global item item0 + it, scanning blocks forward from b
    __device__ __forceinline__ void locate(const Args &a, const TcArgs &t, int b, uint32_t stride) {
        while (b + 1 < t.b1 && t.prefix[b + 1] <= g) ++b;
        item.b = b;
        local = (uint32_t)(g - t.prefix[b]);   // a block has fewer than 2^31 pair-tiles
        enter_block(a, t, stride);
    }
    __device__ __forceinline__ void start(const Args &a, const TcArgs &t, int64_t it) {
        g = t.item0 + it;
        int lo = t.b0, hi = t.b1;   // prefix[lo] <= g < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (t.prefix[mid] <= g) lo = mid; else hi = mid;
        }
        locate(a, t, lo, gridDim.x);
    }
    __device__ __forceinline__ void next(const Args &a, const TcArgs &t) {
        g += gridDim.x;
        local += gridDim.x;
        if (local < count) {
            int carry = 0;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const int d = item.tc[q] + step[q] + carry;
                carry = d >= rad[q];
                item.tc[q] = carry ? d - rad[q] : d;
            }
        } else {
            locate(a, t, item.b, gridDim.x);
        }
    }
};

__device__ __forceinline__ TcRec load_rec(const TcRec *rec, int64_t i) {
    const uint4 *p = reinterpret_cast<const uint4 *>(rec + i);
    TcRec r;
    uint4 *d = reinterpret_cast<uint4 *>(&r);
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = __ldg(p + k);
    return r;
}

// plane row of operand w's tile (chunk 0, plane 0) for a pair-tile
__device__ __forceinline__ int32_t rec_row(const TcRec &r, int w, const Item &item) {
    int32_t v = r.row0[w];
#pragma unroll
    for (int q = 0; q < 6; ++q) v += r.coef[w][q] * item.tc[q];
    return v;
}

// the i-th lowest label (bit) of a mask
constexpr int nth_label(int mask, int i) {
    for (int q = 0; q < 6; ++q)
        if ((mask >> q) & 1) {
            if (i == 0) return q;
            --i;
        }
    return -1;
}

// one drain warp's 16 columns of a term's product for this thread's row: column n = 16 colq +
// c0 + 4 c1 sits at the narrow labels' coordinates (c0, c1, colq); the first term stores, the
// others add (all loads before the stores: the 16 slots are distinct)
template <int MN>
__device__ __forceinline__ void drain16(float *T, int row, int colq, const uint32_t (&r)[16], float alpha, bool first) {
    constexpr int s0 = tc::tstride(nth_label(MN, 0)), s1 = tc::tstride(nth_label(MN, 1));
    float *tr = T + row + tc::tstride(nth_label(MN, 2)) * colq;
    if (first) {
#pragma unroll
        for (int j = 0; j < 16; ++j) tr[s0 * (j & 3) + s1 * (j >> 2)] = alpha * __uint_as_float(r[j]);
    } else {
        float o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) o[j] = tr[s0 * (j & 3) + s1 * (j >> 2)];
#pragma unroll
        for (int j = 0; j < 16; ++j) tr[s0 * (j & 3) + s1 * (j >> 2)] = fmaf(alpha, __uint_as_float(r[j]), o[j]);
    }
}

// the ten three-label masks without label 0
__device__ __forceinline__ void drain_dispatch(int mn, float *T, int row, int colq, const uint32_t (&r)[16],
                                               float alpha, bool first) {
    switch (mn) {
#define COMET_TC_D(v) \
    case v: drain16<v>(T, row, colq, r, alpha, first); break;
        COMET_TC_D(14) COMET_TC_D(22) COMET_TC_D(26) COMET_TC_D(28) COMET_TC_D(38)
        COMET_TC_D(42) COMET_TC_D(44) COMET_TC_D(50) COMET_TC_D(52) COMET_TC_D(56)
#undef COMET_TC_D
        default: break;   // every operand holds three T labels
    }
}

}  // namespace

// Pre-pass: CTA c writes operand c % 2 of term (c / 2) % n_terms of block b0 + c / (2 n_terms),
// one thread per plane row of the tile-blocked layout, 64 bytes per plane (coalesced across the
// warp); rows and summed indices outside the block are zero.
__global__ void __launch_bounds__(256) triples_tc_split_kernel(const Args a, const TcArgs t) {
    const int seg = blockIdx.x, side = seg & 1, p = (seg >> 1) % a.n_terms;
    const int b = t.b0 + seg / (2 * a.n_terms);
    const int32_t *ext_b = a.ext + (int64_t)b * a.n_labels;
    const OpGeo g = op_geo(a.term[p], side, ext_b);
    const float *x = reinterpret_cast<const float *>(a.ops[((int64_t)b * a.n_terms + p) * 2 + side]);
    uint4 *base = reinterpret_cast<uint4 *>(t.planes + (int64_t)t.row0[((int64_t)b * a.n_terms + p) * 2 + side] * tc::ROWB);
    const DbgRange xr = dbg_range(x, (int64_t)g.ext[0] * g.ext[1] * g.ext[2] * g.ed * 4);
    const DbgRange pr = dbg_range(t.planes, t.planes_bytes);
    const int64_t rows = (int64_t)g.nt[0] * g.nt[1] * g.nt[2] * g.rpt;
    for (int64_t R = threadIdx.x; R < rows; R += blockDim.x) {
        const int64_t tile = R / g.rpt;
        const int rr = (int)(R - tile * g.rpt);
        const int t0 = (int)(tile % g.nt[0]), t1 = (int)((tile / g.nt[0]) % g.nt[1]), t2 = (int)(tile / ((int64_t)g.nt[0] * g.nt[1]));
        int c0, c1, c2;
        row_coords(g.wide, rr, c0, c1, c2);
        const int g0 = t0 * g.ts[0] + c0, g1 = t1 * g.ts[1] + c1, g2 = t2 * g.ts[2] + c2;
        const bool valid = g0 < g.ext[0] && g1 < g.ext[1] && g2 < g.ext[2];
        const int64_t ro = valid ? (int64_t)g0 * g.st[0] + (int64_t)g1 * g.st[1] + (int64_t)g2 * g.st[2] : 0;
        for (int ch = 0; ch < g.nch; ++ch) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {   // 16 summed indices (32 bytes per plane) at a time
                uint32_t w[3][8];
#pragma unroll
                for (int j = 0; j < 16; j += 2) {
                    const int k = ch * tc::KCH + half * 16 + j;
                    const float v0 = (valid && k < g.ed && dbg_ok(xr, x + ro + (int64_t)k * g.sd, 4, a.status))
                                         ? x[ro + (int64_t)k * g.sd] : 0.0f;
                    const float v1 = (valid && k + 1 < g.ed && dbg_ok(xr, x + ro + (int64_t)(k + 1) * g.sd, 4, a.status))
                                         ? x[ro + (int64_t)(k + 1) * g.sd] : 0.0f;
                    __nv_bfloat16 h0, m0, l0, h1, m1, l1;
                    split_bf16x3(v0, h0, m0, l0);
                    split_bf16x3(v1, h1, m1, l1);
                    w[0][j >> 1] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                    w[1][j >> 1] = (uint32_t)__bfloat16_as_ushort(m0) | ((uint32_t)__bfloat16_as_ushort(m1) << 16);
                    w[2][j >> 1] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                }
#pragma unroll
                for (int pl = 0; pl < 3; ++pl) {
                    uint4 *dst = base + (((tile * g.nch + ch) * 3 + pl) * g.rpt + rr) * 4 + half * 2;
                    if (!dbg_ok(pr, dst, 32, a.status)) continue;
                    dst[0] = make_uint4(w[pl][0], w[pl][1], w[pl][2], w[pl][3]);
                    dst[1] = make_uint4(w[pl][4], w[pl][5], w[pl][6], w[pl][7]);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(tc::THREADS, 1)
    triples_tc_kernel(const __grid_constant__ CUtensorMap map, const Args a, const TcArgs t) {
    using namespace sm100;
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + (((raw + 1023) & ~1023u) - raw);
    uint8_t *ring = smem;                                            // RING x SLOT
    uint64_t *bars = reinterpret_cast<uint64_t *>(ring + RING * SLOT);
    uint64_t *full = bars, *empty = bars + RING, *tfull = bars + 2 * RING, *tempty = tfull + NACC, *mma_done = tempty + NACC;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    double *s_red = reinterpret_cast<double *>(tmem_slot + 4);     // DRAIN_WARPS partial sums
    int *s_geo = reinterpret_cast<int *>(s_red + DRAIN_WARPS);     // per term: pair-tile strides of
                                                                   // the wide labels 1, 2; narrow mask
    __shared__ float Tsh[TSZ];                                      // the pair-tile

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t tmo = (uint64_t)t.timeout_ns;
    const int64_t n_items = t.n_items;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RING; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int s = 0; s < NACC; ++s) { mbar_init(&tfull[s], 1); mbar_init(&tempty[s], DRAIN_WARPS); }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        fence_barrier_init();
        tma_prefetch_desc(&map);
    }
    if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
    if (threadIdx.x >= 64 && threadIdx.x < 64 + a.n_terms) {
        const TermDev &tm = a.term[threadIdx.x - 64];
        const int sw = (tm.xmask & 1) ? 0 : 1;   // the operand holding label 0
        const int8_t *qw = sw ? tm.y_q : tm.x_q, *rw = sw ? tm.y_rank : tm.x_rank;
        int *g = s_geo + 3 * (threadIdx.x - 64);
        for (int mm = 0; mm < 4; ++mm)
            if (qw[mm] >= 0 && rw[mm] >= 1) g[rw[mm] - 1] = tstride(qw[mm]);
        g[2] = sw ? (tm.xmask & 63) : (63 & ~tm.xmask);   // the other operand's labels
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(t.status, (int)COMET_ERR_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            uint32_t rit = 0;
            bool ok = true, injected = false;
            ItemWalk walk;
            if ((int64_t)blockIdx.x < n_items) walk.start(a, t, blockIdx.x);
            for (int64_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                if (it != (int64_t)blockIdx.x) walk.next(a, t);
                const Item &item = walk.item;
                for (int p = 0; p < a.n_terms && ok; ++p) {
                    const TcRec rec = load_rec(t.rec, (int64_t)item.b * a.n_terms + p);
                    const int32_t wrow = rec_row(rec, 0, item), nrow = rec_row(rec, 1, item);
                    for (int ch = 0; ch < rec.nch && ok; ++ch) {
                        const uint32_t s = rit % RING, rnd = rit / RING;
                        if (rnd > 0 && !mbar_wait(&empty[s], (rnd - 1) & 1, tmo, abort_flag)) { ok = false; break; }
                        mbar_arrive_expect_tx(&full[s], SLOT);
                        ++rit;
                        if ((t.debug_flags & 1) && !injected && blockIdx.x == 0) {
                            injected = true;   // fault injection: this slot's loads are withheld
                            continue;
                        }
                        uint8_t *dst = ring + s * SLOT;
#pragma unroll
                        for (int pl = 0; pl < 3; ++pl) {
                            const int wr = wrow + (ch * 3 + pl) * WROWS, nr = nrow + (ch * 3 + pl) * NROWS;
                            tma_load_2d(&map, &full[s], dst + pl * WPLANE, 0, wr);
                            tma_load_2d(&map, &full[s], dst + pl * WPLANE + BOX * ROWB, 0, wr + BOX);
                            tma_load_2d(&map, &full[s], dst + 3 * WPLANE + pl * NPLANE, 0, nr);
                        }
                    }
                }
            }
            if (!ok) fail();
            // wait (bounded) for every load still in flight before the CTA may exit
            for (uint32_t j = rit > (uint32_t)RING ? rit - RING : 0; j < rit; ++j)
                mbar_wait(&full[j % RING], (j / RING) & 1, tmo, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t idesc = idesc_bf16_f32(WROWS, NROWS);
            uint32_t rit = 0, tcount = 0;
            bool ok = true;
            ItemWalk walk;
            if ((int64_t)blockIdx.x < n_items) walk.start(a, t, blockIdx.x);
            for (int64_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                if (it != (int64_t)blockIdx.x) walk.next(a, t);
                const Item &item = walk.item;
                for (int p = 0; p < a.n_terms && ok; ++p, ++tcount) {
                    const TcRec rec = load_rec(t.rec, (int64_t)item.b * a.n_terms + p);
                    const int ed = rec.ed, nch = rec.nch;
                    const uint32_t ab = tcount % NACC, rnd = tcount / NACC;
                    if (rnd > 0 && !mbar_wait(&tempty[ab], (rnd - 1) & 1, tmo, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d = tmem_base + ab * NROWS;
                    for (int ch = 0; ch < nch; ++ch) {
                        const uint32_t s = rit % RING;
                        if (!mbar_wait(&full[s], (rit / RING) & 1, tmo, abort_flag)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(ring + s * SLOT), sb = sa + 3 * WPLANE;
                        const int kn = min(KCH, ed - ch * KCH), ksteps = (kn + 15) >> 4;
                        for (int ks = 0; ks < ksteps; ++ks) {
                            const uint64_t ah = tile_desc(sa + ks * 32), am = tile_desc(sa + WPLANE + ks * 32),
                                           al = tile_desc(sa + 2 * WPLANE + ks * 32);
                            const uint64_t bh = tile_desc(sb + ks * 32), bm = tile_desc(sb + NPLANE + ks * 32),
                                           bl = tile_desc(sb + 2 * NPLANE + ks * 32);
                            // the small products first, hh last
                            mma_bf16(d, am, bm, idesc, (ch > 0 || ks > 0) ? 1u : 0u);
                            mma_bf16(d, al, bh, idesc, 1);
                            mma_bf16(d, ah, bl, idesc, 1);
                            mma_bf16(d, am, bh, idesc, 1);
                            mma_bf16(d, ah, bm, idesc, 1);
                            mma_bf16(d, ah, bh, idesc, 1);
                        }
                        mma_commit(&empty[s]);
                        ++rit;
                    }
                    if (!ok) break;
                    mma_commit(&tfull[ab]);   // the term's product is complete: the drain may read it
                }
            }
            if (!ok) fail();
            // no MMA may still write tensor memory when it is freed
            mma_commit(mma_done);
            mbar_wait(mma_done, 0, tmo, nullptr);
        }
    } else {
        // ---------------- drain and energy (warps 2 .. 2 + DRAIN_WARPS) ----------------
        const int quad = warp & 3;                         // tensor-memory lanes 32 quad .. + 31
        const int colq = (warp - 2) >> 2;                  // columns 16 colq .. + 15
        const int et = threadIdx.x - 64;                   // 0 .. 32 DRAIN_WARPS - 1
        const int m = quad * 32 + lane;                    // the row this thread drains
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t tcount = 0;
        bool dead = false;   // once set, the warp keeps pace with the named barriers only
        ItemWalk walk;
        if ((int64_t)blockIdx.x < n_items) walk.start(a, t, blockIdx.x);
        for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
            if (it != (int64_t)blockIdx.x) walk.next(a, t);
            const Item &item = walk.item;
            const int32_t *ext_b = a.ext + (int64_t)item.b * a.n_labels;
            for (int p = 0; p < a.n_terms; ++p, ++tcount) {
                const TermDev &tm = a.term[p];
                const uint32_t ab = tcount % NACC, rnd = tcount / NACC;
                uint32_t r[16];
                if (!dead) {
                    bool ok = mbar_wait(&tfull[ab], rnd & 1, tmo, abort_flag);
                    ok = __all_sync(0xffffffffu, ok);   // warp-uniform before the .sync.aligned load
                    if (!ok) {
                        if (lane == 0) fail();
                        dead = true;
                    } else {
                        tc_fence_after();
                        tmem_ld16(tmem_base + lane_base + ab * NROWS + colq * 16, r);
                        tmem_ld_wait();
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty[ab]);
                    }
                }
                if (!dead) {
                    // this row of the term's product (the operand holding label 0: 8 x 4 x 4 rows)
                    // in the pair-tile; the columns' offsets are constants of the other operand's
                    // labels
                    const int *geo = s_geo + 3 * p;
                    const int row = (m & 7) + geo[0] * ((m >> 3) & 3) + geo[1] * (m >> 5);
                    const float alpha = tm.amode == 0 ? 1.0f : tm.amode == 1 ? -1.0f : (float)tm.alpha;
                    drain_dispatch(geo[2], Tsh, row, colq, r, alpha, p == 0);
                }
                named_bar_sync(1, 32 * DRAIN_WARPS);   // every term's additions before the next term's
            }
            // energy of the pair-tile's elements inside the block: thread et holds labels 0..3 at
            // (et & 7, et >> 3 & 3, et >> 5 & 3, et >> 7) and labels 4, 5 at all 16 pairs; D in
            // FP32, T^2 / D summed in FP32 over the 16, then in FP64
            double e_part = 0.0;
            if (!dead) {
                const int c4[4] = {et & 7, (et >> 3) & 3, (et >> 5) & 3, (et >> 7) & 3};
                bool v4 = true;
                float d4 = 0.0f;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int g = item.tc[q] * (q == 0 ? WA : TS) + c4[q];
                    const bool in = g < ext_b[a.t_col[q]];
                    v4 &= in;
                    if (in) d4 += a.sign[q] * reinterpret_cast<const float *>(a.eps[(int64_t)item.b * 6 + q])[g];
                }
                if (v4) {
                    float ev[2][4];
                    int ok2[2];
#pragma unroll
                    for (int q = 4; q < 6; ++q) {
                        const float *eq = reinterpret_cast<const float *>(a.eps[(int64_t)item.b * 6 + q]);
                        ok2[q - 4] = 0;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int g = item.tc[q] * TS + c;
                            const bool in = g < ext_b[a.t_col[q]];
                            ok2[q - 4] |= (int)in << c;
                            ev[q - 4][c] = in ? a.sign[q] * eq[g] : 0.0f;
                        }
                    }
                    const float *tp = Tsh + c4[0] + tstride(1) * c4[1] + tstride(2) * c4[2] + tstride(3) * c4[3];
                    float part = 0.0f;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int cj = u & 3, ck = u >> 2;
                        const bool in = ((ok2[0] >> cj) & 1) && ((ok2[1] >> ck) & 1);
                        const float tv = tp[tstride(4) * cj + tstride(5) * ck];
                        const float v = __fdividef(tv * tv, d4 + (ev[0][cj] + ev[1][ck]));
                        part += in ? v : 0.0f;
                    }
                    e_part = (double)part;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e_part += __shfl_xor_sync(0xffffffffu, e_part, o);
            if (lane == 0) s_red[warp - 2] = e_part;
            named_bar_sync(1, 32 * DRAIN_WARPS);   // the pair-tile is read; partial sums are in
            if (et == 0) {
                double sum = 0.0;
                for (int w = 0; w < DRAIN_WARPS; ++w) sum += s_red[w];
                if (sum != 0.0) atomicAdd(a.energies + item.b, sum);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}

// ---- host side --------------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 tri_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

cudaError_t launch_triples_tc(const Plan &P, const Args &a, TcArgs t, cudaStream_t s) {
    const TriplesPlan &tp = P.tri;
    auto enc = tri_encode_fn();
    if (!enc || tp.tc_max_rows <= 0 || tp.tc_max_rows >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
    // one map over the batch region's plane rows: 32 bf16 per row, 64-row boxes, 64-byte swizzle
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)tc::KCH, (cuuint64_t)tp.tc_max_rows};
    cuuint64_t strides[1] = {(cuuint64_t)tc::ROWB};
    cuuint32_t box[2] = {(cuuint32_t)tc::KCH, (cuuint32_t)tc::BOX};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, t.planes, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(triples_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (size_t bi = 0; bi + 1 < tp.tc_batch.size(); ++bi) {
        t.b0 = tp.tc_batch[bi];
        t.b1 = tp.tc_batch[bi + 1];
        t.item0 = tp.tc_prefix[t.b0];
        t.n_items = tp.tc_prefix[t.b1] - t.item0;
        if (t.n_items == 0) continue;
        int64_t batch_rows = 0;
        for (int b = t.b0; b < t.b1; ++b) batch_rows += tp.tc_rows[b];
        t.planes_bytes = batch_rows * tc::ROWB;
        const unsigned segs = (unsigned)((t.b1 - t.b0) * a.n_terms * 2);
        triples_tc_split_kernel<<<segs, 256, 0, s>>>(a, t);
        const int ctas = (int)std::min<int64_t>(t.n_items, std::max(1, sms));
        triples_tc_kernel<<<ctas, tc::THREADS, tc::SMEM, s>>>(map, a, t);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace comet
