// Batched triples-like contractions in one persistent launch.
//
// Many small contractions of one two-operand expression with uneven extents (the model is the
// 6-D triples output of the CCSD(T) remark in Section 2: T[a,b,c,i,j,k] = sum_d A[d,a,b,i] *
// B[c,d,j,k] per block).  Every block is a GEMM over its merged label groups (the TTGT view of
// Section 2, with the permutations folded into the index arithmetic).  Work items are (block,
// output tile) pairs numbered through prefix sums of the blocks' tile counts, blocks in
// longest-first order; persistent CTAs take items from one atomic counter, so uneven blocks
// balance across the SMs.
//
// Two arithmetic paths:
//   FP64   f64 tensor-core MMA (mma.sync m8n8k4), FP64 accumulation
//   split  the fixed-point three-way bfloat16 split of each operand (split.cuh), written once
//          per block by a pre-pass into GEMM-ready planes; six part products on the tensor
//          cores (mma.sync m16n8k16 bf16, FP32 accumulation) over tiles copied with cp.async;
//          the hh products go to their own accumulator, exact for K <= 1024
// The output T of a block is either consumed in the epilogue (reduce mode: s_b = sum T*W and
// q_b = sum T^2 with a hashed weight W per element, one pair of atomic adds per tile) or stored
// (store mode).
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
#include <vector>

#include "../../include/comet.h"
#include "batched.h"
#include "launch.h"
#include "params.h"
#include "split.cuh"

static_assert(sizeof(comet::BlockDesc) % 16 == 0, "descriptors are copied as 16-byte words");

struct comet_plan_s {
    comet::Plan p;
};

namespace comet {

int prof_begin(int kind, cudaStream_t s);
void prof_end(int idx, cudaStream_t s);
enum { PK_BATCHED_F64_ID = 5, PK_BATCHED_SPLIT_ID = 6 };
void set_error_message(const std::string &s);

// ---- device helpers ----------------------------------------------------------------------------
// MurmurHash3 32-bit finalizer (Appleby, MurmurHash3, public domain)
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ float tri_weight(uint32_t key, uint32_t block, uint32_t lin) {
    const uint32_t h = fmix32(key ^ fmix32(block * 0x9E3779B9u + lin));
    return (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;   // exact in FP32 (24-bit integer)
}

// the same weight from a precomputed block term hb = block * 0x9E3779B9 (32-bit wraparound)
__device__ __forceinline__ float tri_weight_h(uint32_t key, uint32_t hb_plus_lin) {
    const uint32_t h = fmix32(key ^ fmix32(hb_plus_lin));
    return (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
}

// four 8x8 b16 matrices from shared memory; lane l supplies the address of row l%8 of matrix l/8
__device__ __forceinline__ void ldsm_x4(const void *p, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

__device__ __forceinline__ void bmma(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
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
        for (int i = t; i < BN; i += BT) {
            int64_t o0 = 0, o1 = 0;
            if (n0 + i < N) radix_offsets(sd.nb, n0 + i, o0, o1);
            b_col[i] = o0; o_col[i] = o1;
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
                Bs[k][n] = (n0 + n < N && k0 + k < K) ? (double)B[b_col[n] + b_k[k]] : 0.0;
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
                    As[k][m] = (m0 + m < M && k0 + k < K) ? (double)A[a_row[m] + a_k[k]] : 0.0;
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
                            const int64_t lin = o_row[ml] + o_col[nl];
                            if (P.mode == 0) {
                                s += T * (double)tri_weight(P.key, idx, (uint32_t)lin);
                                q += T * T;
                            } else if (out) {
                                out[lin] = (TIn)T;
                            }
                        }
                    }
            }
        }
        if (P.mode == 0) reduce_add(s, q, red, reinterpret_cast<double *>(P.result), idx);
        __syncthreads();
    }
}

// ---- split path --------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit_b() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_b() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Split pre-pass of the batched split path: CTA c writes operand c%2 of block c/2 as three
// bfloat16 planes [3][rows][kpad] (rows in the merged M or N order, K fastest, zero beyond K),
// scaled by the block's exponent.  A warp takes 32 rows at a time: each lane resolves one row's
// source offset, the warp then walks the rows with the lanes along K.
template <typename TIn>
__global__ void __launch_bounds__(256) batched_presplit_kernel(const BatchedParams P) {
    __shared__ int64_t k_off[1024];
    const BlockDesc &d = P.desc[blockIdx.x >> 1];
    const int op = blockIdx.x & 1;
    const Radix &rr = op ? d.nb : d.ma;
    const uint32_t rows = op ? d.N : d.M, K = d.K, kpad = d.kpad;
    const TIn *x = reinterpret_cast<const TIn *>(P.inputs[2 * d.index + (op ^ P.swap)]);
    const int e = P.exps[2 * d.index + op];
    __nv_bfloat16 *planes = reinterpret_cast<__nv_bfloat16 *>(P.ws + (op ? d.b_parts : d.a_parts));
    const int64_t plane = (int64_t)rows * kpad;
    for (uint32_t k = threadIdx.x; k < kpad; k += 256) {
        int64_t o0 = 0, o1 = 0;
        if (k < K) radix_offsets(d.k, k, o0, o1);
        k_off[k] = op ? o1 : o0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t r0 = warp * 32; r0 < rows; r0 += 8 * 32) {
        int64_t my = 0, o1 = 0;
        if (r0 + lane < rows) radix_offsets(rr, r0 + lane, my, o1);
        const uint32_t nr = min(32u, rows - r0);
        for (uint32_t j = 0; j < nr; ++j) {
            const int64_t ro = __shfl_sync(0xffffffffu, my, j);
            const int64_t base = (int64_t)(r0 + j) * kpad;
            for (uint32_t k = lane; k < kpad; k += 32) {
                const TIn v = k < K ? x[ro + k_off[k]] : (TIn)0;
                __nv_bfloat16 h, m, l;
                split3<TIn>(v, e, h, m, l);
                planes[base + k] = h;
                planes[plane + base + k] = m;
                planes[2 * plane + base + k] = l;
            }
        }
    }
}

// Split path main kernel: the operands arrive pre-split (batched_presplit_kernel), so a tile is
// three plane slabs of 32 K values copied with 16-byte cp.async; the M tiles of a strip are
// double-buffered (the copies of tile m+1 run under the MMAs and the epilogue of tile m).
template <int BM, int BN>
struct SplitSmem {
    static constexpr int KP = KCH + 8;                       // 80-byte rows: conflict-free fragments
    static constexpr int A_TILE = 3 * BM * KP;               // bf16 elements
    static constexpr int B_TILE = 3 * BN * KP;
    static constexpr size_t BYTES = (size_t)(2 * A_TILE + B_TILE) * 2;
};

template <int BM, int BN, typename TIn>
__global__ void __launch_bounds__(BT, BM * BN <= 4096 ? 4 : 2) batched_split_kernel(const BatchedParams P) {
    constexpr int MI = BM / 32, NJ = BN / 16;   // m16 / n8 MMA tiles per warp
    using SM = SplitSmem<BM, BN>;
    constexpr int KP = SM::KP;
    extern __shared__ __align__(16) __nv_bfloat16 dsm[];
    __nv_bfloat16 *As0 = dsm, *As1 = dsm + SM::A_TILE, *Bs = dsm + 2 * SM::A_TILE;
    __shared__ int64_t o_row[2][BM], o_col[BN];
    __shared__ __align__(16) BlockDesc sd;
    __shared__ double red[2 * BT / 32];
    __shared__ uint32_t s_item, s_pos;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, wm = warp & 1, wn = warp >> 1;
    const int g = lane >> 2, tq = lane & 3;
    uint32_t item, pos;
    while (next_item(P, item, pos, &s_item, &s_pos)) {
        copy_desc(P.desc + pos, &sd);
        __syncthreads();
        const uint32_t M = sd.M, N = sd.N, K = sd.K, idx = sd.index, kpad = sd.kpad;
        const uint32_t mtiles = (M + BM - 1) / BM;
        const uint32_t n0 = (item - P.prefix[pos]) * BN;
        const int ea = P.exps[2 * idx], eb = P.exps[2 * idx + 1];
        const bool bres = K <= (uint32_t)KCH;
        const __nv_bfloat16 *pa = reinterpret_cast<const __nv_bfloat16 *>(P.ws + sd.a_parts);
        const __nv_bfloat16 *pb = reinterpret_cast<const __nv_bfloat16 *>(P.ws + sd.b_parts);
        const int64_t plane_a = (int64_t)M * kpad, plane_b = (int64_t)N * kpad;
        for (int i = t; i < BN; i += BT) {
            int64_t o0 = 0, o1 = 0;
            if (n0 + i < N) radix_offsets(sd.nb, n0 + i, o0, o1);
            o_col[i] = o1;
        }
        // a [3][R][32] slab of plane rows r0.. at K offset k0 into shared memory (rows beyond
        // `rows` are zero-filled); 4 copies of 16 bytes per row and plane
        auto slab = [&](__nv_bfloat16 *dst, const __nv_bfloat16 *src, int64_t plane, uint32_t rows, uint32_t r0,
                        uint32_t k0, int R) {
            for (int c = t; c < 3 * R * 4; c += BT) {
                const int pl = c / (R * 4), rem = c - pl * R * 4, r = rem >> 2, q = rem & 3;
                const bool ok = r0 + r < rows;
                const __nv_bfloat16 *s = src + pl * plane + (ok ? (int64_t)(r0 + r) * kpad + k0 + q * 8 : 0);
                cp_async16((uint32_t)__cvta_generic_to_shared(dst + (pl * R + r) * KP + q * 8), s, ok ? 16u : 0u);
            }
        };
        auto rows_of = [&](int buf, uint32_t m0) {
            for (int i = t; i < BM; i += BT) {
                int64_t o0 = 0, o1 = 0;
                if (m0 + i < M) radix_offsets(sd.ma, m0 + i, o0, o1);
                o_row[buf][i] = o1;
            }
        };
        if (bres) {
            slab(Bs, pb, plane_b, N, n0, 0, BN);
            slab(As0, pa, plane_a, M, 0, 0, BM);
            cp_async_commit_b();
            rows_of(0, 0);
        }
        const float scale = (float)ldexp(P.alpha, ea + eb);
        float s = 0.0f, q = 0.0f;
        TIn *out = P.mode == 1 ? reinterpret_cast<TIn *const *>(P.result)[idx] : nullptr;
        for (uint32_t mt = 0; mt < mtiles; ++mt) {
            const uint32_t m0 = mt * BM;
            const int buf = mt & 1;
            const __nv_bfloat16 *As = buf ? As1 : As0;
            if (bres) {
                if (mt + 1 < mtiles) {   // prefetch the next M tile into the other buffer
                    slab(buf ? As0 : As1, pa, plane_a, M, m0 + BM, 0, BM);
                    cp_async_commit_b();
                    rows_of(buf ^ 1, m0 + BM);
                    cp_async_wait_b<1>();
                } else {
                    cp_async_wait_b<0>();
                }
                __syncthreads();
            } else {
                __syncthreads();
                rows_of(buf, m0);
            }
            float p0[MI][NJ][4], p1[MI][NJ][4];
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j)
#pragma unroll
                    for (int c = 0; c < 4; ++c) p0[i][j][c] = p1[i][j][c] = 0.0f;
            for (uint32_t k0 = 0; k0 < K; k0 += KCH) {
                if (!bres) {   // long K: one synchronous slab pair per chunk
                    __syncthreads();
                    slab(Bs, pb, plane_b, N, n0, k0, BN);
                    slab(const_cast<__nv_bfloat16 *>(As), pa, plane_a, M, m0, k0, BM);
                    cp_async_commit_b();
                    cp_async_wait_b<0>();
                    __syncthreads();
                }
                const int kmax = (int)min((uint32_t)KCH, K - k0);
#pragma unroll
                for (int ks = 0; ks < KCH / 16; ++ks) {
                    if (ks * 16 >= kmax) break;
                    uint32_t af[3][MI][4], bf[3][NJ][2];
#pragma unroll
                    for (int pl = 0; pl < 3; ++pl) {
                        // A 16x16 fragments: lanes 0-15 rows 0-15 at k, lanes 16-31 the same rows at k+8
#pragma unroll
                        for (int i = 0; i < MI; ++i) {
                            const int r = wm * (BM / 2) + i * 16 + (lane & 15);
                            const int c = ks * 16 + (lane >> 4) * 8;
                            ldsm_x4(As + (pl * BM + r) * KP + c, af[pl][i][0], af[pl][i][1], af[pl][i][2],
                                    af[pl][i][3]);
                        }
                        // B fragments of two n8 tiles: matrix l/8 = (tile j + (l/16), k half (l/8)%2)
#pragma unroll
                        for (int j = 0; j < NJ; j += 2) {
                            const int mi = lane >> 3;
                            const int r = wn * (BN / 2) + (j + (mi >> 1)) * 8 + (lane & 7);
                            const int c = ks * 16 + (mi & 1) * 8;
                            ldsm_x4(Bs + (pl * BN + r) * KP + c, bf[pl][j][0], bf[pl][j][1], bf[pl][j + 1][0],
                                    bf[pl][j + 1][1]);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < MI; ++i)
#pragma unroll
                        for (int j = 0; j < NJ; ++j) {
                            bmma(p1[i][j], af[1][i], bf[1][j]);   // mm
                            bmma(p1[i][j], af[2][i], bf[0][j]);   // lh
                            bmma(p1[i][j], af[0][i], bf[2][j]);   // hl
                            bmma(p1[i][j], af[1][i], bf[0][j]);   // mh
                            bmma(p1[i][j], af[0][i], bf[1][j]);   // hm
                            bmma(p0[i][j], af[0][i], bf[0][j]);   // hh: exact accumulator
                        }
                }
            }
            const int64_t *orow = o_row[buf];
            if (P.mode == 0) {
                // reduce: s and q accumulate the unscaled sums (the scale is applied once per
                // strip); output indices are below 2^32 (the plan refuses larger blocks)
                uint32_t ro[MI][2], co[NJ][2];
#pragma unroll
                for (int i = 0; i < MI; ++i)
#pragma unroll
                    for (int h = 0; h < 2; ++h) ro[i][h] = (uint32_t)orow[wm * (BM / 2) + i * 16 + g + 8 * h];
#pragma unroll
                for (int j = 0; j < NJ; ++j)
#pragma unroll
                    for (int h = 0; h < 2; ++h) co[j][h] = (uint32_t)o_col[wn * (BN / 2) + j * 8 + 2 * tq + h];
                const uint32_t hb = idx * 0x9E3779B9u, key = P.key;
                if (m0 + BM <= M && n0 + BN <= N) {   // interior tile: no bounds per element
#pragma unroll
                    for (int i = 0; i < MI; ++i)
#pragma unroll
                        for (int j = 0; j < NJ; ++j)
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const float u = p0[i][j][c] + p1[i][j][c];
                                s = fmaf(u, tri_weight_h(key, hb + ro[i][c >> 1] + co[j][c & 1]), s);
                                q = fmaf(u, u, q);
                            }
                } else {
#pragma unroll
                    for (int i = 0; i < MI; ++i)
#pragma unroll
                        for (int j = 0; j < NJ; ++j)
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const int ml = wm * (BM / 2) + i * 16 + g + (c >= 2 ? 8 : 0);
                                const int nl = wn * (BN / 2) + j * 8 + 2 * tq + (c & 1);
                                if (m0 + ml < M && n0 + nl < N) {
                                    const float u = p0[i][j][c] + p1[i][j][c];
                                    s = fmaf(u, tri_weight_h(key, hb + ro[i][c >> 1] + co[j][c & 1]), s);
                                    q = fmaf(u, u, q);
                                }
                            }
                }
            } else if (out) {
#pragma unroll
                for (int i = 0; i < MI; ++i)
#pragma unroll
                    for (int j = 0; j < NJ; ++j)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int ml = wm * (BM / 2) + i * 16 + g + (c >= 2 ? 8 : 0);
                            const int nl = wn * (BN / 2) + j * 8 + 2 * tq + (c & 1);
                            if (m0 + ml < M && n0 + nl < N)
                                out[orow[ml] + o_col[nl]] = (TIn)(scale * (p0[i][j][c] + p1[i][j][c]));
                        }
            }
            if (bres) __syncthreads();   // the buffer of this tile is refilled two tiles later
        }
        if (P.mode == 0)
            reduce_add((double)s * scale, (double)q * scale * scale, red, reinterpret_cast<double *>(P.result), idx);
        __syncthreads();
    }
}

// per-block operand scale exponents (split path): CTA c reduces operand c%2 of block c/2
template <typename TIn>
__global__ void __launch_bounds__(256) batched_absmax_kernel(const BatchedParams P) {
    __shared__ float red[8];
    const BlockDesc &d = P.desc[blockIdx.x >> 1];
    const int op = blockIdx.x & 1;
    const int64_t n = op ? d.b_elems : d.a_elems;
    const TIn *x = reinterpret_cast<const TIn *>(P.inputs[2 * d.index + (op ^ P.swap)]);
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) m = fmax(m, fabs((double)x[i]));
    float mf = (float)m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mf = fmaxf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mf;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int i = 0; i < 8; ++i) mm = fmax(mm, (double)red[i]);
        // exact maximum for the exponent: recompute from the FP64 value of the max element
        int e = 0;
        if (mm > 0.0 && !isinf(mm)) { frexp(mm, &e); e -= 1; }
        const_cast<int *>(P.exps)[2 * d.index + op] = e;
    }
}

// ---- host side ---------------------------------------------------------------------------------
struct TileCfg { int bm, bn; };
static const TileCfg kCfgF64[kBatchedCfgF64] = {{64, 64}, {64, 32}, {32, 64}, {32, 32}};
static const TileCfg kCfgSplit[kBatchedCfgSplit] = {{64, 64}, {128, 64}, {64, 128}};

static int n_cfg(const Plan &P) {
    return P.opts.precision == COMET_PREC_SPLIT_BF16 ? kBatchedCfgSplit : kBatchedCfgF64;
}

static TileCfg cfg_of(const Plan &P, int c) {
    return P.opts.precision == COMET_PREC_SPLIT_BF16 ? kCfgSplit[c] : kCfgF64[c];
}

// workspace layout: [counter 256 B][exps 8*n][prefix n_cfg*(n+1)*4][descs n*sizeof(BlockDesc)]
// [split path: the bfloat16 planes of every block's operands]
struct BLayout {
    size_t exps, prefix, desc, parts, total;
};

static BLayout layout_of(int n_blocks, int ncfg, size_t parts_bytes) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    BLayout L;
    L.exps = 256;
    L.prefix = al(L.exps + 8 * (size_t)n_blocks);
    L.desc = al(L.prefix + 4 * (size_t)ncfg * (n_blocks + 1));
    L.parts = al(L.desc + sizeof(BlockDesc) * (size_t)n_blocks);
    L.total = al(L.parts + parts_bytes);
    return L;
}

static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;
static bool g_tune_loaded = false;

static void tune_cache_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("COMET_AUTOTUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {   // one entry per line: "<cfg> <signature>"
        std::istringstream is(line);
        int c;
        std::string sig;
        if (is >> c && std::getline(is, sig) && !sig.empty()) g_tune_cache[sig.substr(1)] = c;
    }
}

static void tune_cache_store(const std::string &sig, int c) {
    g_tune_cache[sig] = c;
    const char *path = std::getenv("COMET_AUTOTUNE_CACHE");
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << c << " " << sig << "\n";
}

// problem class: expression, dtype, precision, block count and the spread of block sizes
static std::string signature(const Plan &P) {
    std::ostringstream o;
    double fmin = 1e300, fmax = 0;
    for (size_t b = 0; b < P.block_flops.size(); ++b) {
        fmin = std::min(fmin, P.block_flops[b]);
        fmax = std::max(fmax, P.block_flops[b]);
    }
    o << P.expr << "|" << (P.dtype == COMET_F32 ? "f32" : "f64") << "|"
      << (P.opts.precision == COMET_PREC_SPLIT_BF16 ? "split" : "f64") << "|n=" << P.n_blocks
      << "|fmin=" << (long long)(fmin / 1e6) << "M|fmax=" << (long long)(fmax / 1e6) << "M";
    return o.str();
}

std::string describe_batched(const Plan &P) {
    std::ostringstream o;
    const TileCfg c = cfg_of(P, P.tile_cfg);
    o << "{\"batched\":true,\"expr\":\"" << P.expr << "\",\"n_blocks\":" << P.n_blocks
      << ",\"precision\":\"" << (P.opts.precision == COMET_PREC_SPLIT_BF16 ? "split_bf16" : "native")
      << "\",\"flops\":" << P.flops << ",\"workspace\":" << P.batched_ws << ",\"tile_cfg\":" << P.tile_cfg
      << ",\"tile\":[" << c.bm << "," << c.bn << "],\"n_tile_cfgs\":" << n_cfg(P)
      << ",\"a_kcontig\":" << P.batched_ak << ",\"b_kcontig\":" << P.batched_bk
      << ",\"swap\":" << P.batched_swap << ",\"signature\":\""
      << signature(P) << "\"}";
    return o.str();
}

static cudaError_t launch_batched(const Plan &P, int cfg, const BatchedParams &bp, cudaStream_t s, int ctas) {
    const bool split = P.opts.precision == COMET_PREC_SPLIT_BF16;
    const bool f32 = P.dtype == COMET_F32;
    const bool ak = P.batched_ak, bk = P.batched_bk;
#define CM_F64(BMv, BNv, T)                                                                         \
    do {                                                                                            \
        if (ak && bk) batched_f64_kernel<BMv, BNv, true, true, T><<<ctas, BT, 0, s>>>(bp);         \
        else if (ak) batched_f64_kernel<BMv, BNv, true, false, T><<<ctas, BT, 0, s>>>(bp);         \
        else if (bk) batched_f64_kernel<BMv, BNv, false, true, T><<<ctas, BT, 0, s>>>(bp);         \
        else batched_f64_kernel<BMv, BNv, false, false, T><<<ctas, BT, 0, s>>>(bp);                \
    } while (0)
#define CM_SPL(BMv, BNv, T)                                                                         \
    do {                                                                                            \
        static const bool attr = [] {                                                               \
            cudaFuncSetAttribute(batched_split_kernel<BMv, BNv, T>,                                 \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,                       \
                                 (int)SplitSmem<BMv, BNv>::BYTES);                                  \
            return true;                                                                            \
        }();                                                                                        \
        (void)attr;                                                                                 \
        batched_split_kernel<BMv, BNv, T><<<ctas, BT, SplitSmem<BMv, BNv>::BYTES, s>>>(bp);        \
    } while (0)
    if (!split) {
        if (f32) {
            switch (cfg) { case 0: CM_F64(64, 64, float); break; case 1: CM_F64(64, 32, float); break;
                           case 2: CM_F64(32, 64, float); break; default: CM_F64(32, 32, float); }
        } else {
            switch (cfg) { case 0: CM_F64(64, 64, double); break; case 1: CM_F64(64, 32, double); break;
                           case 2: CM_F64(32, 64, double); break; default: CM_F64(32, 32, double); }
        }
    } else {
        if (f32) {
            switch (cfg) { case 0: CM_SPL(64, 64, float); break; case 1: CM_SPL(128, 64, float); break;
                           default: CM_SPL(64, 128, float); }
        } else {
            switch (cfg) { case 0: CM_SPL(64, 64, double); break; case 1: CM_SPL(128, 64, double); break;
                           default: CM_SPL(64, 128, double); }
        }
    }
#undef CM_F64
#undef CM_SPL
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
    const BLayout L = layout_of(P.n_blocks, n_cfg(P), P.batched_parts);
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
    cudaError_t e = cudaMemsetAsync(w, 0, 16, s);
    if (e == cudaSuccess && mode == 0) e = cudaMemsetAsync(result, 0, 16 * (size_t)P.n_blocks, s);
    if (e != cudaSuccess) return COMET_ERR_CUDA;
    const bool split = P.opts.precision == COMET_PREC_SPLIT_BF16;
    const int pk = split ? PK_BATCHED_SPLIT_ID : PK_BATCHED_F64_ID;
    int h = prof_begin(pk, s);
    if (split) {
        if (P.dtype == COMET_F32) {
            batched_absmax_kernel<float><<<2 * nb, 256, 0, s>>>(bp);
            batched_presplit_kernel<float><<<2 * nb, 256, 0, s>>>(bp);
        } else {
            batched_absmax_kernel<double><<<2 * nb, 256, 0, s>>>(bp);
            batched_presplit_kernel<double><<<2 * nb, 256, 0, s>>>(bp);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int ctas = (int)std::max<uint32_t>(1, std::min<uint32_t>(bp.total_tiles, (uint32_t)resident_ctas()));
        e = launch_batched(P, cfg, bp, s, ctas);
    }
    prof_end(h, s);
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
    if (!expr || !label_names || !extents || !dtypes) return COMET_ERR_NULL;
    if (n_blocks < 1 || n_labels < 1 || n_labels > 16) return COMET_ERR_ARG;
    for (int l = 0; l < n_labels; ++l) if (!label_names[l]) return COMET_ERR_NULL;
    for (int64_t i = 0; i < (int64_t)n_blocks * n_labels; ++i) if (extents[i] <= 0) return COMET_ERR_SHAPE;
    comet_plan_s *h = new (std::nothrow) comet_plan_s;
    if (!h) return COMET_ERR_INTERNAL;
    Plan &P = h->p;
    std::string err;
    std::vector<comet_extent_t> ex(n_labels);
    for (int l = 0; l < n_labels; ++l) ex[l] = comet_extent_t{label_names[l], extents[l]};
    comet_status_t st;
    try {
        st = build_plan(expr, ex.data(), n_labels, nullptr, 0, dtypes, n_dtypes, opts, &P, &err);
    } catch (...) {
        st = COMET_ERR_INTERNAL;
    }
    if (st == COMET_OK && (P.n_in != 2 || P.op != 0 || P.steps.size() != 1)) {
        st = COMET_ERR_UNSUPPORTED;
        err = "batched plans take one two-operand \"=\" contraction";
    }
    if (st == COMET_OK && !P.steps[0].form.Bt.empty()) {
        st = COMET_ERR_UNSUPPORTED;
        err = "batched plans take no batch labels (labels on both operands and the result)";
    }
    if (st == COMET_OK && (P.slots[0].view || P.slots[1].view || P.slots[2].view)) {
        st = COMET_ERR_UNSUPPORTED;
        err = "batched plans take no repeated labels";
    }
    if (st == COMET_OK && P.opts.precision == COMET_PREC_EMU_F64) {
        st = COMET_ERR_UNSUPPORTED;
        err = "batched plans take the native or the split precision";
    }
    if (st != COMET_OK) {
        set_error_message(err);
        delete h;
        return st;
    }
    // map the caller's label order to the plan's label ids
    std::vector<int> col(P.label_names.size(), -1);
    for (size_t id = 0; id < P.label_names.size(); ++id)
        for (int l = 0; l < n_labels; ++l)
            if (P.label_names[id] == label_names[l]) col[id] = l;
    for (int c : col)
        if (c < 0) { set_error_message("a label of the expression has no extent column"); delete h; return COMET_ERR_LABEL; }
    const Step &s0 = P.steps[0];
    const Slot &sa = P.slots[s0.a], &sb = P.slots[s0.b], &sc = P.slots[s0.c];
    const Slot &sm = s0.form.swap ? sb : sa, &sn = s0.form.swap ? sa : sb;
    P.batched = true;
    P.n_blocks = n_blocks;
    P.block_flops.resize(n_blocks);
    std::vector<BlockDesc> desc(n_blocks);
    std::vector<int64_t> e(P.label_names.size());
    double flops = 0;
    for (int b = 0; b < n_blocks; ++b) {
        for (size_t id = 0; id < e.size(); ++id) e[id] = extents[(int64_t)b * n_labels + col[id]];
        GemmParams g;
        gemm_params_for(e, sm.labels, sn.labels, sc.labels, s0.form, &g);
        if ((uint64_t)g.M * g.N >= (1ull << 32) || g.K > 1024) {
            set_error_message("a block's output exceeds 2^32 elements or its K exceeds 1024");
            delete h;
            return COMET_ERR_UNSUPPORTED;
        }
        BlockDesc &d = desc[b];
        std::memset(&d, 0, sizeof(d));
        d.ma = g.ma; d.nb = g.nb; d.k = g.k;
        d.M = g.M; d.N = g.N; d.K = g.K;
        d.index = (uint32_t)b;
        int64_t na = 1, nbv = 1;
        for (int l : sa.labels) na *= e[l];
        for (int l : sb.labels) nbv *= e[l];
        // the kernels read A = the M operand, B = the N operand; inputs are in expression order
        d.a_elems = s0.form.swap ? nbv : na;
        d.b_elems = s0.form.swap ? na : nbv;
        P.block_flops[b] = 2.0 * g.M * (double)g.N * g.K;
        flops += P.block_flops[b];
        if (b == 0) {
            P.batched_ak = g.k.n > 0 && g.k.s0[0] == 1;
            P.batched_bk = g.k.n > 0 && g.k.s1[0] == 1;
        }
    }
    P.batched_swap = s0.form.swap != 0;
    P.flops = flops;
    P.flops_natural = flops;
    // longest first
    std::vector<int> order(n_blocks);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return P.block_flops[x] > P.block_flops[y]; });
    const int ncfg = n_cfg(P);
    // split path: per-block plane offsets (relative to the workspace), in launch order
    size_t parts = 0;
    if (P.opts.precision == COMET_PREC_SPLIT_BF16) {
        for (int i = 0; i < n_blocks; ++i) {
            BlockDesc &d = desc[order[i]];
            d.kpad = (d.K + 31) / 32 * 32;
            d.a_parts = (int64_t)parts;
            parts += ((size_t)3 * d.M * d.kpad * 2 + 255) / 256 * 256;
            d.b_parts = (int64_t)parts;
            parts += ((size_t)3 * d.N * d.kpad * 2 + 255) / 256 * 256;
        }
    }
    P.batched_parts = parts;
    const BLayout L = layout_of(n_blocks, ncfg, parts);
    for (int i = 0; i < n_blocks && parts; ++i) {
        desc[order[i]].a_parts += (int64_t)L.parts;
        desc[order[i]].b_parts += (int64_t)L.parts;
    }
    P.batched_ws = L.total;
    P.batched_table.assign(L.parts - L.prefix, 0);
    P.batched_prefix.assign(ncfg, std::vector<uint32_t>(n_blocks + 1, 0));
    for (int c = 0; c < ncfg; ++c) {
        const TileCfg tc = cfg_of(P, c);
        uint64_t acc = 0;
        for (int i = 0; i < n_blocks; ++i) {
            const BlockDesc &d = desc[order[i]];
            P.batched_prefix[c][i] = (uint32_t)acc;
            acc += (uint64_t)((d.N + tc.bn - 1) / tc.bn);   // one item per N strip
        }
        if (acc >= (1ull << 32)) {
            set_error_message("more than 2^32 tiles");
            delete h;
            return COMET_ERR_UNSUPPORTED;
        }
        P.batched_prefix[c][n_blocks] = (uint32_t)acc;
        std::memcpy(P.batched_table.data() + 4 * (size_t)c * (n_blocks + 1), P.batched_prefix[c].data(),
                    4 * (size_t)(n_blocks + 1));
    }
    for (int i = 0; i < n_blocks; ++i)
        std::memcpy(P.batched_table.data() + (L.desc - L.prefix) + sizeof(BlockDesc) * (size_t)i, &desc[order[i]],
                    sizeof(BlockDesc));
    if (tile_hint >= ncfg) { delete h; return COMET_ERR_ARG; }
    int cfg = tile_hint;
    if (cfg < 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_cache_load();
        auto it = g_tune_cache.find(signature(P));
        cfg = (it != g_tune_cache.end() && it->second >= 0 && it->second < ncfg) ? it->second : 0;
    }
    P.tile_cfg = cfg;
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
    const BLayout L = layout_of(P.n_blocks, n_cfg(P), P.batched_parts);
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
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_load();
    tune_cache_store(signature(P), win);
    return COMET_OK;
}

}  // extern "C"
