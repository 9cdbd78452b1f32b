// Fused triples accumulation and energy (comet_plan_triples / comet_triples_energy).
//
// The CCSD(T) pattern the paper's Section 3 cites: a six-index block T_b built from two
// four-index operands per term, with several permuted terms summed into the same T_b, and an
// energy E_b = sum T_b^2 / D_b whose denominator is a signed sum of per-label vectors.  Every term
// contracts a single label (the paper's Section 2 contraction with K = that label's extent),
// so each term is a tiny-K outer-product sum and T_b is far larger than the operands: writing
// T_b to memory and reading it back per term would make the path bound by HBM traffic that the
// algorithm does not need.  Here T_b never leaves the SM.  FP32 plans run on the tensor cores
// (k_triples_tc.cu) unless a block's split operands exceed one batch of the workspace; then, and
// for FP64 plans, the FMA kernels of this file run them:
//
//   * a work item is one 4^6 tile of one block; persistent CTAs take items in chunks from one
//     atomic counter, walking the blocks in order;
//   * FP64 (triples_kernel<double>): each of the 256 threads holds 16 elements of the tile in
//     registers, 4 x 4 along two "owned" labels, the other four labels fixed per thread (the
//     FP32 kernel, triples_f32_kernel, further below, holds 2^6 per thread instead);
//   * a step is one term and one chunk of its summed label (16 values for FP64):
//     the X and Y tiles (chunk x 4^3) of step s+1 are copied into shared memory with cp.async
//     while step s runs on the other buffer; each thread adds its 16 dot products into its T
//     elements (a term with alpha = -1 negates them before and after; any other alpha but 1
//     scales the term's X entries in shared memory).  Depending on whether its owned labels sit
//     on X or Y, a thread reads 4 + 4, 16 + 1 or 1 + 16 values per summed index (four code
//     paths);
//   * after the last term, the thread's 16 elements give their T^2 / D, summed in FP64 per
//     thread across the CTA's items of one block and added to E_b once per block change.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/comet.h"
#include "launch.h"
#include "params.h"
#include "plan.hpp"
#include "triples.h"

struct comet_plan_s {
    comet::Plan p;
};

namespace comet {

// the FP32 tensor-core launch sequence (k_triples_tc.cu): per batch, the split pre-pass and the
// main kernel; a carries the device pointers, t the workspace tables and the status word
cudaError_t launch_triples_tc(const Plan &P, const tri::Args &a, tri::TcArgs t, cudaStream_t s);
int prof_begin(int kind, cudaStream_t s);
void prof_end(int idx, cudaStream_t s);
void set_error_message(const std::string &s);

using namespace tri;

using namespace tri;

// Operand tile addressing of one step (term p, summed-label chunk k0): element (kk, r) of the
// tile sits at base + kk * sd + digit0(r) * s0 + digit1(r) * s1 + digit2(r) * s2 (the operand's
// three T labels in its dimension order, 2-bit digits of r), present when kk < kn and each
// digit is below rem (the tile's remaining extent along that label, at most 4).  32-bit offsets:
// every operand has fewer than 2^31 elements (checked when planning).
struct TileAddr {
    int base, sd, s[3], rem[3];
    int n;                     // elements of the operand (debug builds check the staging reads)
};

template <typename T>
constexpr int kc_of() { return sizeof(T) == 4 ? KC : KC / 2; }

__device__ __forceinline__ void cp_async_elem(unsigned dst, const void *src, int bytes) {
    if (bytes == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Step entries of one operand: index idx -> (kk, r) with 8 consecutive kk and 4 consecutive r
// per 32 lanes: with the row pitch = 4 mod 32 floats the lanes of a warp hit 32 different banks.
template <int KCt>
__device__ __forceinline__ void entry(int idx, int &kk, int &r) {
    constexpr int hb = KCt / 8 == 4 ? 2 : 1;   // bits of the high kk part
    const int rest = idx >> 5;
    kk = ((rest & (KCt / 8 - 1)) << 3) | (idx & 7);
    r = ((rest >> hb) << 2) | ((idx >> 3) & 3);
}

// A thread's entries are idx = threadIdx.x + it * NT, it < kc * R / NT.  Since NT is a multiple
// of 32 * kc / 8, all of them have the kk of it = 0 and r = r0 + it * RS (RS = NT / kc, r0 < RS):
// digit 0 of r is fixed, and for RS = 8 digit 1 is h + 2 (it & 1) and digit 2 is it / 2, for
// RS = 16 digit 1 is h and digit 2 is it (h = r0 / 4).  So the row offset along digit 0 and the
// summed label is formed once per step, and each entry adds two stride multiples with
// compile-time factors.
template <typename T>
struct Lane {
    static constexpr int kc = kc_of<T>(), RS = NT / kc, NIT = kc * R / NT;
    static_assert(RS == 8 || RS == 16, "lane pattern");
    int kk, r0, d0, h;
    __device__ __forceinline__ Lane() {
        entry<kc>((int)threadIdx.x, kk, r0);
        d0 = r0 & 3;
        h = r0 >> 2;
    }
    static __device__ __forceinline__ constexpr int dd1(int it) { return RS == 8 ? 2 * (it & 1) : 0; }
    static __device__ __forceinline__ constexpr int d2(int it) { return RS == 8 ? it >> 1 : it; }
};

// issue the asynchronous copies of one operand tile into S (entries outside the tile are not
// written: they only feed T elements outside the block, which the energy skips)
template <typename T>
__device__ __forceinline__ void stage_async(T (*S)[RP], const T *__restrict__ src, const TileAddr &ta, int kn,
                                            int *status) {
    using L = Lane<T>;
    const L ln;
    if (ln.kk >= kn || ln.d0 >= ta.rem[0]) return;
    const T *row = src + (ta.base + ln.kk * ta.sd + ln.d0 * ta.s[0] + ln.h * ta.s[1]);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(&S[ln.kk][ln.r0]);
    const DbgRange rg = dbg_range(src, (int64_t)ta.n * (int64_t)sizeof(T));
#pragma unroll
    for (int it = 0; it < L::NIT; ++it)
        if (ln.h + L::dd1(it) < ta.rem[1] && L::d2(it) < ta.rem[2] &&
            dbg_ok(rg, row + (L::dd1(it) * ta.s[1] + L::d2(it) * ta.s[2]), (int)sizeof(T), status))
            cp_async_elem(dst + (unsigned)(it * L::RS * (int)sizeof(T)),
                          row + (L::dd1(it) * ta.s[1] + L::d2(it) * ta.s[2]), (int)sizeof(T));
}

// addressing of one operand for a step: q / col per dimension (q = -1: the summed label)
__device__ __forceinline__ TileAddr tile_addr(const int8_t *q, const int8_t *col, const int8_t *dig,
                                              const int32_t *ext_b, const int *tbase, const int *text, int k0) {
    TileAddr ta;
    int st = 1;
    ta.base = 0;
    ta.sd = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (q[m] < 0) {
            ta.sd = st;
            ta.base += k0 * st;
        } else {
            const int b0 = tbase[q[m]];
            const int rm = min(TS, text[q[m]] - b0);
            ta.base += b0 * st;
            if (dig[m] == 0) { ta.s[0] = st; ta.rem[0] = rm; }
            if (dig[m] == 1) { ta.s[1] = st; ta.rem[1] = rm; }
            if (dig[m] == 2) { ta.s[2] = st; ta.rem[2] = rm; }
        }
        st *= ext_b[col[m]];
    }
    ta.n = st;
    return ta;
}

// alpha times the X entries this thread copied for a step (after their copies completed)
template <typename T>
__device__ __forceinline__ void scale_own(T (*S)[RP], const TileAddr &ta, int kn, T alpha) {
    using L = Lane<T>;
    const L ln;
    if (ln.kk >= kn || ln.d0 >= ta.rem[0]) return;
    T *row = &S[ln.kk][ln.r0];
#pragma unroll
    for (int it = 0; it < L::NIT; ++it)
        if (ln.h + L::dd1(it) < ta.rem[1] && L::d2(it) < ta.rem[2]) row[it * L::RS] *= alpha;
}

// four consecutive shared-memory values (16-byte aligned): one 128-bit load for FP32, two for FP64
__device__ __forceinline__ void load4(const float *p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const double *p, double (&o)[4]) {
    const double2 v0 = reinterpret_cast<const double2 *>(p)[0], v1 = reinterpret_cast<const double2 *>(p)[1];
    o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
}

// The thread's 16 contributions of one step: acc[u][v] += sum_kk X[kk][rx(u,v)] * Y[kk][ry(u,v)].
// Owned labels are the fastest tile digits: u (or v) runs along 4 consecutive entries.
// case 0: u on X, v on Y; 1: u on Y, v on X; 2: both on X (u, then v = digit 1); 3: both on Y.
template <typename T>
__device__ __forceinline__ void step_compute(const T (*Xs)[RP], const T (*Ys)[RP], int kn, int rx, int ry,
                                             int kase, T (&acc)[16]) {
    constexpr int UK = sizeof(T) == 4 ? 4 : 2;   // summed indices unrolled (FP64: registers)
    if (kase == 0) {
#pragma unroll UK
        for (int kk = 0; kk < kn; ++kk) {
            T xu[4], yv[4];
            load4(&Xs[kk][rx], xu);
            load4(&Ys[kk][ry], yv);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u * 4 + v] = fma(xu[u], yv[v], acc[u * 4 + v]);
        }
    } else if (kase == 1) {
#pragma unroll UK
        for (int kk = 0; kk < kn; ++kk) {
            T yu[4], xv[4];
            load4(&Ys[kk][ry], yu);
            load4(&Xs[kk][rx], xv);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u * 4 + v] = fma(xv[v], yu[u], acc[u * 4 + v]);
        }
    } else if (kase == 2) {
#pragma unroll UK
        for (int kk = 0; kk < kn; ++kk) {
            const T y = Ys[kk][ry];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T xq[4];
                load4(&Xs[kk][rx + 4 * v], xq);
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u * 4 + v] = fma(xq[u], y, acc[u * 4 + v]);
            }
        }
    } else {
#pragma unroll UK
        for (int kk = 0; kk < kn; ++kk) {
            const T x = Xs[kk][rx];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T yq[4];
                load4(&Ys[kk][ry + 4 * v], yq);
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u * 4 + v] = fma(x, yq[u], acc[u * 4 + v]);
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(NT, 3) triples_kernel(const Args a) {
    constexpr int kc = kc_of<T>();
    __shared__ __align__(16) T Xs[2][kc][RP];
    __shared__ __align__(16) T Ys[2][kc][RP];
    __shared__ int32_t s_ext[16];
    __shared__ int64_t s_item;
    __shared__ double s_red[NT / 32];
    __shared__ TermDev s_term[16];
    __shared__ uint16_t s_dig[16][NT];    // per term and thread: rx | ry << 6 | case << 12
    __shared__ TileAddr s_ta[16][2];      // per term of the current tile: X and Y at k0 = 0
    __shared__ const void *s_ops[32];     // the current block's operand pointers
    __shared__ int s_tile[2][12];         // tile bases and block extents per T label, two items
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 16; ++i)
        if (t == i) s_term[i] = a.term[i];
    int f[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) f[j] = (t >> (2 * j)) & 3;
    __syncthreads();
    // tile-row offsets of this thread's fixed labels in each term's X and Y, and where its owned
    // labels sit (the same for every tile)
    for (int p = 0; p < a.n_terms; ++p) {
        const TermDev &tm = s_term[p];
        int rx = 0, ry = 0;
        bool u_on_x = false, v_on_x = false;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int qx = tm.x_q[m], qy = tm.y_q[m];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (qx == a.fixed[j]) rx += f[j] << (2 * tm.x_dig[m]);
                if (qy == a.fixed[j]) ry += f[j] << (2 * tm.y_dig[m]);
            }
            u_on_x |= qx == a.own[0];
            v_on_x |= qx == a.own[1];
        }
        const int kase = u_on_x ? (v_on_x ? 2 : 0) : (v_on_x ? 1 : 3);
        s_dig[p][t] = (uint16_t)(rx | (ry << 6) | (kase << 12));
    }

    int b = 0;                 // current block
    double e_acc = 0.0;
    auto flush = [&](int blk) {   // CTA sum of e_acc into E[blk]
        double v = e_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((t & 31) == 0) s_red[t >> 5] = v;
        __syncthreads();
        if (t == 0) {
            double sum = 0;
            for (int w = 0; w < NT / 32; ++w) sum += s_red[w];
            if (sum != 0.0) atomicAdd(a.energies + blk, sum);
        }
        __syncthreads();
        e_acc = 0.0;
    };
    bool have = false;
    int slot = 0;
    while (true) {
        if (t == 0) s_item = (int64_t)atomicAdd(a.counter, (unsigned long long)CHUNK);
        __syncthreads();
        const int64_t first = s_item;
        __syncthreads();
        if (first >= a.total) break;
        const int64_t last = min(first + (int64_t)CHUNK, a.total);
        for (int64_t item = first; item < last; ++item) {
            // block of this item (blocks are walked in order: search from the current one, or
            // from the start when the chunk lies before it)
            int nb = b;
            if (item < a.prefix[nb]) nb = 0;
            if (item >= a.prefix[nb + 1]) {
                int lo = nb, hi = a.n_blocks;   // prefix[lo] <= item < prefix[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (a.prefix[mid] <= item) lo = mid; else hi = mid;
                }
                nb = lo;
            }
            if (!have || nb != b) {
                if (have) flush(b);
                b = nb;
                have = true;
                if (t < a.n_labels) s_ext[t] = a.ext[(int64_t)b * a.n_labels + t];
                if (t < 2 * a.n_terms) s_ops[t] = a.ops[(int64_t)b * a.n_terms * 2 + t];
                __syncthreads();
            }
            // tile coordinates (first T label fastest; fewer than 2^31 tiles per block), by one
            // thread into the slot the previous item does not read
            const int *tbase = s_tile[slot], *text = s_tile[slot] + 6;
            if (t == 0) {
                int rem = (int)(item - a.prefix[b]);
                for (int q = 0; q < 6; ++q) {
                    const int e = s_ext[a.t_col[q]];
                    const int nt = (e + TS - 1) / TS;
                    const int qt = rem / nt;
                    s_tile[slot][q] = (rem - qt * nt) * TS;
                    s_tile[slot][6 + q] = e;
                    rem = qt;
                }
            }
            slot ^= 1;
            __syncthreads();   // the previous item's steps are done with both buffers and s_ta
            if (t < 2 * a.n_terms) {   // operand addressing of every term for this tile
                const TermDev &tm = s_term[t >> 1];
                s_ta[t >> 1][t & 1] = (t & 1) ? tile_addr(tm.y_q, tm.y_col, tm.y_dig, s_ext, tbase, text, 0)
                                              : tile_addr(tm.x_q, tm.x_col, tm.x_dig, s_ext, tbase, text, 0);
            }
            __syncthreads();
            // a thread whose fixed-label coordinates lie outside the block (the ragged last tile
            // along a label) still copies and meets every barrier, but skips the products: whole
            // warps of such threads free their issue slots
            bool fixed_ok = true;
#pragma unroll
            for (int j = 0; j < 4; ++j) fixed_ok &= tbase[a.fixed[j]] + f[j] < text[a.fixed[j]];
            T acc[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[e] = T(0);
            // steps: (term p, chunk k0) in order; step s+1's tiles are copied while step s runs
            int p = 0, k0 = 0, buf = 0;
            // addressing of term pp's operand (0: X, 1: Y) at summed-label chunk kk0
            auto addr = [&](int pp, int side, int kk0) {
                TileAddr ta = s_ta[pp][side];
                ta.base += kk0 * ta.sd;
                return ta;
            };
            auto issue = [&](int pp, int kk0, int bb) {
                const int K = s_ext[s_term[pp].d_col];
                const int kn = min(kc, K - kk0);
                const T *X = reinterpret_cast<const T *>(s_ops[2 * pp]);
                const T *Y = reinterpret_cast<const T *>(s_ops[2 * pp + 1]);
                stage_async<T>(Xs[bb], X, addr(pp, 0, kk0), kn, a.status);
                stage_async<T>(Ys[bb], Y, addr(pp, 1, kk0), kn, a.status);
                cp_async_commit();
            };
            issue(0, 0, 0);
            while (p < a.n_terms) {
                const int K = s_ext[s_term[p].d_col];
                const int amode = s_term[p].amode;
                const int kn = min(kc, K - k0);
                int pn = p, kn0 = k0 + kc;   // next step
                if (kn0 >= K) { pn = p + 1; kn0 = 0; }
                // alpha = -1: T - S = -(-T + S) in every rounding, so the accumulators are negated
                // around the term instead of scaling its X entries
                const bool neg = amode == 1;
                cp_async_wait_all();
                if (amode == 2) scale_own<T>(Xs[buf], addr(p, 0, k0), kn, (T)s_term[p].alpha);
                __syncthreads();   // step s is in buffer buf; step s-1's reads of buf^1 are done
                if (pn < a.n_terms) issue(pn, kn0, buf ^ 1);
                const int dg = s_dig[p][t];
                if (neg && k0 == 0) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[e] = -acc[e];
                }
                if (fixed_ok) step_compute<T>(Xs[buf], Ys[buf], kn, dg & 63, (dg >> 6) & 63, dg >> 12, acc);
                if (neg && pn != p) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[e] = -acc[e];
                }
                p = pn;
                k0 = kn0;
                buf ^= 1;
            }
            int own_b[2], own_e[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) { own_b[j] = tbase[a.own[j]]; own_e[j] = text[a.own[j]]; }
            // energy of the thread's elements: D = sum_q sign_q eps_q[coordinate q], in the
            // precision of T (FP32: one FP32 reciprocal per element, the tile's 16 terms summed in
            // FP32 and added to the FP64 block sum once; FP64: all in FP64)
            if (fixed_ok) {
                T dfix = T(0);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    dfix += (T)a.fixed_sign[j] *
                            reinterpret_cast<const T *>(a.eps[(int64_t)b * 6 + a.fixed[j]])[tbase[a.fixed[j]] + f[j]];
                const T *e0 = reinterpret_cast<const T *>(a.eps[(int64_t)b * 6 + a.own[0]]);
                const T *e1 = reinterpret_cast<const T *>(a.eps[(int64_t)b * 6 + a.own[1]]);
                T tile_e = T(0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c0 = own_b[0] + u;
                    if (c0 >= own_e[0]) continue;
                    const T d0 = dfix + (T)a.own_sign[0] * e0[c0];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int c1 = own_b[1] + v;
                        if (c1 >= own_e[1]) continue;
                        const T tv = acc[u * 4 + v];
                        tile_e += tv * tv / (d0 + (T)a.own_sign[1] * e1[c1]);
                    }
                }
                e_acc += (double)tile_e;
            }
        }
    }
    if (have) flush(b);
}

// ---------------------------------------------------------------------------------------------
// FP32: one CTA of 64 threads per 4^6 tile, 2^6 elements per thread (triples.h).  Every term is
// then an 8 x 8 outer product per summed index whatever labels its operands hold: the thread
// reads its 8 entries of each operand as four 16-byte shared-memory loads and does 64 FMAs as
// 32 packed ones.  (The 256-thread layout above holds 4 x 4 along two labels: a term with both on
// one operand reads 16 + 1 entries for 16 FMAs, and the kernel is bound by shared-memory
// wavefronts.)

// the three bits of v placed at the set bits of m, lowest first
__host__ __device__ constexpr int deposit3(int v, int m) {
    int r = 0, b = 0;
    for (int j = 0; j < 6; ++j)
        if ((m >> j) & 1) {
            if ((v >> b) & 1) r |= 1 << j;
            ++b;
        }
    return r;
}
template <int M>
struct DepTab {
    int v[8];
    constexpr DepTab() : v() {
        for (int i = 0; i < 8; ++i) v[i] = deposit3(i, M);
    }
};

// the bits of t at the set bits of m, packed from bit 0
__device__ __forceinline__ int extract6(int t, int m) {
    int r = 0, b = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j)
        if ((m >> j) & 1) {
            r |= ((t >> j) & 1) << b;
            ++b;
        }
    return r;
}

// staging addressing of one operand for a tile: element offset of the tile's corner at k0 = 0,
// stride of the summed label, and per rank i (the operand's T labels in T order) the stride and
// the entries left in the tile (at most 4)
struct StageAddr {
    int base, sd, s[3], rem[3];
    int n;                     // elements of the operand (debug builds check the staging reads)
};

__device__ __forceinline__ StageAddr stage_addr(const int8_t *q, const int8_t *col, const int8_t *rank,
                                                const int32_t *ext_b, const int *tbase, const int *text) {
    StageAddr sa;
    int st = 1;
    sa.base = 0;
    sa.sd = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (q[m] < 0) {
            sa.sd = st;
        } else {
            const int b0 = tbase[q[m]];
            const int rm = min(TS, text[q[m]] - b0);
            sa.base += b0 * st;
            if (rank[m] == 0) { sa.s[0] = st; sa.rem[0] = rm; }
            if (rank[m] == 1) { sa.s[1] = st; sa.rem[1] = rm; }
            if (rank[m] == 2) { sa.s[2] = st; sa.rem[2] = rm; }
        }
        st *= ext_b[col[m]];
    }
    sa.n = st;
    return sa;
}

// coordinates of the entry of staged row r along the operand's rank-i label
__device__ __forceinline__ int row_coord(int r, int i) { return 2 * ((r >> (3 + i)) & 1) + ((r >> i) & 1); }

// thread t copies row t of the operand tile for summed indices k0 .. k0 + kn - 1 (rows outside
// the tile are not written: they only feed elements outside the block, which the energy skips)
__device__ __forceinline__ void stage32(float (*S)[RP32], const float *__restrict__ src, const StageAddr &sa, int k0,
                                        int kn, int *status) {
    const int r = (int)threadIdx.x;
    const int c0 = row_coord(r, 0), c1 = row_coord(r, 1), c2 = row_coord(r, 2);
    if (c0 >= sa.rem[0] || c1 >= sa.rem[1] || c2 >= sa.rem[2]) return;
    const float *g = src + (sa.base + k0 * sa.sd + c0 * sa.s[0] + c1 * sa.s[1] + c2 * sa.s[2]);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(&S[0][r]);
    const DbgRange rg = dbg_range(src, (int64_t)sa.n * 4);
#pragma unroll 4
    for (int kk = 0; kk < kn; ++kk)
        if (dbg_ok(rg, g + (int64_t)kk * sa.sd, 4, status))
            cp_async_elem(dst + (unsigned)(kk * RP32 * 4), g + (int64_t)kk * sa.sd, 4);
}

// alpha times the entries this thread copied (after their copies completed)
__device__ __forceinline__ void scale32(float (*S)[RP32], const StageAddr &sa, int kn, float alpha) {
    const int r = (int)threadIdx.x;
    if (row_coord(r, 0) >= sa.rem[0] || row_coord(r, 1) >= sa.rem[1] || row_coord(r, 2) >= sa.rem[2]) return;
    for (int kk = 0; kk < kn; ++kk) S[kk][r] *= alpha;
}

__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t bcast2(float x) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(x));
    return d;
}

// The 64 accumulators as 32 packed pairs: acc[e >> 1] holds elements e (low 32 bits) and e + 1,
// which differ in the low bit of T label 0.  Each packed FMA is two fmaf roundings.
//
// One step of a term: P holds the operand with T label 0 (its labels: mask MP; label 0 is its
// rank 0, so entries 2m and 2m + 1 of the thread's run form a natural pair), B the other one,
// whose values are broadcast to both halves.  Element e gains P[kk][8 hp + p(e)] *
// B[kk][8 hb + b(e)], p(e) / b(e) = the bits of e at the labels of P / B.
template <int MP>
__device__ __forceinline__ void outer32(const float (*P)[RP32], const float (*B)[RP32], int kn, int hp, int hb,
                                        uint64_t (&acc)[32]) {
    constexpr DepTab<MP> dp{};
    constexpr DepTab<63 & ~MP> db{};
    const float *pp = &P[0][8 * hp];
    const float *bp = &B[0][8 * hb];
#pragma unroll 1
    for (int kk = 0; kk < kn; ++kk) {
        const ulonglong2 p0 = *reinterpret_cast<const ulonglong2 *>(pp + kk * RP32);
        const ulonglong2 p1 = *reinterpret_cast<const ulonglong2 *>(pp + kk * RP32 + 4);
        const float4 b0 = *reinterpret_cast<const float4 *>(bp + kk * RP32);
        const float4 b1 = *reinterpret_cast<const float4 *>(bp + kk * RP32 + 4);
        const uint64_t pr[4] = {p0.x, p0.y, p1.x, p1.y};
        const uint64_t bb[8] = {bcast2(b0.x), bcast2(b0.y), bcast2(b0.z), bcast2(b0.w),
                                bcast2(b1.x), bcast2(b1.y), bcast2(b1.z), bcast2(b1.w)};
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int bi = 0; bi < 8; ++bi) {
                const int e2 = (dp.v[2 * m] | db.v[bi]) >> 1;
                acc[e2] = fma2(pr[m], bb[bi], acc[e2]);
            }
    }
}

// the ten three-label masks that hold label 0
__device__ __forceinline__ void outer32_dispatch(int mp, const float (*P)[RP32], const float (*B)[RP32], int kn,
                                                 int hp, int hb, uint64_t (&acc)[32]) {
    switch (mp) {
#define COMET_TRI_M(v) \
    case v: outer32<v>(P, B, kn, hp, hb, acc); break;
        COMET_TRI_M(7) COMET_TRI_M(11) COMET_TRI_M(13) COMET_TRI_M(19) COMET_TRI_M(21)
        COMET_TRI_M(25) COMET_TRI_M(35) COMET_TRI_M(37) COMET_TRI_M(41) COMET_TRI_M(49)
#undef COMET_TRI_M
        default: break;   // the planner gives every operand three T labels
    }
}

__global__ void __launch_bounds__(NT32, CTAS32) triples_f32_kernel(const Args a) {
    __shared__ __align__(16) float Ps[2][KC32][RP32];   // the operand holding T label 0
    __shared__ __align__(16) float Bs[2][KC32][RP32];   // the other one
    __shared__ int32_t s_ext[16];
    __shared__ int64_t s_item;
    __shared__ double s_red[NT32 / 32];
    __shared__ StageAddr s_sa[16][2];     // per term of the current tile: X and Y
    __shared__ const void *s_ops[32];     // the current block's operand pointers
    __shared__ int s_tile[2][12];         // tile bases and block extents per T label, two items
    const int t = threadIdx.x;

    int b = 0;                 // current block
    double e_acc = 0.0;
    auto flush = [&](int blk) {   // CTA sum of e_acc into E[blk]
        double v = e_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((t & 31) == 0) s_red[t >> 5] = v;
        __syncthreads();
        if (t == 0) {
            double sum = 0;
            for (int w = 0; w < NT32 / 32; ++w) sum += s_red[w];
            if (sum != 0.0) atomicAdd(a.energies + blk, sum);
        }
        __syncthreads();
        e_acc = 0.0;
    };
    bool have = false;
    int slot = 0;
    while (true) {
        if (t == 0) s_item = (int64_t)atomicAdd(a.counter, (unsigned long long)CHUNK);
        __syncthreads();
        const int64_t first = s_item;
        __syncthreads();
        if (first >= a.total) break;
        const int64_t last = min(first + (int64_t)CHUNK, a.total);
        for (int64_t item = first; item < last; ++item) {
            int nb = b;
            if (item < a.prefix[nb]) nb = 0;
            if (item >= a.prefix[nb + 1]) {
                int lo = nb, hi = a.n_blocks;   // prefix[lo] <= item < prefix[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (a.prefix[mid] <= item) lo = mid; else hi = mid;
                }
                nb = lo;
            }
            if (!have || nb != b) {
                if (have) flush(b);
                b = nb;
                have = true;
                if (t < a.n_labels) s_ext[t] = a.ext[(int64_t)b * a.n_labels + t];
                if (t < 2 * a.n_terms) s_ops[t] = a.ops[(int64_t)b * a.n_terms * 2 + t];
                __syncthreads();
            }
            const int *tbase = s_tile[slot], *text = s_tile[slot] + 6;
            if (t == 0) {
                int rem = (int)(item - a.prefix[b]);
                for (int q = 0; q < 6; ++q) {
                    const int e = s_ext[a.t_col[q]];
                    const int nt = (e + TS - 1) / TS;
                    const int qt = rem / nt;
                    s_tile[slot][q] = (rem - qt * nt) * TS;
                    s_tile[slot][6 + q] = e;
                    rem = qt;
                }
            }
            slot ^= 1;
            __syncthreads();   // the previous item's steps are done with both buffers and s_sa
            if (t < 2 * a.n_terms) {
                const TermDev &tm = a.term[t >> 1];
                s_sa[t >> 1][t & 1] = (t & 1) ? stage_addr(tm.y_q, tm.y_col, tm.y_rank, s_ext, tbase, text)
                                              : stage_addr(tm.x_q, tm.x_col, tm.x_rank, s_ext, tbase, text);
            }
            __syncthreads();
            // a thread whose 2^6 box lies outside the block along some label (the ragged last
            // tile) still copies and meets every barrier, but skips the products
            bool live = true;
#pragma unroll
            for (int j = 0; j < 6; ++j) live &= tbase[j] + 2 * ((t >> j) & 1) < text[j];
            uint64_t acc[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) acc[e] = 0ull;
            int p = 0, k0 = 0, buf = 0;
            auto issue = [&](int pp, int kk0, int bb) {
                const int K = s_ext[a.term[pp].d_col];
                const int kn = min(KC32, K - kk0);
                const int sp = (a.term[pp].xmask & 1) ? 0 : 1;   // operand holding T label 0
                stage32(Ps[bb], reinterpret_cast<const float *>(s_ops[2 * pp + sp]), s_sa[pp][sp], kk0, kn, a.status);
                stage32(Bs[bb], reinterpret_cast<const float *>(s_ops[2 * pp + 1 - sp]), s_sa[pp][1 - sp], kk0, kn,
                        a.status);
                cp_async_commit();
            };
            issue(0, 0, 0);
            while (p < a.n_terms) {
                const int K = s_ext[a.term[p].d_col];
                const int kn = min(KC32, K - k0);
                int pn = p, kn0 = k0 + KC32;   // next step
                if (kn0 >= K) { pn = p + 1; kn0 = 0; }
                cp_async_wait_all();
                // alpha other than 1 scales the term's X entries (alpha = -1 exactly: the sums
                // are the negated ones in every rounding)
                if (a.term[p].amode != 0) {
                    scale32((a.term[p].xmask & 1) ? Ps[buf] : Bs[buf], s_sa[p][0], kn, (float)a.term[p].alpha);
                }
                __syncthreads();   // step s is in buffer buf; step s-1's reads of buf^1 are done
                if (pn < a.n_terms) issue(pn, kn0, buf ^ 1);
                if (live) {
                    const int m = a.term[p].xmask;
                    const int mp = (m & 1) ? m : 63 & ~m;
                    outer32_dispatch(mp, Ps[buf], Bs[buf], kn, extract6(t, mp), extract6(t, 63 & ~mp), acc);
                }
                p = pn;
                k0 = kn0;
                buf ^= 1;
            }
            // energy: D = sum_j sign_j eps_j[coordinate j], element e at coordinate tbase_j +
            // 2 h_j + (bit j of e); FP32 T^2 / D summed in FP32 over 16 elements, then in FP64
            if (live) {
                float ev[6][2];
                int ok[6];   // bit l: coordinate 2 h_j + l lies inside the block
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    const float *ej = reinterpret_cast<const float *>(a.eps[(int64_t)b * 6 + j]);
                    ok[j] = 0;
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        const int c = tbase[j] + 2 * ((t >> j) & 1) + l;
                        const bool in = c < text[j];
                        ok[j] |= (int)in << l;
                        ev[j][l] = in ? a.sign[j] * ej[c] : 0.f;
                    }
                }
                float d012[8], d345[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    d012[e] = (ev[0][e & 1] + ev[1][(e >> 1) & 1]) + ev[2][e >> 2];
                    d345[e] = (ev[3][e & 1] + ev[4][(e >> 1) & 1]) + ev[5][e >> 2];
                }
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    float part = 0.f;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int e = g * 16 + i;
                        bool in = true;
#pragma unroll
                        for (int j = 0; j < 6; ++j) in &= ((ok[j] >> ((e >> j) & 1)) & 1) != 0;
                        const float te = __uint_as_float((uint32_t)((e & 1) ? acc[e >> 1] >> 32 : acc[e >> 1]));
                        const float v = te * te / (d012[e & 7] + d345[e >> 3]);
                        part += in ? v : 0.f;
                    }
                    e_acc += (double)part;
                }
            }
        }
    }
    if (have) flush(b);
}

}  // namespace comet

using namespace comet;

extern "C" {

comet_status_t comet_plan_triples(const char *const *terms, int n_terms, const char *const *label_names,
                                  int n_labels, int n_blocks, const int64_t *extents, const int *signs,
                                  comet_dtype_t dtype, comet_plan_t *out_plan) {
    if (!out_plan) return COMET_ERR_NULL;
    *out_plan = nullptr;
    comet_plan_s *h = new (std::nothrow) comet_plan_s;
    if (!h) return COMET_ERR_INTERNAL;
    std::string err;
    comet_status_t st;
    try {
        st = plan_triples(terms, n_terms, label_names, n_labels, n_blocks, extents, signs, dtype, &h->p, &err);
    } catch (...) {
        st = COMET_ERR_INTERNAL;
        err = "exception while planning";
    }
    if (st != COMET_OK) {
        set_error_message(err);
        delete h;
        return st;
    }
    *out_plan = h;
    return COMET_OK;
}

comet_status_t comet_triples_prepare(comet_plan_t plan, void *workspace, void *stream) {
    if (!plan || !workspace) return COMET_ERR_NULL;
    const Plan &P = plan->p;
    if (!P.triples) { set_error_message("not a triples plan"); return COMET_ERR_ARG; }
    if ((reinterpret_cast<uintptr_t>(workspace) & 15u) != 0) return COMET_ERR_ALIGN;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(workspace);
    cudaError_t e = cudaMemcpyAsync(w + P.tri.ws_ext, P.tri.ext.data(), P.tri.ext.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + P.tri.ws_prefix, P.tri.prefix.data(), P.tri.prefix.size() * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !P.tri.tc_batch.empty())
        e = cudaMemcpyAsync(w + P.tri.ws_tc_prefix, P.tri.tc_prefix.data(), P.tri.tc_prefix.size() * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !P.tri.tc_batch.empty())
        e = cudaMemcpyAsync(w + P.tri.ws_tc_row0, P.tri.tc_row0.data(), P.tri.tc_row0.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !P.tri.tc_batch.empty())
        e = cudaMemcpyAsync(w + P.tri.ws_tc_rec, P.tri.tc_rec.data(), P.tri.tc_rec.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host tables may go away after the call
    if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return COMET_ERR_CUDA; }
    return COMET_OK;
}

comet_status_t comet_triples_energy(comet_plan_t plan, const void *operands, const void *eps, double *energies,
                                    void *workspace, void *stream) {
    if (!plan || !operands || !eps || !energies || !workspace) return COMET_ERR_NULL;
    const Plan &P = plan->p;
    if (!P.triples) { set_error_message("not a triples plan"); return COMET_ERR_ARG; }
    if ((reinterpret_cast<uintptr_t>(workspace) & 15u) != 0) return COMET_ERR_ALIGN;
    const TriplesPlan &tp = P.tri;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(workspace);
    Args a;
    triples_args(P, &a);
    a.ext = reinterpret_cast<const int32_t *>(w + tp.ws_ext);
    a.prefix = reinterpret_cast<const int64_t *>(w + tp.ws_prefix);
    a.ops = static_cast<const void *const *>(operands);
    a.eps = static_cast<const void *const *>(eps);
    a.energies = energies;
    a.counter = reinterpret_cast<unsigned long long *>(w + tp.ws_counter);
    a.total = tp.prefix.back();
    a.status = device_status_word();
    cudaError_t e = cudaMemsetAsync(energies, 0, sizeof(double) * tp.n_blocks, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.counter, 0, 8, s);
    if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return COMET_ERR_CUDA; }
    if (a.total == 0) return COMET_OK;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>((int64_t)sms * 4, (a.total + CHUNK - 1) / CHUNK);
    int h = prof_begin(PK_TRIPLES_ID, s);
    if (P.dtype == COMET_F32 && !tp.tc_batch.empty()) {
        TcArgs t;
        t.prefix = reinterpret_cast<const int64_t *>(w + tp.ws_tc_prefix);
        t.row0 = reinterpret_cast<const int32_t *>(w + tp.ws_tc_row0);
        t.rec = reinterpret_cast<const TcRec *>(w + tp.ws_tc_rec);
        t.planes = w + tp.ws_tc_planes;
        t.b0 = t.b1 = 0;
        t.item0 = t.n_items = 0;
        t.status = device_status_word();
        // limit of every wait: the plan's, else 2 s; COMET_WAIT_TIMEOUT_MS overrides it (a profiler
        // that replays each kernel many times can stretch a wait past the default)
        int64_t tmo_ms = P.opts.timeout_ms > 0 ? P.opts.timeout_ms : 2000;
        if (const char *env = std::getenv("COMET_WAIT_TIMEOUT_MS")) {
            const long long v = std::atoll(env);
            if (v > 0) tmo_ms = v;
        }
        t.timeout_ns = tmo_ms * 1000000ll;
        // COMET_TRIPLES_DEBUG=1 withholds one ring slot's loads (host-side fault injection: the
        // wait for them runs out and records COMET_ERR_TIMEOUT)
        t.debug_flags = 0;
        if (const char *env = std::getenv("COMET_TRIPLES_DEBUG")) t.debug_flags = std::atoi(env);
        e = t.status ? launch_triples_tc(P, a, t, s) : cudaErrorInvalidValue;
        prof_end(h, s);
        if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return COMET_ERR_CUDA; }
        return COMET_OK;
    } else if (P.dtype == COMET_F32) {
        const int64_t grid32 = std::min<int64_t>((int64_t)sms * CTAS32, (a.total + CHUNK - 1) / CHUNK);
        triples_f32_kernel<<<(unsigned)grid32, NT32, 0, s>>>(a);
    } else {
        triples_kernel<double><<<(unsigned)grid, NT, 0, s>>>(a);
    }
    e = cudaGetLastError();
    prof_end(h, s);
    if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return COMET_ERR_CUDA; }
    return COMET_OK;
}

}  // extern "C"
