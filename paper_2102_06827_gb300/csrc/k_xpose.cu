// Tiled tensor transpose engine (Section 6, "Transpose optimization": choose the loop order so
// that the innermost indices of input and output are innermost, then tile).
//
// GB300 form: the input's leading (stride-1) dims are fused into U and the output's into V.  A
// CTA stages a 64 x 64 (u, v) tile in shared memory: global reads run along U, global writes
// along V, both as 16-byte vectors where the strides allow (8-byte for an FP32 run of even
// extent).  When input and output share the
// same stride-1 dim ("copy mode") the tile needs no transposition and goes straight through
// registers.  The same engine performs three element operations:
//   OP_MOVE   raw 4/8-byte words (bit-exact permutation, comet_transpose)
//   OP_SCALE  out = alpha * in (+ beta * out)  (ta.copy with alpha)
//   OP_SPLIT  x -> three bfloat16 planes hi, mid, lo (split pre-pass of the split-BF16 GEMM)
//   OP_SPLIT6 FP64 x -> six integer-valued bfloat16 planes (pre-pass of the FP64 emulation)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "launch.h"
#include "params.h"
#include "split.cuh"

namespace comet {

enum { OP_MOVE = 0, OP_SCALE = 1, OP_SPLIT = 2, OP_SPLIT6 = 3 };
constexpr int XT = 256;         // threads per CTA

template <int N, typename T>
struct alignas(sizeof(T) * N) Vec {
    T v[N];
};

template <int OP, typename T, int VO>
__device__ __forceinline__ void emit(const XposeParams &p, int64_t off, const T (&x)[VO], int e) {
#ifdef COMET_DEBUG
    if (p.plant && blockIdx.x == 0 && threadIdx.x == 0) off += p.plant;   // test of the range check
#endif
    if constexpr (OP == OP_MOVE) {
        T *o = reinterpret_cast<T *>(p.out) + off;
        if (!dbg_ok(p.dbg_out, o, VO * (int)sizeof(T), p.status)) return;
        Vec<VO, T> w;
#pragma unroll
        for (int q = 0; q < VO; ++q) w.v[q] = x[q];
        *reinterpret_cast<Vec<VO, T> *>(o) = w;
    } else if constexpr (OP == OP_SCALE) {
        T *o = reinterpret_cast<T *>(p.out) + off;
        if (!dbg_ok(p.dbg_out, o, VO * (int)sizeof(T), p.status)) return;
        Vec<VO, T> w;
        if (p.beta != 0.0) {
            Vec<VO, T> old = *reinterpret_cast<const Vec<VO, T> *>(o);
#pragma unroll
            for (int q = 0; q < VO; ++q) w.v[q] = (T)(p.alpha * (double)x[q] + p.beta * (double)old.v[q]);
        } else {
#pragma unroll
            for (int q = 0; q < VO; ++q) w.v[q] = (T)(p.alpha * (double)x[q]);
        }
        *reinterpret_cast<Vec<VO, T> *>(o) = w;
    } else if constexpr (OP == OP_SPLIT) {
        Vec<VO, __nv_bfloat16> h, m, l;
#pragma unroll
        for (int q = 0; q < VO; ++q) split3<T>(x[q], e, h.v[q], m.v[q], l.v[q]);
        __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(p.out) + off;
        if (!dbg_ok(p.dbg_out, o, 2 * (2 * p.out_plane + VO), p.status)) return;   // all three planes
        *reinterpret_cast<Vec<VO, __nv_bfloat16> *>(o) = h;
        *reinterpret_cast<Vec<VO, __nv_bfloat16> *>(o + p.out_plane) = m;
        *reinterpret_cast<Vec<VO, __nv_bfloat16> *>(o + 2 * p.out_plane) = l;
    } else {
        static_assert(sizeof(T) == 8, "the six-way split is for FP64 operands");
        Vec<VO, __nv_bfloat16> sl[6];
#pragma unroll
        for (int q = 0; q < VO; ++q) {
            __nv_bfloat16 v[6];
            split6((double)x[q], e, v);
#pragma unroll
            for (int k = 0; k < 6; ++k) sl[k].v[q] = v[k];
        }
        __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(p.out) + off;
        if (!dbg_ok(p.dbg_out, o, 2 * (5 * p.out_plane + VO), p.status)) return;   // all six planes
#pragma unroll
        for (int k = 0; k < 6; ++k) *reinterpret_cast<Vec<VO, __nv_bfloat16> *>(o + k * p.out_plane) = sl[k];
    }
}

constexpr int XTAB = 256;        // largest tile extent along U, V or R

template <typename OFF>
struct RowOut {
    OFF o;          // output offset of the row's first element
    int32_t s;      // tile position (shared memory) of the row's first element
};

// Transposing mode: tile (u, v, w) of tu x tv x tw.  U is the input's leading run (affine in
// the input with stride su), V the output's (affine in the output with stride sv), R the rest.
// The block first tabulates the input offset of every (v, w) row and the output offset of every
// (u, w) row of its tile, so the two phases below cost one table read per row and no index
// arithmetic per element.  Loads run along u, each thread keeping one u and walking rows; the
// tile sits in shared memory as rows (v + nv*w) of pitch tu|1 (odd, so that the store phase's
// column reads spread over the banks); stores run along v.  OFF is int32_t when every offset
// fits, else int64_t.
template <int OP, typename T, int VI, int VO, typename OFF>
__global__ void __launch_bounds__(XT, 8) xpose_tile_kernel(const XposeParams p) {
    extern __shared__ __align__(16) unsigned char xsm[];
    __shared__ OFF uo[XTAB], vin[XTAB], win[XTAB], wout[XTAB];
    const int t = threadIdx.x;
    const uint32_t tu = p.tu, tv = p.tv, tw = p.tw;
    const uint32_t pitch = tu | 1u;
    T *buf = reinterpret_cast<T *>(xsm);
    OFF *in_row = reinterpret_cast<OFF *>(xsm + align16(tv * tw * pitch * (uint32_t)sizeof(T)));
    RowOut<OFF> *out_row =
        reinterpret_cast<RowOut<OFF> *>(reinterpret_cast<unsigned char *>(in_row) + align16(tv * tw * (uint32_t)sizeof(OFF)));
    const uint32_t b = fd_div(blockIdx.x, p.fd_tiles_u), bu = blockIdx.x - b * p.tiles_u;
    const uint32_t bw = fd_div(b, p.fd_tiles_v), bv = b - bw * p.tiles_v;
    const uint32_t u0 = bu * tu, v0 = bv * tv, w0 = bw * tw;
    const uint32_t nu = min(tu, p.u.total - u0), nv = min(tv, p.v.total - v0), nw = min(tw, p.r.total - w0);
    const int64_t su = p.u.s0[0], sv = p.v.s1[0];
    for (uint32_t i = t; i < nu; i += XT) {
        int64_t a, c;
        radix_offsets(p.u, u0 + i, a, c);
        uo[i] = (OFF)c;
    }
    for (uint32_t i = t; i < nv; i += XT) {
        int64_t a, c;
        radix_offsets(p.v, v0 + i, a, c);
        vin[i] = (OFF)a;
    }
    for (uint32_t i = t; i < nw; i += XT) {
        int64_t a, c;
        radix_offsets(p.r, w0 + i, a, c);
        win[i] = (OFF)a;
        wout[i] = (OFF)c;
    }
    __syncthreads();
    const uint32_t rows_v = nv * nw, rows_u = nu * nw;
    for (uint32_t r = t; r < rows_v; r += XT) {
        const uint32_t w = nv == tv ? fd_div(r, p.fd_tv) : r / nv, v = r - w * nv;
        in_row[r] = (OFF)((int64_t)u0 * su + vin[v] + win[w]);
    }
    for (uint32_t r = t; r < rows_u; r += XT) {
        const uint32_t w = nu == tu ? fd_div(r, p.fd_tu) : r / nu, u = r - w * nu;
        RowOut<OFF> ro;
        ro.o = (OFF)((int64_t)v0 * sv + uo[u] + wout[w]);
        ro.s = (int32_t)(w * nv * pitch + u);
        out_row[r] = ro;
    }
    __syncthreads();
    const int e = (OP == OP_SPLIT || OP == OP_SPLIT6) ? scale_exponent<T>(p.scale_bits) : 0;
    {   // loads: p.ll threads per row, each with a fixed u; batches of rows in flight together
        const uint32_t lanes = p.ll, rpp = p.rpp_l;
        const uint32_t r0 = fd_div(t, p.fd_ll);
        const uint32_t u = (t - r0 * lanes) * VI;
        if constexpr (VI == 1) {
            // element loads as asynchronous copies straight into the tile: every row of the
            // thread is in flight at once and no register holds the data
            if (r0 < rpp && u < nu) {
                const T *__restrict__ src = reinterpret_cast<const T *>(p.in) + (int64_t)u * su;
                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(buf + u);
                for (uint32_t row = r0; row < rows_v; row += rpp) {
                    const uint32_t d = dst + row * pitch * (uint32_t)sizeof(T);
                    if (!dbg_ok(p.dbg_in, src + in_row[row], (int)sizeof(T), p.status)) continue;
                    if (sizeof(T) == 4)
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src + in_row[row]) : "memory");
                    else
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src + in_row[row]) : "memory");
                }
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
        } else if (r0 < rpp && u < nu) {
            const T *__restrict__ src = reinterpret_cast<const T *>(p.in) + (int64_t)u * su;
            T *dst = buf + u;
            // four vectors per batch keep the kernel within 32 registers, so eight blocks fit on
            // an SM: residency matters more here than loads in flight per thread (measured)
            constexpr int UB = 4;
            for (uint32_t row0 = r0; row0 < rows_v; row0 += UB * rpp) {
                Vec<VI, T> x[UB];
#pragma unroll
                for (int j = 0; j < UB; ++j) {
                    const uint32_t row = row0 + j * rpp;
                    if (row < rows_v && dbg_ok(p.dbg_in, src + in_row[row], VI * (int)sizeof(T), p.status))
                        x[j] = *reinterpret_cast<const Vec<VI, T> *>(src + in_row[row]);
                }
#pragma unroll
                for (int j = 0; j < UB; ++j) {
                    const uint32_t row = row0 + j * rpp;
                    if (row < rows_v) {
                        T *d = dst + row * pitch;
#pragma unroll
                        for (int q = 0; q < VI; ++q) d[q] = x[j].v[q];
                    }
                }
            }
        }
    }
    __syncthreads();
    {   // stores: p.sl threads per row, each with a fixed v
        const uint32_t lanes = p.sl, rpp = p.rpp_s;
        const uint32_t r0 = fd_div(t, p.fd_sl);
        const uint32_t v = (t - r0 * lanes) * VO;
        if (r0 < rpp && v < nv) {
            const T *sb = buf + v * pitch;
            const int64_t vo = (int64_t)v * sv;
            constexpr int UL = VO * sizeof(T) >= 16 ? 4 : 8;
#pragma unroll UL
            for (uint32_t row = r0; row < rows_u; row += rpp) {
                const RowOut<OFF> ro = out_row[row];
                T x[VO];
#pragma unroll
                for (int q = 0; q < VO; ++q) x[q] = sb[ro.s + q * pitch];
                emit<OP, T, VO>(p, (int64_t)ro.o + vo, x, e);
            }
        }
    }
}

// Copy mode: input and output share the stride-1 dim U (a single digit, affine on both sides
// with strides su, so), so a tile of tu x tw goes straight through registers.  Rows (the R
// digits) are tabulated per block; each thread keeps one u and walks rows.
template <int OP, typename T, int VW, typename OFF>
__global__ void __launch_bounds__(XT, 6) xpose_copy_kernel(const XposeParams p) {
    __shared__ OFF row_in[XTAB], row_out[XTAB];
    const int t = threadIdx.x;
    const uint32_t tu = p.tu, tw = p.tw;
    const uint32_t bw = fd_div(blockIdx.x, p.fd_tiles_u), bu = blockIdx.x - bw * p.tiles_u;
    const uint32_t u0 = bu * tu, w0 = bw * tw;
    const uint32_t nu = min(tu, p.u.total - u0), nw = min(tw, p.r.total - w0);
    const int64_t su = p.u.s0[0], so = p.u.s1[0];
    for (uint32_t i = t; i < nw; i += XT) {
        int64_t a, c;
        radix_offsets(p.r, w0 + i, a, c);
        row_in[i] = (OFF)(a + (int64_t)u0 * su);
        row_out[i] = (OFF)(c + (int64_t)u0 * so);
    }
    __syncthreads();
    const T *__restrict__ in = reinterpret_cast<const T *>(p.in);
    const int e = (OP == OP_SPLIT || OP == OP_SPLIT6) ? scale_exponent<T>(p.scale_bits) : 0;
    constexpr int UB = VW * sizeof(T) >= 16 ? 4 : 8;
    const uint32_t lanes = p.ll;
    const uint32_t rpp = p.rpp_l;
    const uint32_t r0 = fd_div(t, p.fd_ll);
    const uint32_t u = (t - r0 * lanes) * VW;
    if (!(r0 < rpp && u < nu)) return;
    const T *__restrict__ src = in + (int64_t)u * su;
    const int64_t uo = (int64_t)u * so;
    if constexpr (VW * sizeof(T) <= 8) {
        // element-wise (or 8-byte FP32) rows: every load of the thread goes out at once as an
        // asynchronous copy into its own slots of the tile (no register holds the data), then
        // the thread stores what it copied; no other thread reads these slots, so no block
        // barrier is needed
        extern __shared__ __align__(16) unsigned char csm[];
        T *stage = reinterpret_cast<T *>(csm);
        const uint32_t base = (uint32_t)__cvta_generic_to_shared(stage + u);
        constexpr int VB = VW * (int)sizeof(T);
        for (uint32_t row = r0; row < nw; row += rpp) {
            const uint32_t d = base + row * tu * (uint32_t)sizeof(T);
            if (!dbg_ok(p.dbg_in, src + row_in[row], VB, p.status)) continue;
            if (VB == 4)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src + row_in[row]) : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src + row_in[row]) : "memory");
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
#pragma unroll 4
        for (uint32_t row = r0; row < nw; row += rpp) {
            const Vec<VW, T> w = *reinterpret_cast<const Vec<VW, T> *>(stage + row * tu + u);
            T xs[VW];
#pragma unroll
            for (int q = 0; q < VW; ++q) xs[q] = w.v[q];
            emit<OP, T, VW>(p, (int64_t)row_out[row] + uo, xs, e);
        }
    } else {
        // rows r0, r0 + rpp, ...: a ring of UB loads stays in flight; each store is followed by
        // the load of the row UB passes ahead into the register it freed
        Vec<VW, T> x[UB];
#pragma unroll
        for (int j = 0; j < UB; ++j) {
            const uint32_t row = r0 + j * rpp;
            if (row < nw && dbg_ok(p.dbg_in, src + row_in[row], VW * (int)sizeof(T), p.status))
                x[j] = *reinterpret_cast<const Vec<VW, T> *>(src + row_in[row]);
        }
        for (uint32_t row0 = r0; row0 < nw; row0 += UB * rpp) {
#pragma unroll
            for (int j = 0; j < UB; ++j) {
                const uint32_t row = row0 + j * rpp;
                if (row < nw) {
                    T xs[VW];
#pragma unroll
                    for (int q = 0; q < VW; ++q) xs[q] = x[j].v[q];
                    emit<OP, T, VW>(p, (int64_t)row_out[row] + uo, xs, e);
                    const uint32_t nr = row + UB * rpp;
                    if (nr < nw && dbg_ok(p.dbg_in, src + row_in[nr], VW * (int)sizeof(T), p.status))
                        x[j] = *reinterpret_cast<const Vec<VW, T> *>(src + row_in[nr]);
                }
            }
        }
    }
}

// A single long run (copy mode, R empty), cut into pieces of up to kXposeTile elements: every
// thread strides along u with 16-byte vectors; the ragged tail moves element-wise.
template <int OP, typename T, int VW>
__global__ void __launch_bounds__(XT) xpose_run_kernel(const XposeParams p) {
    const int t = threadIdx.x;
    const uint32_t tu = p.tu;
    const uint32_t u0 = blockIdx.x * tu;
    const uint32_t nu = min(tu, p.u.total - u0);
    const int64_t su = p.u.s0[0], so = p.u.s1[0];
    const T *__restrict__ in = reinterpret_cast<const T *>(p.in);
    const int e = (OP == OP_SPLIT || OP == OP_SPLIT6) ? scale_exponent<T>(p.scale_bits) : 0;
    constexpr int UB = VW * sizeof(T) >= 16 ? 4 : 8;
    const int64_t ri = (int64_t)u0 * su, ro = (int64_t)u0 * so;
    const uint32_t nvec = nu / VW * VW;
    for (uint32_t u00 = t * VW; u00 < nvec; u00 += UB * XT * VW) {
        Vec<VW, T> x[UB];
#pragma unroll
        for (int j = 0; j < UB; ++j) {
            const uint32_t u = u00 + j * XT * VW;
            if (u < nvec && dbg_ok(p.dbg_in, in + ri + (int64_t)u * su, VW * (int)sizeof(T), p.status))
                x[j] = *reinterpret_cast<const Vec<VW, T> *>(in + ri + (int64_t)u * su);
        }
#pragma unroll
        for (int j = 0; j < UB; ++j) {
            const uint32_t u = u00 + j * XT * VW;
            if (u < nvec) {
                T xs[VW];
#pragma unroll
                for (int q = 0; q < VW; ++q) xs[q] = x[j].v[q];
                emit<OP, T, VW>(p, ro + (int64_t)u * so, xs, e);
            }
        }
    }
    if (t < (int)(nu - nvec)) {
        const uint32_t u = nvec + t;
        if (!dbg_ok(p.dbg_in, in + ri + (int64_t)u * su, (int)sizeof(T), p.status)) return;
        T xs[1] = {in[ri + (int64_t)u * su]};
        emit<OP, T, 1>(p, ro + (int64_t)u * so, xs, e);
    }
}

// every element of a dense buffer set to one value: grid-stride 16-byte stores, element tail
template <typename T>
__global__ void __launch_bounds__(256) fill_kernel(T *out, int64_t n, T value) {
    constexpr int W = 16 / sizeof(T);
    Vec<W, T> v;
#pragma unroll
    for (int q = 0; q < W; ++q) v.v[q] = value;
    const int64_t nv = n / W, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += stride)
        reinterpret_cast<Vec<W, T> *>(out)[i] = v;
    for (int64_t i = nv * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) out[i] = value;
}

cudaError_t launch_fill(void *out, int64_t n, double value, int elem_bytes, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>(152 * 8, (n + 256 * 4 - 1) / (256 * 4));
    if (elem_bytes == 4) fill_kernel<float><<<blocks, 256, 0, s>>>(reinterpret_cast<float *>(out), n, (float)value);
    else fill_kernel<double><<<blocks, 256, 0, s>>>(reinterpret_cast<double *>(out), n, value);
    return cudaGetLastError();
}

// max |x| over a dense operand: grid-stride 16-byte loads, warp reduction, one atomic per warp
// on the bit pattern (for non-negative IEEE values the bit order is the numeric order).  `bid`
// and `nb` are this block's index and the block count among the blocks given to the operand.
template <typename T>
__device__ __forceinline__ void absmax_body(const T *__restrict__ x, int64_t n, int64_t bid, int64_t nb,
                                            void *out_bits) {
    constexpr int W = 16 / sizeof(T);
    using U = typename std::conditional<sizeof(T) == 4, unsigned int, unsigned long long>::type;
    T m = 0;
    const int64_t nv = n / W;
    const int64_t stride = nb * blockDim.x;
    for (int64_t i = bid * (int64_t)blockDim.x + threadIdx.x; i < nv; i += stride) {
        Vec<W, T> w = reinterpret_cast<const Vec<W, T> *>(x)[i];
#pragma unroll
        for (int q = 0; q < W; ++q) m = fmax(m, fabs(w.v[q]));
    }
    for (int64_t i = nv * W + bid * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        m = fmax(m, fabs(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) {
        U bits;
        memcpy(&bits, &m, sizeof(U));
        atomicMax(reinterpret_cast<U *>(out_bits), bits);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) absmax_kernel(const T *__restrict__ x, int64_t n, void *out_bits) {
    absmax_body(x, n, blockIdx.x, gridDim.x, out_bits);
}

// both operands of a split step in one launch: blocks [0, blocks0) take x0 (word 0 of out_bits),
// the rest x1 (word 1, 8 bytes further)
template <typename T>
__global__ void __launch_bounds__(256) absmax2_kernel(const T *__restrict__ x0, int64_t n0, const T *__restrict__ x1,
                                                      int64_t n1, int blocks0, void *out_bits) {
    if ((int)blockIdx.x < blocks0) absmax_body(x0, n0, blockIdx.x, blocks0, out_bits);
    else absmax_body(x1, n1, blockIdx.x - blocks0, gridDim.x - blocks0, static_cast<char *>(out_bits) + 8);
}

static int absmax_blocks(int64_t n) { return (int)std::min<int64_t>(152 * 8, (n + 256 * 4 - 1) / (256 * 4)); }

cudaError_t launch_absmax(const void *x, int64_t n, int elem_bytes, void *out_bits, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out_bits, 0, 8, s);
    if (e != cudaSuccess || n == 0) return e;
    const int blocks = absmax_blocks(n);
    if (elem_bytes == 4) absmax_kernel<float><<<blocks, 256, 0, s>>>(reinterpret_cast<const float *>(x), n, out_bits);
    else absmax_kernel<double><<<blocks, 256, 0, s>>>(reinterpret_cast<const double *>(x), n, out_bits);
    return cudaGetLastError();
}

cudaError_t launch_absmax2(const void *x0, int64_t n0, const void *x1, int64_t n1, int elem_bytes, void *out_bits,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out_bits, 0, 16, s);
    const int b0 = absmax_blocks(n0), b1 = absmax_blocks(n1);
    if (e != cudaSuccess || b0 + b1 == 0) return e;
    if (elem_bytes == 4)
        absmax2_kernel<float><<<b0 + b1, 256, 0, s>>>(reinterpret_cast<const float *>(x0), n0,
                                                      reinterpret_cast<const float *>(x1), n1, b0, out_bits);
    else
        absmax2_kernel<double><<<b0 + b1, 256, 0, s>>>(reinterpret_cast<const double *>(x0), n0,
                                                       reinterpret_cast<const double *>(x1), n1, b0, out_bits);
    return cudaGetLastError();
}

// max |x| over a strided view: each thread walks elements through the radix (smallest stride
// first, so neighbouring threads touch neighbouring addresses where the view allows)
template <typename T>
__global__ void __launch_bounds__(256) absmax_view_kernel(const T *__restrict__ x, const Radix r, void *out_bits) {
    using U = typename std::conditional<sizeof(T) == 4, unsigned int, unsigned long long>::type;
    T m = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < r.total; i += gridDim.x * blockDim.x) {
        int64_t o0 = 0, o1 = 0;
        radix_offsets(r, i, o0, o1);
        m = fmax(m, fabs(x[o0]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) {
        U bits;
        memcpy(&bits, &m, sizeof(U));
        atomicMax(reinterpret_cast<U *>(out_bits), bits);
    }
}

cudaError_t launch_absmax_view(const void *x, const Radix &r, int elem_bytes, void *out_bits, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out_bits, 0, 8, s);
    if (e != cudaSuccess || r.total == 0) return e;
    int blocks = (int)std::min<int64_t>(152 * 8, ((int64_t)r.total + 255) / 256);
    if (elem_bytes == 4) absmax_view_kernel<float><<<blocks, 256, 0, s>>>(reinterpret_cast<const float *>(x), r, out_bits);
    else absmax_view_kernel<double><<<blocks, 256, 0, s>>>(reinterpret_cast<const double *>(x), r, out_bits);
    return cudaGetLastError();
}

static uint32_t xpose_grid(const XposeParams &p) {
    return p.tiles_u * p.tiles_v * p.tiles_w;
}

// the shared-memory attribute is set once per kernel instantiation
template <int OP, typename T, int VI, int VO, typename OFF>
static void launch_tile(const XposeParams &p, uint32_t g, size_t smem, cudaStream_t s) {
    static const bool attr = [] {
        cudaFuncSetAttribute(xpose_tile_kernel<OP, T, VI, VO, OFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        return true;
    }();
    (void)attr;
    xpose_tile_kernel<OP, T, VI, VO, OFF><<<g, XT, smem, s>>>(p);
}

// vector widths W (16 bytes), 2 (8 bytes, FP32 only) and 1, chosen at run time
template <int OP, typename T, int VI, typename OFF>
static void launch_tile_vo(const XposeParams &p, int vo, uint32_t g, size_t smem, cudaStream_t s) {
    constexpr int W = 16 / sizeof(T), H = W == 4 ? 2 : 1;
    if (vo >= W) launch_tile<OP, T, VI, W, OFF>(p, g, smem, s);
    else if (W == 4 && vo == 2) launch_tile<OP, T, VI, H, OFF>(p, g, smem, s);
    else launch_tile<OP, T, VI, 1, OFF>(p, g, smem, s);
}

template <int OP, typename T, typename OFF>
static void launch_tile_v(const XposeParams &p, int vi, int vo, uint32_t g, size_t smem, cudaStream_t s) {
    constexpr int W = 16 / sizeof(T), H = W == 4 ? 2 : 1;
    if (vi >= W) launch_tile_vo<OP, T, W, OFF>(p, vo, g, smem, s);
    else if (W == 4 && vi == 2) launch_tile_vo<OP, T, H, OFF>(p, vo, g, smem, s);
    else launch_tile_vo<OP, T, 1, OFF>(p, vo, g, smem, s);
}

template <int OP, typename T>
static cudaError_t launch_op(const XposeParams &p, int vi, int vo, cudaStream_t s) {
    const uint32_t g = xpose_grid(p);
    if (g == 0) return cudaSuccess;
    constexpr int W = 16 / sizeof(T);
    if (vo < 0) {   // copy mode
        const bool wide = -vo >= W && vi >= W;
        if (p.single_run) {
            if (wide) xpose_run_kernel<OP, T, W><<<g, XT, 0, s>>>(p);
            else xpose_run_kernel<OP, T, 1><<<g, XT, 0, s>>>(p);
            return cudaGetLastError();
        }
        const size_t stage = (size_t)p.tu * p.tw * sizeof(T);   // asynchronous rows stage in shared memory
        const bool half = W == 4 && -vo >= 2 && vi >= 2;        // FP32 rows in 8-byte pieces
        if (p.off32) {
            if (wide) xpose_copy_kernel<OP, T, W, int32_t><<<g, XT, 0, s>>>(p);
            else if (half) xpose_copy_kernel<OP, T, (W == 4 ? 2 : 1), int32_t><<<g, XT, stage, s>>>(p);
            else xpose_copy_kernel<OP, T, 1, int32_t><<<g, XT, stage, s>>>(p);
        } else {
            if (wide) xpose_copy_kernel<OP, T, W, int64_t><<<g, XT, 0, s>>>(p);
            else if (half) xpose_copy_kernel<OP, T, (W == 4 ? 2 : 1), int64_t><<<g, XT, stage, s>>>(p);
            else xpose_copy_kernel<OP, T, 1, int64_t><<<g, XT, stage, s>>>(p);
        }
        return cudaGetLastError();
    }
    const size_t smem = xpose_smem_bytes(p, (int)sizeof(T));
    if (smem > 96 * 1024) return cudaErrorInvalidConfiguration;
    if (p.off32) launch_tile_v<OP, T, int32_t>(p, vi, vo, g, smem, s);
    else launch_tile_v<OP, T, int64_t>(p, vi, vo, g, smem, s);
    return cudaGetLastError();
}

cudaError_t launch_move(const XposeParams &p, int elem_bytes, int vi, int vo, cudaStream_t s) {
    if (elem_bytes == 4) return launch_op<OP_MOVE, uint32_t>(p, vi, vo, s);
    return launch_op<OP_MOVE, unsigned long long>(p, vi, vo, s);
}

cudaError_t launch_scale(const XposeParams &p, int elem_bytes, int vi, int vo, cudaStream_t s) {
    if (elem_bytes == 4) return launch_op<OP_SCALE, float>(p, vi, vo, s);
    return launch_op<OP_SCALE, double>(p, vi, vo, s);
}

// The split pre-pass writes bfloat16 planes; its store vectors hold as many bf16 as the input
// vector holds input elements (4 for FP32, 2 for FP64), which keeps every plane's stores
// aligned whenever the input-width condition holds for the output strides and the plane stride.
cudaError_t launch_split(const XposeParams &p, int elem_bytes, int vi, int vo, cudaStream_t s) {
    if (elem_bytes == 4) return launch_op<OP_SPLIT, float>(p, vi, vo, s);
    return launch_op<OP_SPLIT, double>(p, vi, vo, s);
}

// FP64-emulation pre-pass: six integer-valued bfloat16 planes of an FP64 operand
cudaError_t launch_split6(const XposeParams &p, int elem_bytes, int vi, int vo, cudaStream_t s) {
    if (elem_bytes != 8) return cudaErrorInvalidValue;
    return launch_op<OP_SPLIT6, double>(p, vi, vo, s);
}

}  // namespace comet
