// Tiled tensor transpose engine (Section 6, "Transpose optimization": choose the loop order so
// that the innermost indices of input and output are innermost, then tile).
//
// GB300 form: the input's leading (stride-1) dims are fused into U and the output's into V.  A
// CTA stages a 64 x 64 (u, v) tile in shared memory: global reads run along U, global writes
// along V, both as 16-byte vectors where the strides allow.  When input and output share the
// same stride-1 dim ("copy mode") the tile needs no transposition and goes straight through
// registers.  The same engine performs three element operations:
//   OP_MOVE   raw 4/8-byte words (bit-exact permutation, comet_transpose)
//   OP_SCALE  out = alpha * in (+ beta * out)  (ta.copy with alpha)
//   OP_SPLIT  x -> three bfloat16 planes hi, mid, lo (split pre-pass of the split-BF16 GEMM)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "launch.h"
#include "params.h"
#include "split.cuh"

namespace comet {

enum { OP_MOVE = 0, OP_SCALE = 1, OP_SPLIT = 2 };
constexpr int XT = 256;         // threads per CTA

template <int N, typename T>
struct alignas(sizeof(T) * N) Vec {
    T v[N];
};

template <int OP, typename T, int VO>
__device__ __forceinline__ void emit(const XposeParams &p, int64_t off, const T (&x)[VO], int e) {
    if constexpr (OP == OP_MOVE) {
        Vec<VO, T> w;
#pragma unroll
        for (int q = 0; q < VO; ++q) w.v[q] = x[q];
        *reinterpret_cast<Vec<VO, T> *>(reinterpret_cast<T *>(p.out) + off) = w;
    } else if constexpr (OP == OP_SCALE) {
        T *o = reinterpret_cast<T *>(p.out) + off;
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
    } else {
        Vec<VO, __nv_bfloat16> h, m, l;
#pragma unroll
        for (int q = 0; q < VO; ++q) split3<T>(x[q], e, h.v[q], m.v[q], l.v[q]);
        __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(p.out) + off;
        *reinterpret_cast<Vec<VO, __nv_bfloat16> *>(o) = h;
        *reinterpret_cast<Vec<VO, __nv_bfloat16> *>(o + p.out_plane) = m;
        *reinterpret_cast<Vec<VO, __nv_bfloat16> *>(o + 2 * p.out_plane) = l;
    }
}

constexpr int XTAB = 256;        // largest tile extent along U, V or R that uses offset tables

// Transposing mode: tile (u, v, w) of tu x tv x tw.  Loads run along u (input-contiguous),
// stores along v (output-contiguous); the tile sits in shared memory as [w][v][u] with an odd
// row pitch so the column reads of the store phase do not collide in one bank.  Each thread
// keeps one lane position along the contiguous direction and walks rows, so the index work is
// one division per vector.  OFF is int32_t when every offset fits, else int64_t.
template <int OP, typename T, int VI, int VO, typename OFF>
__global__ void __launch_bounds__(XT) xpose_tile_kernel(const XposeParams p) {
    extern __shared__ __align__(16) unsigned char xsm[];
    T *buf = reinterpret_cast<T *>(xsm);
    __shared__ OFF u_in[XTAB], u_out[XTAB], v_in[XTAB], v_out[XTAB], w_in[XTAB], w_out[XTAB];
    const int t = threadIdx.x;
    const uint32_t tu = p.tu, tv = p.tv, tw = p.tw;
    const uint32_t pitch = tu | 1u;
    uint32_t b = blockIdx.x;
    const uint32_t bu = b % p.tiles_u;
    b /= p.tiles_u;
    const uint32_t bv = b % p.tiles_v, bw = b / p.tiles_v;
    const uint32_t u0 = bu * tu, v0 = bv * tv, w0 = bw * tw;
    const uint32_t nu = min(tu, p.u.total - u0), nv = min(tv, p.v.total - v0), nw = min(tw, p.r.total - w0);
    for (uint32_t i = t; i < tu; i += XT) {
        int64_t a = 0, c = 0;
        if (i < nu) radix_offsets(p.u, u0 + i, a, c);
        u_in[i] = (OFF)a; u_out[i] = (OFF)c;
    }
    for (uint32_t i = t; i < tv; i += XT) {
        int64_t a = 0, c = 0;
        if (i < nv) radix_offsets(p.v, v0 + i, a, c);
        v_in[i] = (OFF)a; v_out[i] = (OFF)c;
    }
    for (uint32_t i = t; i < tw; i += XT) {
        int64_t a = 0, c = 0;
        if (i < nw) radix_offsets(p.r, w0 + i, a, c);
        w_in[i] = (OFF)a; w_out[i] = (OFF)c;
    }
    __syncthreads();
    const T *__restrict__ in = reinterpret_cast<const T *>(p.in);
    const int e = (OP == OP_SPLIT) ? scale_exponent<T>(p.scale_bits) : 0;
    // read along u: lanes_l threads per row, each with a fixed u
    {
        const uint32_t lanes = (tu + VI - 1) / VI;
        const uint32_t rpp = XT / lanes;
        const uint32_t r0 = t / lanes;
        const uint32_t u = (t - r0 * lanes) * VI;
        if (r0 < rpp && u < nu) {
            const OFF ui = u_in[u];
            const uint32_t rows = tv * tw;
            // a batch of rows is loaded into registers before any of it is written to shared
            // memory, so the batch's global loads are all in flight together
            constexpr int UB = VI * sizeof(T) >= 16 ? 4 : 8;
            for (uint32_t row0 = r0; row0 < rows; row0 += UB * rpp) {
                Vec<VI, T> x[UB];
                bool ok[UB];
#pragma unroll
                for (int j = 0; j < UB; ++j) {
                    const uint32_t row = row0 + j * rpp;
                    const uint32_t w = fd_div(row, p.fd_tv);
                    const uint32_t v = row - w * tv;
                    ok[j] = row < rows && v < nv && w < nw;
                    if (ok[j]) x[j] = *reinterpret_cast<const Vec<VI, T> *>(in + ((int64_t)w_in[w] + v_in[v] + ui));
                }
#pragma unroll
                for (int j = 0; j < UB; ++j) {
                    if (ok[j]) {
                        T *dst = buf + (row0 + j * rpp) * pitch + u;
#pragma unroll
                        for (int q = 0; q < VI; ++q) dst[q] = x[j].v[q];
                    }
                }
            }
        }
    }
    __syncthreads();
    // write along v: lanes threads per (u, w) row, each with a fixed v
    {
        const uint32_t lanes = (tv + VO - 1) / VO;
        const uint32_t rpp = XT / lanes;
        const uint32_t r0 = t / lanes;
        const uint32_t v = (t - r0 * lanes) * VO;
        if (r0 < rpp && v < nv) {
            const OFF vo = v_out[v];
            const uint32_t rows = tu * tw;
            constexpr int UL = VO * sizeof(T) >= 16 ? 4 : 16;
#pragma unroll UL
            for (uint32_t row = r0; row < rows; row += rpp) {
                const uint32_t w = fd_div(row, p.fd_tu);
                const uint32_t u = row - w * tu;
                if (u < nu && w < nw) {
                    T x[VO];
                    const T *src = buf + (w * tv + v) * pitch + u;
#pragma unroll
                    for (int q = 0; q < VO; ++q) x[q] = src[q * pitch];
                    emit<OP, T, VO>(p, (int64_t)w_out[w] + u_out[u] + vo, x, e);
                }
            }
        }
    }
}

// Copy mode: input and output share the stride-1 dims U, so a tile of tu x tw goes straight
// through registers.  A single fused dim (tu above the table size) is addressed affinely.
template <int OP, typename T, int VW>
__global__ void __launch_bounds__(XT) xpose_copy_kernel(const XposeParams p) {
    __shared__ int64_t u_in[XTAB], u_out[XTAB], w_in[XTAB], w_out[XTAB];
    const int t = threadIdx.x;
    const uint32_t tu = p.tu, tw = p.tw;
    const bool affine = tu > (uint32_t)XTAB;
    const uint32_t bu = blockIdx.x % p.tiles_u, bw = blockIdx.x / p.tiles_u;
    const uint32_t u0 = bu * tu, w0 = bw * tw;
    const uint32_t nu = min(tu, p.u.total - u0), nw = min(tw, p.r.total - w0);
    if (!affine)
        for (uint32_t i = t; i < tu; i += XT) {
            int64_t a = 0, c = 0;
            if (i < nu) radix_offsets(p.u, u0 + i, a, c);
            u_in[i] = a; u_out[i] = c;
        }
    for (uint32_t i = t; i < tw; i += XT) {
        int64_t a = 0, c = 0;
        if (i < nw) radix_offsets(p.r, w0 + i, a, c);
        w_in[i] = a; w_out[i] = c;
    }
    __syncthreads();
    const T *__restrict__ in = reinterpret_cast<const T *>(p.in);
    const int e = (OP == OP_SPLIT) ? scale_exponent<T>(p.scale_bits) : 0;
    const int64_t s_in = p.u.s0[0], s_out = p.u.s1[0];
    const uint32_t n = tu * tw;
    // batches of UB vectors: all loads of a batch are issued before any store, so they are in
    // flight together (the compiler cannot reorder loads from `in` above stores to `out`)
    constexpr int UB = VW * sizeof(T) >= 16 ? 4 : (VW * sizeof(T) >= 8 ? 8 : 16);
    for (uint32_t idx0 = t * VW; idx0 < n; idx0 += UB * XT * VW) {
        Vec<VW, T> x[UB];
        int64_t oo[UB];
        bool ok[UB];
#pragma unroll
        for (int j = 0; j < UB; ++j) {
            const uint32_t idx = idx0 + j * XT * VW;
            const uint32_t w = fd_div(idx, p.fd_tu);
            const uint32_t u = idx - w * tu;
            ok[j] = idx < n && u < nu && w < nw;
            if (ok[j]) {
                const int64_t oi = affine ? (int64_t)(u0 + u) * s_in : (int64_t)u_in[u];
                oo[j] = w_out[w] + (affine ? (int64_t)(u0 + u) * s_out : (int64_t)u_out[u]);
                x[j] = *reinterpret_cast<const Vec<VW, T> *>(in + w_in[w] + oi);
            }
        }
#pragma unroll
        for (int j = 0; j < UB; ++j) {
            if (ok[j]) {
                T xs[VW];
#pragma unroll
                for (int q = 0; q < VW; ++q) xs[q] = x[j].v[q];
                emit<OP, T, VW>(p, oo[j], xs, e);
            }
        }
    }
}

// max |x| over a dense operand: grid-stride 16-byte loads, warp reduction, one atomic per warp
// on the bit pattern (for non-negative IEEE values the bit order is the numeric order)
template <typename T>
__global__ void __launch_bounds__(256) absmax_kernel(const T *__restrict__ x, int64_t n, void *out_bits) {
    constexpr int W = 16 / sizeof(T);
    using U = typename std::conditional<sizeof(T) == 4, unsigned int, unsigned long long>::type;
    T m = 0;
    const int64_t nv = n / W;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += stride) {
        Vec<W, T> w = reinterpret_cast<const Vec<W, T> *>(x)[i];
#pragma unroll
        for (int q = 0; q < W; ++q) m = fmax(m, fabs(w.v[q]));
    }
    for (int64_t i = nv * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        m = fmax(m, fabs(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) {
        U bits;
        memcpy(&bits, &m, sizeof(U));
        atomicMax(reinterpret_cast<U *>(out_bits), bits);
    }
}

cudaError_t launch_absmax(const void *x, int64_t n, int elem_bytes, void *out_bits, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out_bits, 0, 8, s);
    if (e != cudaSuccess || n == 0) return e;
    int blocks = (int)std::min<int64_t>(152 * 8, (n + 256 * 4 - 1) / (256 * 4));
    if (elem_bytes == 4) absmax_kernel<float><<<blocks, 256, 0, s>>>(reinterpret_cast<const float *>(x), n, out_bits);
    else absmax_kernel<double><<<blocks, 256, 0, s>>>(reinterpret_cast<const double *>(x), n, out_bits);
    return cudaGetLastError();
}

static uint32_t xpose_grid(const XposeParams &p) {
    return p.tiles_u * p.tiles_v * p.tiles_w;
}

template <int OP, typename T>
static cudaError_t launch_op(const XposeParams &p, int vi, int vo, cudaStream_t s) {
    const uint32_t g = xpose_grid(p);
    if (g == 0) return cudaSuccess;
    constexpr int W = 16 / sizeof(T);
    if (vo < 0) {   // copy mode
        if (-vo >= W && vi >= W) xpose_copy_kernel<OP, T, W><<<g, XT, 0, s>>>(p);
        else xpose_copy_kernel<OP, T, 1><<<g, XT, 0, s>>>(p);
        return cudaGetLastError();
    }
    const size_t smem = (size_t)p.tw * p.tv * (p.tu | 1u) * sizeof(T);
    auto go = [&](auto kern) {
        static bool set = false;
        if (!set) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
            set = true;
        }
        kern<<<g, XT, smem, s>>>(p);
    };
    if (p.off32) {
        if (vi >= W && vo >= W) go(xpose_tile_kernel<OP, T, W, W, int32_t>);
        else if (vi >= W) go(xpose_tile_kernel<OP, T, W, 1, int32_t>);
        else if (vo >= W) go(xpose_tile_kernel<OP, T, 1, W, int32_t>);
        else go(xpose_tile_kernel<OP, T, 1, 1, int32_t>);
    } else {
        if (vi >= W && vo >= W) go(xpose_tile_kernel<OP, T, W, W, int64_t>);
        else if (vi >= W) go(xpose_tile_kernel<OP, T, W, 1, int64_t>);
        else if (vo >= W) go(xpose_tile_kernel<OP, T, 1, W, int64_t>);
        else go(xpose_tile_kernel<OP, T, 1, 1, int64_t>);
    }
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

}  // namespace comet
