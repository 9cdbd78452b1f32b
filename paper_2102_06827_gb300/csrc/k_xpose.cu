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

namespace comet {

enum { OP_MOVE = 0, OP_SCALE = 1, OP_SPLIT = 2 };
constexpr int TT = 64;          // tile edge (elements)
constexpr int XT = 256;         // threads per CTA

template <int N, typename T>
struct alignas(sizeof(T) * N) Vec {
    T v[N];
};

// Fixed-point three-way split.  The operand is first scaled by 2^-e (e = exponent of its
// largest magnitude, so |x'| < 2); then hi, mid and lo are x' rounded to nearest on the grids
// 2^-6, 2^-14 and 2^-22.  Each part is an integer of magnitude <= 128 times its grid step, so
// it is exact in bfloat16, and a product of two hi parts is an integer multiple of 2^-12 of
// magnitude <= 2^14: up to 1024 of them sum exactly in FP32 whatever the accumulator's
// rounding.  The residuals are exact in the input precision; what remains after lo is below
// 2^-23 of the operand's largest magnitude.
template <typename T>
__device__ __forceinline__ void split3(T x, int e, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
    if constexpr (sizeof(T) == 4) {
        const float xs = ldexpf(x, -e);
        const float fh = rintf(xs * 64.0f) * (1.0f / 64.0f);
        const float r1 = xs - fh;
        const float fm = rintf(r1 * 16384.0f) * (1.0f / 16384.0f);
        const float r2 = r1 - fm;
        const float fl = rintf(r2 * 4194304.0f) * (1.0f / 4194304.0f);
        h = __float2bfloat16_rn(fh);
        m = __float2bfloat16_rn(fm);
        l = __float2bfloat16_rn(fl);
    } else {
        const double xs = ldexp(x, -e);
        const double fh = rint(xs * 64.0) * (1.0 / 64.0);
        const double r1 = xs - fh;
        const double fm = rint(r1 * 16384.0) * (1.0 / 16384.0);
        const double r2 = r1 - fm;
        const double fl = rint(r2 * 4194304.0) * (1.0 / 4194304.0);
        h = __float2bfloat16_rn((float)fh);
        m = __float2bfloat16_rn((float)fm);
        l = __float2bfloat16_rn((float)fl);
    }
}

// exponent e with max|x| in [2^e, 2^(e+1)) from the abs-max bits; 0 for an all-zero (or
// non-finite) operand
template <typename T>
__device__ __forceinline__ int scale_exponent(const void *absmax_bits) {
    if constexpr (sizeof(T) == 4) {
        const float m = __uint_as_float(*reinterpret_cast<const volatile unsigned int *>(absmax_bits));
        if (!(m > 0.0f) || isinf(m)) return 0;
        int e;
        frexpf(m, &e);
        return e - 1;
    } else {
        const double m = __longlong_as_double(
            (long long)*reinterpret_cast<const volatile unsigned long long *>(absmax_bits));
        if (!(m > 0.0) || isinf(m)) return 0;
        int e;
        frexp(m, &e);
        return e - 1;
    }
}

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

template <int OP, typename T, int VI, int VO>
__global__ void __launch_bounds__(XT) xpose_tile_kernel(const XposeParams p) {
    __shared__ T tile[TT][TT + 1];
    __shared__ int64_t u_in[TT], u_out[TT], v_in[TT], v_out[TT];
    const int t = threadIdx.x;
    uint32_t tiles = p.tiles_u * p.tiles_v;
    uint32_t bt = blockIdx.x % tiles;
    uint32_t rc = blockIdx.x / tiles;
    uint32_t u0 = (bt % p.tiles_u) * TT, v0 = (bt / p.tiles_u) * TT;
    if (t < TT) {
        int64_t a = 0, b = 0;
        if (u0 + t < p.u.total) radix_offsets(p.u, u0 + t, a, b);
        u_in[t] = a; u_out[t] = b;
    } else if (t < 2 * TT) {
        int64_t a = 0, b = 0;
        if (v0 + t - TT < p.v.total) radix_offsets(p.v, v0 + t - TT, a, b);
        v_in[t - TT] = a; v_out[t - TT] = b;
    }
    __syncthreads();
    const T *in = reinterpret_cast<const T *>(p.in);
    const int e = (OP == OP_SPLIT) ? scale_exponent<T>(p.scale_bits) : 0;
    uint32_t r_begin = rc * p.r_per_cta;
    uint32_t r_end = min(p.r.total, r_begin + p.r_per_cta);
    for (uint32_t r = r_begin; r < r_end; ++r) {
        int64_t r_in, r_out;
        radix_offsets(p.r, r, r_in, r_out);
        // read along U (input-contiguous)
#pragma unroll 4
        for (int idx = t; idx < TT * TT / VI; idx += XT) {
            int vr = idx / (TT / VI), uc = (idx % (TT / VI)) * VI;
            if (v0 + vr < p.v.total && u0 + uc < p.u.total) {
                Vec<VI, T> w = *reinterpret_cast<const Vec<VI, T> *>(in + r_in + v_in[vr] + u_in[uc]);
#pragma unroll
                for (int q = 0; q < VI; ++q) tile[vr][uc + q] = w.v[q];
            }
        }
        __syncthreads();
        // write along V (output-contiguous)
#pragma unroll 4
        for (int idx = t; idx < TT * TT / VO; idx += XT) {
            int ur = idx / (TT / VO), vc = (idx % (TT / VO)) * VO;
            if (u0 + ur < p.u.total && v0 + vc < p.v.total) {
                T x[VO];
#pragma unroll
                for (int q = 0; q < VO; ++q) x[q] = tile[vc + q][ur];
                emit<OP, T, VO>(p, r_out + u_out[ur] + v_out[vc], x, e);
            }
        }
        __syncthreads();
    }
}

// copy mode: input and output share the stride-1 dim U; V is a second dim for more rows
template <int OP, typename T, int VW>
__global__ void __launch_bounds__(XT) xpose_copy_kernel(const XposeParams p) {
    __shared__ int64_t u_in[TT], u_out[TT], v_in[TT], v_out[TT];
    const int t = threadIdx.x;
    uint32_t tiles = p.tiles_u * p.tiles_v;
    uint32_t bt = blockIdx.x % tiles;
    uint32_t rc = blockIdx.x / tiles;
    uint32_t u0 = (bt % p.tiles_u) * TT, v0 = (bt / p.tiles_u) * TT;
    if (t < TT) {
        int64_t a = 0, b = 0;
        if (u0 + t < p.u.total) radix_offsets(p.u, u0 + t, a, b);
        u_in[t] = a; u_out[t] = b;
    } else if (t < 2 * TT) {
        int64_t a = 0, b = 0;
        if (v0 + t - TT < p.v.total) radix_offsets(p.v, v0 + t - TT, a, b);
        v_in[t - TT] = a; v_out[t - TT] = b;
    }
    __syncthreads();
    const T *in = reinterpret_cast<const T *>(p.in);
    const int e = (OP == OP_SPLIT) ? scale_exponent<T>(p.scale_bits) : 0;
    uint32_t r_begin = rc * p.r_per_cta;
    uint32_t r_end = min(p.r.total, r_begin + p.r_per_cta);
    for (uint32_t r = r_begin; r < r_end; ++r) {
        int64_t r_in, r_out;
        radix_offsets(p.r, r, r_in, r_out);
#pragma unroll 4
        for (int idx = t; idx < TT * TT / VW; idx += XT) {
            int vr = idx / (TT / VW), uc = (idx % (TT / VW)) * VW;
            if (v0 + vr < p.v.total && u0 + uc < p.u.total) {
                Vec<VW, T> w = *reinterpret_cast<const Vec<VW, T> *>(in + r_in + v_in[vr] + u_in[uc]);
                T x[VW];
#pragma unroll
                for (int q = 0; q < VW; ++q) x[q] = w.v[q];
                emit<OP, T, VW>(p, r_out + v_out[vr] + u_out[uc], x, e);
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
    uint64_t tiles = (uint64_t)p.tiles_u * p.tiles_v;
    uint64_t rch = (p.r.total + p.r_per_cta - 1) / p.r_per_cta;
    return (uint32_t)(tiles * rch);
}

template <int OP, typename T>
static cudaError_t launch_op(const XposeParams &p, int vi, int vo, cudaStream_t s) {
    uint32_t g = xpose_grid(p);
    if (g == 0) return cudaSuccess;
    constexpr int W = 16 / sizeof(T);
    if (vo < 0) {   // copy mode
        if (-vo >= W && vi >= W) xpose_copy_kernel<OP, T, W><<<g, XT, 0, s>>>(p);
        else xpose_copy_kernel<OP, T, 1><<<g, XT, 0, s>>>(p);
    } else if (vi >= W && vo >= W) {
        xpose_tile_kernel<OP, T, W, W><<<g, XT, 0, s>>>(p);
    } else if (vi >= W) {
        xpose_tile_kernel<OP, T, W, 1><<<g, XT, 0, s>>>(p);
    } else if (vo >= W) {
        xpose_tile_kernel<OP, T, 1, W><<<g, XT, 0, s>>>(p);
    } else {
        xpose_tile_kernel<OP, T, 1, 1><<<g, XT, 0, s>>>(p);
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
