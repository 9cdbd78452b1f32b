// Tensor-times-vector steps: a binary contraction in which one operand has no free label (all its
// labels are contracted; Section 2's TTGT then degenerates to a matrix-vector product, M = 1 or
// N = 1).  Such a step reads its large operand once and does two flops per element, so it is
// bound by HBM, not by the tensor cores: a tiled tensor-core GEMM would waste all but one row
// of each 128-row tile and would first write split planes of the large operand.
//
//   y[b, n] = alpha * sum_k v[b, k] * X[b, k, n]  (+ beta * y[b, n]),  b over the batch labels
//
// Stage 1: blocks over (n tile, K chunk of 1024) read X in its own memory order -- threads along
// n when X's stride-1 dim is a free label, along k (with a warp reduction per n) when it is a
// contracted one -- and write one partial sum per (chunk, n) in FP64.  FP32 operands use the
// compensated dot product of Ogita, Rump and Oishi (Dot2: TwoProduct by FMA, TwoSum), so the
// chunk sum is as accurate as if computed in twice the working precision; FP64 operands use
// FMA.  Stage 2 adds the chunk partials in FP64 and writes y through the output strides.  With
// v all ones the same kernels sum labels that occur in a single operand (a reduction).
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"
#include "params.h"

namespace comet {

namespace gv {
constexpr int T = 256;
constexpr int KC = 1024;     // k values per chunk
constexpr int NT_N = 128;    // n per block when X is n-contiguous (2 k phases of 128 threads)
constexpr int NT_K = 64;     // n per block when X is k-contiguous (8 warps x 8 n)
}  // namespace gv

template <typename T>
struct Acc;
template <>
struct Acc<float> {   // compensated FP32 sum (Dot2)
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x, float y) {
        const float p = x * y;
        const float e = fmaf(x, y, -p);           // x*y = p + e exactly
        const float t = s + p;
        const float z = t - s;
        const float err = (s - (t - z)) + (p - z);   // s + p = t + err exactly
        s = t;
        c += e + err;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x, double y) { s = fma(x, y, s); }
    __device__ __forceinline__ double value() const { return s; }
};

template <typename T, bool NFAST>
__global__ void __launch_bounds__(gv::T) gemv_partial_kernel(const GemvParams p) {
    using namespace gv;
    __shared__ int64_t k_off[KC];
    __shared__ T vk[KC];
    __shared__ int64_t n_off[NFAST ? NT_N : NT_K];
    __shared__ double red[NFAST ? NT_N : 1];
    const int t = threadIdx.x;
    constexpr int NT = NFAST ? NT_N : NT_K;
    const uint32_t tiles = (p.N + NT - 1) / NT;
    const uint32_t bi = blockIdx.x / tiles, n0 = (blockIdx.x - bi * tiles) * NT, k0 = blockIdx.y * KC;
    const uint32_t nk = min((uint32_t)KC, p.K - k0), nn = min((uint32_t)NT, p.N - n0);
    int64_t bo_v = 0, bo_x = 0;
    radix_offsets(p.bv, bi, bo_v, bo_x);
    const T *v = reinterpret_cast<const T *>(p.v) + bo_v;
    const T *X = reinterpret_cast<const T *>(p.X) + bo_x;
    for (uint32_t i = t; i < (uint32_t)KC; i += gv::T) {
        int64_t ov = 0, ox = 0;
        if (i < nk) radix_offsets(p.k, k0 + i, ov, ox);
        k_off[i] = ox;
        vk[i] = i < nk ? (p.v_ones ? (T)1 : dbg_ok(p.dbg_v, v + ov, (int)sizeof(T), p.status) ? v[ov] : (T)0) : (T)0;
    }
    for (uint32_t i = t; i < (uint32_t)NT; i += gv::T) {
        int64_t ox = 0, oy = 0;
        if (i < nn) radix_offsets(p.n, n0 + i, ox, oy);
        n_off[i] = ox;
    }
    __syncthreads();
    double *out = p.partial + ((size_t)bi * p.nchunks + blockIdx.y) * p.N;
    if (NFAST) {
        // threads along n (contiguous in X), two k phases
        const int tn = t % NT_N, tk = t / NT_N;
        Acc<T> a;
        if ((uint32_t)tn < nn) {
            const T *x = X + n_off[tn];
#pragma unroll 8
            for (uint32_t k = tk; k < nk; k += 2)
                a.add(vk[k], dbg_ok(p.dbg_x, x + k_off[k], (int)sizeof(T), p.status) ? x[k_off[k]] : (T)0);
        }
        if (tk == 1) red[tn] = a.value();
        __syncthreads();
        if (tk == 0 && (uint32_t)tn < nn && dbg_ok(p.dbg_p, out + n0 + tn, 8, p.status))
            out[n0 + tn] = a.value() + red[tn];
    } else {
        // lanes along k (contiguous in X), each warp eight n in turn, warp reduction per n
        const int lane = t & 31, w = t >> 5;
        for (int j = 0; j < NT_K / 8; ++j) {
            const uint32_t tn = w * (NT_K / 8) + j;
            if (tn >= nn) break;   // uniform over the warp
            const T *x = X + n_off[tn];
            Acc<T> a;
#pragma unroll 4
            for (uint32_t k = lane; k < nk; k += 32)
                a.add(vk[k], dbg_ok(p.dbg_x, x + k_off[k], (int)sizeof(T), p.status) ? x[k_off[k]] : (T)0);
            double s = a.value();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0 && dbg_ok(p.dbg_p, out + n0 + tn, 8, p.status)) out[n0 + tn] = s;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) gemv_finish_kernel(const GemvParams p) {
    const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= (uint64_t)p.n_batch * p.N) return;
    const uint32_t bi = (uint32_t)(i / p.N), n = (uint32_t)(i - (uint64_t)bi * p.N);
    double s = 0.0;
    const double *part = p.partial + (size_t)bi * p.nchunks * p.N;
    for (uint32_t c = 0; c < p.nchunks; ++c)
        if (dbg_ok(p.dbg_p, part + (size_t)c * p.N + n, 8, p.status)) s += part[(size_t)c * p.N + n];
    int64_t ox = 0, oy = 0, by = 0, unused = 0;
    radix_offsets(p.n, n, ox, oy);
    radix_offsets(p.by, bi, by, unused);
    T *y = reinterpret_cast<T *>(p.Y) + by + oy;
    if (!dbg_ok(p.dbg_y, y, (int)sizeof(T), p.status)) return;
    const double r = p.alpha * s;
    *y = (T)(p.beta != 0.0 ? r + p.beta * (double)*y : r);
}

cudaError_t launch_gemv(const GemvParams &p, int elem_bytes, cudaStream_t s) {
    using namespace gv;
    if (p.N == 0) return cudaSuccess;
    if (p.K == 0) return cudaErrorInvalidValue;
    const uint64_t tiles = (p.N + (p.n_fast ? NT_N : NT_K) - 1) / (p.n_fast ? NT_N : NT_K);
    if (tiles * p.n_batch >= (1ull << 31) || p.nchunks > 65535) return cudaErrorInvalidValue;
    const dim3 grid1((uint32_t)(tiles * p.n_batch), p.nchunks);
    const uint32_t grid2 = (uint32_t)(((uint64_t)p.n_batch * p.N + 255) / 256);
    if (elem_bytes == 4) {
        if (p.n_fast) gemv_partial_kernel<float, true><<<grid1, gv::T, 0, s>>>(p);
        else gemv_partial_kernel<float, false><<<grid1, gv::T, 0, s>>>(p);
        gemv_finish_kernel<float><<<grid2, 256, 0, s>>>(p);
    } else {
        if (p.n_fast) gemv_partial_kernel<double, true><<<grid1, gv::T, 0, s>>>(p);
        else gemv_partial_kernel<double, false><<<grid1, gv::T, 0, s>>>(p);
        gemv_finish_kernel<double><<<grid2, 256, 0, s>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace comet
