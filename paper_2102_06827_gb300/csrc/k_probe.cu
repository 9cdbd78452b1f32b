// FP64 throughput probes: the denominators of the FP64 rooflines, measured on the GPU at hand.
//
// Each kernel keeps the FP64 pipe busy with independent dependency chains and nothing else
// (no memory traffic inside the timed loop).  The caller times one launch with CUDA events and
// divides the flops this file reports by the elapsed time.  The chain values start from a
// runtime argument and are written out only under a condition that never holds, so the
// compiler can neither fold nor drop the arithmetic.
//
//   kind 0  DFMA: 8 chains per thread, 8 warps per SM sub-partition
//   kind 1  tensor-core f64 MMA m8n8k4   (512 flops per warp instruction)
//   kind 2  tensor-core f64 MMA m16n8k4  (1024 flops)
//   kind 3  tensor-core f64 MMA m16n8k16 (4096 flops)
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/comet.h"

namespace comet {

void set_error_message(const std::string &s);

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) probe_dfma_kernel(double seed, int iters, double *sink) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
    const double m = 0.9999999, d = 1e-9 * seed;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 1234.5678) sink[0] = s;   // never true for the seeds used; keeps the chains alive
}

__global__ void __launch_bounds__(kThreads) probe_dmma884_kernel(double seed, int iters, double *sink) {
    double acc[kChains][2];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c][0] = acc[c][1] = 0.0;
    const double a = seed * 1e-3 * (threadIdx.x & 7), b = seed * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(acc[c][0]), "+d"(acc[c][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c][0] + acc[c][1];
    if (s == 1234.5678) sink[0] = s;
}

__global__ void __launch_bounds__(kThreads) probe_dmma1684_kernel(double seed, int iters, double *sink) {
    double acc[kChains][4];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.0;
    const double a0 = seed * 1e-3, a1 = seed * 2e-3 * (threadIdx.x & 3), b = seed * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
                         "{%0,%1,%2,%3};"
                         : "+d"(acc[c][0]), "+d"(acc[c][1]), "+d"(acc[c][2]), "+d"(acc[c][3])
                         : "d"(a0), "d"(a1), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
    if (s == 1234.5678) sink[0] = s;
}

__global__ void __launch_bounds__(kThreads) probe_dmma16816_kernel(double seed, int iters, double *sink) {
    constexpr int NC = 4;   // 16 accumulator registers per chain set keeps the thread under 128 registers
    double acc[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.0;
    double a[8], b[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed * 1e-3 * (i + (threadIdx.x & 3));
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = seed * 1e-3 * (i + 1);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
            asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
                         "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
                         : "+d"(acc[c][0]), "+d"(acc[c][1]), "+d"(acc[c][2]), "+d"(acc[c][3])
                         : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]),
                           "d"(a[7]), "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NC; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
    if (s == 1234.5678) sink[0] = s;
}

}  // namespace
}  // namespace comet

extern "C" comet_status_t comet_probe_fp64(int kind, int iters, double *flops, void *sink, void *stream) {
    using namespace comet;
    if (!flops || !sink) return COMET_ERR_NULL;
    if (kind < 0 || kind > 3 || iters < 1 || iters > (1 << 24)) return COMET_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms <= 0)
        return COMET_ERR_CUDA;
    const int blocks = sms * 8;   // 64 warps per SM: every sub-partition has 16 warps to switch among
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *out = static_cast<double *>(sink);
    const double warps = (double)blocks * (kThreads / 32);
    switch (kind) {
        case 0:
            probe_dfma_kernel<<<blocks, kThreads, 0, s>>>(1.0, iters, out);
            *flops = 2.0 * (double)blocks * kThreads * kChains * 8.0 * iters;
            break;
        case 1:
            probe_dmma884_kernel<<<blocks, kThreads, 0, s>>>(1.0, iters, out);
            *flops = warps * kChains * 512.0 * iters;
            break;
        case 2:
            probe_dmma1684_kernel<<<blocks, kThreads, 0, s>>>(1.0, iters, out);
            *flops = warps * kChains * 1024.0 * iters;
            break;
        default:
            probe_dmma16816_kernel<<<blocks, kThreads, 0, s>>>(1.0, iters, out);
            *flops = warps * 4 * 4096.0 * iters;
            break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error_message(std::string("FP64 probe: ") + cudaGetErrorString(e));
        return COMET_ERR_CUDA;
    }
    return COMET_OK;
}
