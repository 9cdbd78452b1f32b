// FP64 contraction kernel: the GEMM of the TTGT reformulation (Section 2, C_p = A_p * B_p;
// Section 6 "GEMM optimizations" for the blocking) run directly on the operands' own strided
// layouts.  Row, column and K indices are merged label groups (params.h); every tile load
// decomposes its indices into label digits, so the transposes of TTGT are folded into the
// loads and into the epilogue's stores and no permuted copy is ever written.
//
// Arithmetic: FP64 tensor-core MMA (mma.sync.m8n8k4 f64) with FP64 accumulation; FP32-stored
// operands are widened exactly on load and the result is rounded once on store.
//
// Blocking: TM x TM output tile per CTA (TM = 64; 32 when 64-wide tiles would leave SMs idle),
// K in blocks of 16, four warps of TM/2 x TM/2; the next K block is loaded into registers while
// the current one is multiplied (double-buffered shared memory).
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"
#include "params.h"

namespace comet {

constexpr int FBK = 16, FPAD = 4;
constexpr int FTHREADS = 128;

__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

// A tile: FBM rows (m) x FBK cols (k); element (m,k) at a_row[m] + a_k[k].  The thread map
// follows the contiguous direction of the operand in memory.
template <typename TIn, bool KCONTIG, int TM>
__device__ __forceinline__ void load_tile(const TIn *__restrict__ base, const int64_t *rowoff,
                                          const int64_t *koff, uint32_t row0, uint32_t rows,
                                          uint32_t k0, uint32_t K, double (&r)[TM * FBK / FTHREADS],
                                          const DbgRange &rg, int *status) {
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < TM * FBK / FTHREADS; ++i) {
        int idx = t + i * FTHREADS;
        int m, k;
        if (KCONTIG) { k = idx % FBK; m = idx / FBK; }
        else { m = idx % TM; k = idx / TM; }
        double v = 0.0;
        if (row0 + m < rows && k0 + k < K && dbg_ok(rg, base + rowoff[m] + koff[k], (int)sizeof(TIn), status))
            v = (double)base[rowoff[m] + koff[k]];
        r[i] = v;
    }
}

template <bool KCONTIG, int TM>
__device__ __forceinline__ void store_tile(double (*s)[TM + FPAD], const double (&r)[TM * FBK / FTHREADS]) {
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < TM * FBK / FTHREADS; ++i) {
        int idx = t + i * FTHREADS;
        int m, k;
        if (KCONTIG) { k = idx % FBK; m = idx / FBK; }
        else { m = idx % TM; k = idx / TM; }
        s[k][m] = r[i];
    }
}

template <typename TIn, bool AK, bool BK, int TM>
__global__ void __launch_bounds__(FTHREADS) gemm_f64_kernel(const GemmParams p) {
    constexpr int FBM = TM, FBN = TM, FI = TM / 16, NL = TM * FBK / FTHREADS;
    __shared__ double As[2][FBK][FBM + FPAD];
    __shared__ double Bs[2][FBK][FBN + FPAD];
    __shared__ int64_t a_row[FBM], b_col[FBN], c_row[FBM], c_col[FBN];
    __shared__ int64_t a_k[2][FBK], b_k[2][FBK];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const uint32_t m0 = blockIdx.x * FBM, n0 = blockIdx.y * FBN;
    const TIn *A = reinterpret_cast<const TIn *>(p.A);
    const TIn *B = reinterpret_cast<const TIn *>(p.B);

    if (t < FBM) {
        int64_t o0 = 0, o1 = 0;
        if (m0 + t < p.M) radix_offsets(p.ma, m0 + t, o0, o1);
        a_row[t] = o0; c_row[t] = o1;
    } else if (t < FBM + FBN) {
        int j = t - FBM;
        int64_t o0 = 0, o1 = 0;
        if (n0 + j < p.N) radix_offsets(p.nb, n0 + j, o0, o1);
        b_col[j] = o0; c_col[j] = o1;
    }
    auto k_offsets = [&](int buf, uint32_t k0) {
        if (t < FBK) {
            int64_t o0 = 0, o1 = 0;
            if (k0 + t < p.K) radix_offsets(p.k, k0 + t, o0, o1);
            a_k[buf][t] = o0; b_k[buf][t] = o1;
        }
    };
    k_offsets(0, 0);
    __syncthreads();

    double acc[FI][FI][2];
#pragma unroll
    for (int i = 0; i < FI; ++i)
#pragma unroll
        for (int j = 0; j < FI; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    double ra[NL], rb[NL];
    load_tile<TIn, AK, TM>(A, a_row, a_k[0], m0, p.M, 0, p.K, ra, p.dbg_a, p.status);
    load_tile<TIn, BK, TM>(B, b_col, b_k[0], n0, p.N, 0, p.K, rb, p.dbg_b, p.status);
    store_tile<AK, TM>(As[0], ra);
    store_tile<BK, TM>(Bs[0], rb);
    const uint32_t nkb = (p.K + FBK - 1) / FBK;
    if (nkb > 1) k_offsets(1, FBK);
    __syncthreads();

    for (uint32_t kb = 0; kb < nkb; ++kb) {
        const int cur = kb & 1, nxt = cur ^ 1;
        const bool more = kb + 1 < nkb;
        if (more) {
            load_tile<TIn, AK, TM>(A, a_row, a_k[nxt], m0, p.M, (kb + 1) * FBK, p.K, ra, p.dbg_a, p.status);
            load_tile<TIn, BK, TM>(B, b_col, b_k[nxt], n0, p.N, (kb + 1) * FBK, p.K, rb, p.dbg_b, p.status);
        }
#pragma unroll
        for (int k4 = 0; k4 < FBK / 4; ++k4) {
            const int kk = k4 * 4 + (lane & 3);
            double af[FI], bf[FI];
#pragma unroll
            for (int i = 0; i < FI; ++i) af[i] = As[cur][kk][wm * (TM / 2) + i * 8 + (lane >> 2)];
#pragma unroll
            for (int j = 0; j < FI; ++j) bf[j] = Bs[cur][kk][wn * (TM / 2) + j * 8 + (lane >> 2)];
#pragma unroll
            for (int i = 0; i < FI; ++i)
#pragma unroll
                for (int j = 0; j < FI; ++j) dmma(acc[i][j], af[i], bf[j]);
        }
        if (more) {
            store_tile<AK, TM>(As[nxt], ra);
            store_tile<BK, TM>(Bs[nxt], rb);
        }
        __syncthreads();
        if (kb + 2 < nkb) k_offsets(cur, (kb + 2) * FBK);
        // a_k[cur] is rewritten only after the barrier that ends the use of buffer cur
        __syncthreads();
    }

    // epilogue: C[m,n] = alpha * acc (+ beta * C), stored through the C strides of M and N
    TIn *C = reinterpret_cast<TIn *>(p.C);
#pragma unroll
    for (int i = 0; i < FI; ++i) {
        const int ml = wm * (TM / 2) + i * 8 + (lane >> 2);
        if (m0 + ml >= p.M) continue;
#pragma unroll
        for (int j = 0; j < FI; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int nl = wn * (TM / 2) + j * 8 + (lane & 3) * 2 + h;
                if (n0 + nl >= p.N) continue;
                TIn *dst = C + c_row[ml] + c_col[nl];
                if (!dbg_ok(p.dbg_c, dst, (int)sizeof(TIn), p.status)) continue;
                double v = p.alpha * acc[i][j][h];
                if (p.beta != 0.0) v += p.beta * (double)*dst;
                *dst = (TIn)v;
            }
        }
    }
}

cudaError_t launch_gemm_f64(const GemmParams &p, int elem_bytes, bool a_kcontig, bool b_kcontig,
                            cudaStream_t s) {
    if (p.M == 0 || p.N == 0) return cudaSuccess;
    static int sms = [] {
        int dev = 0, n = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n;
    }();
    // 64-wide tiles unless they would leave SMs idle
    const uint64_t tiles64 = (uint64_t)((p.M + 63) / 64) * ((p.N + 63) / 64);
    const int tm = tiles64 < (uint64_t)sms ? 32 : 64;
    dim3 grid((p.M + tm - 1) / tm, (p.N + tm - 1) / tm);
    if (grid.y > 65535) return cudaErrorInvalidConfiguration;
#define CM_LAUNCH(T, a, b)                                                               \
    do {                                                                                 \
        if (tm == 32) gemm_f64_kernel<T, a, b, 32><<<grid, FTHREADS, 0, s>>>(p);         \
        else gemm_f64_kernel<T, a, b, 64><<<grid, FTHREADS, 0, s>>>(p);                  \
    } while (0)
    if (elem_bytes == 8) {
        if (a_kcontig && b_kcontig) CM_LAUNCH(double, true, true);
        else if (a_kcontig) CM_LAUNCH(double, true, false);
        else if (b_kcontig) CM_LAUNCH(double, false, true);
        else CM_LAUNCH(double, false, false);
    } else {
        if (a_kcontig && b_kcontig) CM_LAUNCH(float, true, true);
        else if (a_kcontig) CM_LAUNCH(float, true, false);
        else if (b_kcontig) CM_LAUNCH(float, false, true);
        else CM_LAUNCH(float, false, false);
    }
#undef CM_LAUNCH
    return cudaGetLastError();
}

}  // namespace comet
