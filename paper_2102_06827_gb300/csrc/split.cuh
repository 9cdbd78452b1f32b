// Fixed-point bfloat16 splits shared by the split pre-passes and the batched kernels.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace comet {

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

// Fixed-point six-way split of an FP64 value (the FP64-emulation pre-pass): x' = x 2^-e
// (|x'| < 2) is rounded to the nearest multiple of 2^-46, X = round(x' 2^46) with |X| <= 2^47,
// and X is written in balanced base 256: X = sum_k s_k 256^(5-k), s_1..s_5 in [-128, 127] and
// |s_0| <= 128, so x' = sum_k s_k 2^-(6+8k) up to 2^-47 and every slice is an integer that
// bfloat16 holds exactly (stored as the integer itself).  Integer arithmetic on the bits only:
// the FP64 pipe of the GPU is not used.
__device__ __forceinline__ void split6(double x, int e, __nv_bfloat16 (&s)[6]) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((bits >> 52) & 0x7FF);
    unsigned long long m = bits & ((1ull << 52) - 1);
    if (E != 0) m |= 1ull << 52;
    // x' 2^46 = m 2^(max(E,1) - 1075 - e + 46): shift right by sh with rounding to nearest
    const int sh = 1029 + e - (E != 0 ? E : 1);
    long long X;
    if (sh <= 0) X = (long long)(m << (-sh < 63 ? -sh : 63));
    else if (sh < 63) X = (long long)((m + (1ull << (sh - 1))) >> sh);
    else X = 0;
    if (bits >> 63) X = -X;
#pragma unroll
    for (int k = 5; k >= 1; --k) {
        const int d = (int)(signed char)(X & 0xFF);
        s[k] = __int2bfloat16_rn(d);
        X = (X - d) >> 8;
    }
    s[0] = __int2bfloat16_rn((int)X);
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

}  // namespace comet
