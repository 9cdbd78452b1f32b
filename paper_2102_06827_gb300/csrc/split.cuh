// Fixed-point three-way bfloat16 split shared by the split pre-pass and the batched kernels.
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
