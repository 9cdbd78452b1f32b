// The weight of the batched triples reduction s_b = sum T*W, q_b = sum T^2.
//
// The 6-D triples outputs are consumed in place, never stored; the weight keeps s_b sensitive
// to every element's value and position.  It is a product of two hashed factors,
//   W(element) = h(key, b, oA) * h(~key, b, oB),
//   h(k, b, x) = (fmix32(k ^ fmix32(b * 0x9E3779B9 + x)) >> 8) * 2^-23 - 1   (in [-1, 1)),
// where oA + oB is the element's column-major offset in T, oA the part that the labels of the
// expression's first operand contribute and oB the part of the second operand's labels.  A
// kernel whose tile rows come from one operand and columns from the other forms one factor
// per row and one per column instead of two hashes per element.
#pragma once
#include <stdint.h>

namespace comet {

// MurmurHash3 32-bit finalizer (Appleby, MurmurHash3, public domain)
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// h(key, b, x) from the block term hb = b * 0x9E3779B9 (32-bit wraparound); exact in FP32
__device__ __forceinline__ float tri_factor(uint32_t key, uint32_t hb, uint32_t x) {
    const uint32_t h = fmix32(key ^ fmix32(hb + x));
    return (float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f;
}

}  // namespace comet
