// Parameter blocks shared by the host planner and the device kernels.
//
// A "group" is an ordered list of labels fused into one GEMM dimension (the merging of
// consecutive indices into one matrix index in the TTGT reformulation, Section 2: (a,b) -> i).
// A group index g decomposes into digits, first label fastest (column-major merging), and each
// digit has a stride in the tensors that hold that label.  Kernels never materialise index
// tables: they decompose g with division by invariant integers.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define CM_HD __host__ __device__ __forceinline__
#else
#define CM_HD inline
#endif

namespace comet {

constexpr int kMaxDigits = 8;   // labels per group / per tensor
constexpr int kMaxRank = 8;

// Unsigned 32-bit division by an invariant divisor (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Fig. 4.1): with l = ceil(log2 d),
// m' = floor(2^32 (2^l - d) / d) + 1, sh1 = min(l,1), sh2 = max(l-1,0):
//   t1 = mulhi(m', n);  q = (t1 + ((n - t1) >> sh1)) >> sh2,  exact for every n < 2^32.
struct FastDiv {
    uint32_t d, m, sh1, sh2;
};

inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    f.m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    f.sh1 = l < 1 ? l : 1;
    f.sh2 = l > 1 ? l - 1 : 0;
    return f;
}

CM_HD uint32_t fd_div(uint32_t n, const FastDiv &f) {
#if defined(__CUDA_ARCH__)
    uint32_t t1 = __umulhi(f.m, n);
#else
    uint32_t t1 = (uint32_t)(((uint64_t)f.m * n) >> 32);
#endif
    return (t1 + ((n - t1) >> f.sh1)) >> f.sh2;
}

// Mixed-radix group with two stride sets (s0, s1): offset0(g) and offset1(g).
struct Radix {
    int n;                         // number of digits (0 = the group has the single index 0)
    uint32_t total;                // product of extents
    uint32_t ext[kMaxDigits];
    FastDiv fd[kMaxDigits];
    int64_t s0[kMaxDigits];
    int64_t s1[kMaxDigits];
};

CM_HD void radix_offsets(const Radix &r, uint32_t g, int64_t &o0, int64_t &o1) {
    int64_t a = 0, b = 0;
#pragma unroll
    for (int d = 0; d < kMaxDigits; ++d) {
        if (d < r.n) {
            uint32_t q = (d + 1 < r.n) ? fd_div(g, r.fd[d]) : 0;
            uint32_t digit = (d + 1 < r.n) ? g - q * r.ext[d] : g;
            a += (int64_t)digit * r.s0[d];
            b += (int64_t)digit * r.s1[d];
            g = q;
        }
    }
    o0 = a;
    o1 = b;
}

// The byte range [lo, hi) of the buffer that one pointer of a launch lies in.  Builds with
// COMET_DEBUG test every global access of the transpose, GEMM and gemv kernels against the
// ranges of their launch and skip (and record) any access outside them; release builds carry
// the ranges and never read them.
struct DbgRange {
    const char *lo, *hi;
};

CM_HD DbgRange dbg_range(const void *base, int64_t bytes) {
    DbgRange r;
    r.lo = static_cast<const char *>(base);
    r.hi = r.lo + (bytes > 0 ? bytes : 0);
    return r;
}

// Pure permutation / element-wise tiled copy (transpose engine).  The tensor's dims are split
// into three groups: U (leading input dims: contiguous reads), V (leading output dims:
// contiguous writes) and R (the rest).  A CTA moves one TU x TV x TW tile of (u, v, r) through
// shared memory: reads run along u, writes along v (along u when V is empty: "copy mode",
// input and output share their stride-1 dim).  s0 = input strides, s1 = output strides.
struct XposeParams {
    Radix u, v, r;
    const void *in;
    void *out;
    int64_t out_plane;             // split pre-pass: element distance between the 3 planes
    const void *scale_bits;        // split pre-pass: device word holding the bits of max |x|
    double alpha;                  // scaled copy: out = alpha * in (+ beta * out)
    double beta;
    uint32_t tu, tv, tw;           // tile extents along U, V and R (tu*tv*tw <= kXposeTile)
    uint32_t tiles_u, tiles_v, tiles_w;
    FastDiv fd_tu, fd_tv, fd_tuv;  // division by tu, tv and tu*tv inside the tile
    uint32_t ll, sl;               // threads per tile row: load phase ceil(tu/vi), store phase ceil(tv/vo)
    uint32_t rpp_l, rpp_s;         // rows per pass of the 256-thread block: 256/ll, 256/sl
    FastDiv fd_ll, fd_sl, fd_tiles_u, fd_tiles_v;
    int off32;                     // every input and output offset is below 2^31
    int single_run;                // copy mode with R empty: one long run, ragged tail allowed
    DbgRange dbg_in, dbg_out;      // debug builds: the buffers of in and out
    int *status;                   // debug builds: device status word for an access out of range
    int64_t plant;                 // debug builds, tests only: added to the first thread's output
                                   // offsets so that the range check must catch them
};

constexpr int kXposeTile = 4096;   // elements per tile (32 KB of FP64, 16 KB of FP32)

CM_HD uint32_t align16(uint32_t b) { return (b + 15u) & ~15u; }

// Dynamic shared memory of the transposing kernel: the (u, v, w) tile with an odd row pitch,
// then the input offsets of its (v, w) rows, then the output offsets and tile positions of its
// (u, w) rows.
CM_HD uint32_t xpose_smem_bytes(const XposeParams &p, int elem_bytes) {
    const uint32_t off = p.off32 ? 4u : 8u;
    const uint32_t rows_v = p.tv * p.tw, rows_u = p.tu * p.tw;
    return align16(rows_v * (p.tu | 1u) * (uint32_t)elem_bytes) + align16(rows_v * off) + align16(rows_u * 2u * off);
}

// Binary contraction as a GEMM over fused groups: C[m,n] = alpha * sum_k A[m,k] B[k,n]
// (+ beta C).  ma: M digits with (A strides, C strides); nb: N digits with (B strides,
// C strides); k: K digits with (A strides, B strides).
struct GemmParams {
    Radix ma, nb, k;
    uint32_t M, N, K;
    const void *A;
    const void *B;
    void *C;
    double alpha, beta;
    int *status;
    int64_t timeout_ns;
    DbgRange dbg_a, dbg_b, dbg_c;  // debug builds: the buffers of A, B and C
};

// Tensor-times-vector step: y[n] = alpha * sum_k v[k] X[k, n] (+ beta y[n]).  n: free digits
// with (X strides, y strides); k: contracted digits with (v strides, X strides).
struct GemvParams {
    Radix n, k;
    Radix bv, by;                  // batch digits: (v strides, X strides) and (y strides, unused)
    uint32_t n_batch;              // product of the batch extents (1 without batch labels)
    uint32_t N, K;
    const void *v;
    const void *X;
    void *Y;
    double alpha, beta;
    int n_fast;                    // 1: X's stride-1 dim is a free digit, 0: a contracted one
    int v_ones;                    // 1: v is all ones (a sum over the k digits of X; v unused)
    uint32_t nchunks;              // ceil(K / 1024)
    double *partial;               // workspace: n_batch x nchunks x N FP64 partial sums
    DbgRange dbg_v, dbg_x, dbg_y, dbg_p;   // debug builds: the buffers of v, X, Y and partial
    int *status;                   // debug builds: device status word
};

#if defined(__CUDACC__)
// True when the `bytes` at p lie inside r.  Debug builds record COMET_ERR_BOUNDS (13) in the
// status word when they do not, and the caller skips the access; release builds: always true.
__device__ __forceinline__ bool dbg_ok(const DbgRange &r, const void *p, int64_t bytes, int *status) {
#ifdef COMET_DEBUG
    const char *c = static_cast<const char *>(p);
    if (c >= r.lo && c + bytes <= r.hi) return true;
    if (status) atomicCAS(status, 0, 13);
    return false;
#else
    (void)r; (void)p; (void)bytes; (void)status;
    return true;
#endif
}
#endif

}  // namespace comet
