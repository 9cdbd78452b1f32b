// Kernel launchers (host functions defined next to their kernels).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/comet.h"
#include "params.h"

namespace comet {

cudaError_t launch_move(const XposeParams &p, int elem_bytes, int vi, int vo, cudaStream_t s);
cudaError_t launch_scale(const XposeParams &p, int elem_bytes, int vi, int vo, cudaStream_t s);
cudaError_t launch_split(const XposeParams &p, int elem_bytes, int vi, int vo, cudaStream_t s);
cudaError_t launch_split6(const XposeParams &p, int elem_bytes, int vi, int vo, cudaStream_t s);

cudaError_t launch_gemm_f64(const GemmParams &p, int elem_bytes, bool a_kcontig, bool b_kcontig,
                            cudaStream_t s);

cudaError_t launch_fill(void *out, int64_t n, double value, int elem_bytes, cudaStream_t s);

// max |x| of a dense operand into *out_bits (zeroed first), as the bits of an input-precision value
cudaError_t launch_absmax(const void *x, int64_t n, int elem_bytes, void *out_bits, cudaStream_t s);
// max |x0| and max |x1| in one launch: words 0 and 1 (8 bytes apart) of out_bits
cudaError_t launch_absmax2(const void *x0, int64_t n0, const void *x1, int64_t n1, int elem_bytes, void *out_bits,
                           cudaStream_t s);
// the same over the r.total elements of a strided view at offsets r (digit strides s0)
cudaError_t launch_absmax_view(const void *x, const Radix &r, int elem_bytes, void *out_bits, cudaStream_t s);

// ksplit > 1: K sliced over more work items, FP32 partials in `partial` (ksplit x tiles x
// 128 x 256 floats) summed by a reduce kernel into C.  ksplit = 1: whole-K tiles, except that a
// partial last wave over the SMs runs in K slices when its partials fit `partial_bytes`.
cudaError_t launch_gemm_split(const GemmParams &p, const void *parts_a, const void *parts_b,
                              int64_t kpad, const void *scale_a, const void *scale_b, int64_t kc,
                              int out_bytes, int debug_flags, cudaStream_t s, int max_ctas,
                              uint32_t ksplit = 1, float *partial = nullptr, int64_t partial_bytes = 0);

cudaError_t launch_gemm_emu(const GemmParams &p, const void *parts_a, const void *parts_b, int64_t kpad,
                            const void *scale_a, const void *scale_b, int debug_flags, cudaStream_t s,
                            int max_ctas);

cudaError_t launch_gemv(const GemvParams &p, int elem_bytes, cudaStream_t s);

// device status word of the current device (set by kernels whose waits run out)
int *device_status_word();

}  // namespace comet
