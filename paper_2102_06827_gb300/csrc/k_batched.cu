// Batched triples-like contractions (placeholder until the persistent kernel lands).
#include <cuda_runtime.h>

#include "../../include/comet.h"
#include "batched.h"

namespace comet {
std::string describe_batched(const Plan &p) { return "{\"batched\":true}"; }
}  // namespace comet

extern "C" {
comet_status_t comet_plan_batched(const char *, int, const char *const *, int, const int64_t *,
                                  const comet_dtype_t *, int, const comet_plan_opts_t *, int,
                                  comet_plan_t *out) {
    if (out) *out = nullptr;
    return COMET_ERR_UNSUPPORTED;
}
int comet_batched_num_tiles(void) { return 0; }
comet_status_t comet_contract_batched(comet_plan_t, const void *const *, int, void *, uint32_t, void *,
                                      void *) {
    return COMET_ERR_UNSUPPORTED;
}
}
