// Batched list ranking and connected components (placeholder until the
// persistent batched kernels land).
#include "common.cuh"
#include "internal.h"

namespace lrcc {

lrcc_status lr_batched_run(Ctx*, const int32_t*, const int64_t*, const int32_t*, int64_t, int32_t*,
                           const Plan&) {
    return LRCC_ERR_ARG;
}
lrcc_status cc_batched_run(Ctx*, const int32_t*, const int32_t*, const int64_t*, const int64_t*, int64_t,
                           int32_t*, const Plan&) {
    return LRCC_ERR_ARG;
}
size_t lr_batched_ws(int64_t) { return 0; }
size_t cc_batched_ws(int64_t) { return 0; }

}  // namespace lrcc
