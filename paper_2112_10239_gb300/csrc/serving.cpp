// Serving loop placeholder (continuous batching is implemented below once the
// synchronous path is validated).
#include "runtime.h"

namespace tlq {
void scheduler_stop(Context*) {}
}  // namespace tlq

using namespace tlq;

extern "C" {
tlq_status tlq_submit(tlq_ctx, tlq_circuit, tlq_ham, const double*, int32_t, int, tlq_precision, double*, double*,
                      tlq_ticket*) {
    set_error("tlq_submit: not available");
    return TLQ_EUNSUPPORTED;
}
tlq_status tlq_poll(tlq_ctx, tlq_ticket, int64_t) {
    set_error("tlq_poll: not available");
    return TLQ_EUNSUPPORTED;
}
tlq_status tlq_serving_stats(tlq_ctx, int64_t*, double*, double*, double*) {
    set_error("tlq_serving_stats: not available");
    return TLQ_EUNSUPPORTED;
}
}
