// Mixed batches of plans in one persistent launch: placeholder.
#include "gft_internal.h"

struct gft_batch_s {
    int dummy = 0;
};

extern "C" {
gft_status gft_batch_create(int32_t, const gft_plan_t*, const int64_t*, uint32_t, gft_batch_t*) {
    gft::set_last_error("mixed batches are not available in this build");
    return GFT_ERR_UNSUPPORTED;
}
gft_status gft_batch_forward(gft_batch_t, const float* const*, float* const*, gft_stream_t) {
    return GFT_ERR_UNSUPPORTED;
}
gft_status gft_batch_get_tile(gft_batch_t, int32_t, int32_t*, int32_t*) { return GFT_ERR_UNSUPPORTED; }
gft_status gft_batch_destroy(gft_batch_t) { return GFT_OK; }
}
