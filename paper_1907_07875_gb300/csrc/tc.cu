// Tensor-core (tcgen05) leaf products for large leaves: placeholder until the
// split-precision kernel lands; every call reports GFT_ERR_UNSUPPORTED.
#include "gft_internal.h"

namespace gft {

void launch_tc(gft_plan_s& p, const float* x, float* y, int64_t batch, bool inverse, cudaStream_t st,
               uint32_t precision) {
    (void)p; (void)x; (void)y; (void)batch; (void)inverse; (void)st; (void)precision;
    fail(GFT_ERR_UNSUPPORTED, "tensor-core precisions are not available in this build");
}

}  // namespace gft
