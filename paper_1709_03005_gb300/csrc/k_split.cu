// Split-precision expansion (placeholder until the tensor-core kernel lands).
#include "hb_api_internal.cuh"

int expand_mixed(hb_ctx *ctx, hb::GroupPair &, double *, cudaStream_t) {
    ctx->err = "HB_MIXED is not available in this build";
    return HB_ERR_UNSUPPORTED;
}

void release_mixed(hb_ctx *) {}
