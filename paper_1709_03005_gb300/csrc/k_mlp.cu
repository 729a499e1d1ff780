// Learned Davidson preconditioner (placeholder until the network lands).
#include "hb_davidson.cuh"

int hb::mlp_weights_for(hb_ctx *ctx, DiagWork *, const double *, int, float **out, cudaStream_t) {
    *out = nullptr;
    ctx->err = "no preconditioner network";
    return HB_ERR_UNSUPPORTED;
}

void hb::release_mlp(hb_ctx *) {}

extern "C" int hb_mlp_set(hb_ctx *ctx, const hb_mlp_weights *) {
    if (ctx) ctx->err = "hb_mlp_set is not available in this build";
    return HB_ERR_UNSUPPORTED;
}
