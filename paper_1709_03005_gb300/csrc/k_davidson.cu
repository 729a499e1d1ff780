// Block Davidson (placeholder until the solver lands).
#include "hb_api_internal.cuh"

extern "C" int hb_diag(hb_ctx *ctx, const hb_blocks *, int32_t, double, int32_t, int32_t, const double *, double *,
                       double *, hb_stats *, void *) {
    if (ctx) ctx->err = "hb_diag is not available in this build";
    return HB_ERR_UNSUPPORTED;
}

extern "C" int hb_mlp_set(hb_ctx *ctx, const hb_mlp_weights *) {
    if (ctx) ctx->err = "hb_mlp_set is not available in this build";
    return HB_ERR_UNSUPPORTED;
}
