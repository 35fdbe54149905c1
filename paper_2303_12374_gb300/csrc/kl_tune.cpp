// kl_tune.cpp -- batched launches, capture and the tuner.
#include "kl_internal.h"

using namespace kl;

extern "C" {

kl_status kl_launch_batched(kl_ctx *ctx, const kl_op *op, int32_t n, const kl_grid *grids,
                            const kl_fields *fields, void *stream)
{
    (void)ctx; (void)op; (void)n; (void)grids; (void)fields; (void)stream;
    return fail(KL_ERR_UNSUPPORTED, "kl_launch_batched: not built yet");
}

kl_status kl_capture(kl_ctx *ctx, const kl_op *op, const kl_grid *grid, const kl_fields *fields,
                     const char *path, void *stream)
{
    (void)ctx; (void)op; (void)grid; (void)fields; (void)path; (void)stream;
    return fail(KL_ERR_UNSUPPORTED, "kl_capture: not built yet");
}

kl_status kl_capture_if_requested(kl_ctx *ctx, const kl_op *op, const kl_grid *grid,
                                  const kl_fields *fields, void *stream)
{
    (void)ctx; (void)op; (void)grid; (void)fields; (void)stream;
    return KL_OK;
}

kl_status kl_tune(kl_ctx *ctx, const char *capture_path, const char *opts, const char *wisdom_path)
{
    (void)ctx; (void)capture_path; (void)opts; (void)wisdom_path;
    return fail(KL_ERR_UNSUPPORTED, "kl_tune: not built yet");
}

}  // extern "C"
