// On-the-fly queries and the serving loop. Placeholder entry points.
#include "internal.h"

struct ServeState {};

int query_edge(abcore_ctx *ctx, int32_t, int32_t, int, int32_t, int32_t, uint8_t *) {
    return ctx->fail(ABCORE_EINVAL, "query_edge: not available");
}
int serve_start(abcore_ctx *ctx, const int32_t *, const int32_t *, int32_t, int32_t) {
    return ctx->fail(ABCORE_EINVAL, "serve: not available");
}
int serve_submit(abcore_ctx *ctx, const abcore_req *, int32_t, uint64_t *) {
    return ctx->fail(ABCORE_EINVAL, "serve: not available");
}
int serve_poll(abcore_ctx *ctx, abcore_resp *, int32_t, int32_t *n_out) {
    *n_out = 0;
    return ctx->fail(ABCORE_EINVAL, "serve: not available");
}
int serve_stop(abcore_ctx *ctx) { return ctx->fail(ABCORE_EINVAL, "serve: not available"); }
void free_serve(abcore_ctx *ctx) { (void)ctx; }
