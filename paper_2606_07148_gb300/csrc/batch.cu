// Batched (alpha, beta)-cores. Placeholder: one peel per pair, in order.
#include "internal.h"

struct BatchState {};

int batch_compute(abcore_ctx *ctx, int32_t n, const int32_t *alphas, const int32_t *betas,
                  uint8_t *d_masks_u, uint8_t *d_masks_v, bool sync_and_check) {
    (void)sync_and_check;
    const Graph &g = ctx->g;
    for (int32_t i = 0; i < n; ++i)
        ABC_TRY(peel_compute(ctx, alphas[i], betas[i], d_masks_u + (size_t)i * g.nU,
                             d_masks_v + (size_t)i * g.nV, true));
    return ABCORE_OK;
}

void free_batch(abcore_ctx *ctx) { (void)ctx; }
