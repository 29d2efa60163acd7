// Query helpers built from the peel: the size of a core, the largest beta with a non-empty
// (alpha, beta)-core (the alpha_offset of the paper's default query, Section 6), and community
// search -- the connected component of the (alpha, beta)-core that contains a query vertex (the
// Remark after GFQ in Section 5).
#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace {

__global__ void k_count_ones(const uint8_t *a, int64_t n, unsigned long long *out) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += a[i] != 0;
    c = (unsigned long long)abc::warp_sum64((long long)c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Membership in internal order from the caller-order masks.
__global__ void k_alive_internal(const int32_t *new2old, int32_t nU, int64_t n, const uint8_t *mask_u,
                                 const uint8_t *mask_v, uint8_t *alive) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = __ldg(&new2old[x]);
        alive[x] = x < nU ? mask_u[o] : mask_v[o];
    }
}

unsigned grid_of(const abcore_ctx *ctx, int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 16));
}

}  // namespace

// Members of the (alpha, beta)-core, with the masks left in the peel's staging buffer.
int core_size(abcore_ctx *ctx, int32_t alpha, int32_t beta, int64_t *size) {
    const Graph &g = ctx->g;
    ABC_TRY(peel_finish(ctx));
    ABC_TRY(peel_prepare(ctx));
    uint8_t *su = ctx->w.stage, *sv = ctx->w.stage + g.nU;
    ABC_TRY(peel_compute(ctx, alpha, beta, su, sv, false, prefer_pruned(ctx, alpha, beta)));
    unsigned long long *cnt = nullptr;
    ABC_TRY(ctx->alloc(&cnt, 1, "core size"));
    unsigned long long h = 0;
    cudaMemsetAsync(cnt, 0, sizeof(h), ctx->stream);
    if (g.n() > 0) k_count_ones<<<grid_of(ctx, g.n()), 256, 0, ctx->stream>>>(ctx->w.stage, g.n(), cnt);
    cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
    int rc = peel_finish(ctx);
    if (!rc) {
        const cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = ctx->cuda_fail(e, "core size");
    }
    ctx->release(cnt);
    if (!rc) *size = (int64_t)h;
    return rc;
}

// Largest beta >= 1 whose (alpha, beta)-core is non-empty, 0 if none: by the nested property
// the core shrinks as beta grows, so a binary search over [1, max V degree] finds it.
int alpha_offset(abcore_ctx *ctx, int32_t alpha, int32_t *beta_out) {
    int32_t lo = 0, hi = ctx->g.maxdegV;  // invariant: core(alpha, lo) non-empty or lo == 0
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo + 1) / 2;
        int64_t sz = 0;
        ABC_TRY(core_size(ctx, alpha, mid, &sz));
        if (sz > 0) lo = mid;
        else hi = mid - 1;
    }
    *beta_out = lo;
    return ABCORE_OK;
}

// The component of the (alpha, beta)-core holding internal vertex q: components of the core's
// induced subgraph (union-find over edges with both ends in the core), then q's one.
int community(abcore_ctx *ctx, int32_t q_internal, int32_t alpha, int32_t beta, uint8_t *d_mask_u, uint8_t *d_mask_v,
              int64_t *size) {
    const Graph &g = ctx->g;
    int64_t sz = 0;
    ABC_TRY(core_size(ctx, alpha, beta, &sz));
    uint8_t *alive = nullptr;
    ABC_TRY(ctx->alloc(&alive, (size_t)std::max<int64_t>(g.n(), 1), "community membership"));
    if (g.n() > 0)
        k_alive_internal<<<grid_of(ctx, g.n()), 256, 0, ctx->stream>>>(g.new2old, g.nU, g.n(), ctx->w.stage,
                                                                       ctx->w.stage + g.nU, alive);
    ctx->stats.launches++;
    int rc = community_compute(ctx, alive, q_internal, d_mask_u, d_mask_v, size);
    ctx->release(alive);
    return rc;
}
