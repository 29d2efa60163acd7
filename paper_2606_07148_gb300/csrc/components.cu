// Connected components of the bipartite graph: the labels GFQ computes in its preprocessing and
// maintains under updates to scope each re-peel to the updated edge's component (Section 5).
//
// One pass of lock-free union-find over the edges (cc_core.cuh): every edge is seen once, from
// its U row. U rows are numbered by non-increasing degree, so the rows split into three ranges
// by length -- hubs (>= 1024 entries: one block per row), medium rows (>= 32: one warp per row)
// and short rows (one thread per row) -- and each range gets a launch shaped for it. A final pass
// compresses every path and names each component by the smallest caller id in it (U vertex u is
// u, V vertex v is nU + v), so labels do not depend on the internal numbering or on the order in
// which the unions happened.
#include <algorithm>

#include "cc_core.cuh"
#include "device.cuh"
#include "internal.h"

namespace {

constexpr int CC_HUB = 1024;    // rows at least this long: one block each
constexpr int CC_MEDIUM = 32;   // rows at least this long: one warp each

__device__ __forceinline__ bool slot_deleted(const uint32_t *tomb, int64_t p) {
    return tomb != nullptr && ((__ldg(&tomb[p >> 5]) >> (p & 31)) & 1u);
}

// An edge counts if its slot is not deleted and, with a `keep` mask, both endpoints are kept.
__device__ __forceinline__ bool edge_kept(const uint32_t *tomb, const uint8_t *keep, int64_t p, int32_t x, int32_t y) {
    return !slot_deleted(tomb, p) && (keep == nullptr || (__ldg(&keep[x]) && __ldg(&keep[y])));
}

__global__ void k_cc_init(int32_t *parent, int64_t n) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        parent[x] = (int32_t)x;
}

// rows [r0, r1): one block per row
__global__ void k_cc_hook_block(const int64_t *off, const int32_t *adj, const uint32_t *tomb, const uint8_t *keep,
                                int32_t *parent,
                                int32_t r0, int32_t r1) {
    for (int32_t x = r0 + blockIdx.x; x < r1; x += gridDim.x) {
        const int64_t s = __ldg(&off[x]), e = __ldg(&off[x + 1]);
        for (int64_t p = s + threadIdx.x; p < e; p += blockDim.x)
            if (edge_kept(tomb, keep, p, x, __ldg(&adj[p]))) abc::cc_unite(parent, x, __ldg(&adj[p]));
    }
}

// rows [r0, r1): one warp per row
__global__ void k_cc_hook_warp(const int64_t *off, const int32_t *adj, const uint32_t *tomb, const uint8_t *keep,
                                int32_t *parent,
                               int32_t r0, int32_t r1) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = r0 + w0; x < r1; x += nw) {
        const int64_t s = __ldg(&off[x]), e = __ldg(&off[x + 1]);
        for (int64_t p = s + lane; p < e; p += 32)
            if (edge_kept(tomb, keep, p, (int32_t)x, __ldg(&adj[p]))) abc::cc_unite(parent, (int32_t)x, __ldg(&adj[p]));
    }
}

// rows [r0, r1): one thread per row
__global__ void k_cc_hook_thread(const int64_t *off, const int32_t *adj, const uint32_t *tomb, const uint8_t *keep,
                                int32_t *parent,
                                 int32_t r0, int32_t r1) {
    for (int64_t x = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < r1; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = __ldg(&off[x]), e = __ldg(&off[x + 1]);
        for (int64_t p = s; p < e; ++p)
            if (edge_kept(tomb, keep, p, (int32_t)x, __ldg(&adj[p]))) abc::cc_unite(parent, (int32_t)x, __ldg(&adj[p]));
    }
}

// Compress every path (parent[x] = root) and record, per root, the smallest caller id.
__global__ void k_cc_roots(int32_t *parent, const int32_t *new2old, int32_t nU, int64_t n, int32_t *minc,
                           unsigned long long *ncomp) {
    unsigned long long roots = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = abc::cc_find(parent, (int32_t)x);
        parent[x] = r;
        const int32_t caller = __ldg(&new2old[x]) + (x >= nU ? nU : 0);
        atomicMin(&minc[r], caller);
        roots += (r == x) ? 1 : 0;
    }
    roots = (unsigned long long)abc::warp_sum64((long long)roots);
    if ((threadIdx.x & 31) == 0 && roots) atomicAdd(ncomp, roots);
}

// Labels in the caller's order.
__global__ void k_cc_emit(const int32_t *old2new, const int32_t *parent, const int32_t *minc, int32_t nU, int32_t nV,
                          int32_t *lab_u, int32_t *lab_v) {
    const int64_t n = (int64_t)nU + nV;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = __ldg(&minc[__ldg(&parent[__ldg(&old2new[i])])]);
        if (i < nU) lab_u[i] = l;
        else lab_v[i - nU] = l;
    }
}

// Community of vertex q: members of the core (alive[x]) in q's component of the core.
__global__ void k_community(const int32_t *old2new, const int32_t *parent, const uint8_t *alive, int32_t q_internal,
                            int32_t nU, int32_t nV, uint8_t *mask_u, uint8_t *mask_v, unsigned long long *size) {
    const int64_t n = (int64_t)nU + nV;
    const int32_t rq = abc::cc_find(const_cast<int32_t *>(parent), q_internal);
    const bool qin = __ldg(&alive[q_internal]) != 0;
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = __ldg(&old2new[i]);
        const uint8_t in = (qin && __ldg(&alive[x]) && abc::cc_find(const_cast<int32_t *>(parent), x) == rq) ? 1 : 0;
        if (i < nU) mask_u[i] = in;
        else mask_v[i - nU] = in;
        c += in;
    }
    c = (unsigned long long)abc::warp_sum64((long long)c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(size, c);
}

}  // namespace

int community_compute(abcore_ctx *ctx, const uint8_t *d_alive, int32_t q_internal, uint8_t *d_mask_u,
                      uint8_t *d_mask_v, int64_t *size) {
    const Graph &g = ctx->g;
    const int64_t n = g.n();
    int32_t *parent = nullptr;
    unsigned long long *cnt = nullptr;
    ABC_TRY(ctx->alloc(&parent, (size_t)std::max<int64_t>(n, 1), "community forest"));
    int rc = ctx->alloc(&cnt, 1, "community size");
    if (!rc) rc = cc_hook_base(ctx, parent, nullptr, ctx->stream, d_alive);
    unsigned long long h = 0;
    if (!rc) {
        const unsigned gi = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 16));
        cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), ctx->stream);
        k_community<<<gi, 256, 0, ctx->stream>>>(g.old2new, parent, d_alive, q_internal, g.nU, g.nV, d_mask_u, d_mask_v, cnt);
        ctx->stats.launches++;
        cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
        const cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = ctx->cuda_fail(e, "community");
    }
    ctx->release(parent);
    ctx->release(cnt);
    if (!rc && size) *size = (int64_t)h;
    return rc;
}

int cc_hook_base(abcore_ctx *ctx, int32_t *parent, const uint32_t *tomb, cudaStream_t st, const uint8_t *keep) {
    const Graph &g = ctx->g;
    const int64_t n = g.n();
    const unsigned gi = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 16));
    k_cc_init<<<gi, 256, 0, st>>>(parent, n);
    ctx->stats.launches++;
    return cc_hook_rows(ctx, parent, tomb, st, keep);
}

int cc_hook_rows(abcore_ctx *ctx, int32_t *parent, const uint32_t *tomb, cudaStream_t st, const uint8_t *keep) {
    const Graph &g = ctx->g;
    // U rows by length (internal U ids are sorted by non-increasing degree)
    const int32_t h = (int32_t)std::min<int64_t>(cnt_ge(g.cntU_ge, CC_HUB), g.nU);
    const int32_t w = (int32_t)std::min<int64_t>(cnt_ge(g.cntU_ge, CC_MEDIUM), g.nU);
    if (h > 0) k_cc_hook_block<<<(unsigned)std::min<int64_t>(h, (int64_t)ctx->num_sms * 8), 256, 0, st>>>(g.off, g.adj, tomb, keep, parent, 0, h);
    if (w > h) {
        const int64_t warps = w - h;
        k_cc_hook_warp<<<(unsigned)std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)ctx->num_sms * 16), 256, 0, st>>>(
            g.off, g.adj, tomb, keep, parent, h, w);
    }
    if (g.nU > w) {
        const int64_t rows = g.nU - w;
        k_cc_hook_thread<<<(unsigned)std::min<int64_t>((rows + 255) / 256, (int64_t)ctx->num_sms * 16), 256, 0, st>>>(
            g.off, g.adj, tomb, keep, parent, w, g.nU);
    }
    ctx->stats.launches += 3;
    ABC_CU(cudaGetLastError());
    return ABCORE_OK;
}

int cc_emit(abcore_ctx *ctx, int32_t *parent, int32_t *d_lab_u, int32_t *d_lab_v, int64_t *ncomp, cudaStream_t st) {
    const Graph &g = ctx->g;
    const int64_t n = g.n();
    int32_t *minc = nullptr;
    unsigned long long *cnt = nullptr;
    ABC_TRY(ctx->alloc(&minc, (size_t)std::max<int64_t>(n, 1), "component labels"));
    int rc = ctx->alloc(&cnt, 1, "component count");
    unsigned long long h = 0;
    if (!rc) {
        const unsigned gi = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 16));
        cudaMemsetAsync(minc, 0x7f, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1), st);
        cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
        k_cc_roots<<<gi, 256, 0, st>>>(parent, g.new2old, g.nU, n, minc, cnt);
        if (n > 0) k_cc_emit<<<gi, 256, 0, st>>>(g.old2new, parent, minc, g.nU, g.nV, d_lab_u, d_lab_v);
        ctx->stats.launches += 2;
        cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st);
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = ctx->cuda_fail(e, "components");
    }
    ctx->release(minc);
    ctx->release(cnt);
    if (!rc && ncomp) *ncomp = (int64_t)h;
    return rc;
}

int components_compute(abcore_ctx *ctx, int32_t *d_lab_u, int32_t *d_lab_v, int64_t *ncomp) {
    int32_t *parent = nullptr;
    ABC_TRY(ctx->alloc(&parent, (size_t)std::max<int64_t>(ctx->g.n(), 1), "component forest"));
    int rc = cc_hook_base(ctx, parent, nullptr, ctx->stream);
    if (!rc) rc = cc_emit(ctx, parent, d_lab_u, d_lab_v, ncomp, ctx->stream);
    ctx->release(parent);
    return rc;
}
