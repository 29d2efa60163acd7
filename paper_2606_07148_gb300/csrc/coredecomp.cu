// Core numbers (Definition 2) and the layout that lets the single query prune with them
// (Lemma 1; Algorithm 2, GCC+).
//
// core(x) is the largest k with x in the (k, k)-core. The decomposition peels (k, k)-cores for
// k = 2, 3, ... in one cooperative launch: step k queues every live vertex whose live-neighbour
// count is k - 1 and cascades with bound k on both layers; every vertex that falls during step k
// has core number k - 1 (isolated vertices have 0, and nothing falls at k = 1). Each step reuses
// the single peel's ticket-queue cascade; steps are separated by bounded grid barriers, and the
// launch ends once every vertex has fallen. Within a step only vertices of degree >= k can still
// be live, and they form a prefix of each layer (layers are numbered by non-increasing degree):
// the step scan reads vertices of degree >= k - 1, decrements go to vertices of degree >= k.
//
// GCC+ then needs, for thresholds dl <= dq, the vertices with core >= dq (certain members) and
// core >= dl (possible members) as prefixes: a second copy of the graph is built with each layer
// numbered by non-increasing core number (ties in degree order), and per-layer tables of how many
// vertices have core >= t.
#include <algorithm>
#include <chrono>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "peel_core.cuh"

namespace {

using abc::LaneStats;
using abc::WarpSmem;

constexpr int CORE_THREADS = 256;

struct CoreArgs {
    const int64_t *off;
    const int32_t *adj;
    int32_t nU, nV;
    int32_t *cnt, *plen;
    unsigned long long *q;
    long long qcap;
    PeelCtl *ctl;
    unsigned *bar;
    uint32_t *flags;
    int32_t *core;                  // [n] core number by internal id
    const int64_t *cntU_ge, *cntV_ge;  // vertices with degree >= t (device copies of the host tables)
    int32_t maxdeg;                 // max(maxdegU, maxdegV)
    unsigned long long nonisolated; // vertices of degree >= 1
    unsigned long long *removed;
    int32_t chunk, batch_entries, flush_steps;
    unsigned long long timeout_ns;
};

__global__ void __launch_bounds__(CORE_THREADS) k_core(CoreArgs C) {
    __shared__ WarpSmem smem[CORE_THREADS / 32];
    const int G = gridDim.x;
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t n = (int64_t)C.nU + C.nV;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)G * blockDim.x;

    PeelArgs a{};
    a.off = C.off;
    a.adj = C.adj;
    a.cnt = C.cnt;
    a.plen = C.plen;
    a.q = C.q;
    a.qcap = C.qcap;
    a.ctl = C.ctl;
    a.nU = C.nU;
    a.nV = C.nV;
    a.chunk = C.chunk;
    a.batch_entries = C.batch_entries;
    a.flush_steps = C.flush_steps;
    a.timeout_ns = C.timeout_ns;
    a.skip_zero = 0;
    a.corev = C.core;
    a.removed = C.removed;
    a.flags = C.flags;
    a.flag_first = 0;
    a.flag_count = G;
    const int grab_div = max(1, G * (CORE_THREADS / 32) / 8);
    LaneStats ls;

    // every count starts at the full degree, and a fallen vertex walks its whole row
    for (int64_t x = t0; x < n; x += nthreads) {
        const int32_t d = (int32_t)(__ldg(&C.off[x + 1]) - __ldg(&C.off[x]));
        C.cnt[x] = d;
        C.plen[x] = d;
        C.core[x] = 0;
    }
    if (!abc::group_barrier(C.bar, G, C.ctl, false, C.timeout_ns)) goto out;
    for (int32_t k = 2; k <= C.maxdeg + 1; ++k) {
        // live vertices of degree >= k - 1 whose count is exactly k - 1 fall now
        const int32_t sU = (int32_t)C.cntU_ge[k - 1], sV = (int32_t)C.cntV_ge[k - 1];
        a.pU = (int32_t)C.cntU_ge[k];
        a.pV = (int32_t)C.cntV_ge[k];
        a.thrU = a.thrV = k;
        a.step = k - 1;
        a.epoch = (uint32_t)k;
        {
            int pc = 0;
            const int64_t tot = (int64_t)sU + sV;
            for (int64_t b = t0 - lane; b < tot; b += nthreads) {
                const int64_t i = b + lane;
                bool fall = false;
                int32_t x = 0;
                if (i < tot) {
                    x = i < sU ? (int32_t)i : (int32_t)(C.nU + (i - sU));
                    fall = __ldcg(&C.cnt[x]) == k - 1;
                }
                abc::push_add(a, smem[wib].push, pc, fall, x, fall && __ldcg(&C.plen[x]) > 0 ? 1 : 0, ls);
            }
            abc::push_flush(a, smem[wib].push, pc);
        }
        if (!abc::group_barrier(C.bar, G, C.ctl, false, C.timeout_ns)) goto out;
        (void)abc::cascade_loop(a, smem[wib], ls, grab_div, blockIdx.x == 0 && wib == 0);
        // the barrier's last arriver records whether every vertex has fallen
        if (!abc::group_barrier(C.bar, G, C.ctl, true, C.timeout_ns, C.removed, C.nonisolated)) goto out;
        if (*(volatile unsigned *)(C.bar + 16)) break;
    }
out:
    abc::flush_stats(a, ls);
}

__global__ void k_core_max(const int32_t *a, int64_t n, int *out) {
    int mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, a[i]);
    for (int d = 16; d >= 1; d >>= 1) mx = max(mx, __shfl_xor_sync(ABC_FULL, mx, d));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

__global__ void k_core_by_caller(const int32_t *core, const int32_t *new2old, int32_t nU, int64_t n, int32_t *out) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        out[__ldg(&new2old[x]) + (x >= nU ? nU : 0)] = core[x];
}

// per layer: hist[t] = vertices with core number t
__global__ void k_core_hist(const int32_t *core_caller, int32_t nU, int64_t n, int32_t maxcore, int64_t *histU,
                            int64_t *histV) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = min(core_caller[i], maxcore);
        atomicAdd((unsigned long long *)(i < nU ? &histU[c] : &histV[c]), 1ull);
    }
}

}  // namespace

void free_pruning(abcore_ctx *ctx) {
    Pruning &p = ctx->pr;
    free_graph_of(ctx, p.gc);
    ctx->release(p.core_caller);
    p.coreU_ge.clear();
    p.coreV_ge.clear();
    p.maxcore = 0;
    p.ready = false;
}

// Core numbers of the loaded graph into core_caller (unified caller ids). The peel workspace
// (counts, prefixes, queue) is borrowed.
static int core_decompose(abcore_ctx *ctx, int32_t *core_caller, int32_t *maxcore_out) {
    const Graph &g = ctx->g;
    const int64_t n = g.n();
    ABC_TRY(peel_finish(ctx));
    ABC_TRY(peel_prepare(ctx));
    PeelWork &w = ctx->w;
    int32_t *core = nullptr;
    int64_t *dU = nullptr, *dV = nullptr;
    unsigned *bar = nullptr;
    uint32_t *flags = nullptr;
    unsigned long long *removed = nullptr;
    int rc = ABCORE_OK;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_core, CORE_THREADS, 0);
    const int grid = std::max(per_sm, 1) * ctx->num_sms;
    const int32_t maxdeg = std::max(g.maxdegU, g.maxdegV);
    // degree tables padded to maxdeg + 2 entries on both layers
    std::vector<int64_t> hU((size_t)maxdeg + 2, 0), hV((size_t)maxdeg + 2, 0);
    for (int32_t t = 0; t <= maxdeg + 1; ++t) {
        hU[t] = cnt_ge(g.cntU_ge, t);
        hV[t] = cnt_ge(g.cntV_ge, t);
    }
    const unsigned long long nonisolated = (unsigned long long)(cnt_ge(g.cntU_ge, 1) + cnt_ge(g.cntV_ge, 1));
#define STEP(x)            \
    do {                   \
        rc = (x);          \
        if (rc) goto done; \
    } while (0)
    STEP(ctx->alloc(&core, (size_t)std::max<int64_t>(n, 1), "core numbers"));
    STEP(ctx->alloc(&dU, hU.size(), "degree table"));
    STEP(ctx->alloc(&dV, hV.size(), "degree table"));
    STEP(ctx->alloc(&bar, 64, "core barrier"));
    STEP(ctx->alloc(&flags, (size_t)grid * 32, "core close flags"));
    STEP(ctx->alloc(&removed, 1, "core removed"));
    {
        ABC_CU(cudaMemcpyAsync(dU, hU.data(), sizeof(int64_t) * hU.size(), cudaMemcpyHostToDevice, ctx->stream));
        ABC_CU(cudaMemcpyAsync(dV, hV.data(), sizeof(int64_t) * hV.size(), cudaMemcpyHostToDevice, ctx->stream));
        ABC_CU(cudaMemsetAsync(bar, 0, 64 * sizeof(unsigned), ctx->stream));
        ABC_CU(cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (size_t)grid * 32, ctx->stream));
        ABC_CU(cudaMemsetAsync(removed, 0, sizeof(unsigned long long), ctx->stream));
        PeelCtl *ctl = w.ctl + w.next;  // a free slot of the peel's control ring
        ABC_CU(cudaMemsetAsync(ctl, 0, sizeof(PeelCtl), ctx->stream));
        if (w.q_dirty) {
            ABC_CU(cudaMemsetAsync(w.q, 0xff, sizeof(unsigned long long) * (size_t)w.qcap, ctx->stream));
            w.q_dirty = false;
        }
        CoreArgs C{};
        C.off = g.off;
        C.adj = g.adj;
        C.nU = g.nU;
        C.nV = g.nV;
        C.cnt = w.cnt;
        C.plen = w.plen;
        C.q = w.q;
        C.qcap = w.qcap;
        C.ctl = ctl;
        C.bar = bar;
        C.flags = flags;
        C.core = core;
        C.cntU_ge = dU;
        C.cntV_ge = dV;
        C.maxdeg = maxdeg;
        C.nonisolated = nonisolated;
        C.removed = removed;
        C.chunk = std::max(ctx->prm.chunk, 32);
        C.batch_entries = ctx->prm.batch_entries;
        C.flush_steps = ctx->prm.flush_steps;
        C.timeout_ns = (unsigned long long)ctx->prm.timeout_ms * 1000000ull;
        void *args[] = {&C};
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(CORE_THREADS);
        cfg.stream = ctx->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ABC_CU(cudaLaunchKernelExC(&cfg, (const void *)k_core, args));
        ctx->stats.launches++;
        int err = 0;
        ABC_CU(cudaMemcpyAsync(&err, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        ABC_CU(cudaStreamSynchronize(ctx->stream));
        if (err) {
            w.q_dirty = true;
            rc = ctx->fail(err == ABCORE_ETIMEDOUT ? ABCORE_ETIMEDOUT : err, "core decomposition: device error %d", err);
            goto done;
        }
        const unsigned gi = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 16));
        k_core_by_caller<<<gi, 256, 0, ctx->stream>>>(core, g.new2old, g.nU, n, core_caller);
        int *d_max = nullptr;
        STEP(ctx->alloc(&d_max, 1, "max core"));
        cudaMemsetAsync(d_max, 0, sizeof(int), ctx->stream);
        int h_max = 0;
        if (n > 0) k_core_max<<<gi, 256, 0, ctx->stream>>>(core, n, d_max);
        cudaMemcpyAsync(&h_max, d_max, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
        const cudaError_t e = cudaStreamSynchronize(ctx->stream);
        ctx->release(d_max);
        if (e != cudaSuccess) {
            rc = ctx->cuda_fail(e, "core decomposition");
            goto done;
        }
        *maxcore_out = h_max;
    }
done:
    cudaStreamSynchronize(ctx->stream);
    ctx->release(core);
    ctx->release(dU);
    ctx->release(dV);
    ctx->release(bar);
    ctx->release(flags);
    ctx->release(removed);
    return rc;
#undef STEP
}

int prepare_pruning(abcore_ctx *ctx) {
    Pruning &p = ctx->pr;
    if (p.ready) return ABCORE_OK;
    free_pruning(ctx);
    const Graph &g = ctx->g;
    const int64_t n = g.n();
    const auto t0 = std::chrono::steady_clock::now();
    ABC_TRY(ctx->alloc(&p.core_caller, (size_t)std::max<int64_t>(n, 1), "core numbers"));
    int32_t maxcore = 0;
    int rc = core_decompose(ctx, p.core_caller, &maxcore);
    if (rc) {
        free_pruning(ctx);
        return rc;
    }
    const auto t1 = std::chrono::steady_clock::now();
    // per-layer tables: vertices with core >= t
    int64_t *hist = nullptr;
    rc = ctx->alloc(&hist, 2 * ((size_t)maxcore + 1), "core histogram");
    if (!rc) {
        std::vector<int64_t> h(2 * ((size_t)maxcore + 1), 0);
        cudaMemsetAsync(hist, 0, sizeof(int64_t) * h.size(), ctx->stream);
        const unsigned gi = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 16));
        if (n > 0) k_core_hist<<<gi, 256, 0, ctx->stream>>>(p.core_caller, g.nU, n, maxcore, hist, hist + maxcore + 1);
        cudaMemcpyAsync(h.data(), hist, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost, ctx->stream);
        const cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = ctx->cuda_fail(e, "core histogram");
        p.coreU_ge.assign((size_t)maxcore + 2, 0);
        p.coreV_ge.assign((size_t)maxcore + 2, 0);
        for (int32_t t = maxcore; t >= 0; --t) {
            p.coreU_ge[t] = p.coreU_ge[t + 1] + h[t];
            p.coreV_ge[t] = p.coreV_ge[t + 1] + h[maxcore + 1 + t];
        }
    }
    ctx->release(hist);
    // the graph again, each layer numbered by non-increasing core number
    int32_t *eu = nullptr, *ev = nullptr;
    if (!rc) rc = ctx->alloc(&eu, (size_t)std::max<int64_t>(g.m, 1), "core layout edges");
    if (!rc) rc = ctx->alloc(&ev, (size_t)std::max<int64_t>(g.m, 1), "core layout edges");
    if (!rc) rc = csr_edges(ctx, g, eu, ev);
    if (!rc) rc = build_graph(ctx, p.gc, g.nU, g.nV, g.m, eu, ev, p.core_caller, maxcore);
    ctx->release(eu);
    ctx->release(ev);
    if (rc) {
        free_pruning(ctx);
        return rc;
    }
    const auto t2 = std::chrono::steady_clock::now();
    p.maxcore = maxcore;
    p.decomp_ms = std::chrono::duration<float, std::milli>(t1 - t0).count();
    p.layout_ms = std::chrono::duration<float, std::milli>(t2 - t1).count();
    p.ready = true;
    return ABCORE_OK;
}
