// C-ABI entry points of the abcore library (declared and documented in include/abcore.h).
// This file validates arguments, moves caller buffers between host and device, and hands the
// work to the builder (build.cu), the peel (peel.cu), the batch scheduler (batch.cu) and the
// serving loop (serve.cu).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"

namespace {

bool ptr_on_device(uint32_t flags) { return (flags & ABCORE_PTR_DEVICE) != 0; }

int require_graph(abcore_ctx *ctx) {
    if (!ctx->g.loaded) return ctx->fail(ABCORE_ENOTLOADED, "no graph loaded");
    return ABCORE_OK;
}

void drop_derived(abcore_ctx *ctx) {
    free_batch(ctx);
    free_serve(ctx);
    free_gfq(ctx);
    free_peel(ctx);
}

int check_sizes(abcore_ctx *ctx, int32_t nU, int32_t nV, int64_t m) {
    if (nU < 0 || nV < 0 || m < 0) return ctx->fail(ABCORE_EINVAL, "negative size");
    if ((int64_t)nU + nV > (int64_t)INT32_MAX - 1)
        return ctx->fail(ABCORE_EINVAL, "nU + nV must be below 2^31 - 1");
    if (m > (int64_t)nU * (int64_t)nV) return ctx->fail(ABCORE_EINVAL, "more edges than vertex pairs");
    return ABCORE_OK;
}

}  // namespace

extern "C" {

int abcore_create(abcore_ctx **out, int device, void *cuda_stream) {
    if (!out) return ABCORE_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return ABCORE_ECUDA;
    }
    if (device < 0 || device >= ndev) return ABCORE_EINVAL;
    abcore_ctx *ctx = new (std::nothrow) abcore_ctx();
    if (!ctx) return ABCORE_ENOMEM;
    ctx->device = device;
    if (const char *lv = getenv("ABCORE_LOG")) ctx->prm.log_level = std::max(0, std::min(2, atoi(lv)));
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete ctx;
        return ABCORE_ECUDA;
    }
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return ABCORE_ECUDA;
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    return ABCORE_OK;
}

int abcore_destroy(abcore_ctx *ctx) {
    if (!ctx) return ABCORE_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_derived(ctx);
    free_graph(ctx);
    for (auto &p : ctx->alloc_sizes) cudaFree(p.first);
    ctx->alloc_sizes.clear();
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return ABCORE_OK;
}

const char *abcore_last_error(abcore_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

int abcore_load_edges(abcore_ctx *ctx, int32_t nU, int32_t nV, int64_t m, const int32_t *eu,
                      const int32_t *ev, uint32_t flags) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(check_sizes(ctx, nU, nV, m));
    if (m > 0 && (!eu || !ev)) return ctx->fail(ABCORE_EINVAL, "NULL edge array");
    ABC_TRY(abcore_sync(ctx));
    drop_derived(ctx);
    const int32_t *deu = eu, *dev = ev;
    int32_t *tu = nullptr, *tv = nullptr;
    if (!ptr_on_device(flags) && m > 0) {
        ABC_TRY(ctx->alloc(&tu, (size_t)m, "edge upload"));
        int rc = ctx->alloc(&tv, (size_t)m, "edge upload");
        if (rc) { ctx->release(tu); return rc; }
        cudaError_t e1 = cudaMemcpyAsync(tu, eu, sizeof(int32_t) * m, cudaMemcpyHostToDevice, ctx->stream);
        cudaError_t e2 = cudaMemcpyAsync(tv, ev, sizeof(int32_t) * m, cudaMemcpyHostToDevice, ctx->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            ctx->release(tu); ctx->release(tv);
            return ctx->cuda_fail(e1 != cudaSuccess ? e1 : e2, "edge upload");
        }
        deu = tu;
        dev = tv;
    }
    int rc = build_graph_from_device_edges(ctx, nU, nV, m, deu, dev);
    cudaStreamSynchronize(ctx->stream);
    ctx->release(tu);
    ctx->release(tv);
    return rc;
}

int abcore_load_csr(abcore_ctx *ctx, int32_t nU, int32_t nV, const int64_t *offU, const int32_t *adjU,
                    const int64_t *offV, const int32_t *adjV, uint32_t flags) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    if (nU < 0 || nV < 0) return ctx->fail(ABCORE_EINVAL, "negative size");
    if (!offU) return ctx->fail(ABCORE_EINVAL, "NULL offU");
    ABC_TRY(abcore_sync(ctx));
    const bool dev = ptr_on_device(flags);
    int64_t m = 0;
    if (dev) ABC_CU(cudaMemcpy(&m, offU + nU, sizeof(int64_t), cudaMemcpyDeviceToHost));
    else m = offU[nU];
    ABC_TRY(check_sizes(ctx, nU, nV, m));
    if (m > 0 && !adjU) return ctx->fail(ABCORE_EINVAL, "NULL adjU");
    drop_derived(ctx);
    int64_t *doff = nullptr, *doffv = nullptr;
    int32_t *dadj = nullptr, *drow = nullptr, *dadjv = nullptr, *drowv = nullptr;
    int rc = ABCORE_OK;
    do {
        if ((rc = ctx->alloc(&doff, (size_t)nU + 1, "csr upload"))) break;
        if ((rc = ctx->alloc(&dadj, (size_t)m, "csr upload"))) break;
        if ((rc = ctx->alloc(&drow, (size_t)m, "csr rows"))) break;
        const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        cudaError_t e = cudaMemcpyAsync(doff, offU, sizeof(int64_t) * (nU + 1), kind, ctx->stream);
        if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(dadj, adjU, sizeof(int32_t) * m, kind, ctx->stream);
        if (e != cudaSuccess) { rc = ctx->cuda_fail(e, "csr upload"); break; }
        if ((rc = check_csr_offsets(ctx, nU, doff, m))) break;
        if ((rc = expand_csr_to_edges(ctx, nU, doff, dadj, m, drow))) break;
        if ((rc = build_graph_from_device_edges(ctx, nU, nV, m, drow, dadj))) break;
        if (offV && (flags & ABCORE_VALIDATE)) {
            if (!adjV && m > 0) { rc = ctx->fail(ABCORE_EINVAL, "NULL adjV"); break; }
            if ((rc = ctx->alloc(&doffv, (size_t)nV + 1, "csr upload"))) break;
            if ((rc = ctx->alloc(&dadjv, (size_t)m, "csr upload"))) break;
            if ((rc = ctx->alloc(&drowv, (size_t)m, "csr rows"))) break;
            e = cudaMemcpyAsync(doffv, offV, sizeof(int64_t) * (nV + 1), kind, ctx->stream);
            if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(dadjv, adjV, sizeof(int32_t) * m, kind, ctx->stream);
            if (e != cudaSuccess) { rc = ctx->cuda_fail(e, "csr upload"); break; }
            if ((rc = check_csr_offsets(ctx, nV, doffv, m))) break;
            if ((rc = expand_csr_to_edges(ctx, nV, doffv, dadjv, m, drowv))) break;
            // U side gives (u = drow, v = dadj); V side gives (v = drowv, u = dadjv)
            if ((rc = compare_edge_sets(ctx, nV, m, drow, dadj, dadjv, drowv))) break;
        }
    } while (0);
    cudaStreamSynchronize(ctx->stream);
    ctx->release(doff); ctx->release(dadj); ctx->release(drow);
    ctx->release(doffv); ctx->release(dadjv); ctx->release(drowv);
    if (rc) free_graph(ctx);
    return rc;
}

int abcore_compute(abcore_ctx *ctx, int32_t alpha, int32_t beta, uint8_t *mask_u, uint8_t *mask_v,
                   uint32_t flags) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    const Graph &g = ctx->g;
    if (alpha < 0 || beta < 0) return ctx->fail(ABCORE_EINVAL, "alpha and beta must be >= 0");
    if ((g.nU > 0 && !mask_u) || (g.nV > 0 && !mask_v)) return ctx->fail(ABCORE_EINVAL, "NULL mask");
    const bool dev = ptr_on_device(flags);
    if ((flags & ABCORE_ASYNC) && !dev) return ctx->fail(ABCORE_EINVAL, "ABCORE_ASYNC needs device pointers");
    ABC_TRY(serve_materialize(ctx));
    if (g.n() == 0) return ABCORE_OK;
    if (ctx->prm.algo == 2 && !ctx->pr.ready) {
        ABC_TRY(peel_finish(ctx));
        ABC_TRY(prepare_pruning(ctx));
    }
    const bool pruned = prefer_pruned(ctx, alpha, beta);
    if (dev) return peel_compute(ctx, alpha, beta, mask_u, mask_v, !(flags & ABCORE_ASYNC), pruned);
    ABC_TRY(peel_finish(ctx));
    ABC_TRY(peel_prepare(ctx));
    uint8_t *su = ctx->w.stage, *sv = ctx->w.stage + g.nU;
    ABC_TRY(peel_compute(ctx, alpha, beta, su, sv, false, pruned));
    if (g.nU) ABC_CU(cudaMemcpyAsync(mask_u, su, (size_t)g.nU, cudaMemcpyDeviceToHost, ctx->stream));
    if (g.nV) ABC_CU(cudaMemcpyAsync(mask_v, sv, (size_t)g.nV, cudaMemcpyDeviceToHost, ctx->stream));
    return peel_finish(ctx);
}

int abcore_compute_batch(abcore_ctx *ctx, int32_t n, const int32_t *alphas, const int32_t *betas,
                         uint8_t *masks_u, uint8_t *masks_v, uint32_t flags) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    const Graph &g = ctx->g;
    if (n < 0) return ctx->fail(ABCORE_EINVAL, "negative pair count");
    if (n == 0) return ABCORE_OK;
    if (!alphas || !betas) return ctx->fail(ABCORE_EINVAL, "NULL threshold array");
    for (int32_t i = 0; i < n; ++i)
        if (alphas[i] < 0 || betas[i] < 0) return ctx->fail(ABCORE_EINVAL, "alpha and beta must be >= 0");
    if ((g.nU > 0 && !masks_u) || (g.nV > 0 && !masks_v)) return ctx->fail(ABCORE_EINVAL, "NULL mask");
    const bool dev = ptr_on_device(flags);
    if ((flags & ABCORE_ASYNC) && !dev) return ctx->fail(ABCORE_EINVAL, "ABCORE_ASYNC needs device pointers");
    ABC_TRY(serve_materialize(ctx));
    if (g.n() == 0) return ABCORE_OK;
    ABC_TRY(peel_finish(ctx));
    if (dev) return batch_compute(ctx, n, alphas, betas, masks_u, masks_v, !(flags & ABCORE_ASYNC));
    uint8_t *du = nullptr, *dv = nullptr;
    ABC_TRY(ctx->alloc(&du, (size_t)n * g.nU, "batch masks"));
    int rc = ctx->alloc(&dv, (size_t)n * g.nV, "batch masks");
    if (!rc) rc = batch_compute(ctx, n, alphas, betas, du, dv, true);
    if (!rc && g.nU) {
        cudaError_t e = cudaMemcpyAsync(masks_u, du, (size_t)n * g.nU, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) rc = ctx->cuda_fail(e, "batch mask download");
    }
    if (!rc && g.nV) {
        cudaError_t e = cudaMemcpyAsync(masks_v, dv, (size_t)n * g.nV, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) rc = ctx->cuda_fail(e, "batch mask download");
    }
    cudaStreamSynchronize(ctx->stream);
    ctx->release(du);
    ctx->release(dv);
    return rc;
}

int abcore_core_numbers(abcore_ctx *ctx, int32_t *core_u, int32_t *core_v, int32_t *max_core, uint32_t flags) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    const Graph &g = ctx->g;
    if ((g.nU > 0 && !core_u) || (g.nV > 0 && !core_v)) return ctx->fail(ABCORE_EINVAL, "NULL core array");
    ABC_TRY(serve_materialize(ctx));
    ABC_TRY(peel_finish(ctx));
    if (g.n() == 0) {
        if (max_core) *max_core = 0;
        return ABCORE_OK;
    }
    ABC_TRY(prepare_pruning(ctx));
    const cudaMemcpyKind kind = ptr_on_device(flags) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (g.nU) ABC_CU(cudaMemcpyAsync(core_u, ctx->pr.core_caller, sizeof(int32_t) * g.nU, kind, ctx->stream));
    if (g.nV)
        ABC_CU(cudaMemcpyAsync(core_v, ctx->pr.core_caller + g.nU, sizeof(int32_t) * g.nV, kind, ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    if (max_core) *max_core = ctx->pr.maxcore;
    return ABCORE_OK;
}

int abcore_components(abcore_ctx *ctx, int32_t *label_u, int32_t *label_v, int64_t *n_components,
                      uint32_t flags) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    const Graph &g = ctx->g;
    if ((g.nU > 0 && !label_u) || (g.nV > 0 && !label_v)) return ctx->fail(ABCORE_EINVAL, "NULL label array");
    ABC_TRY(peel_finish(ctx));
    if (g.n() == 0) {
        if (n_components) *n_components = 0;
        return ABCORE_OK;
    }
    int32_t *du = label_u, *dv = label_v, *tmp = nullptr;
    if (!ptr_on_device(flags)) {
        ABC_TRY(ctx->alloc(&tmp, (size_t)g.n(), "component labels"));
        du = tmp;
        dv = tmp + g.nU;
    }
    int rc = ctx->gfq ? serve_materialize(ctx) : ABCORE_OK;  // queried updates become the CSR first
    if (!rc) rc = ctx->serve ? serve_components(ctx, du, dv, n_components) : components_compute(ctx, du, dv, n_components);
    if (!rc && tmp) {
        cudaError_t e = cudaSuccess;
        if (g.nU) e = cudaMemcpyAsync(label_u, du, sizeof(int32_t) * g.nU, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && g.nV)
            e = cudaMemcpyAsync(label_v, dv, sizeof(int32_t) * g.nV, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = ctx->cuda_fail(e, "component label download");
    }
    ctx->release(tmp);
    return rc;
}

int abcore_alpha_offset(abcore_ctx *ctx, int32_t alpha, int32_t *beta_offset) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    // with alpha = 0 the upper layer alone is a core for every beta: no offset exists
    if (alpha < 1 || !beta_offset) return ctx->fail(ABCORE_EINVAL, "alpha must be >= 1 and beta_offset non-NULL");
    ABC_TRY(serve_materialize(ctx));
    if (ctx->g.n() == 0) {
        *beta_offset = 0;
        return ABCORE_OK;
    }
    return alpha_offset(ctx, alpha, beta_offset);
}

int abcore_default_query(abcore_ctx *ctx, int32_t *delta, int32_t *alpha, int32_t *alpha_off, int32_t *beta) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    if (!delta || !alpha || !alpha_off || !beta) return ctx->fail(ABCORE_EINVAL, "NULL output");
    ABC_TRY(serve_materialize(ctx));
    ABC_TRY(peel_finish(ctx));
    int32_t d = 0;
    if (ctx->g.n() > 0) {
        ABC_TRY(prepare_pruning(ctx));
        d = ctx->pr.maxcore;
    }
    // Section 6: alpha = 0.4 delta and beta = 0.6 alpha_offset, both rounded down (in integers,
    // so no rounding of 0.4 or 0.6 enters); alpha stays at least 1, the smallest alpha for which
    // an offset is defined
    const int32_t a = std::max<int32_t>(1, (int32_t)((2ll * d) / 5));
    int32_t off = 0;
    if (ctx->g.n() > 0) ABC_TRY(alpha_offset(ctx, a, &off));
    *delta = d;
    *alpha = a;
    *alpha_off = off;
    *beta = (int32_t)((3ll * off) / 5);
    return ABCORE_OK;
}

int abcore_community(abcore_ctx *ctx, int32_t layer, int32_t id, int32_t alpha, int32_t beta, uint8_t *mask_u,
                     uint8_t *mask_v, int64_t *size, uint32_t flags) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    const Graph &g = ctx->g;
    if (alpha < 0 || beta < 0) return ctx->fail(ABCORE_EINVAL, "alpha and beta must be >= 0");
    if (layer != 0 && layer != 1) return ctx->fail(ABCORE_EINVAL, "layer must be 0 (U) or 1 (V)");
    if (id < 0 || id >= (layer == 0 ? g.nU : g.nV)) return ctx->fail(ABCORE_EINVAL, "vertex id out of range");
    if ((g.nU > 0 && !mask_u) || (g.nV > 0 && !mask_v)) return ctx->fail(ABCORE_EINVAL, "NULL mask");
    ABC_TRY(serve_materialize(ctx));
    ABC_TRY(peel_finish(ctx));
    int32_t q = 0;
    ABC_CU(cudaMemcpyAsync(&q, g.old2new + (layer == 0 ? 0 : g.nU) + id, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    uint8_t *du = mask_u, *dv = mask_v, *tmp = nullptr;
    if (!ptr_on_device(flags)) {
        ABC_TRY(ctx->alloc(&tmp, (size_t)g.n(), "community masks"));
        du = tmp;
        dv = tmp + g.nU;
    }
    int rc = community(ctx, q, alpha, beta, du, dv, size);
    if (!rc && tmp) {
        cudaError_t e = cudaSuccess;
        if (g.nU) e = cudaMemcpyAsync(mask_u, du, (size_t)g.nU, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && g.nV) e = cudaMemcpyAsync(mask_v, dv, (size_t)g.nV, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = ctx->cuda_fail(e, "community mask download");
    }
    ctx->release(tmp);
    return rc;
}

int abcore_autotune(abcore_ctx *ctx, int32_t n, const int32_t *alphas, const int32_t *betas, uint32_t what,
                    double *best_ms) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    if (n <= 0 || !alphas || !betas) return ctx->fail(ABCORE_EINVAL, "autotune needs at least one (alpha, beta)");
    if (what & ~ABCORE_TUNE_BATCH) return ctx->fail(ABCORE_EINVAL, "unknown autotune target");
    if (!(what & ABCORE_TUNE_BATCH) && n > CTL_RING) return ctx->fail(ABCORE_EINVAL, "at most %d queries per sample", CTL_RING);
    for (int32_t i = 0; i < n; ++i)
        if (alphas[i] < 0 || betas[i] < 0) return ctx->fail(ABCORE_EINVAL, "alpha and beta must be >= 0");
    ABC_TRY(serve_materialize(ctx));
    ABC_TRY(peel_finish(ctx));
    if (ctx->g.n() == 0) {
        if (best_ms) *best_ms = 0;
        return ABCORE_OK;
    }
    return autotune(ctx, n, alphas, betas, what, best_ms);
}

int abcore_measure_atomics(abcore_ctx *ctx, int64_t array_bytes, double *with_return, double *without_return) {
    if (!ctx || !with_return || !without_return) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    if (array_bytes < 4096 || array_bytes > ((int64_t)4 << 30))
        return ctx->fail(ABCORE_EINVAL, "array_bytes must be in [4 KiB, 4 GiB]");
    ABC_TRY(peel_finish(ctx));
    return measure_atomics(ctx, array_bytes, with_return, without_return);
}

int abcore_sync(abcore_ctx *ctx) {
    if (!ctx) return ABCORE_EINVAL;
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(peel_finish(ctx));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    return ABCORE_OK;
}

int abcore_query_edge(abcore_ctx *ctx, int32_t u, int32_t v, int op, int32_t alpha, int32_t beta,
                      uint8_t *in_core) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    if (!in_core) return ctx->fail(ABCORE_EINVAL, "NULL in_core");
    if (u < 0 || u >= ctx->g.nU || v < 0 || v >= ctx->g.nV) return ctx->fail(ABCORE_EINVAL, "vertex id out of range");
    if (op != ABCORE_INSERT && op != ABCORE_DELETE) return ctx->fail(ABCORE_EINVAL, "op must be insert or delete");
    if (alpha < 0 || beta < 0) return ctx->fail(ABCORE_EINVAL, "alpha and beta must be >= 0");
    ABC_TRY(peel_finish(ctx));
    return query_edge(ctx, u, v, op, alpha, beta, in_core);
}

int abcore_serve_start(abcore_ctx *ctx, const int32_t *ta, const int32_t *tb, int32_t nt, int32_t slots) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    if (nt <= 0 || !ta || !tb) return ctx->fail(ABCORE_EINVAL, "need at least one target");
    for (int32_t i = 0; i < nt; ++i)
        if (ta[i] < 0 || tb[i] < 0) return ctx->fail(ABCORE_EINVAL, "alpha and beta must be >= 0");
    if (slots < 1) return ctx->fail(ABCORE_EINVAL, "ring_slots must be >= 1");
    ABC_TRY(peel_finish(ctx));
    return serve_start(ctx, ta, tb, nt, slots);
}

int abcore_serve_submit(abcore_ctx *ctx, const abcore_req *reqs, int32_t n, uint64_t *seq_out) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    if (n < 0 || (n > 0 && !reqs)) return ctx->fail(ABCORE_EINVAL, "bad request array");
    return serve_submit(ctx, reqs, n, seq_out);
}

int abcore_serve_poll(abcore_ctx *ctx, abcore_resp *out, int32_t max, int32_t *n_out) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    if (!n_out || max < 0 || (max > 0 && !out)) return ctx->fail(ABCORE_EINVAL, "bad response buffer");
    return serve_poll(ctx, out, max, n_out);
}

int abcore_serve_stop(abcore_ctx *ctx) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    return serve_stop(ctx);
}

int abcore_get_stats(abcore_ctx *ctx, abcore_stats *out) {
    if (!ctx || !out) return ABCORE_EINVAL;
    *out = ctx->stats;
    out->device_bytes = ctx->dev_bytes;
    out->peak_device_bytes = ctx->peak_bytes;
    int64_t sv[4];
    serve_counters(ctx, sv);
    out->serve_regions = sv[0];
    out->serve_region_vertices = sv[1];
    out->serve_cascades = sv[2];
    out->serve_cascade_vertices = sv[3];
    return ABCORE_OK;
}

int abcore_set_param(abcore_ctx *ctx, const char *name, int64_t value) {
    if (!ctx || !name) return ABCORE_EINVAL;
    ctx->err.clear();
    Params &p = ctx->prm;
    const std::string k(name);
    if (k == "chunk") {
        if (value < 32 || value > (1 << 20)) return ctx->fail(ABCORE_EINVAL, "chunk must be in [32, 2^20]");
        p.chunk = (int)value;
        free_peel(ctx);
        free_batch(ctx);
    } else if (k == "batch_entries") {
        if (value < 128 || value > (1 << 24)) return ctx->fail(ABCORE_EINVAL, "batch_entries must be in [128, 2^24]");
        ABC_TRY(abcore_sync(ctx));
        p.batch_entries = (int)value;
        free_batch(ctx);
    } else if (k == "packed_counts") {
        if (value < 0 || value > 1) return ctx->fail(ABCORE_EINVAL, "packed_counts must be 0 or 1");
        ABC_TRY(abcore_sync(ctx));
        p.packed_counts = (int)value;
        free_batch(ctx);
    } else if (k == "count_swizzle") {
        if (value < 0 || value > 1) return ctx->fail(ABCORE_EINVAL, "count_swizzle must be 0 or 1");
        ABC_TRY(abcore_sync(ctx));
        p.count_swizzle = (int)value;
        free_batch(ctx);
    } else if (k == "round0_variant") {
        if (value < 0 || value > 5) return ctx->fail(ABCORE_EINVAL, "round0_variant must be 0..5");
        ABC_TRY(abcore_sync(ctx));
        p.round0_variant = (int)value;
    } else if (k == "round0_hub") {
        // two layers' tables of ints in one block's shared memory (at most 227 KB)
        if (value < 0 || value > 28672) return ctx->fail(ABCORE_EINVAL, "round0_hub must be 0..28672");
        ABC_TRY(abcore_sync(ctx));
        p.round0_hub = (int)value;
    } else if (k == "pdl") {
        if (value < 0 || value > 1) return ctx->fail(ABCORE_EINVAL, "pdl must be 0 or 1");
        ABC_TRY(abcore_sync(ctx));
        p.pdl = (int)value;
    } else if (k == "round0") {
        if (value < 0 || value > 1) return ctx->fail(ABCORE_EINVAL, "round0 must be 0 or 1");
        ABC_TRY(abcore_sync(ctx));
        p.round0 = (int)value;
    } else if (k == "flush_steps") {
        if (value < 1 || value > (1 << 20)) return ctx->fail(ABCORE_EINVAL, "flush_steps must be in [1, 2^20]");
        ABC_TRY(abcore_sync(ctx));
        p.flush_steps = (int)value;
        free_batch(ctx);
    } else if (k == "batch_entries_small") {
        if (value != 0 && (value < 128 || value > (1 << 24)))
            return ctx->fail(ABCORE_EINVAL, "batch_entries_small must be 0 or in [128, 2^24]");
        ABC_TRY(abcore_sync(ctx));
        p.batch_entries_small = (int)value;
    } else if (k == "local_rounds") {
        if (value < 0 || value > 4096) return ctx->fail(ABCORE_EINVAL, "local_rounds must be 0..4096");
        ABC_TRY(abcore_sync(ctx));
        p.local_rounds = (int)value;
    } else if (k == "grab_div") {
        if (value < 0) return ctx->fail(ABCORE_EINVAL, "grab_div must be >= 0");
        p.grab_div = (int)value;
    } else if (k == "blocks_per_sm") {
        if (value < 0 || value > 32) return ctx->fail(ABCORE_EINVAL, "blocks_per_sm must be in [0, 32]");
        p.blocks_per_sm = (int)value;
        ctx->cascade_blocks = 0;
        free_batch(ctx);
    } else if (k == "mode") {
        if (value < -1 || value > 3) return ctx->fail(ABCORE_EINVAL, "mode must be -1..3");
        p.mode = (int)value;
    } else if (k == "timeout_ms") {
        if (value < 1) return ctx->fail(ABCORE_EINVAL, "timeout_ms must be >= 1");
        p.timeout_ms = value;
    } else if (k == "emit_bitmap_min_pct") {
        if (value < 0 || value > 101) return ctx->fail(ABCORE_EINVAL, "emit_bitmap_min_pct must be 0..101");
        p.emit_bitmap_min_pct = (int)value;
    } else if (k == "emit_scatter_max_pct") {
        if (value < 0 || value > 100) return ctx->fail(ABCORE_EINVAL, "emit_scatter_max_pct must be 0..100");
        p.emit_scatter_max_pct = (int)value;
    } else if (k == "probe_bytes") {
        if (value < 1) return ctx->fail(ABCORE_EINVAL, "probe_bytes must be >= 1");
        p.probe_bytes = (double)value;
    } else if (k == "batch_wave") {
        if (value < 0 || value > 32) return ctx->fail(ABCORE_EINVAL, "batch_wave must be 0..32");
        p.batch_wave = (int)value;
        free_batch(ctx);
    } else if (k == "batch_plain_below") {
        if (value < 0 || value > INT32_MAX) return ctx->fail(ABCORE_EINVAL, "batch_plain_below must be >= 0");
        ABC_TRY(abcore_sync(ctx));
        p.batch_plain_below = (int)value;
        free_batch(ctx);
    } else if (k == "batch_seed") {
        if (value < 0 || value > 1) return ctx->fail(ABCORE_EINVAL, "batch_seed must be 0 or 1");
        p.batch_seed = (int)value;
        free_batch(ctx);
    } else if (k == "hub_degree") {
        if (value < 0) return ctx->fail(ABCORE_EINVAL, "hub_degree must be >= 0");
        ABC_TRY(abcore_sync(ctx));
        p.hub_degree = (int)std::min<int64_t>(value, INT32_MAX);
        free_batch(ctx);
    } else if (k == "timing") {
        if (value < 0 || value > 1) return ctx->fail(ABCORE_EINVAL, "timing must be 0 or 1");
        ABC_TRY(abcore_sync(ctx));
        p.timing = (int)value;
    } else if (k == "timing_kinds") {
        if (value < 0 || value > 0xff) return ctx->fail(ABCORE_EINVAL, "timing_kinds must be in [0, 255]");
        ABC_TRY(abcore_sync(ctx));
        p.timing_kinds = (int)value;
    } else if (k == "serve_inserts") {
        if (value < 1 || value > (1 << 29)) return ctx->fail(ABCORE_EINVAL, "serve_inserts must be in [1, 2^29]");
        p.serve_inserts = value;
    } else if (k == "log_level") {
        if (value < 0 || value > 2) return ctx->fail(ABCORE_EINVAL, "log_level must be 0..2");
        p.log_level = (int)value;
    } else if (k == "query_scope") {
        if (value < 0 || value > 1) return ctx->fail(ABCORE_EINVAL, "query_scope must be 0 (certificate) or 1 (component)");
        p.query_scope = (int)value;
    } else if (k == "algo") {
        if (value < 0 || value > 2) return ctx->fail(ABCORE_EINVAL, "algo must be 0 (auto), 1 (GCC) or 2 (GCC+)");
        p.algo = (int)value;
    } else if (k == "reset_stats") {
        ABC_TRY(abcore_sync(ctx));
        const int32_t mode = ctx->stats.mode, grid = ctx->stats.grid_blocks;
        ctx->stats = abcore_stats{};
        ctx->stats.mode = mode;
        ctx->stats.grid_blocks = grid;
    } else if (k == "debug_stall_slots") {
        if (value < 0 || value > 32) return ctx->fail(ABCORE_EINVAL, "debug_stall_slots must be 0..32");
        p.debug_stall_slots = (int)value;
    } else {
        return ctx->fail(ABCORE_EINVAL, "unknown parameter '%s'", name);
    }
    return ABCORE_OK;
}

int abcore_get_param(abcore_ctx *ctx, const char *name, int64_t *value) {
    if (!ctx || !name || !value) return ABCORE_EINVAL;
    const Params &p = ctx->prm;
    const std::string k(name);
    if (k == "chunk") *value = p.chunk;
    else if (k == "grab_div") *value = p.grab_div;
    else if (k == "local_rounds") *value = p.local_rounds;
    else if (k == "batch_entries_small") *value = p.batch_entries_small;
    else if (k == "batch_entries") *value = p.batch_entries;
    else if (k == "flush_steps") *value = p.flush_steps;
    else if (k == "packed_counts") *value = p.packed_counts;
    else if (k == "round0") *value = p.round0;
    else if (k == "round0_variant") *value = p.round0_variant;
    else if (k == "round0_hub") *value = p.round0_hub;
    else if (k == "count_swizzle") *value = p.count_swizzle;
    else if (k == "pdl") *value = p.pdl;
    else if (k == "blocks_per_sm") *value = p.blocks_per_sm;
    else if (k == "mode") *value = p.mode;
    else if (k == "timeout_ms") *value = p.timeout_ms;
    else if (k == "emit_scatter_max_pct") *value = p.emit_scatter_max_pct;
    else if (k == "emit_bitmap_min_pct") *value = p.emit_bitmap_min_pct;
    else if (k == "probe_bytes") *value = (int64_t)p.probe_bytes;
    else if (k == "batch_wave") *value = p.batch_wave;
    else if (k == "hub_degree") *value = p.hub_degree;
    else if (k == "timing") *value = p.timing;
    else if (k == "timing_kinds") *value = p.timing_kinds;
    else if (k == "serve_inserts") *value = p.serve_inserts;
    else if (k == "algo") *value = p.algo;
    else if (k == "query_scope") *value = p.query_scope;
    else if (k == "batch_seed") *value = p.batch_seed;
    else if (k == "batch_plain_below") *value = p.batch_plain_below;
    else if (k == "log_level") *value = p.log_level;
    else return ctx->fail(ABCORE_EINVAL, "unknown parameter '%s'", name);
    return ABCORE_OK;
}

int abcore_graph_info(abcore_ctx *ctx, int32_t *nU, int32_t *nV, int64_t *m, int32_t *max_deg_u,
                      int32_t *max_deg_v) {
    if (!ctx) return ABCORE_EINVAL;
    ABC_TRY(require_graph(ctx));
    if (nU) *nU = ctx->g.nU;
    if (nV) *nV = ctx->g.nV;
    if (m) *m = ctx->g.m;
    if (max_deg_u) *max_deg_u = ctx->g.maxdegU;
    if (max_deg_v) *max_deg_v = ctx->g.maxdegV;
    return ABCORE_OK;
}

int abcore_export_csr(abcore_ctx *ctx, int64_t *off, int32_t *adj, int32_t *new2old, uint32_t flags) {
    if (!ctx) return ABCORE_EINVAL;
    ctx->err.clear();
    ABC_CU(cudaSetDevice(ctx->device));
    ABC_TRY(require_graph(ctx));
    ABC_TRY(abcore_sync(ctx));
    ABC_TRY(serve_materialize(ctx));
    const Graph &g = ctx->g;
    const cudaMemcpyKind kind = ptr_on_device(flags) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (off) ABC_CU(cudaMemcpyAsync(off, g.off, sizeof(int64_t) * (g.n() + 1), kind, ctx->stream));
    if (adj && g.m) ABC_CU(cudaMemcpyAsync(adj, g.adj, sizeof(int32_t) * 2 * g.m, kind, ctx->stream));
    if (new2old && g.n()) ABC_CU(cudaMemcpyAsync(new2old, g.new2old, sizeof(int32_t) * g.n(), kind, ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    return ABCORE_OK;
}

}  // extern "C"
