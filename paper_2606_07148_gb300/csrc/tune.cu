// Autotuner: picks the launch and cascade parameters by measuring them on the loaded graph.
//
// The peel's speed depends on the graph and the thresholds in ways a fixed rule misses: how many
// blocks share an SM (occupancy against per-warp registers), how many adjacency entries one
// work item carries (the unit a warp takes from the queue), how long a row must be before its
// count is found by search rather than by the violator stream (the hub threshold), how a layer's
// counts are taken at all (the stream/search switch, weighted by the cost of one search probe),
// and when survivors are scattered into zeroed masks rather than gathered. The batch adds how
// many chains share the GPU at once, below which alpha pairs are left to single peels, and
// whether chains are seeded from smaller-alpha chains. The tuner runs coordinate descent over these, timing each
// setting with CUDA events on the context's stream on a sample of (alpha, beta) queries, with the
// L2 flushed (a 256 MB write) before every timed run, and leaves the fastest setting on the
// context. Every setting computes the same cores: only time changes.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace {

struct Knob {
    const char *name;
    std::vector<int64_t> values;
};

struct Timer {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    uint8_t *flush = nullptr;
    size_t flush_bytes = 0;
};

// One timed pass over the sample: best of `reps` runs of the whole sample, L2 flushed before
// each run. Returns milliseconds, or a negative value on error (ctx->err set).
double time_sample(abcore_ctx *ctx, Timer &T, bool batch, int32_t n, const int32_t *al, const int32_t *be,
                   uint8_t *mu, uint8_t *mv, int reps) {
    // warm-up (plans, graphs, workspaces)
    if (batch) {
        if (batch_compute(ctx, n, al, be, mu, mv, true)) return -1;
    } else {
        for (int32_t i = 0; i < n; ++i)
            if (peel_compute(ctx, al[i], be[i], mu, mv, false, prefer_pruned(ctx, al[i], be[i]))) return -1;
        if (peel_finish(ctx)) return -1;
    }
    double best = 1e30;
    for (int r = 0; r < reps; ++r) {
        if (cudaMemsetAsync(T.flush, r & 0xff, T.flush_bytes, ctx->stream) != cudaSuccess) return -1;
        cudaEventRecord(T.e0, ctx->stream);
        if (batch) {
            if (batch_compute(ctx, n, al, be, mu, mv, false)) return -1;
        } else {
            for (int32_t i = 0; i < n; ++i)
                if (peel_compute(ctx, al[i], be[i], mu, mv, false, prefer_pruned(ctx, al[i], be[i]))) return -1;
        }
        cudaEventRecord(T.e1, ctx->stream);
        if (batch) {
            if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return -1;
        } else if (peel_finish(ctx)) {
            return -1;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, T.e0, T.e1);
        best = std::min(best, (double)ms);
    }
    return best;
}

}  // namespace

int autotune(abcore_ctx *ctx, int32_t n, const int32_t *alphas, const int32_t *betas, uint32_t what,
             double *best_ms) {
    const Graph &g = ctx->g;
    const bool batch = (what & ABCORE_TUNE_BATCH) != 0;
    std::vector<Knob> knobs;
    if (batch) {
        // splits between single peels and chains at the sample's own alphas: none, then below
        // each of its smallest distinct alphas in turn
        std::vector<int64_t> split{0};
        std::vector<int32_t> al(alphas, alphas + n);
        std::sort(al.begin(), al.end());
        al.erase(std::unique(al.begin(), al.end()), al.end());
        for (size_t i = 0; i + 1 < al.size() && i < 6; ++i) split.push_back((int64_t)al[i] + 1);
        knobs.push_back({"batch_plain_below", split});
        knobs.push_back({"batch_seed", {0, 1}});
        knobs.push_back({"batch_wave", {2, 4, 8, 16}});
        knobs.push_back({"blocks_per_sm", {0, 2, 3}});
        knobs.push_back({"chunk", {512, 1024, 2048}});
    } else {
        knobs.push_back({"blocks_per_sm", {0, 3, 2}});
        knobs.push_back({"chunk", {256, 512, 1024, 2048}});
        knobs.push_back({"grab_div", {0, 64, 512}});
        knobs.push_back({"batch_entries", {1024, 4096, 16384}});
        knobs.push_back({"batch_entries_small", {0, 512, 1024}});
        knobs.push_back({"flush_steps", {1, 4, 16}});
        knobs.push_back({"hub_degree", {0, 64, 256, 1024}});
        knobs.push_back({"probe_bytes", {12, 16, 24, 32, 64}});
        knobs.push_back({"emit_scatter_max_pct", {0, 5, 25}});
        knobs.push_back({"emit_bitmap_min_pct", {0, 50, 101}});
        knobs.push_back({"round0", {0, 1}});
        knobs.push_back({"round0_variant", {0, 2, 4, 5}});
        knobs.push_back({"round0_hub", {8192, 16384, 28672}});
    }
    Timer T;
    uint8_t *mu = nullptr, *mv = nullptr;
    const size_t mbytes = batch ? (size_t)n : 1;
    ABC_TRY(ctx->alloc(&mu, mbytes * (size_t)std::max(g.nU, 1), "tuning masks"));
    int rc = ctx->alloc(&mv, mbytes * (size_t)std::max(g.nV, 1), "tuning masks");
    T.flush_bytes = (size_t)256 << 20;
    if (!rc) rc = ctx->alloc(&T.flush, T.flush_bytes, "L2 flush buffer");
    if (!rc && (cudaEventCreate(&T.e0) != cudaSuccess || cudaEventCreate(&T.e1) != cudaSuccess))
        rc = ctx->fail(ABCORE_ECUDA, "autotune: event creation failed");
    const int reps = 5;
    double best = -1;
    if (!rc) {
        best = time_sample(ctx, T, batch, n, alphas, betas, mu, mv, reps);
        if (best < 0) rc = ctx->err.empty() ? ctx->fail(ABCORE_ECUDA, "autotune: a timed run failed") : ABCORE_ECUDA;
    }
    // coordinate descent, up to three sweeps
    for (int sweep = 0; sweep < 3 && !rc; ++sweep) {
        bool moved = false;
        for (const Knob &k : knobs) {
            int64_t cur = 0;
            abcore_get_param(ctx, k.name, &cur);
            int64_t keep = cur;
            for (int64_t v : k.values) {
                if (v == cur) continue;
                if ((rc = abcore_set_param(ctx, k.name, v))) break;
                const double t = time_sample(ctx, T, batch, n, alphas, betas, mu, mv, reps);
                if (t < 0) {
                    rc = ABCORE_ECUDA;
                    break;
                }
                // a margin keeps timing noise from moving settings (a batch of chains varies
                // more from run to run than a single peel)
                if (t < best * (batch ? 0.95 : 0.985)) {
                    best = t;
                    keep = v;
                    moved = true;
                }
            }
            if (rc) break;
            rc = abcore_set_param(ctx, k.name, keep);
            if (rc) break;
        }
        if (!moved) break;
    }
    if (T.e0) cudaEventDestroy(T.e0);
    if (T.e1) cudaEventDestroy(T.e1);
    cudaStreamSynchronize(ctx->stream);
    ctx->release(mu);
    ctx->release(mv);
    ctx->release(T.flush);
    if (!rc && best_ms) *best_ms = best;
    return rc;
}
