// Host-side internals of the abcore library: the context, the device-resident graph, the
// per-query workspace, tuning parameters and the functions each translation unit provides.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/abcore.h"

// Device-side control block of one peel (queue counters, error word, counters for stats).
// Each hot word sits on its own 128-byte line: pushers add to tail, workers add to done, idle
// warps poll both, and tickets come from head.
struct PeelCtl {
    unsigned long long head;   // next queue ticket to hand out
    unsigned long long pad0[15];
    unsigned long long tail;   // queue slots reserved by pushers
    unsigned long long pad1[15];
    unsigned long long done;   // queue slots fully processed
    unsigned long long pad2[15];
    int err;                   // first error code (0 = none)
    int pad3[31];
    unsigned long long l0n;    // candidates found below their bound by the count init (round0)
    unsigned long long pad4[15];
    unsigned long long st[12]; // stat counters, see ST_* below
    unsigned long long ph[4];  // with PeelArgs::phases: globaltimer ns at the cascade's start, when
                               // the last block saw the queue drained, and when the last block
                               // finished the mask emission
};
enum {
    ST_INIT = 0,     // candidate vertices initialised
    ST_PROBES = 1,   // adjacency words read by the in-candidate degree search
    ST_STREAM = 2,   // adjacency entries streamed from initial violators
    ST_ENTRIES = 3,  // adjacency entries read by the cascade
    ST_DECS = 4,     // atomic decrements
    ST_PUSHES = 5,   // vertices queued
    ST_ITEMS = 6,    // cascade work items processed
    ST_STEPS = 7,    // chain steps (batch)
    ST_SDECS = 8,    // atomic decrements issued by the violator stream
    ST_SCAN = 9,     // candidates checked after the violator stream
    ST_HUBDECS = 10, // first-round decrements summed in a block's shared hub table
    ST_HUBFLUSH = 11, // atomics that wrote those tables' sums back to the counts
};

// Everything a peel kernel needs, passed by value.
// marks a U row in the second half of a round0 list entry (the row length is below 2^31)
constexpr long long L0_UPPER = 1ll << 62;

struct PeelArgs {
    const int64_t *off;      // [n+1] row offsets, internal unified ids
    const int32_t *adj;      // [2m] neighbours, each row ascending
    int32_t *cnt;            // count of live candidate neighbours (the atomic target), one slot per
                             // vertex (cnt_slot); with `packed`, uint16 counts, two per 32-bit word
    int32_t packed;
    // count layout: with swz, vertex x's count lives at slot swizzle(x) -- per layer, the odd
    // multiplicative hash of the layer-local id modulo the power-of-two range just above the
    // layer's candidate prefix (U slots [0, swz_mask_u], V slots swz_base_v + [0, swz_mask_v]) --
    // so the counts of the hubs (the lowest ids of the degree-ordered layers, which draw most
    // decrements) fall on different L2 lines and slices instead of a few neighbouring ones, while
    // the candidates' counts stay at least half as dense as in vertex order (and in L2); only
    // candidates' counts are ever touched. Without swz, slot x.
    int32_t swz;
    uint32_t swz_mask_u, swz_mask_v;
    int64_t swz_base_v;
    int32_t *plen;           // [n] row prefix a removed candidate walks (candidate neighbours)
    unsigned long long *q;   // [qcap] work queue of (vertex << 32 | chunk); ~0 = empty slot
    long long qcap;
    PeelCtl *ctl;
    int32_t nU, nV;
    int32_t pU, pV;          // candidate prefixes: U [0,pU), V [nU, nU+pV)
    int32_t cU, cV;          // vertices below these (U [0,cU), V [nU, nU+cV)) are certain members:
                             // never counted, decremented or removed (0 for the plain peel)
    int32_t thrU, thrV;      // alpha, beta
    // U rows' plen counts neighbours below nU + pV_rows; when a batch chain's step has narrowed
    // the V prefix (pV < pV_rows), a fallen U vertex walks only its row's entries below nU + pV,
    // found by a row search that starts from the share frac_rows (0: never narrowed)
    int32_t pV_rows;
    float frac_rows;
    int32_t chunk;           // adjacency entries per work item
    int32_t batch_entries;   // entries one warp walks per batch at most (the rest is re-queued)
    int32_t flush_steps;     // steps a pending push may wait before its warp flushes
    int32_t grab_div;        // queue items per grab = clamp(available / grab_div, 1, 32)
    int32_t local_rounds = 256; // batches one warp may chain on its own pushes (cascade_loop)
    int32_t phases = 0;      // 1: k_cascade records its phase times in PeelCtl::ph
    unsigned long long *trace = nullptr; // diagnostics: the watcher warp samples the queue here
                                         // instead of taking work (cascade_loop)
    int32_t batch_entries_small = 0; // > 0: the batch limit of a warp whose grab left the queue
                                     // nearly empty (fewer than grab_div * 8 items behind it), so
                                     // that warps with nothing to do take over what it defers
    int32_t searchU;         // 1: U counts by searching U rows; 0: by streaming V violators
    int32_t searchV;         // 1: V counts by searching V rows; 0: by streaming U violators
    int32_t hubcutU;         // U ids below this count by search whatever searchU says (and the
    int32_t hubcutV;         // violator stream skips them); V likewise for ids nU + [0, hubcutV)
    unsigned long long timeout_ns;
    // mask emission
    const int32_t *old2new;  // [n] caller id (layer base + id) -> internal id
    const int32_t *new2old;  // [n] internal id -> caller per-layer id
    uint8_t *mask_u, *mask_v;
    int32_t emit;            // 0 none, 1 gather over all vertices, 2 scatter of live candidates
    int32_t skip_zero;       // 1: no decrements toward a layer whose threshold is 0
    // batched chains: a vertex queued during chain step `step` records it in
    // lvl[vertex * lvl_stride + lvl_col] (lvl == nullptr: no record)
    uint8_t *lvl;
    int32_t lvl_stride, lvl_col, step;
    // seeding of a batch chain (seed_col >= 0): a candidate outside the same step's core of the
    // chain whose lvl column that is (its lvl <= step) is known dead and queued whatever its
    // count; dead_own then makes a crossing check the vertex's own lvl column first, so a vertex
    // queued that way is never queued twice
    int32_t dead_own, seed_col;
    int32_t *corev;          // if set, a vertex queued during `step` gets corev[vertex] = step
    // round0: the count init lists its violators in l0 (not the queue); k_round0 walks their rows
    // with atomics that return nothing, and the scan then queues every other candidate below its
    // bound (see peel.cu)
    // (an entry is {first adjacency index, row length | L0_UPPER for a U row})
    int32_t round0;
    longlong2 *l0;
    unsigned long long *removed;  // if set, counts the vertices queued
    // if set: a bitmap over caller ids (bit layer base + caller id) of the candidates this peel
    // removes, set when the cascade takes a fallen vertex's first chunk (round0: when the count
    // init lists it) and read, then cleared, by the caller-order mask gather
    uint32_t *fallen;
    // scatter emission: a bitmap over caller ids (same layout) in which the cascade's last phase
    // sets the survivors' bits; k_expand writes both masks from it and clears it
    uint32_t *sbits;
    // queue closing: flag line of block b at flags[b * 32]; the watcher writes `epoch` (nonzero,
    // new for every cascade) into the lines of blocks [flag_first, flag_first + flag_count)
    uint32_t *flags;
    int32_t flag_first, flag_count;
    uint32_t epoch;
};

struct Params {
    int chunk = 1024;
    int batch_entries = 1024;  // see PeelArgs (1024 kept a 94k-candidate, 18-level cascade 4.5x
                               // faster than 4096; the autotuner may raise it)
    int flush_steps = 4;
    int packed_counts = 1;     // batch chains keep 16-bit counts when every degree fits
    int round0 = 0;            // single peel: walk the initial candidate violators' rows with
                               // no-return atomics when a layer counts by search (k_round0), instead
                               // of queueing them. Pays where the cascade is bound by atomic
                               // throughput (1.5B edges, (64,64): 2.01 -> 1.74 ms); costs where it is
                               // latency-bound (80M edges, (50,50): 0.30 -> 0.53 ms). The autotuner
                               // decides per workload.
    int round0_variant = 0;    // k_round0's compiled (entries per lane per step, blocks per SM) pair:
                               // 0 (8, any), 1 (4, 8), 2 (16, 4), 3 (8, 8); 4: rows four at a time;
                               // 5: rows four at a time, hub decrements summed in shared memory
    int round0_hub = 16384;    // variant 5: hub counts per layer kept in each block's table
    int count_swizzle = 1;     // single peel: counts in the swizzled layout (see PeelArgs::swz); 0: in
                               // vertex order (batch chains always keep vertex order)
    int pdl = 1;               // single peel: launch the kernels after the count init as
                               // programmatic dependents of the one before (each waits for its
                               // predecessor on the device; the launch latency overlaps its tail)
    int grab_div = 0;          // 0 = automatic (resident warps / 8)
    int local_rounds = 256;    // single peel: see PeelArgs::local_rounds
    int batch_entries_small = 512; // single peel: see PeelArgs::batch_entries_small (0: off)
    int threads = 256;
    int blocks_per_sm = 0;     // 0 = occupancy calculator
    int mode = -1;             // -1 auto; else bit 0 searchU, bit 1 searchV
    long long timeout_ms = 4000;
    int emit_scatter_max_pct = 5;  // scatter masks when |P| <= this % of n
    int emit_bitmap_min_pct = 0;   // gather: test removal in the caller-order bitmap when |P| >= this
                                   // % of n (each removal then sets its bit), else read the count
    double probe_bytes = 32.0;     // cost model: bytes charged per search probe
    int batch_plain_below = 0; // abcore_compute_batch: pairs with alpha below this are peeled one by one
                               // with the single (plain) peel instead of in chains; the autotuner
                               // picks it (small alphas leave chains with huge U candidate sets)
    int batch_seed = 0;        // 1: a batch chain is seeded from the finished chain of the next
                               // smaller alpha with the same betas (its non-members are queued at
                               // once); measured no faster on the power-law grids, so off by default
    int batch_wave = 4;        // chains sharing the GPU at once (0 = as many as fit, up to 32);
                               // 4 measured best on a 500M-edge graph (counts stay closer to L2)
    int debug_stall_slots = 0; // test hook: queue slots reserved but never written
    int timing = 0;            // 1: CUDA events around each launch, summed into stats.kernel_ms
    int timing_kinds = 0xff;   // single peel: the kernel kinds (bit ABCORE_K_*) timed. An event
                               // between two kernels costs the step about as much as a launch, so
                               // a measurement may time only the kind it reports.
    int64_t serve_inserts = 1 << 20;  // inserted edges each served target's pool first holds (it
                                      // doubles whenever an insert does not fit)
    int log_level = 0;         // diagnostics on stderr: 0 none, 1 plans and events, 2 also the
                               // batch's per-step timeline (initial value from ABCORE_LOG)
    int query_scope = 0;       // abcore_query_edge: 0 the certificate scope (serving loop), 1 the
                               // paper's scope -- the endpoints' components re-peeled from scratch
    int algo = 0;              // abcore_compute: 0 GCC+ when core numbers are prepared and it has
                               // fewer vertices to peel, else GCC; 1 always GCC; 2 always GCC+
                               // (prepares core numbers on first use)
    int hub_degree = 256;      // candidates of at least this degree always count by search: the
                               // violator stream would hit each of them that many times, and
                               // atomics on one address serialise (0 = off)
};

struct Graph {
    bool loaded = false;
    int32_t nU = 0, nV = 0;
    int64_t m = 0;
    int64_t *off = nullptr;      // [n+1]
    int32_t *adj = nullptr;      // [2m]
    int32_t *new2old = nullptr;  // [n]
    int32_t *old2new = nullptr;  // [n]
    int32_t maxdegU = 0, maxdegV = 0;
    // host tables indexed by degree threshold t (0..maxdeg+1):
    // cnt_ge[t] = #vertices with degree >= t, edges_ge[t] = sum of their degrees
    std::vector<int64_t> cntU_ge, edgesU_ge, cntV_ge, edgesV_ge;
    int64_t n() const { return (int64_t)nU + nV; }
};

constexpr int CTL_RING = 64;  // peels that may be in flight (ABCORE_ASYNC) before a forced wait

// Host-side record of one peel in flight, turned into stats when it finishes.
struct SlotInfo {
    int64_t cands = 0, n = 0;
    int emit = 0;
    int32_t alpha = 0, beta = 0;
    bool timed = false, has_init = false, has_stream = false;
    unsigned kinds = 0;  // kernel kinds timed (bit ABCORE_K_*) when timed
};

struct PeelWork {
    int64_t n = 0, qcap = 0;
    int32_t *cnt = nullptr;        // [cnt_slots] (each layer's power-of-two range, see PeelArgs::swz)
    int64_t cnt_slots = 0;
    int32_t *plen = nullptr;       // [n]
    unsigned long long *q = nullptr;
    PeelCtl *ctl = nullptr;        // [CTL_RING] device control blocks
    PeelCtl *ctl_host = nullptr;   // [CTL_RING] pinned readback
    unsigned long long *trace = nullptr; // [CTL_RING][TRACE_WORDS] queue samples (log level 2)
    bool pending[CTL_RING] = {};
    SlotInfo info[CTL_RING];
    cudaEvent_t ev[CTL_RING][4] = {};  // created on first timed use: before init, after init,
                                       // before cascade, after cascade
    int next = 0, last = -1;
    uint8_t *stage = nullptr;      // [n] staging for host-pointer masks
    bool q_dirty = false;          // queue not known to be all-empty
    uint32_t *flags = nullptr;     // [grid * 32] per-block queue-closed flags (epochs)
    int flag_blocks = 0;
    longlong2 *l0 = nullptr;       // [n] initial candidate violators' rows (round0)
    uint32_t *fallen = nullptr;    // [(n + 31) / 32] removed-candidate bitmap (all zero between peels)
    bool fallen_dirty = false;     // a failed peel may have left bits set
    uint32_t epoch = 0;            // last cascade epoch handed out
};

// Algorithm 2 (GCC+) preprocessing: core numbers (Definition 2) and a copy of the graph whose
// layers are numbered by non-increasing core number, so that for thresholds dl <= dq the vertices
// with core >= dq (certain members) and core >= dl (the only possible members) are prefixes.
struct Pruning {
    bool ready = false;
    Graph gc;                                 // core-ordered graph (degree order breaks ties)
    int32_t *core_caller = nullptr;           // [n] core number by unified caller id
    std::vector<int64_t> coreU_ge, coreV_ge;  // vertices of each layer with core >= t, t = 0..maxcore+1
    int32_t maxcore = 0;
    float decomp_ms = 0.f, layout_ms = 0.f;   // time of the last preparation
};

struct BatchState;
struct ServeState;
struct GfqState;

struct abcore_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    std::string err;
    Graph g;
    Pruning pr;
    PeelWork w;
    Params prm;
    abcore_stats stats{};
    int64_t dev_bytes = 0, peak_bytes = 0;
    int cascade_blocks = 0;
    int init_blocks = 0;     // resident k_init blocks (occupancy x SMs)
    int scan_blocks = 0;     // resident k_scan blocks
    int expand_blocks = 0;   // resident k_expand blocks
    int gather_blocks = 0;   // resident k_gather blocks
    size_t hub_smem = 0;     // dynamic shared memory k_round0_hub has been allowed so far
    BatchState *batch = nullptr;
    ServeState *serve = nullptr;
    GfqState *gfq = nullptr;   // on-the-fly queries with the component scope (query_scope = 1)
    bool pending_async = false;

    // diagnostics at `level` or below the "log_level" parameter, one line on stderr
    void log(int level, const char *fmt, ...) {
        if (prm.log_level < level) return;
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        fprintf(stderr, "[abcore] %s\n", buf);
    }
    int fail(int code, const char *fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
    int cuda_fail(cudaError_t e, const char *what) {
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return fail(ABCORE_ENOMEM, "%s: out of device memory", what);
        }
        return fail(ABCORE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    }
    template <class T>
    int alloc(T **p, size_t count, const char *what) {
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) return cuda_fail(e, what);
        *p = (T *)q;
        dev_bytes += (int64_t)bytes;
        if (dev_bytes > peak_bytes) peak_bytes = dev_bytes;
        alloc_sizes.push_back({q, (int64_t)bytes});
        return ABCORE_OK;
    }
    template <class T>
    void release(T *&p) {
        if (!p) return;
        for (size_t i = 0; i < alloc_sizes.size(); ++i)
            if (alloc_sizes[i].first == (void *)p) {
                dev_bytes -= alloc_sizes[i].second;
                alloc_sizes[i] = alloc_sizes.back();
                alloc_sizes.pop_back();
                break;
            }
        cudaFree((void *)p);
        p = nullptr;
    }
    std::vector<std::pair<void *, int64_t>> alloc_sizes;
};

#define ABC_CU(call)                                              \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call);  \
    } while (0)

#define ABC_TRY(call)                  \
    do {                               \
        int rc_ = (call);              \
        if (rc_ != ABCORE_OK) return rc_; \
    } while (0)

// build.cu -- device CSR builder
int build_graph_from_device_edges(abcore_ctx *ctx, int32_t nU, int32_t nV, int64_t m,
                                  const int32_t *d_eu, const int32_t *d_ev);
int expand_csr_to_edges(abcore_ctx *ctx, int32_t nU, const int64_t *d_off, const int32_t *d_adj,
                        int64_t m, int32_t *d_eu);
int check_csr_offsets(abcore_ctx *ctx, int32_t nrows, const int64_t *d_off, int64_t m);
int compare_edge_sets(abcore_ctx *ctx, int32_t nV, int64_t m, const int32_t *eu1, const int32_t *ev1,
                      const int32_t *eu2, const int32_t *ev2);
void free_graph(abcore_ctx *ctx);  // the loaded graph and everything derived from it
void free_graph_of(abcore_ctx *ctx, Graph &g);
// Build `g` from m distinct caller-id edges; each layer numbered by non-increasing degree, or, with
// d_rank (per unified caller id, values 0..maxrank), by non-increasing rank with ties in degree order.
int build_graph(abcore_ctx *ctx, Graph &g, int32_t nU, int32_t nV, int64_t m, const int32_t *d_eu,
                const int32_t *d_ev, const int32_t *d_rank, int32_t maxrank);
int csr_edges(abcore_ctx *ctx, const Graph &g, int32_t *d_eu, int32_t *d_ev);  // caller-id edge list

// query.cu -- core size, alpha_offset (the paper's default query), community search
int core_size(abcore_ctx *ctx, int32_t alpha, int32_t beta, int64_t *size);
int alpha_offset(abcore_ctx *ctx, int32_t alpha, int32_t *beta_out);
int community(abcore_ctx *ctx, int32_t q_internal, int32_t alpha, int32_t beta, uint8_t *d_mask_u, uint8_t *d_mask_v,
              int64_t *size);

// probe.cu -- random-atomic throughput
int measure_atomics(abcore_ctx *ctx, int64_t array_bytes, double *with_return, double *without_return);

// tune.cu -- autotuner
int autotune(abcore_ctx *ctx, int32_t n, const int32_t *alphas, const int32_t *betas, uint32_t what,
             double *best_ms);

// coredecomp.cu -- core numbers and the GCC+ layout
int prepare_pruning(abcore_ctx *ctx);
void free_pruning(abcore_ctx *ctx);

// peel.cu -- single (alpha, beta)-core
int peel_prepare(abcore_ctx *ctx);
int peel_compute(abcore_ctx *ctx, int32_t alpha, int32_t beta, uint8_t *d_mask_u, uint8_t *d_mask_v,
                 bool sync_and_check, bool pruned = false);
int peel_finish(abcore_ctx *ctx);
bool prefer_pruned(const abcore_ctx *ctx, int32_t alpha, int32_t beta);
void free_peel(abcore_ctx *ctx);
int pick_mode(const abcore_ctx *ctx, int32_t alpha, int32_t beta, int32_t pU, int32_t pV);
int cascade_grid(abcore_ctx *ctx);

// batch.cu
int batch_compute(abcore_ctx *ctx, int32_t n, const int32_t *alphas, const int32_t *betas,
                  uint8_t *d_masks_u, uint8_t *d_masks_v, bool sync_and_check);
void free_batch(abcore_ctx *ctx);

// serve.cu
int query_edge(abcore_ctx *ctx, int32_t u, int32_t v, int op, int32_t alpha, int32_t beta,
               uint8_t *in_core);
int serve_start(abcore_ctx *ctx, const int32_t *ta, const int32_t *tb, int32_t nt, int32_t slots);
int serve_submit(abcore_ctx *ctx, const abcore_req *reqs, int32_t n, uint64_t *seq_out);
int serve_poll(abcore_ctx *ctx, abcore_resp *out, int32_t max, int32_t *n_out);
int serve_stop(abcore_ctx *ctx);
int serve_materialize(abcore_ctx *ctx);  // rebuild the CSR if served or queried updates changed the graph
void free_serve(abcore_ctx *ctx);
void free_gfq(abcore_ctx *ctx);
int serve_components(abcore_ctx *ctx, int32_t *d_lab_u, int32_t *d_lab_v, int64_t *ncomp);
// the serving loop's re-peel counters summed over targets: regions, region vertices, cascades,
// cascaded vertices (zeros when not serving; read while the loop runs they may lag)
void serve_counters(abcore_ctx *ctx, int64_t out[4]);

// components.cu -- connected components (union-find)
int cc_hook_base(abcore_ctx *ctx, int32_t *parent, const uint32_t *tomb, cudaStream_t st,
                 const uint8_t *keep = nullptr);
// the unions of cc_hook_base without resetting the forest first (base rows minus tombstones,
// edges with both endpoints kept)
int cc_hook_rows(abcore_ctx *ctx, int32_t *parent, const uint32_t *tomb, cudaStream_t st, const uint8_t *keep);
int community_compute(abcore_ctx *ctx, const uint8_t *d_alive, int32_t q_internal, uint8_t *d_mask_u,
                      uint8_t *d_mask_v, int64_t *size);
int cc_emit(abcore_ctx *ctx, int32_t *parent, int32_t *d_lab_u, int32_t *d_lab_v, int64_t *ncomp, cudaStream_t st);
int components_compute(abcore_ctx *ctx, int32_t *d_lab_u, int32_t *d_lab_v, int64_t *ncomp);

// The swizzled count layout of a graph with nU upper and nV lower vertices: per layer a
// power-of-two slot range (masks), the V range after the U range; returns the slots needed.
__host__ __device__ static inline int64_t swz_layout(int32_t nU, int32_t nV, uint32_t *mask_u, uint32_t *mask_v,
                                                     int64_t *base_v) {
    auto pow2 = [](int32_t k) {
        uint32_t p = 1;
        while ((int64_t)p < (int64_t)k) p <<= 1;
        return p;
    };
    const uint32_t su = pow2(nU), sv = pow2(nV);
    *mask_u = su - 1;
    *mask_v = sv - 1;
    *base_v = su;
    return (int64_t)su + sv;
}

// Fill a PeelArgs' count layout for candidate prefixes of pU and pV vertices (swizzled when
// `on`); it fits any count array laid out for the whole layers (swz_layout of nU, nV).
__host__ __device__ static inline void set_count_layout(PeelArgs &a, int32_t pU, int32_t pV, bool on) {
    a.swz = on ? 1 : 0;
    swz_layout(pU, pV, &a.swz_mask_u, &a.swz_mask_v, &a.swz_base_v);
}

static inline int64_t cnt_ge(const std::vector<int64_t> &t, int32_t thr) {
    if (thr <= 0) return t.empty() ? 0 : t[0];
    if ((size_t)thr >= t.size()) return 0;
    return t[thr];
}
