/*
 * abcore.h -- exact (alpha, beta)-core computation on bipartite graphs, on one GB300 (sm_103a).
 *
 * A bipartite graph G = (U u L, E) with E a subset of U x L (Section 3 of the paper) is loaded
 * once onto the GPU. The (alpha, beta)-core (Definition 1) is the maximal vertex set in which
 * every upper (U) vertex has at least alpha neighbours and every lower (L, here "V") vertex
 * has at least beta neighbours inside the set. It is unique, so every result of this library
 * is exact and bit-for-bit reproducible: a membership mask byte is 1 for a member, 0 otherwise.
 *
 * Conventions for every call:
 *  - Return value: ABCORE_OK (0) or a negative ABCORE_E* code. After an error,
 *    abcore_last_error(ctx) describes it; the context stays usable unless the code is
 *    ABCORE_ECUDA.
 *  - Vertex ids at the interface are per layer: u in [0, nU), v in [0, nV).
 *  - Pointer arguments are host pointers unless the call's flags contain ABCORE_PTR_DEVICE, in
 *    which case they are device pointers on the context's device. The caller owns every buffer
 *    it passes; the library copies inputs and never keeps a caller pointer after returning.
 *  - All device work is ordered on the context's stream. Calls block until their results are
 *    ready, except abcore_compute / abcore_compute_batch with ABCORE_PTR_DEVICE | ABCORE_ASYNC,
 *    which return once the work is enqueued; abcore_sync then waits and reports its status.
 *  - A context is not thread-safe: use one context per host thread.
 */
#ifndef ABCORE_H
#define ABCORE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define ABCORE_OK           0
#define ABCORE_EINVAL     (-1)  /* bad argument: negative threshold, id out of range, ...      */
#define ABCORE_ENOTLOADED (-2)  /* no graph has been loaded into the context                  */
#define ABCORE_ENOMEM     (-3)  /* device or host allocation failed                           */
#define ABCORE_EEXIST     (-4)  /* insert of an edge already present / duplicate input edge   */
#define ABCORE_ENOENT     (-5)  /* delete of an edge that is not present                      */
#define ABCORE_ECUDA      (-6)  /* a CUDA runtime call failed                                 */
#define ABCORE_ETIMEDOUT  (-7)  /* a bounded device-side wait expired; the work was abandoned */
#define ABCORE_EBUSY      (-8)  /* request ring full; retry after polling completions         */

/* ---- flags ----------------------------------------------------------------------------- */
#define ABCORE_PTR_HOST   0u    /* pointer arguments are host memory (default)               */
#define ABCORE_PTR_DEVICE 1u    /* pointer arguments are device memory of the ctx's device   */
#define ABCORE_VALIDATE   2u    /* load: check the second CSR layer against the first         */
#define ABCORE_ASYNC      4u    /* compute with device pointers: return after enqueueing      */

/* ---- edge update kinds (abcore_query_edge, abcore_req.op) ------------------------------ */
#define ABCORE_INSERT 0
#define ABCORE_DELETE 1

typedef struct abcore_ctx abcore_ctx;

/* Kernel kinds, indexing abcore_stats.kernel_launches / kernel_ms. */
#define ABCORE_K_INIT    0  /* candidate counts (row search or full degree)              */
#define ABCORE_K_STREAM  1  /* streaming the initial violators' rows                     */
#define ABCORE_K_CASCADE 2  /* work-queue cascade plus mask emission                     */
#define ABCORE_K_BATCH   3  /* batched chains                                            */
#define ABCORE_K_SERVE   4  /* on-the-fly queries and the serving loop                   */
#define ABCORE_K_KINDS   8

/* Device counters accumulated over compute calls since the context was created or since
 * abcore_set_param(ctx, "reset_stats", 1), plus memory figures. kernel_ms is filled only while
 * the "timing" parameter is 1: CUDA events are then recorded on the context's stream around
 * each launch. */
typedef struct {
    int64_t peels;           /* single peels run (a batch counts each chain step)             */
    int64_t candidates;      /* sum of |P|: vertices meeting their bound on full degree        */
    int64_t init_vertices;   /* candidates whose live-candidate count was set                  */
    int64_t search_probes;   /* 32-byte adjacency sectors read while searching candidate rows  */
    int64_t stream_entries;  /* adjacency entries streamed from the initial violators' rows    */
    int64_t entries;         /* adjacency entries read by the cascade                          */
    int64_t decrements;      /* atomic count decrements, all kernels                           */
    int64_t stream_decrements; /* of which issued while streaming the initial violators' rows  */
    int64_t scanned;         /* candidates checked for violations after that stream            */
    int64_t pushes;          /* vertices queued for removal                                    */
    int64_t items;           /* cascade work items (row chunks) processed                      */
    int64_t emit_gathered;   /* mask bytes written by a gather over every vertex               */
    int64_t emit_scattered;  /* candidates checked by a scatter of survivors into zeroed masks */
    int64_t mask_zeroed;     /* mask bytes written from the survivor bitmap after a scatter    */
    int64_t launches;        /* kernels launched                                               */
    int64_t kernel_launches[ABCORE_K_KINDS];  /* timed launches per kernel kind                */
    double kernel_ms[ABCORE_K_KINDS];         /* device milliseconds per kernel kind           */
    int32_t mode;            /* last peel: bit 0 U counts by search, bit 1 V counts by search  */
    int32_t grid_blocks;     /* blocks of the persistent cascade launch                        */
    int64_t device_bytes;    /* device memory held by the context now                          */
    int64_t peak_device_bytes;
    int64_t round0_rows;     /* candidates already below their bound when counted, whose rows
                                the first round walked without returns ("round0")              */
    int64_t scope_queries;   /* on-the-fly queries answered with the component scope            */
    int64_t scope_vertices;  /* vertices those queries re-peeled (their components' sizes)      */
    int64_t serve_regions;   /* served inserts that grew a region to peel (summed over targets) */
    int64_t serve_region_vertices; /* vertices in those regions                                 */
    int64_t serve_cascades;  /* served deletes that cascaded inside a target core              */
    int64_t serve_cascade_vertices; /* vertices those cascades removed                          */
    int64_t hub_decrements;  /* of stream_decrements, those summed in a block's shared-memory hub
                                table (round0_variant 5) instead of going to L2 one by one      */
    int64_t hub_flushes;     /* L2 atomics that wrote those tables back to the counts           */
} abcore_stats;

/* ---- lifecycle ------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t to order all work
 * on (cudaStreamLegacy and cudaStreamPerThread are accepted), or NULL for a stream the context
 * creates and owns. Device buffers passed to later calls must be ready in that stream's order.
 * *out receives the context. */
int abcore_create(abcore_ctx **out, int device, void *cuda_stream);

/* Release every device and host resource of the context. NULL is accepted. */
int abcore_destroy(abcore_ctx *ctx);

/* Text of the last error on this context ("" if none). Valid until the next call on ctx. */
const char *abcore_last_error(abcore_ctx *ctx);

/* ---- graph loading (Section 3: CSR storage; Section 4.1: flat continuous ids) ----------- */

/* Load a graph from m distinct edges (eu[i], ev[i]), eu[i] in [0,nU), ev[i] in [0,nV).
 * The device CSR builder stores both layers (U->V rows and V->U rows, int64 offsets, int32
 * ids, each row sorted), renumbering vertices within each layer by non-increasing degree;
 * results are always reported in the caller's ids. Replaces any previously loaded graph.
 * Errors: EINVAL (negative sizes, id out of range), EEXIST (an edge given twice), ENOMEM. */
int abcore_load_edges(abcore_ctx *ctx, int32_t nU, int32_t nV, int64_t m,
                      const int32_t *eu, const int32_t *ev, uint32_t flags);

/* Load a graph given as the CSR of the U layer: offU[nU+1] (offU[0] = 0, non-decreasing),
 * adjU[offU[nU]] holding V ids. offV/adjV (the V layer, U ids) may be NULL; when given with
 * ABCORE_VALIDATE they must describe the same edge set, else EINVAL. Rows need not be
 * sorted. Same errors as abcore_load_edges. */
int abcore_load_csr(abcore_ctx *ctx, int32_t nU, int32_t nV,
                    const int64_t *offU, const int32_t *adjU,
                    const int64_t *offV, const int32_t *adjV, uint32_t flags);

/* ---- (alpha, beta)-core computation (Definition 1; Algorithm 1, the GCC peel) ----------- */

/* Compute the (alpha, beta)-core of the loaded graph. mask_u[nU] and mask_v[nV] receive one
 * byte per vertex: 1 if in the core, else 0. alpha, beta >= 0 (0 = no constraint on that
 * layer). Errors: EINVAL (negative threshold, NULL mask), ENOTLOADED, ETIMEDOUT. */
int abcore_compute(abcore_ctx *ctx, int32_t alpha, int32_t beta,
                   uint8_t *mask_u, uint8_t *mask_v, uint32_t flags);

/* Core numbers (Definition 2: the largest k with the vertex in the (k, k)-core) of every vertex,
 * in the caller's ids: core_u[nU], core_v[nV]; *max_core (may be NULL) receives the largest.
 * The first call after a graph is loaded (or changed by served updates) runs the preprocessing
 * of Algorithm 2 (GCC+) on the device: the core decomposition, then a second copy of the graph
 * with each layer numbered by non-increasing core number (another CSR's worth of device
 * memory). abcore_compute may then prune with Lemma 1: vertices with core < min(alpha, beta)
 * are out, those with core >= max(alpha, beta) are in, and only the rest are peeled. The
 * "algo" parameter decides: 0 (default) prunes a query only when that leaves fewer vertices to
 * peel than the plain peel's degree prefixes; 1 never prunes; 2 always prunes, and prepares
 * the core numbers itself on first use. Errors: EINVAL (NULL array), ENOTLOADED, ENOMEM,
 * ETIMEDOUT. */
int abcore_core_numbers(abcore_ctx *ctx, int32_t *core_u, int32_t *core_v, int32_t *max_core,
                        uint32_t flags);

/* alpha_offset of the paper's default query (Section 6): the largest beta >= 1 whose
 * (alpha, beta)-core is non-empty, or 0 if none is. Found by binary search over beta with the
 * peel (the core shrinks as beta grows, by the nested property). With the default query
 * alpha = 0.4 * delta (delta = the largest core number, abcore_core_numbers' max_core) and
 * beta = 0.6 * alpha_offset. alpha must be at least 1 (with alpha = 0 the upper layer alone is
 * a core for every beta). Errors: EINVAL, ENOTLOADED, ETIMEDOUT. */
int abcore_alpha_offset(abcore_ctx *ctx, int32_t alpha, int32_t *beta_offset);

/* The paper's default query (Section 6): delta is the largest core number (Definition 2),
 * alpha = floor(0.4 * delta) (at least 1), alpha_offset is abcore_alpha_offset(alpha), and
 * beta = floor(0.6 * alpha_offset). The products are taken in integers (2 * delta / 5 and
 * 3 * alpha_offset / 5), so the results are exact. Runs the core decomposition on first use, as
 * abcore_core_numbers does. An empty graph gives delta = 0, alpha = 1, alpha_offset = beta = 0.
 * Errors: EINVAL (a NULL output), ENOTLOADED, ENOMEM, ETIMEDOUT. */
int abcore_default_query(abcore_ctx *ctx, int32_t *delta, int32_t *alpha, int32_t *alpha_offset,
                         int32_t *beta);

/* Community search (Section 5, the Remark after GFQ): the connected component of the
 * (alpha, beta)-core that contains vertex `id` of layer `layer` (0 = U, 1 = V). mask_u[nU] and
 * mask_v[nV] receive 1 for its members; all zero if the vertex is not in the core. *size (may
 * be NULL) receives the member count. Errors: EINVAL (bad layer, id or threshold, NULL mask),
 * ENOTLOADED, ENOMEM, ETIMEDOUT. */
int abcore_community(abcore_ctx *ctx, int32_t layer, int32_t id, int32_t alpha, int32_t beta,
                     uint8_t *mask_u, uint8_t *mask_v, int64_t *size, uint32_t flags);

/* Compute n cores at once (Lemma 1 and Algorithm 2 generalised: pairs sharing alpha are peeled
 * as one chain of increasing beta, each core seeded from the one containing it). Pair i is
 * (alphas[i], betas[i]); its masks are rows i of masks_u (n x nU, row-major) and masks_v
 * (n x nV). Results equal n separate abcore_compute calls, whatever the pair order. The
 * launch is captured once as a CUDA graph per pair list and replayed on later calls.
 * Errors: as abcore_compute. */
int abcore_compute_batch(abcore_ctx *ctx, int32_t n, const int32_t *alphas, const int32_t *betas,
                         uint8_t *masks_u, uint8_t *masks_v, uint32_t flags);

/* ---- autotuning ---------------------------------------------------------------------------- */

#define ABCORE_TUNE_PEEL  0u  /* tune abcore_compute on the sample, one call per pair           */
#define ABCORE_TUNE_BATCH 1u  /* tune abcore_compute_batch on the sample, one batch of n pairs  */

/* Pick the launch and cascade parameters by measurement on the loaded graph: blocks per SM,
 * adjacency entries per work item ("chunk"), the queue's grab divisor, the hub degree above
 * which counts always come from a row search, the probe cost that steers the per-layer choice
 * between searching candidate rows and streaming violator rows, the scatter-versus-gather
 * switch of the mask emission, and for batches the number of chains sharing the GPU. Coordinate
 * descent; every setting is timed with CUDA events on the context's stream, best of three runs
 * of the whole sample with L2 flushed before each. The fastest setting stays on the context
 * (abcore_set_param changes it again); *best_ms (may be NULL) receives its sample time. Results
 * never depend on these parameters. Takes a few hundred timed runs of the sample.
 * Errors: EINVAL (empty sample, negative threshold, more than 64 pairs for ABCORE_TUNE_PEEL),
 * ENOTLOADED, ENOMEM, ETIMEDOUT. */
int abcore_autotune(abcore_ctx *ctx, int32_t n, const int32_t *alphas, const int32_t *betas,
                    uint32_t what, double *best_ms);

/* Wait for work enqueued with ABCORE_ASYNC and return its status: the first error of any of
 * those calls. After an error, the masks of every call enqueued since the previous successful
 * abcore_sync are undefined (a failed peel can leave work state behind for the peels queued after
 * it); the context itself stays usable, and later calls start from clean state. */
int abcore_sync(abcore_ctx *ctx);

/* ---- on-the-fly query (Section 5, GFQ) --------------------------------------------------- */

/* Apply the edge update (u, v) -- op ABCORE_INSERT or ABCORE_DELETE -- to the loaded graph
 * (it persists), then set *in_core to 1 iff both u and v belong to the (alpha, beta)-core of
 * the updated graph, else 0. The "query_scope" parameter picks what is re-peeled; both give the
 * same answers:
 *   0 (default): only the region the update can affect, from the target core kept by the
 *      serving loop (a delete cascades inside the core; an insert peels the non-core vertices
 *      reachable along the removal certificate; see abcore_serve_start);
 *   1: the paper's scope -- the connected component(s) of u and v in the updated graph, peeled
 *      from scratch (Algorithm 1 on the component's induced subgraph). The component forest is
 *      kept current: an insert unites two components, a delete recomputes the components of the
 *      one it may split. abcore_stats.scope_vertices counts the vertices re-peeled.
 * Errors: EINVAL, ENOTLOADED, EEXIST (insert of a present edge), ENOENT (delete of an
 * absent edge); on those the graph is unchanged and *in_core reports the current core. */
int abcore_query_edge(abcore_ctx *ctx, int32_t u, int32_t v, int op, int32_t alpha, int32_t beta,
                      uint8_t *in_core);

/* ---- connected components (Section 5: the component labels GFQ keeps) ------------------- */

/* Connected components of the current graph (served updates included). label_u[nU] and
 * label_v[nV] receive each vertex's component label: the smallest unified caller id in its
 * component, where U vertex u is u and V vertex v is nU + v (so labels do not depend on how
 * the library numbers vertices inside). An isolated vertex is a component of its own.
 * *n_components (may be NULL) receives the number of components. Computed on the device by
 * lock-free union-find over the edges. While serving, the loop keeps the component forest
 * current: an insert unites two components at once; after a delete, which may split one, this
 * call recomputes the forest from the current graph. The call waits until every submitted
 * update has been applied. Errors: EINVAL (NULL label array), ENOTLOADED, ENOMEM. */
int abcore_components(abcore_ctx *ctx, int32_t *label_u, int32_t *label_v, int64_t *n_components,
                      uint32_t flags);

/* ---- serving: continuously batched update/query stream ---------------------------------- */

typedef struct {
    int32_t op;       /* ABCORE_INSERT or ABCORE_DELETE                                  */
    int32_t u, v;     /* per-layer endpoint ids                                          */
    int32_t target;   /* index into the targets given to abcore_serve_start              */
    uint64_t tag;     /* caller's value, echoed in the response                          */
} abcore_req;

typedef struct {
    uint64_t seq;     /* arrival sequence number assigned by abcore_serve_submit          */
    uint64_t tag;     /* the request's tag                                                */
    int32_t status;   /* ABCORE_OK, ABCORE_EEXIST or ABCORE_ENOENT                        */
    uint8_t in_core;  /* both endpoints in the target core after this update              */
    uint8_t u_in;     /* u in the target core after this update                          */
    uint8_t v_in;     /* v in the target core after this update                          */
    uint8_t pad;
} abcore_resp;

/* Start serving with n_targets (alpha, beta) targets and a request ring of ring_slots entries.
 * Updates are applied in submission order and every answer is the one the update would get
 * if requests were processed one at a time, so answers do not depend on timing or batching.
 * Each target keeps its own device view of the updates; inserted edges live in a pool per target,
 * first sized by the "serve_inserts" parameter (default 2^20 inserts, 32 bytes each). Requests
 * are admitted by memory: an insert that does not fit its target's pool is held back, with the
 * view unchanged, until the library has doubled that pool (from the next submit, poll or stop
 * call), and is then processed in its turn -- answers are the same as with a large pool. Held
 * requests keep their ring slots, so submits meanwhile may return EBUSY. If the device has no
 * memory for the larger pool, that call returns ABCORE_ENOMEM and the requests keep waiting (a
 * later call tries again); the session stays usable. */
int abcore_serve_start(abcore_ctx *ctx, const int32_t *target_alphas, const int32_t *target_betas,
                       int32_t n_targets, int32_t ring_slots);

/* Submit n requests; seq_out[i] (may be NULL) receives their sequence numbers. Returns EBUSY,
 * submitting nothing, if the ring lacks room for all n. */
int abcore_serve_submit(abcore_ctx *ctx, const abcore_req *reqs, int32_t n, uint64_t *seq_out);

/* Copy up to max finished responses, in sequence order, to out; *n_out receives the count. */
int abcore_serve_poll(abcore_ctx *ctx, abcore_resp *out, int32_t max, int32_t *n_out);

/* Finish every submitted request, then stop serving. */
int abcore_serve_stop(abcore_ctx *ctx);

/* ---- introspection ----------------------------------------------------------------------- */

/* Accumulated counters (see abcore_stats) and the context's device memory. */
int abcore_get_stats(abcore_ctx *ctx, abcore_stats *out);

/* Set a parameter by name; EINVAL if the name is unknown or the value out of range. Results
 * never depend on any of them (except the actions and "query_scope", which picks an equivalent
 * algorithm). Defaults in brackets; abcore_autotune sets the starred ones.
 *
 * Single peel:
 *   "algo" [0]          0 auto, 1 GCC (plain peel, Algorithm 1), 2 GCC+ (pruned by core numbers,
 *                       Algorithm 2; needs abcore_core_numbers first); auto takes GCC+ when it leaves
 *                       fewer vertices than GCC.
 *   "mode" [-1]         per-layer count init: -1 cost model, 0..3 bit 0 U by row search, bit 1 V.
 *   "hub_degree"* [256] rows of at least this degree always count by search (0: none).
 *   "probe_bytes"* [32] the cost model's price of a search probe (steers search vs stream).
 *   "round0"* [0]       1: walk the initial violators' rows with no-return decrements first.
 *   "round0_variant"* [0] that walk's form: 0..3 lane-per-entry (entries in flight / blocks an SM:
 *                       8/any, 4/8, 16/4, 8/8), 4 four rows per warp, 5 the same in one 1024-thread
 *                       block per SM summing hub decrements in shared memory.
 *   "round0_hub"* [16384] hubs per layer in variant 5's table (0..28672).
 *   "count_swizzle" [1] counts in the per-layer multiplicative slot order (0: vertex order).
 *   "pdl" [1]           later kernels launch as programmatic dependents of the one before.
 *   "emit_scatter_max_pct"* [5] scatter the survivors when the candidates are at most this
 *                       percentage of the vertices, else gather over caller ids.
 *   "emit_bitmap_min_pct"* [0] the gather tests removal in a bitmap when the candidates are at
 *                       least this percentage of the vertices (101: never; by count instead).
 * Cascade (single peel; chunk, grab_div, batch_entries and flush_steps also in batch chains):
 *   "blocks_per_sm"* [0] resident blocks an SM for the cascade and the batch (0: as many as fit;
 *                       batch: 2 selects the batch kernel compiled for two blocks an SM).
 *   "chunk"* [1024]     adjacency entries per work item (32..2^20).
 *   "grab_div"* [0]     queue items per grab = backlog / grab_div, 1..32 (0: resident warps / 8).
 *   "batch_entries"* [1024] entries a warp walks per batch (128..2^24; the rest is re-queued).
 *   "batch_entries_small"* [512] the limit when a warp's grab leaves the queue nearly empty (0 off).
 *   "local_rounds" [256] batches a warp may chain on its own pushes (0..4096).
 *   "flush_steps"* [4]  steps a buffered push may wait before its warp flushes.
 * Batch:
 *   "batch_wave"* [4]   chains per wave (0..32; 0: all at once).
 *   "batch_plain_below"* [0] pairs with alpha below this run as single peels, not chains.
 *   "batch_seed"* [0]   1: seed each chain from the finished chain of the next smaller alpha.
 *   "packed_counts" [1] chains keep 16-bit counts whenever every degree fits.
 * Serving and queries:
 *   "serve_inserts" [2^20] initial inserted-edge pool per target (1..2^29; grows on demand).
 *   "query_scope" [0]   abcore_query_edge re-peels 0 the certificate-bounded region, 1 the
 *                       endpoints' connected components (the paper's scope).
 * Diagnostics and limits:
 *   "timeout_ms" [4000] limit of every bounded device wait, in milliseconds (>= 1).
 *   "timing" [0]        1: CUDA events around each launch, summed into abcore_stats.kernel_ms.
 *   "timing_kinds" [0xff] single peel: bit ABCORE_K_* set for each kind timed (an event between two
 *                       kernels costs the step about as much as a launch).
 *   "log_level" [0 or ABCORE_LOG] 0 none, 1 plans and events, 2 also timelines (on stderr).
 *   "debug_stall_slots" [0] test hook: reserve this many queue slots that nothing fills, so the
 *                       next cascade's bounded wait expires (reported as ABCORE_ETIMEDOUT).
 * Actions (no value to read back): "reset_stats" zeroes abcore_stats' counters. */
int abcore_set_param(abcore_ctx *ctx, const char *name, int64_t value);

/* Throughput of random 32-bit atomicSub on this device, per second, with the old value returned
 * (the cascade's crossing test needs it) and without: 2^26 operations over an int array of the
 * largest power-of-two size up to array_bytes (in [4 KiB, 4 GiB]; below the L2's size the array
 * stays in L2), best of three timed runs after one warm-up. This is the ceiling of a cascade
 * whose counts sit in L2. Errors: EINVAL, ENOMEM, ECUDA. */
int abcore_measure_atomics(abcore_ctx *ctx, int64_t array_bytes, double *with_return,
                           double *without_return);

/* Current value of a tuning parameter (the names abcore_set_param takes, except the actions
 * "reset_stats" and "debug_stall_slots"); EINVAL if unknown. */
int abcore_get_param(abcore_ctx *ctx, const char *name, int64_t *value);

/* Graph sizes of the loaded graph; any pointer may be NULL. */
int abcore_graph_info(abcore_ctx *ctx, int32_t *nU, int32_t *nV, int64_t *m,
                      int32_t *max_deg_u, int32_t *max_deg_v);

/* Copy out the device CSR as stored: off[nU+nV+1] and adj[2m] over internal unified ids
 * (U vertices 0..nU-1, V vertices nU..nU+nV-1, each layer ordered by non-increasing degree),
 * and new2old[nU+nV], the caller's per-layer id of each internal vertex. */
int abcore_export_csr(abcore_ctx *ctx, int64_t *off, int32_t *adj, int32_t *new2old, uint32_t flags);

/* ---- allocation-free variant (an interface convenience; the paper has no counterpart) ------ */

/* Limits of abcore_compute_static, whose working memory is a fixed array inside the library. */
#define ABCORE_STATIC_MAX_VERTICES (1 << 20)
#define ABCORE_STATIC_MAX_ITEMS    ((1 << 20) + (1 << 16))

/* The (alpha, beta)-core without allocating anything: no cudaMalloc, cudaFree or allocating
 * library routine is called, and no abcore_ctx is needed (the call runs on the current device).
 * It is meant for callers that cannot allocate device memory at run time -- code running inside
 * another framework that owns the device's memory pool, plugins that must not grow a host
 * process's device footprint, or programs that reserve all device memory up front.
 *   off[nU+nV+1], adj[off[nU+nV]]: the graph in unified ids, on the current device and owned by
 *     the caller: rows 0..nU-1 are the upper vertices and list lower vertices as nU + v, rows
 *     nU..nU+nV-1 are the lower vertices and list upper vertices u; every edge appears in both
 *     rows; rows may be in any order. adj must hold off[nU+nV] entries.
 *   mask_u[nU], mask_v[nV]: device buffers receiving 1 for core members, else 0.
 *   cuda_stream: the cudaStream_t to run on (NULL = the legacy default stream). The call reads two
 *     small values back from the device (the graph's size check, then the status) and waits for
 *     its stream each time, so its results are ready when it returns.
 * Working memory is one file-scope device array of about 13 MiB, held by every GPU that loads
 * this library until the process exits. Rejected with ABCORE_EINVAL: graphs above
 * ABCORE_STATIC_MAX_VERTICES vertices; graphs whose rows need more than ABCORE_STATIC_MAX_ITEMS
 * queue items, a row of length d needing ceil(d / 1024) of them (the test is exact: the sum of
 * ceil(d / 1024) over all nU + nV rows, so at the vertex limit rows of up to 1024 entries always
 * fit); a negative off[0] or decreasing offsets; an adjacency id outside [0, nU + nV) (found while
 * peeling: the masks are then undefined). The first call on each device looks up the array's
 * device address; make that first call before any stream capture. Every call shares the array
 * and it keeps the last call's contents (each call clears what must start empty), so calls that
 * overlap on the GPU -- from several host threads or streams at once -- race and must not be made.
 * Returns ABCORE_OK, ABCORE_EINVAL, ABCORE_ECUDA, ABCORE_ETIMEDOUT (a bounded device wait expired),
 * or ABCORE_ENOMEM if the removal queue overflowed -- which the size check rules out, so it would
 * mean an internal fault. */
int abcore_compute_static(int32_t nU, int32_t nV, const int64_t *off, const int32_t *adj,
                          int32_t alpha, int32_t beta, uint8_t *mask_u, uint8_t *mask_v,
                          void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ABCORE_H */
