// Batched (alpha, beta)-cores: many pairs over one graph in one persistent launch, replayed as a
// CUDA graph.
//
// Nested property (Section 4.2, the basis of Lemma 1): if alpha' >= alpha and beta' >= beta then
// core(alpha', beta') lies inside core(alpha, beta); and for any vertex set S containing
// core(alpha, beta), peeling G[S] gives the same core as peeling G. Algorithm 2 (GCC+) uses this
// with core numbers; here it is applied along chains: pairs that share alpha are sorted by beta,
// and one chain peels (alpha, beta_0) and then raises the V bound step by step, each step
// starting from the previous step's core. A vertex is removed at most once per chain, so a
// chain costs at most one full peel, whatever its length. The step at which each vertex falls
// is recorded (lvl), and the masks of all the chain's pairs follow from it:
//     x in core(alpha, beta_j)  <=>  x is a step-0 candidate and lvl[x] > j.
//
// The chains run concurrently, each on its own group of blocks of one cooperative launch. Inside
// a group, steps are separated by a bounded group barrier; the cascade of each step reuses the
// single peel's work queue (peel_core.cuh). A second kernel writes every pair's masks in the
// caller's ids. Memsets, both launches and the status read-back are captured once per pair list
// as a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "peel_core.cuh"

namespace {

using abc::LaneStats;
using abc::WarpSmem;

constexpr int BATCH_THREADS = 256;
constexpr int MAX_CHAINS_PER_WAVE = 32;
constexpr int MAX_STEPS = 255;
// timeline of one chain (log level 2): its start, then three marks per step
constexpr int PROF_STRIDE = 1 + 3 * MAX_STEPS;
__host__ __device__ constexpr int prof_at(int step, int phase) { return 1 + 3 * step + phase; }

struct ChainDev {
    int32_t alpha;
    int32_t nsteps;
    int32_t beta_off;        // betas[beta_off .. beta_off + nsteps): ascending V bounds
    int32_t pU0, pV0;        // step-0 candidate prefixes
    int32_t searchU, searchV;
    int32_t hubcutU, hubcutV;
    int32_t first_block, nblocks;
    int32_t col;             // column of this chain in lvl
    int32_t seed_col;        // column of a finished chain with a smaller alpha and the same betas
                             // (its step-j core contains this chain's), or -1
    int64_t sa, ea, sb, eb;  // step-0 violator slices (see stream_range)
};

struct ChainMem {
    int32_t *cnt;
    int32_t *plen;
    unsigned long long *q;
    PeelCtl *ctl;
    unsigned *bar;           // group barrier: [0] arrivals, [32] generation
    uint32_t *ulive;         // bitmap over the U prefix: candidates a step's U scan must look at
};

struct BatchArgs {
    const int64_t *off;
    const int32_t *adj;
    int32_t nU, nV;
    const ChainDev *chains;
    const ChainMem *mem;
    const int32_t *betas;
    const int32_t *pvs;      // per beta: the V candidate prefix (vertices of degree >= beta)
    const float *fracs;      // per beta: the share of a U row's step-0 candidate entries below it
                             // (where the search for a fallen U row's new end starts)
    int32_t nchains;
    uint8_t *lvl;
    int32_t lvl_stride;
    int32_t chunk;
    int32_t batch_entries, flush_steps;
    int32_t packed;          // 16-bit counts (every degree below 2^16)
    int32_t swz;             // counts in the swizzled layout (PeelArgs::swz)
    uint32_t *flags;
    long long qcap;
    unsigned long long timeout_ns;
    // optional timeline: prof[c * PROF_STRIDE + 0] = globaltimer when chain c's block 0 starts,
    // then per step j three marks (prof_at): after its V walk (step 0: the count init), after its
    // U scan (step 0: the first round), after its cascade
    // (j = 0) and when its step j - 1 has closed (j >= 1); nullptr: not recorded
    unsigned long long *prof;
};

// Compiled for two occupancies: three blocks an SM (80 registers a thread, some spilled) or two
// (no spills); "blocks_per_sm" = 2 picks the second.
template <int MINB>
__global__ void __launch_bounds__(BATCH_THREADS, MINB) k_batch(BatchArgs B) {
    __shared__ WarpSmem smem[BATCH_THREADS / 32];
    __shared__ unsigned s_hubs[abc::WALK_HUBS];  // the V walk's U-hub tallies (fall_walk_v)
    int c = 0;
    while (c + 1 < B.nchains && (int)blockIdx.x >= B.chains[c + 1].first_block) ++c;
    const ChainDev cd = B.chains[c];
    const ChainMem mem = B.mem[c];
    const int G = cd.nblocks;
    const int r = (int)blockIdx.x - cd.first_block;
    const int wib = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < abc::WALK_HUBS; i += blockDim.x) s_hubs[i] = 0u;
    // (init_range's first barrier orders these stores before any walk)

    PeelArgs a{};
    a.off = B.off;
    a.adj = B.adj;
    a.cnt = mem.cnt;
    a.packed = B.packed;
    set_count_layout(a, cd.pU0, cd.pV0, B.swz != 0);  // later steps' candidates are prefixes of these
    a.plen = mem.plen;
    a.q = mem.q;
    a.qcap = B.qcap;
    a.ctl = mem.ctl;
    a.nU = B.nU;
    a.nV = B.nV;
    a.pU = cd.pU0;
    a.pV = cd.pV0;
    a.thrU = cd.alpha;
    a.thrV = B.betas[cd.beta_off];
    a.chunk = B.chunk;
    a.batch_entries = B.batch_entries;
    a.flush_steps = B.flush_steps;
    a.searchU = cd.searchU;
    a.searchV = cd.searchV;
    a.hubcutU = cd.hubcutU;
    a.hubcutV = cd.hubcutV;
    a.timeout_ns = B.timeout_ns;
    a.skip_zero = 0;  // a V bound of 0 may rise later: keep every count exact
    a.lvl = B.lvl;
    a.lvl_stride = B.lvl_stride;
    a.lvl_col = cd.col;
    a.seed_col = cd.seed_col;
    a.dead_own = cd.seed_col >= 0 ? 1 : 0;
    a.step = 0;
    a.flags = B.flags;
    a.flag_first = cd.first_block;
    a.flag_count = G;
    a.epoch = 1;
    const int grab_div = max(1, G * (BATCH_THREADS / 32) / 8);

    const int64_t t0 = (int64_t)r * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)G * blockDim.x;
    LaneStats ls;
    unsigned long long probes = 0, inits = 0, ents = 0, sdecs = 0;

    unsigned long long *prof = B.prof != nullptr && r == 0 && threadIdx.x == 0 ? B.prof + (size_t)c * PROF_STRIDE
                                                                               : nullptr;
    if (prof) prof[0] = abc::now_ns();
    abc::init_range(a, smem[wib].push, t0, nthreads, ls, probes, inits);
    if (!abc::group_barrier(mem.bar, G, mem.ctl, false, B.timeout_ns)) goto out;
    if (prof) prof[prof_at(0, 0)] = abc::now_ns();
    if (cd.ea > cd.sa || cd.eb > cd.sb) {
        const unsigned long long d0 = ls.decs;
        abc::stream_range(a, cd.sa, cd.ea, cd.sb, cd.eb, t0, nthreads, ls, ents);
        sdecs = ls.decs - d0;
        ls.decs = d0;
        if (!abc::group_barrier(mem.bar, G, mem.ctl, false, B.timeout_ns)) goto out;
        unsigned long long scanned = 0;
        abc::scan_range(a, smem[wib].push, t0, nthreads, ls, scanned);
        if (!abc::group_barrier(mem.bar, G, mem.ctl, false, B.timeout_ns)) goto out;
    }
    if (prof) prof[prof_at(0, 1)] = abc::now_ns();
    // A failed cascade leaves its code in ctl->err. Every warp still reaches the barrier, so no
    // block waits on warps that left, and the barrier reports the error to all of them.
    (void)abc::cascade_loop<false>(a, smem[wib], ls, grab_div, r == 0 && wib == 0);
    if (!abc::group_barrier(mem.bar, G, mem.ctl, true, B.timeout_ns)) goto out;
    if (prof) prof[prof_at(0, 2)] = abc::now_ns();
    for (int j = 1; j < cd.nsteps; ++j) {
        const int32_t prev = a.thrV;
        const int32_t pv_prev = a.pV;
        a.thrV = B.betas[cd.beta_off + j];
        a.step = j;
        a.epoch = (uint32_t)j + 1;
        // the V candidates shrink to degree >= the new bound. The live V vertices of the previous
        // prefix that miss it (all those past the new prefix among them, their degree being below
        // it; with a seed chain, also those outside its step-j core) fall first, their rows walked
        // with decrements that return nothing; the U candidates those decrements took below alpha
        // are then queued; the cascade does the rest. A fallen U vertex walks only its entries
        // inside the new prefix (process_items).
        a.pV = B.pvs[cd.beta_off + j];
        a.pV_rows = cd.pV0;
        a.frac_rows = B.fracs[cd.beta_off + j];
        {
            unsigned long long e0 = 0, d0 = 0;
            abc::fall_walk_v(a, smem[wib], pv_prev, prev, a.dead_own != 0, t0, nthreads, ls, e0, d0, s_hubs);
            ents += e0;
            sdecs += d0;
        }
        if (!abc::group_barrier(mem.bar, G, mem.ctl, false, B.timeout_ns)) goto out;
        if (prof) prof[prof_at(j, 0)] = abc::now_ns();
        {
            unsigned long long sc = 0;
            abc::fall_scan_u(a, smem[wib], t0, nthreads, ls, sc, mem.ulive, j == 1);
        }
        if (!abc::group_barrier(mem.bar, G, mem.ctl, false, B.timeout_ns)) goto out;
        if (prof) prof[prof_at(j, 1)] = abc::now_ns();
        (void)abc::cascade_loop<false>(a, smem[wib], ls, grab_div, r == 0 && wib == 0);
        if (!abc::group_barrier(mem.bar, G, mem.ctl, true, B.timeout_ns)) goto out;
        if (prof) prof[prof_at(j, 2)] = abc::now_ns();
    }
out:
    abc::flush_stats(a, ls);
    {
        unsigned long long v[4] = {inits, probes, ents, sdecs};
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = (unsigned long long)abc::warp_sum64((long long)v[i]);
        if ((threadIdx.x & 31) == 0) {
            if (v[0]) atomicAdd(&a.ctl->st[ST_INIT], v[0]);
            if (v[1]) atomicAdd(&a.ctl->st[ST_PROBES], v[1]);
            if (v[2]) atomicAdd(&a.ctl->st[ST_STREAM], v[2]);
            if (v[3]) atomicAdd(&a.ctl->st[ST_SDECS], v[3]);
        }
        if (r == 0 && threadIdx.x == 0) atomicAdd(&a.ctl->st[ST_STEPS], (unsigned long long)cd.nsteps);
    }
}

struct PairRef {
    int32_t chain;  // index into the wave's chains
    int32_t step;
    int32_t pv;     // V candidate prefix of the pair's beta
};

// Masks of every pair of a wave, in the caller's ids: one thread per vertex, one byte per pair.
__global__ void __launch_bounds__(256) k_batch_emit(const int32_t *__restrict__ old2new, int32_t nU, int32_t nV,
                                                    const uint8_t *__restrict__ lvl, int32_t lvl_stride,
                                                    const ChainDev *__restrict__ chains, int32_t nchains,
                                                    const PairRef *__restrict__ pairs, const int32_t *__restrict__ pidx,
                                                    int32_t npairs, uint8_t *__restrict__ masks_u,
                                                    uint8_t *__restrict__ masks_v) {
    extern __shared__ int32_t sh[];
    int32_t *pU0 = sh, *col = sh + nchains;
    int32_t *pc = sh + 2 * nchains, *ps = pc + npairs, *pi = ps + npairs, *pv = pi + npairs;
    for (int i = threadIdx.x; i < nchains; i += blockDim.x) {
        pU0[i] = chains[i].pU0;
        col[i] = chains[i].col;
    }
    for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
        pc[i] = pairs[i].chain;
        ps[i] = pairs[i].step;
        pi[i] = pidx[i];
        pv[i] = pairs[i].pv;
    }
    __syncthreads();
    const int64_t n = (int64_t)nU + nV;
    if (lvl_stride == 4 && (nU & 3) == 0 && (nV & 3) == 0 &&
        ((reinterpret_cast<uintptr_t>(masks_u) | reinterpret_cast<uintptr_t>(masks_v)) & 3) == 0) {
        // four consecutive caller ids per thread (16-byte id load, one 4-byte store per pair), and
        // each vertex's removal steps in one 4-byte row (at most four chains a wave)
        const int4 *o4 = reinterpret_cast<const int4 *>(old2new);
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n / 4; q += (int64_t)gridDim.x * blockDim.x) {
            const int64_t i = 4 * q;
            const int4 xv = __ldg(&o4[q]);
            const int32_t xs[4] = {xv.x, xv.y, xv.z, xv.w};
            const bool upper = i < nU;  // nU is a multiple of four: the quad is in one layer
            uint32_t rows[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) rows[j] = __ldg(reinterpret_cast<const uint32_t *>(lvl + (size_t)xs[j] * 4));
            for (int p = 0; p < npairs; ++p) {
                const int ch = pc[p];
                const unsigned sh = 8u * (unsigned)col[ch];
                uint32_t bytes = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool cand = upper ? (xs[j] < pU0[ch]) : (xs[j] - nU < pv[p]);
                    const bool in = cand && (int)((rows[j] >> sh) & 0xffu) > ps[p];
                    bytes |= (in ? 1u : 0u) << (8 * j);
                }
                if (upper) *reinterpret_cast<uint32_t *>(masks_u + (size_t)pi[p] * nU + i) = bytes;
                else *reinterpret_cast<uint32_t *>(masks_v + (size_t)pi[p] * nV + (i - nU)) = bytes;
            }
        }
        return;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = __ldg(&old2new[i]);
        const bool upper = i < nU;
        const uint8_t *row = lvl + (size_t)x * lvl_stride;
        for (int p = 0; p < npairs; ++p) {
            const int ch = pc[p];
            // a candidate of the pair that had not fallen by its step (V vertices that left the
            // prefix at a later step are never queued: the prefix test places them)
            const bool cand = upper ? (x < pU0[ch]) : (x - nU < pv[p]);
            const uint8_t v = (cand && __ldg(&row[col[ch]]) > ps[p]) ? 1 : 0;
            if (upper) masks_u[(size_t)pi[p] * nU + i] = v;
            else masks_v[(size_t)pi[p] * nV + (i - nU)] = v;
        }
    }
}

}  // namespace

// One wave: up to MAX_CHAINS_PER_WAVE chains sharing the device at once.
struct Wave {
    std::vector<ChainDev> chains;
    std::vector<PairRef> pairs;
    std::vector<int32_t> pidx;   // caller pair index of each PairRef
    ChainDev *d_chains = nullptr;
    PairRef *d_pairs = nullptr;
    int32_t *d_pidx = nullptr;
    int grid = 0;
};

struct BatchState {
    // key of the captured graph
    std::vector<int32_t> key_a, key_b;
    uint8_t *key_mu = nullptr, *key_mv = nullptr;
    int64_t key_graph_n = -1, key_graph_m = -1;
    int key_chunk = 0;
    // plan
    std::vector<Wave> waves;
    std::vector<int32_t> betas, pvs;
    std::vector<float> fracs;
    int32_t *d_betas = nullptr;
    int32_t *d_pvs = nullptr;
    float *d_fracs = nullptr;
    bool lvl_global = false;            // every chain has its own lvl column (seeding; cleared once per call)
    int nmem = 0;                       // chain workspaces allocated
    std::vector<ChainMem> mem;
    ChainMem *d_mem = nullptr;
    uint8_t *lvl = nullptr;
    int lvl_stride = 0;
    uint32_t *flags = nullptr;          // [grid * 32] per-block queue-closed flags (epochs)
    PeelCtl *ctl_host = nullptr;        // pinned: [waves x MAX_CHAINS_PER_WAVE]
    long long qcap = 0;
    bool q_dirty = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = true;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    unsigned long long *prof = nullptr;  // [waves x MAX_CHAINS_PER_WAVE x PROF_STRIDE] (log level 2)
};

static void destroy_plan(abcore_ctx *ctx, BatchState *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    for (auto &w : b->waves) {
        ctx->release(w.d_chains);
        ctx->release(w.d_pairs);
        ctx->release(w.d_pidx);
    }
    b->waves.clear();
    ctx->release(b->d_betas);
    ctx->release(b->d_pvs);
    ctx->release(b->d_fracs);
    ctx->release(b->prof);
    if (b->ctl_host) cudaFreeHost(b->ctl_host);
    b->ctl_host = nullptr;
    b->key_a.clear();
    b->key_b.clear();
    b->key_graph_n = -1;
}

void free_batch(abcore_ctx *ctx) {
    BatchState *b = ctx->batch;
    if (!b) return;
    cudaStreamSynchronize(ctx->stream);
    destroy_plan(ctx, b);
    for (auto &m : b->mem) {
        ctx->release(m.cnt);
        ctx->release(m.plen);
        ctx->release(m.q);
        ctx->release(m.ctl);
        ctx->release(m.bar);
        ctx->release(m.ulive);
    }
    ctx->release(b->d_mem);
    ctx->release(b->lvl);
    ctx->release(b->flags);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
    ctx->batch = nullptr;
}

static void (*batch_kernel(abcore_ctx *ctx))(BatchArgs) {
    return ctx->prm.blocks_per_sm == 2 ? k_batch<2> : k_batch<3>;
}

static int batch_grid(abcore_ctx *ctx) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(ctx), BATCH_THREADS, 0);
    if (ctx->prm.blocks_per_sm > 0) per_sm = std::min(per_sm, ctx->prm.blocks_per_sm);
    return std::max(per_sm, 1) * ctx->num_sms;
}

// The removal-step record, n rows of `stride` bytes.
static int ensure_lvl(abcore_ctx *ctx, BatchState *b, int stride) {
    if (b->lvl && b->lvl_stride == stride) return ABCORE_OK;
    ctx->release(b->lvl);
    b->lvl_stride = stride;
    return ctx->alloc(&b->lvl, (size_t)std::max<int64_t>(ctx->g.n(), 1) * stride, "batch levels");
}

constexpr int MAX_LVL_COLS = 64;  // chains with a column of their own in lvl (beyond: one per wave slot)

// Build the plan for a pair list: chains by alpha, waves, seeds, slices, device tables.
//
// Chains are sorted by alpha. Without seeding, each wave takes the next chains in that order and
// chains share lvl columns by their slot in the wave. With seeding (and at most MAX_LVL_COLS
// chains), every chain has its own column and the chains are dealt to waves round-robin (chain k
// runs in wave k mod W), so a chain's smaller-alpha neighbours mostly ran in earlier waves: with
// the same beta steps, the closest such chain's step-j core contains this chain's (the nested
// property in alpha), and its non-members are queued as known dead.
static int make_plan(abcore_ctx *ctx, BatchState *b, int32_t n, const int32_t *alphas, const int32_t *betas) {
    const Graph &g = ctx->g;
    std::map<int32_t, std::vector<int32_t>> by_alpha;
    for (int32_t i = 0; i < n; ++i)
        if (alphas[i] >= ctx->prm.batch_plain_below) by_alpha[alphas[i]].push_back(betas[i]);
    struct Chain {
        int32_t alpha;
        std::vector<int32_t> betas;
    };
    std::vector<Chain> chains;
    for (auto &kv : by_alpha) {
        std::vector<int32_t> bs = kv.second;
        std::sort(bs.begin(), bs.end());
        bs.erase(std::unique(bs.begin(), bs.end()), bs.end());
        for (size_t s = 0; s < bs.size(); s += MAX_STEPS)
            chains.push_back({kv.first, std::vector<int32_t>(bs.begin() + s, bs.begin() + std::min(bs.size(), s + MAX_STEPS))});
    }
    const int C = (int)chains.size();
    const int grid = batch_grid(ctx);
    int per_wave = std::max(1, std::min({MAX_CHAINS_PER_WAVE, grid, b->nmem}));
    if (ctx->prm.batch_wave > 0) per_wave = std::min(per_wave, ctx->prm.batch_wave);
    const int NW = (C + per_wave - 1) / per_wave;
    const bool own_cols = ctx->prm.batch_seed && C <= MAX_LVL_COLS;
    b->lvl_global = own_cols;
    const int stride = ((own_cols ? C : per_wave) + 3) / 4 * 4;
    ABC_TRY(ensure_lvl(ctx, b, stride));
    b->betas.clear();
    b->pvs.clear();
    b->fracs.clear();
    b->waves.assign(NW, Wave{});
    std::vector<int> wave_of(C), slot_of(C), col_of(C);
    for (int k = 0; k < C; ++k) {
        wave_of[k] = own_cols ? k % NW : k / per_wave;
        slot_of[k] = own_cols ? k / NW : k % per_wave;
        col_of[k] = own_cols ? k : slot_of[k];
    }
    int seeded = 0;
    for (int k = 0; k < C; ++k) {
        const Chain &ch = chains[k];
        Wave &wave = b->waves[wave_of[k]];
        ChainDev d{};
        d.alpha = ch.alpha;
        d.nsteps = (int32_t)ch.betas.size();
        d.beta_off = (int32_t)b->betas.size();
        b->betas.insert(b->betas.end(), ch.betas.begin(), ch.betas.end());
        const int32_t beta0 = ch.betas[0];
        for (size_t j = 0; j < ch.betas.size(); ++j) {
            const int32_t bj = ch.betas[j];
            b->pvs.push_back((int32_t)cnt_ge(g.cntV_ge, bj));
            // where the search for a fallen U row's end inside the new prefix starts: the share of
            // the step-0 prefix's entries that lie below the new bound
            const double eb = (double)std::max<int64_t>(cnt_ge(g.edgesV_ge, ch.betas[0]), 1);
            b->fracs.push_back((float)((double)cnt_ge(g.edgesV_ge, bj) / eb));
        }
        d.pU0 = (int32_t)cnt_ge(g.cntU_ge, ch.alpha);
        d.pV0 = (int32_t)cnt_ge(g.cntV_ge, beta0);
        const int mode = pick_mode(ctx, ch.alpha, beta0, d.pU0, d.pV0);
        // U counts by row search: a U vertex's plen is then its row's end inside the step-0 V
        // prefix, where the search for its end inside a later step's prefix ends
        d.searchU = 1;
        d.searchV = (mode >> 1) & 1;
        d.hubcutU = 0;
        d.hubcutV = ctx->prm.hub_degree > 0 ? (int32_t)std::min<int64_t>(cnt_ge(g.cntV_ge, ctx->prm.hub_degree), d.pV0) : 0;
        if (!d.searchV && d.pV0 > 0) {
            d.sb = cnt_ge(g.edgesU_ge, ch.alpha);
            d.eb = g.m;
        }
        d.col = col_of[k];
        d.seed_col = -1;
        if (own_cols && ctx->prm.batch_seed) {
            for (int s2 = k - 1; s2 >= 0; --s2)
                if (wave_of[s2] < wave_of[k] && chains[s2].alpha < ch.alpha && chains[s2].betas == ch.betas) {
                    d.seed_col = col_of[s2];
                    seeded++;
                    break;
                }
        }
        wave.chains.push_back(d);
    }
    for (auto &wave : b->waves) {
        const int cw = (int)wave.chains.size();
        wave.grid = grid;
        int first = 0;
        for (int k = 0; k < cw; ++k) {
            ChainDev &d = wave.chains[k];
            d.nblocks = grid / cw + (k < grid % cw ? 1 : 0);
            d.first_block = first;
            first += d.nblocks;
        }
    }
    // pair -> (wave, chain in wave, step); pairs left to single peels have no chain
    for (int32_t i = 0; i < n; ++i) {
        if (alphas[i] < ctx->prm.batch_plain_below) continue;
        int ci = 0;
        for (; ci < C; ++ci) {
            if (chains[ci].alpha != alphas[i]) continue;
            const auto &bs = chains[ci].betas;
            if (std::binary_search(bs.begin(), bs.end(), betas[i])) break;
        }
        const auto &bs = chains[ci].betas;
        const int step = (int)(std::lower_bound(bs.begin(), bs.end(), betas[i]) - bs.begin());
        b->waves[wave_of[ci]].pairs.push_back({slot_of[ci], step, (int32_t)cnt_ge(g.cntV_ge, betas[i])});
        b->waves[wave_of[ci]].pidx.push_back(i);
    }
    ABC_TRY(ctx->alloc(&b->d_betas, b->betas.size(), "batch betas"));
    ABC_CU(cudaMemcpy(b->d_betas, b->betas.data(), sizeof(int32_t) * b->betas.size(), cudaMemcpyHostToDevice));
    ABC_TRY(ctx->alloc(&b->d_pvs, b->pvs.size(), "batch prefixes"));
    ABC_CU(cudaMemcpy(b->d_pvs, b->pvs.data(), sizeof(int32_t) * b->pvs.size(), cudaMemcpyHostToDevice));
    ABC_TRY(ctx->alloc(&b->d_fracs, b->fracs.size(), "batch prefix shares"));
    ABC_CU(cudaMemcpy(b->d_fracs, b->fracs.data(), sizeof(float) * b->fracs.size(), cudaMemcpyHostToDevice));
    for (auto &w : b->waves) {
        ABC_TRY(ctx->alloc(&w.d_chains, w.chains.size(), "batch chains"));
        ABC_TRY(ctx->alloc(&w.d_pairs, std::max<size_t>(w.pairs.size(), 1), "batch pairs"));
        ABC_TRY(ctx->alloc(&w.d_pidx, std::max<size_t>(w.pidx.size(), 1), "batch pairs"));
        ABC_CU(cudaMemcpy(w.d_chains, w.chains.data(), sizeof(ChainDev) * w.chains.size(), cudaMemcpyHostToDevice));
        if (!w.pairs.empty()) {
            ABC_CU(cudaMemcpy(w.d_pairs, w.pairs.data(), sizeof(PairRef) * w.pairs.size(), cudaMemcpyHostToDevice));
            ABC_CU(cudaMemcpy(w.d_pidx, w.pidx.data(), sizeof(int32_t) * w.pidx.size(), cudaMemcpyHostToDevice));
        }
    }
    ABC_CU(cudaMallocHost(&b->ctl_host, sizeof(PeelCtl) * MAX_CHAINS_PER_WAVE * b->waves.size()));
    if (ctx->prm.log_level >= 2)
        ABC_TRY(ctx->alloc(&b->prof, b->waves.size() * MAX_CHAINS_PER_WAVE * PROF_STRIDE, "batch timeline"));
    ctx->log(1, "batch plan: %d pairs, %d chains in %d waves of up to %d, grid %d blocks, %d seeded chains", n, C,
             (int)b->waves.size(), per_wave, grid, seeded);
    return ABCORE_OK;
}

// Counts of the batch's chains are 16-bit when every degree fits (parameter "packed_counts").
static bool batch_packed(const abcore_ctx *ctx) {
    return ctx->prm.packed_counts && std::max(ctx->g.maxdegU, ctx->g.maxdegV) <= 65535;
}

// Chain workspaces: counts, queue, control block and barrier per concurrent chain, plus lvl.
static int ensure_memory(abcore_ctx *ctx, BatchState *b, int want_chains) {
    const Graph &g = ctx->g;
    const int64_t n = g.n();
    const int grid = batch_grid(ctx);
    const long long qcap = n + (2 * g.m) / std::max(ctx->prm.chunk, 1) + 1024 +
                           (long long)MAX_STEPS * 2 * grid * (BATCH_THREADS / 32) * 32 / std::max(want_chains, 1) + 4096;
    if (b->nmem >= want_chains && b->qcap >= qcap) return ABCORE_OK;
    for (auto &m : b->mem) {
        ctx->release(m.cnt);
        ctx->release(m.plen);
        ctx->release(m.q);
        ctx->release(m.ctl);
        ctx->release(m.bar);
        ctx->release(m.ulive);
    }
    b->mem.clear();
    ctx->release(b->d_mem);
    b->nmem = 0;
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    const double per_chain = (batch_packed(ctx) ? 6.0 : 8.0) * n + 8.0 * qcap + 1.0 * n;  // counts + prefixes, queue, levels
    int fit = (int)std::max(1.0, 0.6 * (double)freeb / per_chain);
    const int chains = std::max(1, std::min(want_chains, fit));
    b->qcap = qcap;
    b->mem.resize(chains);
    for (int c = 0; c < chains; ++c) {
        ChainMem &m = b->mem[c];
        // counts in the swizzled layout need each layer's power-of-two range
        uint32_t mu = 0, mv = 0;
        int64_t bv = 0;
        const int64_t slots = std::max(n, swz_layout(g.nU, g.nV, &mu, &mv, &bv));
        // (32 slots of padding: the U scan reads whole 32-vertex words of counts)
        ABC_TRY(ctx->alloc(&m.cnt, (size_t)(batch_packed(ctx) ? slots / 2 + 17 : slots + 32), "batch counts"));
        ABC_TRY(ctx->alloc(&m.ulive, (size_t)(g.nU / 32 + 1), "batch live U bitmap"));
        ABC_TRY(ctx->alloc(&m.plen, (size_t)std::max<int64_t>(n, 1), "batch prefixes"));
        ABC_TRY(ctx->alloc(&m.q, (size_t)qcap, "batch queue"));
        ABC_TRY(ctx->alloc(&m.ctl, 1, "batch control"));
        ABC_TRY(ctx->alloc(&m.bar, 64, "batch barrier"));
        ABC_CU(cudaMemsetAsync(m.q, 0xff, sizeof(unsigned long long) * (size_t)qcap, ctx->stream));
        ABC_CU(cudaMemsetAsync(m.bar, 0, 64 * sizeof(unsigned), ctx->stream));
    }
    ABC_TRY(ctx->alloc(&b->d_mem, chains, "batch chain table"));
    ABC_CU(cudaMemcpy(b->d_mem, b->mem.data(), sizeof(ChainMem) * chains, cudaMemcpyHostToDevice));
    if (!b->flags) ABC_TRY(ctx->alloc(&b->flags, (size_t)grid * 32, "batch close flags"));
    b->nmem = chains;
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    return ABCORE_OK;
}

// Enqueue the whole batch on the stream (captured into a graph on first use).
static int enqueue_batch(abcore_ctx *ctx, BatchState *b, uint8_t *d_mu, uint8_t *d_mv) {
    const Graph &g = ctx->g;
    const int64_t n = g.n();
    if (b->lvl_global) ABC_CU(cudaMemsetAsync(b->lvl, 0xff, (size_t)n * b->lvl_stride, ctx->stream));
    for (size_t wi = 0; wi < b->waves.size(); ++wi) {
        Wave &w = b->waves[wi];
        const int cw = (int)w.chains.size();
        for (int c = 0; c < cw; ++c) {
            ABC_CU(cudaMemsetAsync(b->mem[c].ctl, 0, sizeof(PeelCtl), ctx->stream));
            ABC_CU(cudaMemsetAsync(b->mem[c].bar, 0, 64 * sizeof(unsigned), ctx->stream));
        }
        if (!b->lvl_global) ABC_CU(cudaMemsetAsync(b->lvl, 0xff, (size_t)n * b->lvl_stride, ctx->stream));
        ABC_CU(cudaMemsetAsync(b->flags, 0, sizeof(uint32_t) * (size_t)w.grid * 32, ctx->stream));
        BatchArgs B{};
        B.off = g.off;
        B.adj = g.adj;
        B.nU = g.nU;
        B.nV = g.nV;
        B.chains = w.d_chains;
        B.mem = b->d_mem;
        B.betas = b->d_betas;
        B.pvs = b->d_pvs;
        B.fracs = b->d_fracs;
        B.nchains = cw;
        B.lvl = b->lvl;
        B.lvl_stride = b->lvl_stride;
        B.chunk = std::max(ctx->prm.chunk, 32);
        B.flags = b->flags;
        B.batch_entries = ctx->prm.batch_entries;
        B.packed = batch_packed(ctx) ? 1 : 0;
        // chains keep counts in vertex order: every step scans all of a chain's candidates in
        // order, which the swizzled layout would turn into random sector reads (measured slower)
        B.swz = 0;
        B.flush_steps = ctx->prm.flush_steps;
        B.qcap = b->qcap;
        B.timeout_ns = (unsigned long long)ctx->prm.timeout_ms * 1000000ull;
        B.prof = b->prof ? b->prof + wi * MAX_CHAINS_PER_WAVE * PROF_STRIDE : nullptr;
        void *args[] = {&B};
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(w.grid);
        cfg.blockDim = dim3(BATCH_THREADS);
        cfg.stream = ctx->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ABC_CU(cudaLaunchKernelExC(&cfg, (const void *)batch_kernel(ctx), args));
        ctx->stats.launches++;
        if (!w.pairs.empty()) {
            const int np = (int)w.pairs.size();
            const size_t shm = sizeof(int32_t) * (2 * cw + 4 * np);
            if (shm > 200 * 1024) return ctx->fail(ABCORE_EINVAL, "too many pairs in one batch wave");
            if (shm > 48 * 1024)
                ABC_CU(cudaFuncSetAttribute(k_batch_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
            const int eg = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8);
            k_batch_emit<<<std::max(eg, 1), 256, shm, ctx->stream>>>(g.old2new, g.nU, g.nV, b->lvl, b->lvl_stride,
                                                                     w.d_chains, cw, w.d_pairs, w.d_pidx, np, d_mu, d_mv);
            ctx->stats.launches++;
        }
        for (int c = 0; c < cw; ++c)
            ABC_CU(cudaMemcpyAsync(b->ctl_host + wi * MAX_CHAINS_PER_WAVE + c, b->mem[c].ctl, sizeof(PeelCtl),
                                   cudaMemcpyDeviceToHost, ctx->stream));
    }
    return ABCORE_OK;
}

int batch_compute(abcore_ctx *ctx, int32_t n, const int32_t *alphas, const int32_t *betas, uint8_t *d_masks_u,
                  uint8_t *d_masks_v, bool sync_and_check) {
    const Graph &g = ctx->g;
    if (!ctx->batch) ctx->batch = new BatchState();
    BatchState *b = ctx->batch;
    const bool same = b->exec && b->key_mu == d_masks_u && b->key_mv == d_masks_v && b->key_graph_n == g.n() &&
                      b->key_graph_m == g.m && b->key_chunk == ctx->prm.chunk &&
                      b->key_a == std::vector<int32_t>(alphas, alphas + n) &&
                      b->key_b == std::vector<int32_t>(betas, betas + n);
    if (!same || !b->use_graph) {
        destroy_plan(ctx, b);
        std::map<int32_t, int> na;
        for (int32_t i = 0; i < n; ++i)
            if (alphas[i] >= ctx->prm.batch_plain_below) na[alphas[i]]++;
        int want = std::min<int>((int)na.size(), MAX_CHAINS_PER_WAVE);
        if (ctx->prm.batch_wave > 0) want = std::min(want, ctx->prm.batch_wave);
        if (want > 0) {
            ABC_TRY(ensure_memory(ctx, b, want));
            ABC_TRY(make_plan(ctx, b, n, alphas, betas));
        } else {
            b->waves.clear();
        }
        b->key_a.assign(alphas, alphas + n);
        b->key_b.assign(betas, betas + n);
        b->key_mu = d_masks_u;
        b->key_mv = d_masks_v;
        b->key_graph_n = g.n();
        b->key_graph_m = g.m;
        b->key_chunk = ctx->prm.chunk;
        if (b->use_graph) {
            cudaStreamCaptureStatus cs;
            ABC_CU(cudaStreamIsCapturing(ctx->stream, &cs));
            if (cs == cudaStreamCaptureStatusNone &&
                cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const int64_t l0 = ctx->stats.launches;
                int rc = enqueue_batch(ctx, b, d_masks_u, d_masks_v);
                cudaGraph_t graph = nullptr;
                cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
                ctx->stats.launches = l0;
                if (rc == ABCORE_OK && e == cudaSuccess &&
                    cudaGraphInstantiate(&b->exec, graph, 0) == cudaSuccess) {
                    b->graph = graph;
                } else {
                    if (graph) cudaGraphDestroy(graph);
                    cudaGetLastError();
                    b->exec = nullptr;
                    b->use_graph = false;  // capture refused: launch directly from now on
                }
            } else {
                cudaGetLastError();
                b->use_graph = false;
            }
        }
    }
    if (b->q_dirty) {
        for (auto &m : b->mem) ABC_CU(cudaMemsetAsync(m.q, 0xff, sizeof(unsigned long long) * (size_t)b->qcap, ctx->stream));
        b->q_dirty = false;
    }
    const bool timed = ctx->prm.timing != 0;
    if (timed) {
        if (!b->ev0) ABC_CU(cudaEventCreate(&b->ev0));
        if (!b->ev1) ABC_CU(cudaEventCreate(&b->ev1));
        ABC_CU(cudaEventRecord(b->ev0, ctx->stream));
    }
    if (b->exec) {
        ABC_CU(cudaGraphLaunch(b->exec, ctx->stream));
        for (auto &w : b->waves) ctx->stats.launches += 1 + (w.pairs.empty() ? 0 : 1);
    } else {
        ABC_TRY(enqueue_batch(ctx, b, d_masks_u, d_masks_v));
    }
    // pairs of small alpha are peeled one at a time by the single peel, always the plain one (the
    // batch stays index-free): there a chain would walk far more rows than the separate peels,
    // whose degree prefixes leave most of them out
    int plain_rc = ABCORE_OK;
    bool plain_any = false;
    for (int32_t i = 0; i < n && !plain_rc; ++i) {
        if (alphas[i] >= ctx->prm.batch_plain_below) continue;
        plain_any = true;
        plain_rc = peel_compute(ctx, alphas[i], betas[i], d_masks_u + (size_t)i * g.nU, d_masks_v + (size_t)i * g.nV,
                                false, false);
    }
    if (timed) ABC_CU(cudaEventRecord(b->ev1, ctx->stream));
    ABC_CU(cudaGetLastError());
    (void)sync_and_check;
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    if (plain_any) {
        const int frc = peel_finish(ctx);
        if (!plain_rc) plain_rc = frc;
    }
    if (plain_rc) return plain_rc;
    int first_err = 0;
    abcore_stats &s = ctx->stats;
    for (size_t wi = 0; wi < b->waves.size(); ++wi)
        for (size_t c = 0; c < b->waves[wi].chains.size(); ++c) {
            const PeelCtl &pc = b->ctl_host[wi * MAX_CHAINS_PER_WAVE + c];
            if (pc.err && !first_err) first_err = pc.err;
            s.peels += (int64_t)pc.st[ST_STEPS];
            s.candidates += b->waves[wi].chains[c].pU0 + b->waves[wi].chains[c].pV0;
            s.init_vertices += (int64_t)pc.st[ST_INIT];
            s.search_probes += (int64_t)pc.st[ST_PROBES];
            s.stream_entries += (int64_t)pc.st[ST_STREAM];
            s.entries += (int64_t)pc.st[ST_ENTRIES];
            s.decrements += (int64_t)pc.st[ST_DECS] + (int64_t)pc.st[ST_SDECS];
            s.stream_decrements += (int64_t)pc.st[ST_SDECS];
            s.pushes += (int64_t)pc.st[ST_PUSHES];
            s.items += (int64_t)pc.st[ST_ITEMS];
        }
    for (auto &w : b->waves) s.emit_gathered += (int64_t)w.pairs.size() * g.n();
    if (b->prof && ctx->prm.log_level >= 2) {
        // per chain: the wave, alpha, and each step's duration in microseconds (step 0 includes
        // the count init and the first round)
        std::vector<unsigned long long> h(b->waves.size() * MAX_CHAINS_PER_WAVE * PROF_STRIDE);
        if (cudaMemcpy(h.data(), b->prof, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost) == cudaSuccess) {
            for (size_t wi = 0; wi < b->waves.size(); ++wi)
                for (size_t c = 0; c < b->waves[wi].chains.size(); ++c) {
                    const ChainDev &cd = b->waves[wi].chains[c];
                    const unsigned long long *t = h.data() + (wi * MAX_CHAINS_PER_WAVE + c) * PROF_STRIDE;
                    std::string line;
                    char tmp[64];
                    unsigned long long prev = t[0];
                    for (int j = 0; j < cd.nsteps; ++j) {
                        const unsigned long long a0 = t[prof_at(j, 0)], a1 = t[prof_at(j, 1)], a2 = t[prof_at(j, 2)];
                        snprintf(tmp, sizeof(tmp), " %.0f/%.0f/%.0f", (double)(a0 - prev) / 1e3, (double)(a1 - a0) / 1e3,
                                 (double)(a2 - a1) / 1e3);
                        line += tmp;
                        prev = a2;
                    }
                    ctx->log(2, "batch wave %zu chain alpha=%d blocks=%d total %.1f us; steps (walk/scan/cascade us):%s", wi,
                             cd.alpha, cd.nblocks, (double)(t[prof_at(cd.nsteps - 1, 2)] - t[0]) / 1e3, line.c_str());
                }
        }
    }
    if (timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess) {
            s.kernel_ms[ABCORE_K_BATCH] += ms;
            s.kernel_launches[ABCORE_K_BATCH]++;
        }
    }
    if (first_err) {
        b->q_dirty = true;
        if (first_err == ABCORE_ETIMEDOUT)
            return ctx->fail(ABCORE_ETIMEDOUT, "batch: a bounded device wait expired (limit %lld ms)",
                             (long long)ctx->prm.timeout_ms);
        return ctx->fail(first_err, "batch: device reported error %d", first_err);
    }
    return ABCORE_OK;
}
