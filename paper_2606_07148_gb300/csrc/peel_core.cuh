// Cascade machinery shared by the single, batched and served peels.
//
// The peel (Algorithm 1, the GCC peel phase) removes a vertex x and lowers the live-neighbour
// count of every candidate neighbour y; y is removed when its count crosses below its bound.
// Here the crossing is detected exactly once per vertex: atomicSub returns the old count, and
// only the decrement that takes it from thr(y) to thr(y) - 1 queues y. Because the core is the
// unique fixpoint, the order of removals does not matter, so instead of rounds separated by
// barriers the removals flow through one device-wide work queue: warps grab queued row chunks,
// decrement, and queue the vertices they cause to fall, until a termination check proves the
// queue drained (every reserved slot processed, nothing in flight).
//
// Queue items are (vertex << 32 | chunk index); a row of length L is split into
// ceil(L / chunk) items so a hub's neighbours spread over many warps. Empty slots hold ~0ull;
// the consumer of a slot writes ~0ull back, so the queue is all-empty between peels.
#pragma once

#include "device.cuh"
#include "internal.h"

namespace abc {

constexpr unsigned long long EMPTY = ~0ull;
// one close flag per block, each on its own 128-byte line
constexpr int FLAG_STRIDE = 32;
constexpr int MAX_GRAB = 32;
constexpr int TRACE_SAMPLES = 2048;  // queue samples kept per traced cascade
constexpr int TRACE_BLOCKS = 2048;   // blocks whose exit and emission end times are kept
// header (sample count, watcher start ns), samples, then per block: cascade exit, emission end
constexpr int TRACE_WORDS = 4 + 4 * TRACE_SAMPLES + 2 * TRACE_BLOCKS;

// Per-warp buffer of fallen vertices waiting to be queued (see push_add).
template <int CAP>
struct PushBuf {
    static_assert(CAP >= 64, "a flush must leave room for one warp's pushes");
    int32_t y[CAP];  // vertex
    int32_t c[CAP];  // first chunk index
    int32_t n[CAP];  // item count: chunks [c, c + n)
};

struct WarpSmem {
    long long start[MAX_GRAB];  // first adjacency index of each grabbed item
    int excl[MAX_GRAB];         // exclusive prefix of item lengths
    int upper[MAX_GRAB];        // 1 if the item's row belongs to a U vertex
    PushBuf<256> push;
};

struct LaneStats {
    unsigned long long entries = 0, decs = 0, pushes = 0, items = 0;
};

// Adjacency is read once per peel: load it with the evict-first (streaming) policy so it does
// not push the counts -- the atomics' working set -- out of L2.
__device__ __forceinline__ int32_t ld_adj(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ int4 ld_adj4(const int4 *p) { return __ldcs(p); }

// A violator-stream entry y skips a hub: its count came from a search and already excludes
// every initial violator.
__device__ __forceinline__ bool stream_skips(const PeelArgs &a, int32_t y, bool upper_row) {
    return upper_row ? (y - a.nU < a.hubcutV) : (y < a.hubcutU);
}

// Candidate test and bound of a neighbour y seen from a row of layer `upper_row`.
__device__ __forceinline__ bool cand_of(const PeelArgs &a, int32_t y, bool upper_row, int32_t &thr) {
    if (upper_row) {
        thr = a.thrV;
        return y < a.nU + a.pV && y >= a.nU + a.cV;
    }
    thr = a.thrU;
    return y < a.pU && y >= a.cU;
}

// Counts, as int32 or (packed, when every degree fits 16 bits) as uint16 halves of 32-bit words:
// half the footprint keeps more of them in L2. A packed decrement subtracts from the word holding
// the count; a count is never decremented below zero (each decrement stands for a distinct live
// neighbour falling), so no borrow crosses into the other half.
// Slot of vertex x's count (PeelArgs::swz): the odd multiplier makes the per-layer map a
// bijection of the layer's power-of-two range.
constexpr unsigned long long SWZ_MUL = 0x9E3779B1ull;
__device__ __forceinline__ int64_t cnt_slot(const PeelArgs &a, int32_t x) {
    if (!a.swz) return x;
    if (x < a.nU) return (int64_t)(((unsigned long long)(uint32_t)x * SWZ_MUL) & a.swz_mask_u);
    return a.swz_base_v + (int64_t)(((unsigned long long)(uint32_t)(x - a.nU) * SWZ_MUL) & a.swz_mask_v);
}
__device__ __forceinline__ int cnt_load(const PeelArgs &a, int32_t x) {
    const int64_t s = cnt_slot(a, x);
    return a.packed ? (int)__ldcg(reinterpret_cast<const unsigned short *>(a.cnt) + s) : __ldcg(&a.cnt[s]);
}
__device__ __forceinline__ void cnt_store(const PeelArgs &a, int32_t x, int v) {
    const int64_t s = cnt_slot(a, x);
    if (a.packed) reinterpret_cast<unsigned short *>(a.cnt)[s] = (unsigned short)v;
    else a.cnt[s] = v;
}
__device__ __forceinline__ int cnt_dec(const PeelArgs &a, int32_t x) {  // returns the old count
    const int64_t s = cnt_slot(a, x);
    if (!a.packed) return atomicSub(&a.cnt[s], 1);
    const unsigned sh = (unsigned)(s & 1) << 4;
    const unsigned old = atomicSub(reinterpret_cast<unsigned *>(a.cnt) + (s >> 1), 1u << sh);
    return (int)((old >> sh) & 0xffffu);
}
__device__ __forceinline__ void cnt_dec_noret(const PeelArgs &a, int32_t x) {
    const int64_t s = cnt_slot(a, x);
    if (!a.packed) atomicAdd(&a.cnt[s], -1);
    else atomicSub(reinterpret_cast<unsigned *>(a.cnt) + (s >> 1), 1u << ((unsigned)(s & 1) << 4));
}
// v decrements of x's count at once (v never exceeds the count, as above), no return.
__device__ __forceinline__ void cnt_sub_noret(const PeelArgs &a, int32_t x, int v) {
    const int64_t s = cnt_slot(a, x);
    if (!a.packed) atomicAdd(&a.cnt[s], -v);
    else atomicSub(reinterpret_cast<unsigned *>(a.cnt) + (s >> 1), (unsigned)v << ((unsigned)(s & 1) << 4));
}

// Row length that a removed candidate x must still walk: the candidate prefix length kept in
// plen[x] (the full degree when its layer's counts came from the full rows).
__device__ __forceinline__ int row_len_of(const PeelArgs &a, int32_t y) { return __ldcg(&a.plen[y]); }

// Pushes are buffered per warp and queued in bulk: one atomicAdd on the queue's tail reserves
// the slots of many fallen vertices at once (tail is a single hot word that every pusher hits).
//
// Warp-collective: queue the buffered vertices (pb.*[0, pc)) and empty the buffer.
template <int CAP>
__device__ __forceinline__ void push_flush(const PeelArgs &a, PushBuf<CAP> &pb, int &pc) {
    if (pc == 0) return;
    __syncwarp();
    const int lane = threadIdx.x & 31;
    int mine = 0;
    for (int i = lane; i < pc; i += 32) mine += pb.n[i];
    const int incl = warp_incl_scan(mine);
    const int total = __shfl_sync(ABC_FULL, incl, 31);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.ctl->tail, (unsigned long long)total);
    base = __shfl_sync(ABC_FULL, base, 0);
    if (base + (unsigned long long)total > (unsigned long long)a.qcap) {
        if (lane == 0) set_error(&a.ctl->err, ABCORE_ENOMEM);
    } else {
        unsigned long long pos = base + (unsigned long long)(incl - mine);
        for (int i = lane; i < pc; i += 32) {
            const unsigned long long hi = (unsigned long long)(uint32_t)pb.y[i] << 32;
            const int nch = pb.n[i];
            const unsigned c0 = (unsigned)pb.c[i];
            for (int c = 0; c < nch; ++c) st_relaxed(&a.q[pos + c], hi | (c0 + (unsigned)c));
            pos += (unsigned long long)nch;
        }
    }
    __syncwarp();
    pc = 0;
}

// Block-collective push_flush: one atomic on tail reserves the slots of all the block's warps
// (for kernels whose every warp flushes at the end at about the same time).
template <int CAP>
__device__ __forceinline__ void push_flush_block(const PeelArgs &a, PushBuf<CAP> &pb, int &pc) {
    __shared__ unsigned long long s_qbase;
    __shared__ int s_wtot[32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    __syncwarp();
    int mine = 0;
    for (int i = lane; i < pc; i += 32) mine += pb.n[i];
    const int incl = warp_incl_scan(mine);
    const int total = __shfl_sync(ABC_FULL, incl, 31);
    if (lane == 0) s_wtot[wib] = total;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long bt = 0;
        for (int w = 0; w < nwb; ++w) bt += (unsigned long long)s_wtot[w];
        unsigned long long b0 = bt ? atomicAdd(&a.ctl->tail, bt) : 0ull;
        if (bt && b0 + bt > (unsigned long long)a.qcap) {
            set_error(&a.ctl->err, ABCORE_ENOMEM);
            b0 = ~0ull;
        }
        s_qbase = b0;
    }
    __syncthreads();
    const unsigned long long b0 = s_qbase;
    if (b0 != ~0ull && total > 0) {
        unsigned long long pos = b0 + (unsigned long long)(incl - mine);
        for (int w = 0; w < wib; ++w) pos += (unsigned long long)s_wtot[w];
        for (int i = lane; i < pc; i += 32) {
            const unsigned long long hi = (unsigned long long)(uint32_t)pb.y[i] << 32;
            const int nch = pb.n[i];
            const unsigned c0 = (unsigned)pb.c[i];
            for (int c = 0; c < nch; ++c) st_relaxed(&a.q[pos + c], hi | (c0 + (unsigned)c));
            pos += (unsigned long long)nch;
        }
    }
    __syncthreads();
    pc = 0;
}

// Warp-collective: lanes with `want` queue nch items of vertex y, chunks [c0, c0 + nch); nch == 0
// queues nothing. With `fallen`, y is a vertex that has just fallen (it is counted, and its
// removal step recorded). Flushes when the buffer is nearly full.
// Record removed candidate x (caller id o within its layer) in the caller-order bitmap.
__device__ __forceinline__ void mark_fallen(const PeelArgs &a, int32_t x, int32_t o) {
    const uint32_t u = (uint32_t)(x < a.nU ? o : a.nU + o);
    atomicOr(&a.fallen[u >> 5], 1u << (u & 31));
}

// Whether vertex x has not fallen in this chain yet (always true outside batch chains).
__device__ __forceinline__ bool chain_alive(const PeelArgs &a, int32_t x) {
    return a.lvl == nullptr || __ldcg(&a.lvl[(size_t)x * a.lvl_stride + a.lvl_col]) == 0xFF;
}

// Whether candidate x is known to be outside this step's core before any count is looked at.
__device__ __forceinline__ bool known_dead(const PeelArgs &a, int32_t x) {
    if (a.lvl == nullptr) return false;
    const uint8_t *row = a.lvl + (size_t)x * a.lvl_stride;
    return (a.dead_own && __ldcg(&row[a.lvl_col]) != 0xFF) ||
           (a.seed_col >= 0 && __ldcg(&row[a.seed_col]) <= (uint8_t)a.step);
}

template <int CAP>
__device__ __forceinline__ void push_add(const PeelArgs &a, PushBuf<CAP> &pb, int &pc, bool want, int32_t y, int nch,
                                         LaneStats &ls, bool fallen = true, int c0 = 0) {
    if (want && fallen) {
        ls.pushes++;
        // a removal with an empty row is never queued, so nothing else would record it
        if (nch == 0 && a.fallen != nullptr) mark_fallen(a, y, __ldg(&a.new2old[y]));
        if (a.lvl) {
            // the step a vertex first falls at
            uint8_t *l = a.lvl + (size_t)y * a.lvl_stride + a.lvl_col;
            if (*l == 0xFF) *l = (uint8_t)a.step;
        }
        if (a.corev) a.corev[y] = a.step;
    }
    if (a.removed) {
        const unsigned fm = __ballot_sync(ABC_FULL, want && fallen);
        if (fm && (threadIdx.x & 31) == 0) atomicAdd(a.removed, (unsigned long long)__popc(fm));
    }
    const bool keep = want && nch > 0;
    const unsigned pm = __ballot_sync(ABC_FULL, keep);
    if (pm == 0) return;
    if (keep) {
        const int i = pc + __popc(pm & lanemask_lt());
        pb.y[i] = y;
        pb.c[i] = c0;
        pb.n[i] = nch;
    }
    pc += __popc(pm);
    if (pc > CAP - 32) push_flush(a, pb, pc);
}

__device__ __forceinline__ int chunks_of(int len, int chunk) { return (len + chunk - 1) / chunk; }


// Length of the prefix of the sorted row adj[s, e) (s < e) holding ids below `bound`: the row's
// candidate neighbours. The search reads whole 32-byte sectors (the 8 entries of the aligned
// sector, clipped to the open range) and starts at s + frac * (e - s), frac being the share of
// the whole layer's adjacency entries that lie below the bound -- where the boundary of a row
// whose neighbours are drawn like everyone else's falls. From there it gallops outward in
// doubling steps until the boundary is bracketed, then bisects. The result does not depend on
// frac; a good guess settles most rows in one sector where bisection reads log2(length / 8).
// `probes` counts the sectors read.
__device__ __forceinline__ int row_prefix(const int32_t *__restrict__ adj, int64_t s, int64_t e, int32_t bound,
                                          float frac, unsigned long long &probes) {
    const int32_t *row = adj + s;
    const int d = (int)(e - s);
    int lo = 0, hi = d;  // the boundary (first index holding an id >= bound, or d) is in [lo, hi]
    int p = (int)(frac * (float)d);
    p = p < 0 ? 0 : (p >= d ? d - 1 : p);
    const int mis = (int)((reinterpret_cast<uintptr_t>(row) >> 2) & 7);  // entries past a sector start
    int dist = 8;
    int dir = 0;  // 0: first probe; +1 / -1: galloping right / left; 2: bracketed, bisecting
    while (lo < hi) {  // p is in [lo, hi): every pass shrinks the range
        const int w = ((p + mis) & ~7) - mis;
        const int w0 = max(w, lo), w1 = min(w + 8, hi);
        int below = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = w + k;
            if (i >= w0 && i < w1) below += __ldg(&row[i]) < bound ? 1 : 0;
        }
        probes++;
        if (below > 0 && below < w1 - w0) return w0 + below;
        const int want = below == 0 ? -1 : 1;
        if (below == 0) hi = w0;
        else lo = w1;
        if (lo >= hi) break;
        if (dir == 0 || dir == want) {
            dir = want;
            // (a row is shorter than 2^31, so w1 - 1 + dist stays in range: dist < 2 * d)
            p = want > 0 ? w1 - 1 + dist : w0 - dist;
            dist <<= 1;
            p = p < lo ? lo : (p >= hi ? hi - 1 : p);
        } else {
            dir = 2;
        }
        if (dir == 2) p = lo + ((hi - lo) >> 1);
    }
    return lo;
}

// Entries handled per lane per step by the streaming and cascade loops: the loads, then the
// atomics, of one step are independent, so they overlap instead of waiting one at a time.
constexpr int ILP = 4;

// Two limits shape a warp's batch (PeelArgs): batch_entries, the entries one warp walks per
// batch at most -- items beyond go back to the queue for other warps (a warp holding 32 chunks of
// hub rows would otherwise walk them alone while others idle); and flush_steps, the steps a
// pending push may wait before its warp flushes (a batch producing few pushes would otherwise
// hold them, and the cascade's next level, until it ends).

// Warp-collective: process the items held by the lanes (`it` == EMPTY: none), spreading the
// row chunks' entries evenly over the lanes (warp-level load balancing over an exclusive scan).
//
// A vertex that falls during the cascade is queued as one item, chunk 0; whoever takes chunk 0
// of a row longer than one chunk queues the row's other chunks. (The pusher would otherwise
// have to read the fallen vertex's row length, one more dependent memory round trip per push.)
//
// Pushes still buffered when the batch ends are left in sm.push (pc entries) for the caller.
template <bool PIPE>
__device__ __forceinline__ void process_items(const PeelArgs &a, unsigned long long it, WarpSmem &sm,
                                              LaneStats &ls, int &pc, int lim) {
    const int lane = threadIdx.x & 31;
    long long start = 0;
    int len = 0, upper = 0, more = 0, c = 0;
    int32_t x = 0, o = -1;
    if (it != EMPTY) {
        x = (int32_t)(it >> 32);
        c = (int)(it & 0xffffffffu);
        if (a.fallen != nullptr && c == 0) o = __ldg(&a.new2old[x]);  // caller id, for the bitmap
        int rl = row_len_of(a, x);
        const long long s0 = __ldg(&a.off[x]);
        // a chain step with a narrower V prefix: a U row's candidates are its entries below it
        if (x < a.nU && a.pV < a.pV_rows && rl > 0) {
            unsigned long long probes = 0;
            rl = row_prefix(a.adj, s0, s0 + rl, a.nU + a.pV, a.frac_rows, probes);
        }
        // a count of 0 means every candidate neighbour has fallen and decremented this vertex
        // already: walking its row would only decrement fallen vertices, so the walk is skipped
        if (rl > 0 && cnt_load(a, x) == 0) rl = 0;
        start = s0 + (long long)c * a.chunk;
        len = min(a.chunk, rl - c * a.chunk);
        if (len < 0) len = 0;
        if (c == 0 && rl > a.chunk) more = chunks_of(rl, a.chunk) - 1;
        upper = x < a.nU;
    }
    int incl = warp_incl_scan(len);
    // items past `lim` entries (never the first non-empty one) go back to the queue untouched;
    // a kept chunk 0 of a long row queues the row's other chunks
    const bool defer = incl - len >= lim && it != EMPTY;
    push_add(a, sm.push, pc, defer, x, 1, ls, /*fallen=*/false, /*c0=*/c);
    push_add(a, sm.push, pc, more > 0 && !defer, x, more, ls, /*fallen=*/false, /*c0=*/1);
    if (defer) len = 0;
    if (it != EMPTY && !defer) ls.items++;
    if (o >= 0 && !defer) mark_fallen(a, x, o);
    push_flush(a, sm.push, pc);
    incl = warp_incl_scan(len);
    const int L = __shfl_sync(ABC_FULL, incl, 31);
    sm.start[lane] = start;
    sm.excl[lane] = incl - len;
    sm.upper[lane] = upper;
    __syncwarp();
    int j = 0, since = 0;
    // With PIPE (software pipelining), the adjacency entries of step b + 32 * ILP are loaded
    // before the atomics of step b are issued, so each step waits for one memory round trip
    // instead of two; it costs registers (kernels already short of them leave it off).
    int32_t ny[ILP];
    int32_t nthr[ILP];
    bool nhit[ILP];
    auto load_step = [&](int b) {
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            const int e = b + 32 * u + lane;
            nhit[u] = false;
            ny[u] = 0;
            nthr[u] = 0;
            if (e < L) {
                while (j + 1 < 32 && sm.excl[j + 1] <= e) ++j;
                ny[u] = ld_adj(&a.adj[sm.start[j] + (e - sm.excl[j])]);
                nthr[u] = sm.upper[j];  // layer of the row, resolved below
                nhit[u] = true;
            }
        }
    };
    if (PIPE) load_step(0);
    for (int b = 0; b < L; b += 32 * ILP) {
        if (!PIPE) load_step(b);
        int32_t y[ILP];
        int32_t thr[ILP];
        bool hit[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            y[u] = ny[u];
            thr[u] = nthr[u];
            hit[u] = nhit[u];
        }
        if (PIPE && b + 32 * ILP < L) load_step(b + 32 * ILP);
        int old[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            if (hit[u]) {
                ls.entries++;
                int32_t t;
                hit[u] = cand_of(a, y[u], thr[u] != 0, t) && (t > 0 || !a.skip_zero);
                thr[u] = t;
            }
        }
#pragma unroll
        for (int u = 0; u < ILP; ++u) old[u] = hit[u] ? cnt_dec(a, y[u]) : 0;
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            if (hit[u]) ls.decs++;
            // the crossing decrement: y had a count of 1 or more, so its row is not empty (a vertex a
            // seeded chain step queued as known dead may still cross: it is not queued twice)
            push_add(a, sm.push, pc, hit[u] && old[u] == thr[u] && (a.dead_own == 0 || chain_alive(a, y[u])), y[u], 1, ls);
        }
        ++since;
        if (pc >= 32 || (pc > 0 && since >= a.flush_steps)) {
            push_flush(a, sm.push, pc);
            since = 0;
        }
    }
    __syncwarp();
}

// Warp-collective: if the buffered pushes make at most 32 items, hand lane l the l-th of them and
// empty the buffer (true); otherwise leave the buffer alone (false).
__device__ __forceinline__ bool take_local(WarpSmem &sm, int &pc, unsigned long long &it) {
    const int lane = threadIdx.x & 31;
    int mine = 0;
    for (int i = lane; i < pc; i += 32) mine += sm.push.n[i];
    const int total = __shfl_sync(ABC_FULL, warp_incl_scan(mine), 31);
    if (total > 32) return false;
    // entry i covers items [first_i, first_i + n_i) in buffer order
    it = EMPTY;
    int first = 0;
    for (int i = 0; i < pc; ++i) {
        const int nn = sm.push.n[i];
        if (lane >= first && lane < first + nn)
            it = ((unsigned long long)(uint32_t)sm.push.y[i] << 32) | (unsigned)(sm.push.c[i] + (lane - first));
        first += nn;
    }
    __syncwarp();
    pc = 0;
    return true;
}

// `head` is set to CLOSED when the queue drains; a ticket grab that returns CLOSED or more ends
// the holder's loop.
constexpr unsigned long long CLOSED = 1ull << 62;

__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The watcher closes a drained (or failed) queue: head moves to CLOSED, so no warp can take a
// ticket any more, and every block of the launch (or chain) gets the closing epoch in its own
// flag line. Warp-collective.
__device__ __forceinline__ void close_queue(const PeelArgs &a) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) atomicExch(&a.ctl->head, CLOSED);
    for (int i = lane; i < a.flag_count; i += 32)
        st_relaxed_u32(a.flags + (size_t)(a.flag_first + i) * FLAG_STRIDE, a.epoch);
    __syncwarp();
}

// Block-collective cascade loop (every warp of the block calls it): returns 1 when the queue
// drained, 0 on error.
//
// Work is handed out by ticket: lane 0 takes k consecutive slot numbers with one atomicAdd on
// `head` (k grows with the visible backlog), and lane l owns slot base + l. Pushers fill slots
// in reservation order, so a ticket below `tail` is filled soon. Items are processed as soon as
// any lane's slot is filled; lanes still waiting keep their tickets (holding items while
// waiting could starve the very pushes that fill the remaining slots).
//
// Termination: one warp of the launch (the watcher) reads done and tail while it is idle.
// done == tail means nothing is in flight, so nothing can be queued any more (done is read
// before tail; both only grow and done <= tail, so equality at those two reads proves the queue
// drained). The watcher then closes the queue (close_queue). Each block's first warp polls only
// its block's own flag line, and every warp that learns of the close (from the flag, from a
// CLOSED grab, or from an error) passes the news to the block's other warps in shared memory;
// tickets still waiting are at or above tail and were never filled, so their slots are empty
// and can simply be abandoned. Thousands of idle warps thus never poll the words that the
// pushers' atomics need. Every waiting warp still checks the error word, and whether `done`
// moves, on every 64th idle poll: with no progress for timeout_ns it records ABCORE_ETIMEDOUT and
// leaves. A watcher that sees an error closes the queue so that everyone leaves promptly.
template <bool PIPE = true>
__device__ __forceinline__ int cascade_loop(const PeelArgs &a, WarpSmem &sm, LaneStats &ls, int grab_div,
                                            bool watcher) {
    __shared__ volatile uint32_t s_closed;  // == a.epoch once this block learnt of the close
    const int lane = threadIdx.x & 31;
    const bool leader = (threadIdx.x >> 5) == 0;
    if (threadIdx.x == 0) s_closed = 0;
    // the block holding a tracing watcher (which takes no work)
    const int obs = __syncthreads_or(watcher && a.trace != nullptr) ? 1 : 0;
    // The first grab is one atomic on head for the whole block: at launch every warp would grab
    // at once, and thousands of atomics on that one word take turns.
    __shared__ unsigned long long s_base;
    __shared__ int s_k, s_lim;
    if (threadIdx.x == 0) {
        s_k = 0;
        s_lim = a.batch_entries;
        const int nwk = (int)(blockDim.x >> 5) - obs;
        const unsigned long long t = ld_relaxed(&a.ctl->tail);
        const unsigned long long h = ld_relaxed(&a.ctl->head);
        if (nwk > 0 && t > h && h < CLOSED) {
            const unsigned long long kk = (t - h) / (unsigned long long)grab_div;
            const int k = (int)(kk < 1 ? 1 : (kk > MAX_GRAB ? MAX_GRAB : kk));
            const unsigned long long total = (unsigned long long)k * (unsigned long long)nwk;
            const unsigned long long base = atomicAdd(&a.ctl->head, total);
            if (base < CLOSED) {
                if (base + total > (unsigned long long)a.qcap) {
                    set_error(&a.ctl->err, ABCORE_ENOMEM);
                } else {
                    s_base = base;
                    s_k = k;
                    if (a.batch_entries_small > 0 && t < base + total + (unsigned long long)grab_div * 8ull)
                        s_lim = a.batch_entries_small;
                }
            }
        }
    }
    __syncthreads();
    if (watcher && a.trace != nullptr) {
        // Diagnostics: the watcher takes no work; its lane 0 samples done, tail and head about
        // every microsecond (the first TRACE_SAMPLES samples are kept) until the queue drains,
        // fails or stalls for timeout_ns, then closes it as the watcher would.
        int verdict = 0;
        if (lane == 0) {
            const unsigned long long t0 = now_ns();
            a.trace[1] = t0;
            unsigned long long idle_since = t0, last_done = ~0ull, k = 0;
            for (;;) {
                const unsigned long long d = ld_acquire(&a.ctl->done);
                const unsigned long long tl = ld_acquire(&a.ctl->tail);
                const unsigned long long h = ld_relaxed(&a.ctl->head);
                const unsigned long long tn = now_ns();
                if (k < (unsigned long long)TRACE_SAMPLES) {
                    unsigned long long *smp = a.trace + 4 + 4 * k;
                    smp[0] = tn - t0;
                    smp[1] = d;
                    smp[2] = tl;
                    smp[3] = h;
                }
                ++k;
                if (ld_relaxed_i32(&a.ctl->err) != 0) {
                    verdict = 3;
                    break;
                }
                if (d == tl) {
                    verdict = 1;
                    break;
                }
                if (d != last_done) {
                    last_done = d;
                    idle_since = tn;
                } else if (tn - idle_since > a.timeout_ns) {
                    set_error(&a.ctl->err, ABCORE_ETIMEDOUT);
                    verdict = 3;
                    break;
                }
                __nanosleep(1000);
            }
            a.trace[0] = k < (unsigned long long)TRACE_SAMPLES ? k : (unsigned long long)TRACE_SAMPLES;
        }
        verdict = __shfl_sync(ABC_FULL, verdict, 0);
        close_queue(a);
        if (lane == 0) s_closed = a.epoch;
        return verdict == 1 ? 1 : 0;
    }
    const uint32_t *myflag = a.flags + (size_t)blockIdx.x * FLAG_STRIDE;
    unsigned long long idle_since = now_ns(), last_done = ~0ull;
    int st = 2;  // this lane's ticket: 0 waiting, 2 none
    int lim = a.batch_entries;  // entries per batch, chosen at each grab
    unsigned long long my = 0;
    if (s_k > 0) {  // this warp's share of the block's first grab
        my = s_base + (unsigned long long)(((int)(threadIdx.x >> 5) - obs) * s_k + lane);
        st = lane < s_k ? 0 : 2;
        lim = s_lim;
    }
    unsigned sleep_ns = 32;
    unsigned idle_polls = 0;
    for (;;) {
        if (__ballot_sync(ABC_FULL, st == 0) == 0) {  // no ticket held: take new ones
            unsigned long long base = 0;
            int k = 1, closed = 0;
            if (lane == 0) {
                if (s_closed == a.epoch) {
                    closed = 1;
                } else {
                    const unsigned long long t = ld_relaxed(&a.ctl->tail);
                    const unsigned long long h = ld_relaxed(&a.ctl->head);
                    if (t > h) {
                        const unsigned long long kk = (t - h) / (unsigned long long)grab_div;
                        k = (int)(kk < 1 ? 1 : (kk > MAX_GRAB ? MAX_GRAB : kk));
                    }
                    base = atomicAdd(&a.ctl->head, (unsigned long long)k);
                    // little left behind this grab: other warps are likely idle, so keep batches
                    // short and let them take what this one defers
                    lim = a.batch_entries;
                    if (a.batch_entries_small > 0 &&
                        t < base + (unsigned long long)k + (unsigned long long)grab_div * 8ull)
                        lim = a.batch_entries_small;
                    if (base >= CLOSED) closed = 1;
                    else if (base + (unsigned long long)k > (unsigned long long)a.qcap) {
                        // tickets past the end of the queue: only an overflowed queue gets here
                        set_error(&a.ctl->err, ABCORE_ENOMEM);
                        closed = 2;
                    }
                    if (closed) closed |= ld_relaxed_i32(&a.ctl->err) != 0 ? 2 : 0;
                }
            }
            closed = __shfl_sync(ABC_FULL, closed, 0);
            if (closed) {
                if (watcher && (closed & 2)) close_queue(a);
                if (lane == 0) s_closed = a.epoch;  // tell the block's waiting warps
                return (closed & 2) ? 0 : 1;
            }
            base = __shfl_sync(ABC_FULL, base, 0);
            k = __shfl_sync(ABC_FULL, k, 0);
            lim = __shfl_sync(ABC_FULL, lim, 0);
            my = base + (unsigned long long)lane;
            st = lane < k ? 0 : 2;
        }
        unsigned long long it = EMPTY;
        if (st == 0) {
            it = ld_relaxed(&a.q[my]);
            if (it != EMPTY) {
                st_relaxed(&a.q[my], EMPTY);
                st = 2;
            }
        }
        const unsigned have = __ballot_sync(ABC_FULL, it != EMPTY);
        if (have != 0) {
            // Work-first: what a batch leaves queued, if one warp can take it all, this warp takes
            // next, skipping the queue's round trip (in the deep, narrow levels of a cascade that
            // round trip is most of each level's latency). The batch's slots count as done only
            // after the whole chain, so the queue cannot look drained meanwhile.
            int pc = 0;
            process_items<PIPE>(a, it, sm, ls, pc, lim);
            for (int round = 0; pc > 0; ++round) {
                unsigned long long nxt = EMPTY;
                if (round >= a.local_rounds || !take_local(sm, pc, nxt)) {
                    push_flush(a, sm.push, pc);
                    break;
                }
                process_items<PIPE>(a, nxt, sm, ls, pc, lim);
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicAdd(&a.ctl->done, (unsigned long long)__popc(have));
            idle_since = now_ns();
            sleep_ns = 32;
            continue;
        }
        // nothing arrived: has the queue closed (drained, or failed)?
        int verdict = 0;  // 0 keep waiting, 1 drained, 3 error
        if (lane == 0) {
            if (s_closed == a.epoch) {
                verdict = 1;
            } else if (leader && ld_relaxed_u32(myflag) == a.epoch) {
                s_closed = a.epoch;
                verdict = 1;
            }
            if (verdict == 1 && ld_relaxed_i32(&a.ctl->err) != 0) verdict = 3;
            if (verdict == 0 && (watcher || (++idle_polls & 63) == 0)) {
                const unsigned long long d = ld_acquire(&a.ctl->done);
                const unsigned long long tcur = ld_acquire(&a.ctl->tail);
                if (ld_relaxed_i32(&a.ctl->err) != 0) verdict = 3;
                else if (watcher && d == tcur) verdict = 1;
                else if (d != last_done) {  // the device is making progress: restart the clock
                    last_done = d;
                    idle_since = now_ns();
                } else if (now_ns() - idle_since > a.timeout_ns) {
                    set_error(&a.ctl->err, ABCORE_ETIMEDOUT);
                    verdict = 3;
                }
            }
        }
        verdict = __shfl_sync(ABC_FULL, verdict, 0);
        if (verdict != 0) {
            if (watcher) close_queue(a);
            if (lane == 0) s_closed = a.epoch;  // tell the block's waiting warps
            return verdict == 1 ? 1 : 0;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 256) sleep_ns <<= 1;
    }
}

// Bounded barrier over the `G` blocks of one group (a batch chain, or a whole launch). The last block to arrive can run `fixup`
// while every other block of the group waits. Returns false if the group saw an error.
//
// With `watch`, the last block to arrive also records whether *watch has reached `limit` in
// bar[16], which every block can read once the barrier has passed (it changes only at the next
// such barrier, so all blocks read the same value).
__device__ __forceinline__ bool group_barrier(unsigned *bar, int G, PeelCtl *ctl, bool fixup, unsigned long long timeout_ns,
                                              const unsigned long long *watch = nullptr,
                                              unsigned long long limit = 0) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *genp = bar + 32;
        const unsigned gen = *genp;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == (unsigned)G - 1) {
            atomicExch(bar, 0u);
            if (watch) bar[16] = ld_relaxed(watch) >= limit ? 1u : 0u;
            if (fixup) {
                // the cascade closed the queue: every reserved slot [0, tail) was processed and
                // emptied by its consumer, and the tickets it voided, [tail, old head), were never
                // filled; so the whole queue is empty and the next step starts at slot 0 (a step
                // never needs more room than one peel, however many steps the chain has)
                atomicExch(&ctl->tail, 0ull);
                atomicExch(&ctl->head, 0ull);
                atomicExch(&ctl->done, 0ull);
            }
            __threadfence();
            atomicAdd(bar + 32, 1u);
        } else {
            const unsigned long long t0 = now_ns();
            unsigned sl = 32;
            while (*genp == gen) {
                if (now_ns() - t0 > timeout_ns) {
                    set_error(&ctl->err, ABCORE_ETIMEDOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(sl);
                if (sl < 512) sl <<= 1;
            }
        }
        __threadfence();
        if (ld_relaxed_i32(&ctl->err) != 0) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// Candidate counts (the scan phase): thread t of nthreads handles candidates t, t + nthreads, ...
// Per layer, the count is either the row prefix below the other layer's candidate boundary
// (binary search in the sorted row) or the full degree (to be corrected by stream_range).
// Candidates already below their bound are queued. Warp-collective; `t0` is warp-aligned.
template <int CAP>
__device__ __forceinline__ void init_range(const PeelArgs &a, PushBuf<CAP> &pb, int64_t t0, int64_t nthreads,
                                           LaneStats &ls, unsigned long long &probes, unsigned long long &inits) {
    // each lane takes INIT_ILP candidates per pass, so their offset loads are in flight together
    constexpr int INIT_ILP = 4;
    const int64_t nu = (int64_t)a.pU - a.cU, P = nu + (a.pV - a.cV);  // uncertain candidates
    const int lane = threadIdx.x & 31;
    int pc = 0;
    // the share of U-row entries that are V candidates (the candidates' total degree over m), and
    // of V-row entries that are U candidates: each row search starts from it
    const int64_t mU = __ldg(&a.off[a.nU]), mV = __ldg(&a.off[(int64_t)a.nU + a.nV]) - mU;
    const float fracU = mU > 0 ? (float)(__ldg(&a.off[(int64_t)a.nU + a.pV]) - mU) / (float)mU : 0.f;
    const float fracV = mV > 0 ? (float)__ldg(&a.off[a.pU]) / (float)mV : 0.f;
    for (int64_t b = t0 - lane; b < P; b += nthreads * INIT_ILP) {
        int32_t x[INIT_ILP];
        int64_t s[INIT_ILP], e[INIT_ILP];
#pragma unroll
        for (int k = 0; k < INIT_ILP; ++k) {
            const int64_t i = b + lane + k * nthreads;
            x[k] = -1;
            s[k] = e[k] = 0;
            if (i < P) {
                x[k] = i < nu ? (int32_t)(a.cU + i) : (int32_t)(a.nU + a.cV + (i - nu));
                s[k] = __ldg(&a.off[x[k]]);
                e[k] = __ldg(&a.off[x[k] + 1]);
            }
        }
        bool viol[INIT_ILP];
        int len[INIT_ILP];
#pragma unroll
        for (int k = 0; k < INIT_ILP; ++k) {
            viol[k] = false;
            len[k] = 0;
            const bool upper = x[k] >= 0 && x[k] < a.nU;
            if (x[k] >= 0) {
                const bool hubx = upper ? x[k] < a.hubcutU : x[k] - a.nU < a.hubcutV;
                if ((upper ? a.searchU : a.searchV) || hubx) {
                    // candidate neighbours form the row's prefix below the other layer's bound
                    const int32_t bound = upper ? a.nU + a.pV : a.pU;
                    len[k] = e[k] == s[k] ? 0 : row_prefix(a.adj, s[k], e[k], bound, upper ? fracU : fracV, probes);
                } else {
                    len[k] = (int)(e[k] - s[k]);
                }
                viol[k] = len[k] < (upper ? a.thrU : a.thrV) || known_dead(a, x[k]);
                cnt_store(a, x[k], len[k]);
                a.plen[x[k]] = len[k];
                inits++;
            }
        }
        if (a.round0) {
            // listed for k_round0 instead of queued: one reservation on the list's shared counter
            // for the warp's violators of all INIT_ILP passes
            unsigned vm[INIT_ILP];
            int tot = 0;
#pragma unroll
            for (int k = 0; k < INIT_ILP; ++k) {
                vm[k] = __ballot_sync(ABC_FULL, viol[k]);
                tot += __popc(vm[k]);
            }
            if (tot) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&a.ctl->l0n, (unsigned long long)tot);
                base = __shfl_sync(ABC_FULL, base, 0);
#pragma unroll
                for (int k = 0; k < INIT_ILP; ++k) {
                    if (viol[k]) {
                        const bool upper = x[k] < a.nU;
                        if (a.fallen != nullptr) mark_fallen(a, x[k], __ldg(&a.new2old[x[k]]));
                        // the row's first entry, length and layer: k_round0 needs nothing more
                        a.l0[base + __popc(vm[k] & lanemask_lt())] =
                            make_longlong2(s[k], (long long)len[k] | (upper ? L0_UPPER : 0));
                        ls.pushes++;
                    }
                    base += (unsigned long long)__popc(vm[k]);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < INIT_ILP; ++k)
                push_add(a, pb, pc, viol[k], x[k] < 0 ? 0 : x[k], len[k] > 0 ? 1 : 0, ls);  // chunk 0
        }
    }
    push_flush(a, pb, pc);
}

// One adjacency entry y of an initial violator's row: lower y's count if y is a candidate that
// counts by degree. No value is returned: whether a count fell below its bound is decided by
// scan_range once the whole stream is done (atomics without a return run faster).
__device__ __forceinline__ void stream_entry(const PeelArgs &a, int32_t y, bool from_upper, bool valid,
                                             LaneStats &ls) {
    int32_t thr = 0;
    if (valid && cand_of(a, y, from_upper, thr) && (thr > 0 || !a.skip_zero) && !stream_skips(a, y, from_upper)) {
        cnt_dec_noret(a, y);
        ls.decs++;
    }
}

// Stream the rows of the initial violators (the first peel round): slice A = adj[sa, ea) holds
// V rows (entries are U ids), slice B = adj[sb, eb) holds U rows. Interior read with 16-byte
// loads. Warp-collective; `t0` is this thread's index among nthreads (a multiple of 32).
__device__ __forceinline__ void stream_range(const PeelArgs &a, int64_t sa, int64_t ea, int64_t sb, int64_t eb,
                                             int64_t t0, int64_t nthreads, LaneStats &ls,
                                             unsigned long long &ents) {
    const int lane = threadIdx.x & 31;
    for (int sl = 0; sl < 2; ++sl) {
        const int64_t s = sl == 0 ? sa : sb, e = sl == 0 ? ea : eb;
        if (e <= s) continue;
        const bool from_upper = sl == 1;
        const int64_t a0 = min((s + 3) & ~(int64_t)3, e);
        const int64_t a1 = max(e & ~(int64_t)3, a0);
        const int64_t nh = (a0 - s) + (e - a1);
        for (int64_t b = t0 - lane; b < nh; b += nthreads) {
            const int64_t i = b + lane;
            const bool valid = i < nh;
            int32_t y = 0;
            if (valid) {
                const int64_t pos = i < (a0 - s) ? s + i : a1 + (i - (a0 - s));
                y = ld_adj(&a.adj[pos]);
                ents++;
            }
            stream_entry(a, y, from_upper, valid, ls);
        }
        const int64_t nv = (a1 - a0) >> 2;
        const int4 *v4 = reinterpret_cast<const int4 *>(a.adj + a0);
        // two 16-byte loads per lane per step
        for (int64_t b = 2 * (t0 - lane); b < nv; b += 2 * nthreads) {
            const int64_t i0 = b + lane, i1 = b + 32 + lane;
            const bool v0 = i0 < nv, v1 = i1 < nv;
            int4 q0 = make_int4(0, 0, 0, 0), q1 = make_int4(0, 0, 0, 0);
            if (v0) q0 = ld_adj4(&v4[i0]);
            if (v1) q1 = ld_adj4(&v4[i1]);
            ents += (v0 ? 4 : 0) + (v1 ? 4 : 0);
            stream_entry(a, q0.x, from_upper, v0, ls);
            stream_entry(a, q0.y, from_upper, v0, ls);
            stream_entry(a, q0.z, from_upper, v0, ls);
            stream_entry(a, q0.w, from_upper, v0, ls);
            stream_entry(a, q1.x, from_upper, v1, ls);
            stream_entry(a, q1.y, from_upper, v1, ls);
            stream_entry(a, q1.z, from_upper, v1, ls);
            stream_entry(a, q1.w, from_upper, v1, ls);
        }
    }
}

// After the violator stream: queue the candidates counted by degree whose count fell below
// their bound (hubs and searched layers were queued by init_range). Warp-collective; `t0` is
// this thread's index among nthreads.
template <int CAP, bool BLOCK = false>
__device__ __forceinline__ void scan_range(const PeelArgs &a, PushBuf<CAP> &pb, int64_t t0, int64_t nthreads,
                                           LaneStats &ls, unsigned long long &scanned) {
    const int lane = threadIdx.x & 31;
    int pc = 0;
    // U ids [u0, pU) and V ids nU + [v0, pV): the candidates counted by degree, or with round0
    // every uncertain candidate (the ones round0 already walked have plen below their bound)
    const int64_t u0 = a.round0 ? a.cU : (a.searchU ? a.pU : max(a.hubcutU, a.cU));
    const int64_t v0 = a.round0 ? a.cV : (a.searchV ? a.pV : max(a.hubcutV, a.cV));
    const int64_t nu = a.pU - u0, total = nu + (a.pV - v0);
    // SCAN_ILP candidates per lane per pass, so their count loads are in flight together
    constexpr int SCAN_ILP = 4;
    for (int64_t b = t0 - lane; b < total; b += nthreads * SCAN_ILP) {
        int32_t x[SCAN_ILP];
        int c[SCAN_ILP];
#pragma unroll
        for (int k = 0; k < SCAN_ILP; ++k) {
            const int64_t i = b + lane + k * nthreads;
            x[k] = -1;
            c[k] = 0;
            if (i < total) {
                x[k] = i < nu ? (int32_t)(u0 + i) : (int32_t)(a.nU + v0 + (i - nu));
                c[k] = cnt_load(a, x[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < SCAN_ILP; ++k) {
            bool viol = false;
            int nch = 0;
            if (x[k] >= 0) {
                const int thr = x[k] < a.nU ? a.thrU : a.thrV;
                // (a candidate the count init queued as known dead is not queued twice)
                viol = c[k] < thr && !(a.dead_own && !chain_alive(a, x[k]));
                if (viol) {
                    const int pl = __ldcg(&a.plen[x[k]]);
                    if (a.round0 && pl < thr) viol = false;  // an initial violator: round0 walked it
                    else nch = pl > 0 ? 1 : 0;               // chunk 0 (see process_items)
                }
                scanned++;
            }
            push_add(a, pb, pc, viol, x[k] < 0 ? 0 : x[k], nch, ls);
        }
    }
    if (BLOCK) push_flush_block(a, pb, pc);
    else push_flush(a, pb, pc);
}

// A batch chain's step with a higher V bound (thrV, prefix a.pV), run before its cascade: every
// live V candidate of the previous prefix [nU, nU + pv_prev) whose count misses the new bound --
// all those past the new prefix among them, their degree being below it -- falls now. Its fall is
// recorded (lvl) and its row is walked at once by the warp, lanes sharing out the 32 vertices'
// entries evenly, with decrements that return nothing: no crossing is looked for here, the U scan
// after it (fall_scan_u) finds every U candidate these decrements took below alpha. A vertex whose
// count is 0 has no live neighbour left and walks nothing. With `by_lvl` a V vertex is live iff
// its lvl is unset (seeded chains queue known-dead vertices whatever their count); otherwise iff
// its count meets the previous bound prev_thrV. Warp-collective; `t0` is warp-aligned.
// Block-collective when `tab` is set: decrements of the first WALK_HUBS U ids (the U hubs: ids
// follow degree, and a row's first entries are its hub neighbours) go to the block's shared tally
// `tab`, added to the counts (and the tally zeroed) once the block's walk is done. In vertex
// order the hubs' counts share a few L2 lines that every walking warp would otherwise hit; no
// crossing is looked for during the walk, so only the counts after it matter.
constexpr int WALK_HUBS = 2048;
__device__ __forceinline__ void fall_walk_v(const PeelArgs &a, WarpSmem &sm, int32_t pv_prev, int32_t prev_thrV,
                                            bool by_lvl, int64_t t0, int64_t nthreads, LaneStats &ls,
                                            unsigned long long &ents, unsigned long long &decs,
                                            unsigned *tab = nullptr) {
    const int lane = threadIdx.x & 31;
    // WILP groups of 32 vertices per warp per pass: all their count loads are issued first (one
    // vertex at a time would leave every lane waiting on a load per vertex), then each group's
    // falling rows are walked in turn
    constexpr int WILP = 4;
    for (int64_t b0 = t0 - lane; b0 < pv_prev; b0 += nthreads * WILP) {
        int cg[WILP];
#pragma unroll
        for (int k = 0; k < WILP; ++k) {
            const int64_t i = b0 + lane + k * nthreads;
            cg[k] = i < pv_prev ? cnt_load(a, (int32_t)(a.nU + i)) : 0;
        }
#pragma unroll 1
        for (int k = 0; k < WILP; ++k) {
            const int64_t b = b0 + k * nthreads;  // warp-uniform
            if (b >= pv_prev) break;
            const int64_t i = b + lane;
            const int32_t x = (int32_t)(a.nU + (i < pv_prev ? i : 0));
            bool fall = false;
            int len = 0;
            long long s = 0;
            if (i < pv_prev) {
                const int c = cg[k];
                const bool live = by_lvl ? chain_alive(a, x) : c >= prev_thrV;
                fall = live && (c < a.thrV || (a.seed_col >= 0 && known_dead(a, x)));
                if (fall) {
                    a.lvl[(size_t)x * a.lvl_stride + a.lvl_col] = (uint8_t)a.step;
                    ls.pushes++;
                    if (c > 0) {
                        len = __ldcg(&a.plen[x]);
                        s = __ldg(&a.off[x]);
                    }
                }
            }
            const int incl = warp_incl_scan(len);
            const int L = __shfl_sync(ABC_FULL, incl, 31);
            if (L == 0) continue;
            sm.start[lane] = s;
            sm.excl[lane] = incl - len;
            __syncwarp();
            int j = 0;
            for (int e0 = 0; e0 < L; e0 += 32 * ILP) {
                int32_t y[ILP];
#pragma unroll
                for (int u = 0; u < ILP; ++u) {
                    const int e = e0 + 32 * u + lane;
                    y[u] = -1;
                    if (e < L) {
                        while (j + 1 < 32 && sm.excl[j + 1] <= e) ++j;
                        y[u] = ld_adj(&a.adj[sm.start[j] + (e - sm.excl[j])]);
                    }
                }
#pragma unroll
                for (int u = 0; u < ILP; ++u) {
                    if (y[u] < 0) continue;
                    ents++;
                    if (y[u] < a.pU && y[u] >= a.cU) {  // a U candidate
                        if (tab != nullptr && y[u] < WALK_HUBS) atomicAdd(&tab[y[u]], 1u);
                        else cnt_dec_noret(a, y[u]);
                        decs++;
                    }
                }
            }
            __syncwarp();
        }
    }
    if (tab != nullptr) {
        __syncthreads();
        for (int i = threadIdx.x; i < WALK_HUBS; i += blockDim.x) {
            const unsigned v = tab[i];
            if (v != 0u) {
                cnt_sub_noret(a, i, (int)v);
                tab[i] = 0u;
            }
        }
    }
}

// After fall_walk_v: every U candidate that was live (lvl unset) and whose count is now below
// alpha falls, queued for the cascade. Each lane takes the 32 candidates of one word of `live`, a
// bitmap over the U prefix: with `full` every candidate of the prefix, else only those whose bit
// is set. The word is rewritten to hold the ones whose count still meets alpha (a fallen vertex's
// count stays below alpha, so the bits left set cover every live vertex, and later scans skip the
// rest). The 32 counts come in 16-byte loads (vertex order, which batch chains keep); a removal
// step is read only for a count below alpha. A U vertex live at a step has a live neighbour
// inside the step-0 V prefix, so its row prefix is never empty: it is queued as one item.
// Warp-collective; `t0` is warp-aligned; the count array holds at least 32 slots past the prefix.
__device__ __forceinline__ void fall_scan_u(const PeelArgs &a, WarpSmem &sm, int64_t t0, int64_t nthreads,
                                            LaneStats &ls, unsigned long long &scanned, uint32_t *live, bool full) {
    const int lane = threadIdx.x & 31;
    int pc = 0;
    const int64_t nwords = ((int64_t)a.pU + 31) >> 5;
    for (int64_t w = t0; w - lane < nwords; w += nthreads) {
        uint32_t bits = 0;
        if (w < nwords) {
            if (full) {
                const int64_t x0 = w << 5;
                const int64_t lo = max((int64_t)a.cU - x0, (int64_t)0), hi = min((int64_t)a.pU - x0, (int64_t)32);
                bits = lo >= hi ? 0u : ((hi == 32 ? ~0u : ((1u << hi) - 1u)) & ~((1u << lo) - 1u));
            } else {
                bits = __ldcg(&live[w]);
            }
        }
        uint32_t low = 0;
        if (bits != 0u) {
            // the word's 32 counts: 64 bytes (16-bit counts) or 128 bytes
            int c[32];
            if (a.packed) {
                const uint4 *p4 = reinterpret_cast<const uint4 *>(reinterpret_cast<const unsigned short *>(a.cnt) + (w << 5));
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const uint4 q = __ldcg(&p4[v]);
                    const uint32_t h[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        c[8 * v + 2 * t] = (int)(h[t] & 0xffffu);
                        c[8 * v + 2 * t + 1] = (int)(h[t] >> 16);
                    }
                }
            } else {
                const int4 *p4 = reinterpret_cast<const int4 *>(a.cnt + (w << 5));
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const int4 q = __ldcg(&p4[v]);
                    c[4 * v] = q.x;
                    c[4 * v + 1] = q.y;
                    c[4 * v + 2] = q.z;
                    c[4 * v + 3] = q.w;
                }
            }
#pragma unroll
            for (int b = 0; b < 32; ++b)
                if (((bits >> b) & 1u) && c[b] < a.thrU) low |= 1u << b;
            scanned += (unsigned long long)__popc(bits);
        }
        // of those below alpha, the ones still live fall now
        uint32_t fallm = 0;
        if (low != 0u) {
#pragma unroll
            for (int b = 0; b < 32; ++b)
                if (((low >> b) & 1u) && chain_alive(a, (int32_t)((w << 5) + b))) fallm |= 1u << b;
        }
        if (w < nwords && (full || low != 0u)) live[w] = bits & ~low;
        while (__ballot_sync(ABC_FULL, fallm != 0u)) {
            const bool has = fallm != 0u;
            const int32_t x = has ? (int32_t)((w << 5) + (__ffs(fallm) - 1)) : 0;
            push_add(a, sm.push, pc, has, x, 1, ls);
            fallm &= fallm - 1u;
        }
    }
    push_flush(a, sm.push, pc);
}

// Block-collective flush_stats.
__device__ __forceinline__ void flush_stats_block(const PeelArgs &a, LaneStats &ls) {
    const unsigned long long v[4] = {ls.entries, ls.decs, ls.pushes, ls.items};
    unsigned long long *const d[4] = {&a.ctl->st[ST_ENTRIES], &a.ctl->st[ST_DECS], &a.ctl->st[ST_PUSHES],
                                      &a.ctl->st[ST_ITEMS]};
    block_add<4>(v, d);
}

__device__ __forceinline__ void flush_stats(const PeelArgs &a, LaneStats &ls) {
    unsigned long long v[4] = {ls.entries, ls.decs, ls.pushes, ls.items};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        unsigned long long x = (unsigned long long)warp_sum64((long long)v[i]);
        v[i] = x;
    }
    if ((threadIdx.x & 31) == 0) {
        if (v[0]) atomicAdd(&a.ctl->st[ST_ENTRIES], v[0]);
        if (v[1]) atomicAdd(&a.ctl->st[ST_DECS], v[1]);
        if (v[2]) atomicAdd(&a.ctl->st[ST_PUSHES], v[2]);
        if (v[3]) atomicAdd(&a.ctl->st[ST_ITEMS], v[3]);
    }
}

}  // namespace abc
