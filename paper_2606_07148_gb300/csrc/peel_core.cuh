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
constexpr int MAX_GRAB = 32;

struct WarpSmem {
    long long start[MAX_GRAB];  // first adjacency index of each grabbed item
    int excl[MAX_GRAB];         // exclusive prefix of item lengths
    int upper[MAX_GRAB];        // 1 if the item's row belongs to a U vertex
};

struct LaneStats {
    unsigned long long entries = 0, decs = 0, pushes = 0, items = 0;
};

// Candidate test and bound of a neighbour y seen from a row of layer `upper_row`.
__device__ __forceinline__ bool cand_of(const PeelArgs &a, int32_t y, bool upper_row, int32_t &thr) {
    if (upper_row) {
        thr = a.thrV;
        return y < a.nU + a.pV;
    }
    thr = a.thrU;
    return y < a.pU;
}

// Row length that a removed candidate x must still walk: the candidate prefix length kept in
// cp[x].y (the full degree when its layer's counts came from the full rows).
__device__ __forceinline__ int row_len_of(const PeelArgs &a, int32_t y) { return __ldcg(&a.cp[y].y); }

// Warp-collective: lanes with `want` queue vertex y as nch items (nch may be 0).
__device__ __forceinline__ void warp_push(const PeelArgs &a, bool want, int32_t y, int nch, LaneStats &ls) {
    const unsigned pm = __ballot_sync(ABC_FULL, want);
    if (pm == 0) return;
    const int lane = threadIdx.x & 31;
    if (!want) nch = 0;
    else ls.pushes++;
    const int incl = warp_incl_scan(nch);
    const int total = __shfl_sync(ABC_FULL, incl, 31);
    if (total == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.ctl->tail, (unsigned long long)total);
    base = __shfl_sync(ABC_FULL, base, 0);
    if (base + (unsigned long long)total > (unsigned long long)a.qcap) {
        if (lane == 0) set_error(&a.ctl->err, ABCORE_ENOMEM);
        return;
    }
    unsigned long long pos = base + (unsigned long long)(incl - nch);
    for (int i = 0; i < nch; ++i)
        st_relaxed(&a.q[pos + i], ((unsigned long long)(uint32_t)y << 32) | (unsigned)i);
}

__device__ __forceinline__ int chunks_of(int len, int chunk) { return (len + chunk - 1) / chunk; }

// Warp-collective: process queue slots [h, h + k), k <= 32.
__device__ __forceinline__ void process_items(const PeelArgs &a, unsigned long long h, int k, WarpSmem &sm,
                                              LaneStats &ls, unsigned long long deadline) {
    const int lane = threadIdx.x & 31;
    long long start = 0;
    int len = 0, upper = 0;
    if (lane < k && h + lane < (unsigned long long)a.qcap) {
        unsigned long long *slot = &a.q[h + lane];
        unsigned long long it = ld_relaxed(slot);
        while (it == EMPTY) {
            if (now_ns() > deadline) {
                set_error(&a.ctl->err, ABCORE_ETIMEDOUT);
                break;
            }
            __nanosleep(32);
            it = ld_relaxed(slot);
        }
        if (it != EMPTY) {
            st_relaxed(slot, EMPTY);
            const int32_t x = (int32_t)(it >> 32);
            const int c = (int)(it & 0xffffffffu);
            const int rl = row_len_of(a, x);
            start = __ldg(&a.off[x]) + (long long)c * a.chunk;
            len = min(a.chunk, rl - c * a.chunk);
            if (len < 0) len = 0;
            upper = x < a.nU;
            ls.items++;
        }
    }
    const int incl = warp_incl_scan(len);
    const int L = __shfl_sync(ABC_FULL, incl, 31);
    if (lane < MAX_GRAB) {
        sm.start[lane] = start;
        sm.excl[lane] = incl - len;
        sm.upper[lane] = upper;
    }
    __syncwarp();
    int j = 0;
    for (int b = 0; b < L; b += 32) {
        const int e = b + lane;
        bool push = false;
        int32_t y = 0;
        int nch = 0;
        if (e < L) {
            while (j + 1 < k && sm.excl[j + 1] <= e) ++j;
            const long long pos = sm.start[j] + (e - sm.excl[j]);
            y = __ldg(&a.adj[pos]);
            ls.entries++;
            int32_t thr;
            if (cand_of(a, y, sm.upper[j] != 0, thr) && thr > 0) {
                const int old = atomicSub(&a.cp[y].x, 1);
                ls.decs++;
                if (old == thr) {
                    push = true;
                    nch = chunks_of(row_len_of(a, y), a.chunk);
                }
            }
        }
        warp_push(a, push, y, nch, ls);
    }
    __syncwarp();
}

// Warp-collective cascade loop: returns 1 when the queue drained, 0 on error.
__device__ __forceinline__ int cascade_loop(const PeelArgs &a, WarpSmem &sm, LaneStats &ls, int grab_div) {
    const int lane = threadIdx.x & 31;
    unsigned long long idle_since = now_ns(), last_done = ~0ull;
    for (;;) {
        int state = 2;  // 0 work, 1 finished, 2 retry, 3 error
        unsigned long long h = 0;
        int k = 0;
        if (lane == 0) {
            const unsigned long long head = ld_relaxed(&a.ctl->head);
            const unsigned long long tail = ld_relaxed(&a.ctl->tail);
            if (head < tail) {
                unsigned long long avail = tail - head;
                unsigned long long kk = avail / (unsigned long long)grab_div;
                if (kk < 1) kk = 1;
                if (kk > MAX_GRAB) kk = MAX_GRAB;
                if (atomicCAS(&a.ctl->head, head, head + kk) == head) {
                    h = head;
                    k = (int)kk;
                    state = 0;
                }
            } else {
                const unsigned long long d = ld_acquire(&a.ctl->done);
                const unsigned long long t2 = ld_acquire(&a.ctl->tail);
                if (d == t2) state = 1;
                else if (ld_relaxed_i32(&a.ctl->err) != 0) state = 3;
                else {
                    if (d != last_done) {  // the device is making progress: restart the clock
                        last_done = d;
                        idle_since = now_ns();
                    }
                    if (now_ns() - idle_since > a.timeout_ns) {
                        set_error(&a.ctl->err, ABCORE_ETIMEDOUT);
                        state = 3;
                    } else {
                        __nanosleep(64);
                    }
                }
            }
        }
        state = __shfl_sync(ABC_FULL, state, 0);
        if (state == 1) return 1;
        if (state == 3) return 0;
        if (state == 2) continue;
        h = __shfl_sync(ABC_FULL, h, 0);
        k = __shfl_sync(ABC_FULL, k, 0);
        process_items(a, h, k, sm, ls, now_ns() + a.timeout_ns);
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(&a.ctl->done, (unsigned long long)k);
        idle_since = now_ns();
        if (ld_relaxed_i32(&a.ctl->err) != 0) return 0;
    }
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
