// On-the-fly (alpha, beta)-core queries under edge updates (Section 5, GFQ) and the device-resident,
// continuously batched serving loop.
//
// Question answered for update k (Section 3, on-the-fly query problem): apply the insert or delete
// of e = (u, v), then report whether e lies in the (alpha, beta)-core of the updated graph. The
// core is vertex-induced, so that is "u and v are both in the core" (the endpoint bits are
// returned too). Answers follow arrival order exactly, as if requests ran one at a time.
//
// Scope of the re-peel. GFQ re-peels the connected component of the update (Section 5). This
// engine keeps each target core C and its in-core degrees and re-peels a smaller region that
// still gives exactly the core of the updated graph G':
//  * delete (u, v) with both in C: the new core lies inside C, so only a cascade inside C,
//    started at u and v, is needed; a delete with an endpoint outside C changes nothing;
//  * insert (u, v): the new core contains C. To find what joins, each target keeps a removal
//    certificate: a level rho(w) for every vertex w outside C such that fewer than thr(w) of
//    w's neighbours are in C or have rho >= rho(w) (peeling by increasing rho then removes
//    every non-core vertex, which proves C is the whole core). Take the new members in order of
//    rho: each one is an endpoint of e or has a new member with smaller rho as a neighbour,
//    since otherwise its neighbours in the new core would all lie in C or at rho >= its own,
//    too few. So every new member is reached from the endpoints along edges of strictly
//    increasing rho. That region R (non-core vertices meeting their degree bound) is peeled
//    level by level with C held fixed; its survivors join C, and the levels at which the others
//    fall, offset past every rho in use, become their new rho. Vertices outside R keep valid
//    certificates: a neighbour in R had rho at least theirs, and its new rho is larger still.
//    If both endpoints are in C, nothing can join.
//  * The delete cascade assigns rho the same way (its levels, offset past every rho in use).
//
// Data on the device. The base CSR (internal, degree-ordered ids) is shared and never changes.
// Each target keeps its own view of the updates -- tombstone bits over base adjacency slots, a
// list of inserted neighbours per vertex, current degrees -- plus its core mask and in-core
// counts, so the targets never wait for one another: each target is one block of the serving
// kernel and applies every update in order to its own view.
//
// Requests travel through a ring in pinned, device-mapped host memory; each block polls the
// published request count, processes requests in sequence, and the block owning a request's
// target writes its response into a mapped completion ring. The kernel leaves after an idle
// spell without requests (a bounded wait) and the host relaunches it on the next submit or
// poll; every other wait is bounded as well and ends in ABCORE_ETIMEDOUT.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "cc_core.cuh"
#include "device.cuh"
#include "internal.h"

namespace {

constexpr int SERVE_THREADS = 256;
constexpr int SERVE_WARPS = SERVE_THREADS / 32;

struct TargetDev {
    int32_t alpha, beta;
    uint8_t *M;        // [n] core membership
    int32_t *cnt;      // [n] members: in-core degree; region vertices: region count
    int32_t *deg;      // [n] degree in the current graph
    uint32_t *tomb;    // [ceil(2m / 32)] deleted base adjacency slots
    // inserted neighbours: vertex x owns the pool segment [ins[x].x, ins[x].x + capacity) and
    // uses its first ins[x].y slots (-1 = none yet); a deleted one is overwritten with -1. A full
    // segment is copied into a new one of twice the capacity (2, 4, 8, ...).
    int2 *ins;         // [n] {segment start, entries used}
    int32_t *pool;     // [pool_cap]
    int32_t *pool_top; // pool entries handed out
    int32_t pool_cap;
    int32_t *mark;     // [n] epoch tags for region / cascade membership
    int32_t *q;        // [2n] scratch queue (a region, then the region vertices it peels)
    int32_t *epoch;    // persisted epoch counter
    int64_t *rho;      // [n] removal certificate level of non-core vertices (RHO_CORE in C)
    int64_t *base;     // next unused certificate level (64-bit: every re-peel raises it by its
                       // level count plus one, so a long session would run a 32-bit level out)
    unsigned long long *st;  // [4] regions grown, region vertices, cascades, vertices cascaded
};

constexpr int64_t RHO_CORE = 0x7fffffffffffffffll;
// Certificate levels never reach this: a re-peel that would pass it stops the session with
// ABCORE_ENOMEM instead of wrapping (2^62 levels are far beyond any session's reach).
constexpr int64_t RHO_LIMIT = 1ll << 62;

struct ServeArgs {
    const int64_t *off;
    const int32_t *adj;
    const int32_t *old2new;
    int32_t nU, nV;
    TargetDev *targets;
    int32_t ntargets;
    const abcore_req *req;              // mapped host ring
    abcore_resp *resp;                  // mapped host ring
    unsigned long long *resp_seq;       // mapped: seq + 1 once resp[slot] is valid
    const unsigned long long *submitted;  // mapped: requests published by the host
    const int *stop;                    // mapped: host asks the loop to leave once idle
    unsigned long long *progress_host;  // mapped: requests processed, per target
    unsigned long long *progress_dev;   // device: requests processed, per target
    unsigned long long *exit_at;        // device: ~0, or the request count every block stops at
    int *err;                           // device: first error
    int *grow;                          // device, per target: 1 once its inserted-edge pool is full
    int32_t *comp;                      // component union-find over the current graph
    int *comp_stale;                    // set once a delete may have split a component
    int32_t slots;
    unsigned long long idle_ns, timeout_ns;
};

__device__ __forceinline__ unsigned long long ld_sys(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_sys_i32(const int *p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_sys(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ bool tomb_get(const uint32_t *t, int64_t p) { return (t[p >> 5] >> (p & 31)) & 1u; }
__device__ __forceinline__ void tomb_set(uint32_t *t, int64_t p, bool on) {
    if (on) atomicOr(&t[p >> 5], 1u << (p & 31));
    else atomicAnd(&t[p >> 5], ~(1u << (p & 31)));
}

// Block-collective search of `key` in the ascending row adj[s, e): its position or -1.
__device__ int64_t cta_find(const int32_t *adj, int64_t s, int64_t e, int32_t key) {
    __shared__ int64_t lo_s, hi_s, found_s;
    __shared__ int32_t sval[SERVE_THREADS];
    if (threadIdx.x == 0) {
        lo_s = s;
        hi_s = e;
        found_s = -1;
    }
    __syncthreads();
    for (;;) {
        const int64_t lo = lo_s, hi = hi_s, len = hi - lo;
        if (len <= (int64_t)SERVE_THREADS * 4) {
            for (int64_t p = lo + threadIdx.x; p < hi; p += SERVE_THREADS)
                if (__ldg(&adj[p]) == key) found_s = p;
            __syncthreads();
            break;
        }
        const int64_t pos = lo + (len * threadIdx.x) / SERVE_THREADS;
        sval[threadIdx.x] = __ldg(&adj[pos]);
        __syncthreads();
        const int32_t v = sval[threadIdx.x];
        if (threadIdx.x == 0 && v > key) hi_s = lo;  // key below the row: empty interval
        if (v <= key && (threadIdx.x == SERVE_THREADS - 1 || sval[threadIdx.x + 1] > key)) {
            lo_s = pos;
            hi_s = threadIdx.x == SERVE_THREADS - 1 ? hi : lo + (len * (threadIdx.x + 1)) / SERVE_THREADS;
        }
        __syncthreads();
    }
    const int64_t r = found_s;
    __syncthreads();
    return r;
}

__device__ __forceinline__ int32_t thr_of(const ServeArgs &A, const TargetDev &S, int32_t z) {
    return z < A.nU ? S.alpha : S.beta;
}

// Capacity of an inserted-neighbour segment holding `used` entries.
__device__ __forceinline__ int32_t ins_capacity(int32_t used) {
    int32_t c = 2;
    while (c < used) c <<= 1;
    return c;
}

// Visit the current neighbours of w: base row minus tombstones, plus live inserted neighbours.
// Warp-collective: lanes stride the base row, then the inserted segment.
template <class F>
__device__ __forceinline__ void for_neighbours(const ServeArgs &A, const TargetDev &S, int32_t w, F f) {
    const int lane = threadIdx.x & 31;
    const int64_t s = __ldg(&A.off[w]), e = __ldg(&A.off[w + 1]);
    for (int64_t p = s + lane; p < e; p += 32)
        if (!tomb_get(S.tomb, p)) f(__ldg(&A.adj[p]));
    const int2 seg = S.ins[w];
    for (int32_t i = lane; i < seg.y; i += 32) {
        const int32_t z = S.pool[seg.x + i];
        if (z >= 0) f(z);
    }
}

// Block-collective: position in the pool of inserted neighbour `key` of x, or -1.
__device__ int32_t ins_find(const TargetDev &S, int32_t x, int32_t key) {
    __shared__ int32_t found_s;
    if (threadIdx.x == 0) found_s = -1;
    __syncthreads();
    const int2 seg = S.ins[x];
    for (int32_t i = threadIdx.x; i < seg.y; i += SERVE_THREADS)
        if (S.pool[seg.x + i] == key) found_s = seg.x + i;  // live entries are distinct
    __syncthreads();
    const int32_t r = found_s;
    __syncthreads();
    return r;
}

// Block-collective: append y to x's inserted neighbours, moving the segment to one of twice the
// capacity when it is full. Returns false (and records ABCORE_ENOMEM) if the pool is exhausted.
__device__ bool ins_append(const ServeArgs &A, TargetDev &S, int32_t x, int32_t y) {
    __shared__ int32_t from_s, to_s;
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
        const int2 seg = S.ins[x];
        ok_s = 1;
        from_s = -1;
        to_s = seg.x;
        if (seg.x < 0 || seg.y == ins_capacity(seg.y)) {
            const int32_t cap = seg.x < 0 ? 2 : 2 * ins_capacity(seg.y);
            const int32_t at = atomicAdd(S.pool_top, cap);
            if (at > S.pool_cap - cap) {
                abc::set_error(A.err, ABCORE_ENOMEM);
                ok_s = 0;
            } else {
                from_s = seg.x;
                to_s = at;
            }
        }
    }
    __syncthreads();
    const int2 seg = S.ins[x];
    if (ok_s && from_s >= 0)
        for (int32_t i = threadIdx.x; i < seg.y; i += SERVE_THREADS) S.pool[to_s + i] = S.pool[from_s + i];
    __syncthreads();
    if (threadIdx.x == 0 && ok_s) {
        S.pool[to_s + seg.y] = y;
        S.ins[x] = make_int2(to_s, seg.y + 1);
    }
    const bool ok = ok_s != 0;
    __syncthreads();
    return ok;
}

// Process queue entries level by level: each warp takes entries of the current level,
// `body(w)` may push new entries through `push`. Block-collective.
struct BlockQueue {
    int32_t *q;
    int *tail;  // shared
};

__device__ __forceinline__ void bq_push(BlockQueue &Q, int32_t z) { Q.q[atomicAdd(Q.tail, 1)] = z; }

// Cascade inside the core after a delete: members whose in-core count fell below their bound
// leave, lowering their member neighbours' counts (queued on the exact crossing). Vertices
// leaving at cascade level L get certificate level base + L.
__device__ void delete_cascade(const ServeArgs &A, TargetDev &S, int32_t x, int32_t y) {
    __shared__ int tail;
    __shared__ int64_t base_s;
    BlockQueue Q{S.q, &tail};
    if (threadIdx.x == 0) {
        tail = 0;
        base_s = *S.base;
        const int32_t cx = --S.cnt[x], cy = --S.cnt[y];
        if (cx < thr_of(A, S, x)) { S.M[x] = 0; Q.q[tail++] = x; }
        if (cy < thr_of(A, S, y)) { S.M[y] = 0; Q.q[tail++] = y; }
    }
    __syncthreads();
    int head = 0, level = 0;
    const int warp = threadIdx.x >> 5;
    while (head < tail) {
        const int end = tail;
        __syncthreads();
        for (int i = head + warp; i < end; i += SERVE_WARPS) {
            const int32_t w = S.q[i];
            if ((threadIdx.x & 31) == 0) S.rho[w] = base_s + level;
            for_neighbours(A, S, w, [&](int32_t z) {
                if (S.M[z]) {
                    const int old = atomicSub(&S.cnt[z], 1);
                    if (old == thr_of(A, S, z)) {
                        S.M[z] = 0;
                        bq_push(Q, z);
                    }
                }
            });
        }
        __syncthreads();
        head = end;
        ++level;
    }
    if (threadIdx.x == 0 && tail > 0) {
        *S.base = base_s + level + 1;
        if (*S.base > RHO_LIMIT) abc::set_error(A.err, ABCORE_ENOMEM);
        S.st[2] += 1;
        S.st[3] += (unsigned long long)tail;
    }
    __syncthreads();
}

// Region growth and peel after an insert with an endpoint outside the core (see the header).
__device__ void insert_region(const ServeArgs &A, TargetDev &S, int32_t x, int32_t y, int32_t ep) {
    __shared__ int tail;
    __shared__ int64_t base_s;
    BlockQueue Q{S.q, &tail};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        tail = 0;
        base_s = *S.base;
        const int32_t ends[2] = {x, y};
        for (int i = 0; i < 2; ++i) {
            const int32_t z = ends[i];
            // a non-core endpoint below its bound on degree can neither join nor lose its
            // certificate (at most deg < thr neighbours can count)
            if (S.M[z] || S.deg[z] < thr_of(A, S, z) || S.mark[z] == ep) continue;
            S.mark[z] = ep;
            Q.q[tail++] = z;
        }
    }
    __syncthreads();
    if (tail == 0) return;
    // grow R along edges of strictly increasing rho through non-core vertices meeting their bound
    int head = 0;
    while (head < tail) {
        const int end = tail;
        __syncthreads();
        for (int i = head + warp; i < end; i += SERVE_WARPS) {
            const int32_t w = S.q[i];
            const int64_t rw = S.rho[w];
            for_neighbours(A, S, w, [&](int32_t z) {
                if (!S.M[z] && S.rho[z] > rw && S.deg[z] >= thr_of(A, S, z)) {
                    const int old = atomicExch(&S.mark[z], ep);
                    if (old != ep) bq_push(Q, z);
                }
            });
        }
        __syncthreads();
        head = end;
    }
    const int R = tail;
    // region counts: neighbours in C or in R
    for (int i = warp; i < R; i += SERVE_WARPS) {
        const int32_t w = S.q[i];
        int c = 0;
        for_neighbours(A, S, w, [&](int32_t z) { c += (S.M[z] || S.mark[z] == ep) ? 1 : 0; });
        for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(ABC_FULL, c, d);
        if (lane == 0) S.cnt[w] = c;
    }
    __syncthreads();
    // peel R level by level with C fixed; region vertices falling at level L get tag ep + 1 and
    // certificate level base + L
    if (threadIdx.x == 0) tail = R;
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += SERVE_THREADS) {
        const int32_t w = S.q[i];
        if (S.cnt[w] < thr_of(A, S, w)) {
            S.mark[w] = ep + 1;
            bq_push(Q, w);
        }
    }
    __syncthreads();
    head = R;
    int level = 0;
    while (head < tail) {
        const int end = tail;
        __syncthreads();
        for (int i = head + warp; i < end; i += SERVE_WARPS) {
            const int32_t w = S.q[i];
            if (lane == 0) S.rho[w] = base_s + level;
            for_neighbours(A, S, w, [&](int32_t z) {
                if (S.mark[z] == ep) {
                    const int old = atomicSub(&S.cnt[z], 1);
                    if (old == thr_of(A, S, z)) {
                        S.mark[z] = ep + 1;
                        bq_push(Q, z);
                    }
                }
            });
        }
        __syncthreads();
        head = end;
        ++level;
    }
    // survivors join C; their old-core neighbours gain one in-core neighbour per edge
    for (int i = warp; i < R; i += SERVE_WARPS) {
        const int32_t w = S.q[i];
        if (S.mark[w] != ep) continue;
        for_neighbours(A, S, w, [&](int32_t z) {
            if (S.M[z] && S.mark[z] != ep) atomicAdd(&S.cnt[z], 1);
        });
    }
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += SERVE_THREADS) {
        const int32_t w = S.q[i];
        if (S.mark[w] == ep) {
            S.M[w] = 1;
            S.rho[w] = RHO_CORE;
        }
    }
    if (threadIdx.x == 0) {
        *S.base = base_s + level + 1;
        if (*S.base > RHO_LIMIT) abc::set_error(A.err, ABCORE_ENOMEM);
        S.st[0] += 1;
        S.st[1] += (unsigned long long)R;
    }
    __syncthreads();
}

// Pool entries an append to a segment needs: a new segment of 2, or twice the room of a full one.
__device__ __forceinline__ int64_t append_need(int2 seg) {
    if (seg.x < 0) return 2;
    const int32_t cap = ins_capacity(seg.y);
    return seg.y == cap ? 2 * (int64_t)cap : 0;
}

// Whether an edge (x, y) fits in the target's inserted-edge pool (the two appends together).
__device__ __forceinline__ int pool_room(const TargetDev &S, int32_t x, int32_t y) {
    return (int64_t)*S.pool_top + append_need(S.ins[x]) + append_need(S.ins[y]) <= (int64_t)S.pool_cap;
}

// process_update's answer when the target's pool has no room for an insert (not a status the
// caller sees: the request is held back and processed again once the pool has grown)
constexpr int POOL_FULL = 1;

// The edge change of one update on a view: presence test, then tombstone / inserted-segment
// change and degrees. Returns the status, or POOL_FULL with the view unchanged.
__device__ int apply_update(const ServeArgs &A, TargetDev &S, int op, int32_t x, int32_t y) {
    __shared__ int status_s;
    const int64_t px = cta_find(A.adj, __ldg(&A.off[x]), __ldg(&A.off[x + 1]), y);
    int64_t py = -1;
    int32_t qx = -1;  // pool position of y among x's inserted neighbours
    if (px >= 0) py = cta_find(A.adj, __ldg(&A.off[y]), __ldg(&A.off[y + 1]), x);
    else qx = ins_find(S, x, y);
    __shared__ int present_s;  // read once, before anything below writes the view
    if (threadIdx.x == 0) present_s = px >= 0 ? !tomb_get(S.tomb, px) : qx >= 0;
    __syncthreads();
    const bool present = present_s != 0;
    int st = ABCORE_OK;
    if (op == ABCORE_INSERT && present) st = ABCORE_EEXIST;
    if (op == ABCORE_DELETE && !present) st = ABCORE_ENOENT;
    if (st == ABCORE_OK && op == ABCORE_INSERT && px < 0) {
        // admission by memory: the new edge needs room in both endpoints' pool segments. With no
        // room, nothing changes and the request waits for the host to grow the pool.
        __shared__ int room_s;
        if (threadIdx.x == 0) room_s = pool_room(S, x, y);
        __syncthreads();
        if (!room_s) return POOL_FULL;
    }
    if (st == ABCORE_OK) {
        if (op == ABCORE_INSERT) {
            if (px >= 0) {
                if (threadIdx.x == 0) {
                    tomb_set(S.tomb, px, false);
                    tomb_set(S.tomb, py, false);
                }
            } else if (!ins_append(A, S, x, y) || !ins_append(A, S, y, x)) {
                st = ABCORE_ENOMEM;  // cannot happen after pool_room; the error ends the loop
            }
            if (threadIdx.x == 0 && st == ABCORE_OK) {
                S.deg[x]++;
                S.deg[y]++;
            }
        } else {
            if (px >= 0) {
                if (threadIdx.x == 0) {
                    tomb_set(S.tomb, px, true);
                    tomb_set(S.tomb, py, true);
                }
            } else {
                const int32_t qy = ins_find(S, y, x);
                if (threadIdx.x == 0) {
                    S.pool[qx] = -1;
                    S.pool[qy] = -1;
                }
            }
            if (threadIdx.x == 0) {
                S.deg[x]--;
                S.deg[y]--;
            }
        }
    }
    if (threadIdx.x == 0) status_s = st;
    __syncthreads();
    const int r = status_s;
    __syncthreads();
    return r;
}

// One update against one target's view: the edge change (apply_update), then the scoped re-peel.
// Returns the status (or POOL_FULL, with the view unchanged); *bits = (u in C) | (v in C) << 1.
__device__ int process_update(const ServeArgs &A, TargetDev &S, int op, int32_t x, int32_t y, int32_t ep,
                              int *bits) {
    const int st = apply_update(A, S, op, x, y);
    if (st == POOL_FULL) return st;
    if (st == ABCORE_OK) {
        const bool mx = S.M[x], my = S.M[y];
        __syncthreads();
        if (op == ABCORE_INSERT) {
            if (mx && my) {
                if (threadIdx.x == 0) {
                    S.cnt[x]++;
                    S.cnt[y]++;
                }
            } else {
                insert_region(A, S, x, y, ep);
            }
        } else if (mx && my) {
            delete_cascade(A, S, x, y);
        }
    }
    __syncthreads();
    *bits = (S.M[x] ? 1 : 0) | (S.M[y] ? 2 : 0);
    __syncthreads();
    return st;
}

__global__ void __launch_bounds__(SERVE_THREADS) k_serve(ServeArgs A) {
    __shared__ int state_s;  // 0 work, 1 leave
    __shared__ abcore_req r_s;
    TargetDev S = A.targets[blockIdx.x];
    const int t = blockIdx.x;
    unsigned long long k = A.progress_dev[t];
    int32_t ep = *S.epoch;
    for (;;) {
        if (threadIdx.x == 0) {
            state_s = 0;
            const unsigned long long t0 = abc::now_ns();
            unsigned sl = 64;
            for (;;) {
                if (abc::ld_relaxed_i32(A.err)) {  // an error (a full pool) ends the session
                    state_s = 1;
                    break;
                }
                const unsigned long long ex = abc::ld_relaxed(A.exit_at);
                if (k >= ex) {  // the loop is closing at request count ex
                    state_s = 1;
                    break;
                }
                const unsigned long long sub = ld_sys(A.submitted);
                if (k < sub) break;
                if (ld_sys_i32(A.stop) || abc::now_ns() - t0 > A.idle_ns) {
                    // stop request or idle spell: close the loop for every block at count `sub`,
                    // so no block handles a request the others skip; the host relaunches later
                    atomicCAS(A.exit_at, ~0ull, sub);
                    continue;
                }
                __nanosleep(sl);
                if (sl < 2048) sl <<= 1;
            }
            if (state_s == 0) {
                const abcore_req *rq = A.req + (k % (unsigned long long)A.slots);
                volatile const int32_t *w = reinterpret_cast<volatile const int32_t *>(rq);
                r_s.op = w[0];
                r_s.u = w[1];
                r_s.v = w[2];
                r_s.target = w[3];
                r_s.tag = *reinterpret_cast<volatile const uint64_t *>(&rq->tag);
            }
        }
        __syncthreads();
        if (state_s != 0) break;
        const abcore_req r = r_s;
        const int32_t x = __ldg(&A.old2new[r.u]);
        const int32_t y = __ldg(&A.old2new[A.nU + r.v]);
        ep += 2;
        int bits = 0;
        const int st = process_update(A, S, r.op, x, y, ep, &bits);
        if (st == POOL_FULL) {
            // hold request k back: the loop closes at k for every block, the host grows this
            // target's pool and relaunches, and k is processed then (its answer is unchanged)
            if (threadIdx.x == 0) {
                A.grow[t] = 1;
                atomicMin(A.exit_at, k);
            }
            break;
        }
        if (threadIdx.x == 0) {
            // component labels (kept by the first target's block): an insert joins the two
            // components; a delete may split one, which the next label request recomputes
            if (t == 0 && st == ABCORE_OK) {
                if (r.op == ABCORE_INSERT) abc::cc_unite(A.comp, x, y);
                else *A.comp_stale = 1;
            }
            if (r.target == t) {
                abcore_resp *o = A.resp + (k % (unsigned long long)A.slots);
                o->seq = k;
                o->tag = r.tag;
                o->status = st;
                o->u_in = (uint8_t)(bits & 1);
                o->v_in = (uint8_t)((bits >> 1) & 1);
                o->in_core = (uint8_t)(bits == 3);
                o->pad = 0;
                __threadfence_system();
                st_sys(&A.resp_seq[k % (unsigned long long)A.slots], k + 1);
            }
            A.progress_dev[t] = k + 1;
            __threadfence_system();
            st_sys(&A.progress_host[t], k + 1);
        }
        ++k;
        __syncthreads();
    }
    if (threadIdx.x == 0) *S.epoch = ep;
}

// Target state by a level-synchronous peel of the current CSR: membership, in-core counts,
// degrees, an empty update view, and the removal certificate (rho = the round a vertex falls).
__global__ void k_lv_init(const int64_t *off, int32_t nU, int32_t nV, TargetDev S, int32_t *front,
                          unsigned *nfront) {
    const int64_t n = (int64_t)nU + nV;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = (int32_t)(off[x + 1] - off[x]);
        const int32_t thr = x < nU ? S.alpha : S.beta;
        S.cnt[x] = d;
        S.deg[x] = d;
        S.ins[x] = make_int2(-1, 0);
        S.mark[x] = 0;
        if (d < thr) {
            S.rho[x] = 0;
            S.M[x] = 0;
            front[atomicAdd(nfront, 1u)] = (int32_t)x;
        } else {
            S.rho[x] = RHO_CORE;
            S.M[x] = 1;
        }
    }
}

__global__ void k_lv_round(const int64_t *off, const int32_t *adj, int32_t nU, TargetDev S, const int32_t *fin,
                           unsigned nin, int32_t *fout, unsigned *nout, int32_t round) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nin;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t w = fin[i];
        for (int64_t p = off[w] + lane; p < off[w + 1]; p += 32) {
            const int32_t y = adj[p];
            if (S.rho[y] != RHO_CORE) continue;  // already removed
            const int32_t thr = y < nU ? S.alpha : S.beta;
            const int old = atomicSub(&S.cnt[y], 1);
            if (old == thr) {
                S.rho[y] = round + 1;
                S.M[y] = 0;
                fout[atomicAdd(nout, 1u)] = y;
            }
        }
    }
}

// Edges of the current graph (view of target 0) in caller ids, for rebuilding the CSR.
__global__ void k_collect_edges(const int64_t *off, const int32_t *adj, const int32_t *new2old, int32_t nU,
                                TargetDev S, int32_t *eu, int32_t *ev, unsigned long long *count) {
    const int64_t m = off[nU];
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        if (tomb_get(S.tomb, p)) continue;
        // row of p: binary search in off[0..nU]
        int32_t lo = 0, hi = nU - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (off[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        const unsigned long long i = atomicAdd(count, 1ull);
        eu[i] = new2old[lo];
        ev[i] = new2old[adj[p]];
    }
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nU; x += (int64_t)gridDim.x * blockDim.x) {
        const int2 seg = S.ins[x];
        for (int32_t i = 0; i < seg.y; ++i) {
            const int32_t z = S.pool[seg.x + i];
            if (z < 0) continue;
            const unsigned long long k = atomicAdd(count, 1ull);
            eu[k] = new2old[x];
            ev[k] = new2old[z];
        }
    }
}

// Union the inserted edges of the current graph (view of target 0) into a component forest.
__global__ void k_cc_inserted(int32_t nU, TargetDev S, int32_t *parent) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nU; x += (int64_t)gridDim.x * blockDim.x) {
        const int2 seg = S.ins[x];
        for (int32_t i = 0; i < seg.y; ++i) {
            const int32_t z = S.pool[seg.x + i];
            if (z >= 0) abc::cc_unite(parent, (int32_t)x, z);
        }
    }
}

// ---- GFQ with the paper's scope (Section 5): after an update, the connected components of its
// endpoints are peeled again from scratch on the current graph (an ablation of the certificate
// scope above; both give the exact core of the updated graph). One view of the updates (no core
// state: each query re-peels), the component forest, and a level-synchronous peel over the
// component(s), a warp per frontier vertex.

// The update's edge change on the view; ids[0], ids[1] receive the endpoints' internal ids.
__global__ void __launch_bounds__(SERVE_THREADS) k_gfq_apply(ServeArgs A, TargetDev V, int op, int32_t u, int32_t v,
                                                             int32_t *ids, int *status) {
    const int32_t x = __ldg(&A.old2new[u]);
    const int32_t y = __ldg(&A.old2new[A.nU + v]);
    const int st = apply_update(A, V, op, x, y);
    if (threadIdx.x == 0) {
        ids[0] = x;
        ids[1] = y;
        *status = st;
    }
}

// An insert unites the endpoints' components.
__global__ void k_gfq_unite(int32_t *parent, const int32_t *ids) { abc::cc_unite(parent, ids[0], ids[1]); }

// Before a delete is accounted for: keep[x] = 1 for the vertices of the endpoints' component.
__global__ void k_gfq_mark(int32_t *parent, int64_t n, const int32_t *ids, uint8_t *keep) {
    const int32_t r = abc::cc_find(parent, ids[0]);
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        keep[x] = abc::cc_find(parent, (int32_t)x) == r ? 1 : 0;
}

// ... then that component's forest is reset, to be rebuilt from its remaining edges.
__global__ void k_gfq_reset(int32_t *parent, int64_t n, const uint8_t *keep) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        if (keep[x]) parent[x] = (int32_t)x;
}

// Inserted edges of kept vertices (each seen from its U endpoint) rejoin the forest.
__global__ void k_gfq_hook_inserted(int32_t nU, TargetDev V, int32_t *parent, const uint8_t *keep) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nU; x += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[x]) continue;
        const int2 seg = V.ins[x];
        for (int32_t i = 0; i < seg.y; ++i) {
            const int32_t z = V.pool[seg.x + i];
            if (z >= 0) abc::cc_unite(parent, (int32_t)x, z);
        }
    }
}

// Start of the re-peel: vertices of the endpoints' components get their current degree as count;
// those below their bound form the first frontier. Everything else is outside the scope.
__global__ void k_gfq_init(int32_t *parent, int64_t n, int32_t nU, const int32_t *ids, int32_t alpha, int32_t beta,
                           const int32_t *deg, int32_t *cnt, uint8_t *alive, int32_t *front, unsigned *nfront,
                           unsigned long long *scope) {
    const int32_t ru = abc::cc_find(parent, ids[0]), rv = abc::cc_find(parent, ids[1]);
    unsigned long long k = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = abc::cc_find(parent, (int32_t)x);
        if (r != ru && r != rv) {
            alive[x] = 0;
            continue;
        }
        ++k;
        const int32_t d = deg[x];
        cnt[x] = d;
        if (d >= (x < nU ? alpha : beta)) {
            alive[x] = 1;
        } else {
            alive[x] = 0;
            front[atomicAdd(nfront, 1u)] = (int32_t)x;
        }
    }
    k = (unsigned long long)abc::warp_sum64((long long)k);
    if ((threadIdx.x & 31) == 0 && k) atomicAdd(scope, k);
}

// One peel round over the view: each removed vertex lowers its live neighbours' counts; the
// decrement that crosses a bound removes the neighbour (exactly once) into the next frontier.
__global__ void k_gfq_round(ServeArgs A, TargetDev V, int32_t alpha, int32_t beta, int32_t *cnt, uint8_t *alive,
                            const int32_t *fin, unsigned nin, int32_t *fout, unsigned *nout) {
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < nin; i += nw) {
        const int32_t w = fin[i];
        for_neighbours(A, V, w, [&](int32_t z) {
            if (!alive[z]) return;
            const int old = atomicSub(&cnt[z], 1);
            if (old == (z < A.nU ? alpha : beta)) {
                alive[z] = 0;
                fout[atomicAdd(nout, 1u)] = z;
            }
        });
    }
}

// Current degree of every vertex of the base graph (the view starts empty).
__global__ void k_gfq_deg(const int64_t *off, int64_t n, int32_t *deg, int2 *ins) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        deg[x] = (int32_t)(off[x + 1] - off[x]);
        ins[x] = make_int2(-1, 0);
    }
}

}  // namespace

struct ServeState {
    std::vector<int32_t> alphas, betas;
    std::vector<TargetDev> tdev;
    TargetDev *d_targets = nullptr;
    std::vector<void *> bufs;  // device buffers to release
    int32_t slots = 0;
    // mapped host memory
    abcore_req *h_req = nullptr;
    abcore_resp *h_resp = nullptr;
    unsigned long long *h_resp_seq = nullptr;
    unsigned long long *h_ctl = nullptr;  // [0] submitted, [8] stop (int), [16..] progress per target
    abcore_req *d_req = nullptr;
    abcore_resp *d_resp = nullptr;
    unsigned long long *d_resp_seq = nullptr, *d_ctl = nullptr;
    unsigned long long *d_progress = nullptr, *d_exit_at = nullptr;
    int *d_err = nullptr;
    int *d_grow = nullptr;              // per target: its pool must grow before it can go on
    int64_t pool_grows = 0;
    int32_t *d_comp = nullptr;          // component union-find (see k_serve)
    int *d_comp_stale = nullptr;
    unsigned long long next_seq = 0, consumed = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t loop_done = nullptr;
    bool loop_launched = false;
    bool dirty = false;  // updates applied since the CSR was built
    int64_t pool_cap = 0;
};

static int64_t *ctl_stop_ptr(unsigned long long *ctl) { return (int64_t *)(ctl + 8); }

static bool loop_running(ServeState *s) {
    if (!s->loop_launched) return false;
    const cudaError_t e = cudaEventQuery(s->loop_done);
    if (e == cudaErrorNotReady) {
        cudaGetLastError();  // "not ready" is a status, not an error: keep it out of later checks
        return true;
    }
    return false;
}

static unsigned long long min_progress(ServeState *s) {
    unsigned long long mn = ~0ull;
    for (size_t t = 0; t < s->alphas.size(); ++t) {
        const unsigned long long p = __atomic_load_n(&s->h_ctl[16 + t], __ATOMIC_ACQUIRE);
        mn = std::min(mn, p);
    }
    return mn;
}

static int launch_loop(abcore_ctx *ctx, ServeState *s) {
    const Graph &g = ctx->g;
    ServeArgs A{};
    A.off = g.off;
    A.adj = g.adj;
    A.old2new = g.old2new;
    A.nU = g.nU;
    A.nV = g.nV;
    A.targets = s->d_targets;
    A.ntargets = (int32_t)s->alphas.size();
    A.req = s->d_req;
    A.resp = s->d_resp;
    A.resp_seq = s->d_resp_seq;
    A.submitted = s->d_ctl;
    A.stop = (const int *)(s->d_ctl + 8);
    A.progress_host = s->d_ctl + 16;
    A.progress_dev = s->d_progress;
    A.exit_at = s->d_exit_at;
    A.err = s->d_err;
    A.grow = s->d_grow;
    A.comp = s->d_comp;
    A.comp_stale = s->d_comp_stale;
    A.slots = s->slots;
    A.idle_ns = 200ull * 1000000ull;
    A.timeout_ns = (unsigned long long)ctx->prm.timeout_ms * 1000000ull;
    cudaGetLastError();
    ABC_CU(cudaMemsetAsync(s->d_exit_at, 0xff, sizeof(unsigned long long), s->stream));
    k_serve<<<A.ntargets, SERVE_THREADS, 0, s->stream>>>(A);
    ABC_CU(cudaGetLastError());
    ABC_CU(cudaEventRecord(s->loop_done, s->stream));
    s->loop_launched = true;
    ctx->stats.launches++;
    return ABCORE_OK;
}

static int check_device_error(abcore_ctx *ctx, ServeState *s) {
    if (s->loop_launched && !loop_running(s)) {
        int e = 0;
        ABC_CU(cudaMemcpy(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e == ABCORE_ENOMEM) return ctx->fail(ABCORE_ENOMEM, "serve: certificate level limit reached");
        if (e) return ctx->fail(e, "serve: device reported error %d", e);
    }
    return ABCORE_OK;
}

// Grow the inserted-edge pool of every target whose loop block stopped for lack of room (the
// loop has finished): a pool of twice the entries, the used prefix copied over. If the device
// has no memory for it, the call reports ABCORE_ENOMEM and the target's requests keep waiting;
// a later call tries again.
static int grow_pools(abcore_ctx *ctx, ServeState *s) {
    const int nt = (int)s->tdev.size();
    std::vector<int> want(nt, 0);
    ABC_CU(cudaMemcpyAsync(want.data(), s->d_grow, sizeof(int) * nt, cudaMemcpyDeviceToHost, s->stream));
    ABC_CU(cudaStreamSynchronize(s->stream));
    for (int t = 0; t < nt; ++t) {
        if (!want[t]) continue;
        TargetDev &T = s->tdev[t];
        int32_t top = 0;
        ABC_CU(cudaMemcpyAsync(&top, T.pool_top, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
        ABC_CU(cudaStreamSynchronize(s->stream));
        const int64_t ncap = std::min<int64_t>(2 * (int64_t)T.pool_cap, INT32_MAX);
        if (ncap <= T.pool_cap)
            return ctx->fail(ABCORE_ENOMEM, "serve: target %d's inserted-edge pool is at its 2^31-entry limit", t);
        int32_t *np = nullptr;
        const int rc = ctx->alloc(&np, (size_t)ncap, "serve inserted pool");
        if (rc) return ctx->fail(rc, "serve: target %d's inserted-edge pool cannot grow to %lld entries; its "
                                     "requests wait until device memory frees up", t, (long long)ncap);
        ABC_CU(cudaMemcpyAsync(np, T.pool, sizeof(int32_t) * (size_t)std::max(top, 0), cudaMemcpyDeviceToDevice,
                               s->stream));
        ABC_CU(cudaStreamSynchronize(s->stream));
        for (auto &b : s->bufs)
            if (b == (void *)T.pool) b = (void *)np;
        ctx->release(T.pool);
        T.pool = np;
        T.pool_cap = (int32_t)ncap;
        ABC_CU(cudaMemcpyAsync(s->d_targets + t, &T, sizeof(TargetDev), cudaMemcpyHostToDevice, s->stream));
        want[t] = 0;
        ABC_CU(cudaMemcpyAsync(s->d_grow + t, &want[t], sizeof(int), cudaMemcpyHostToDevice, s->stream));
        ABC_CU(cudaStreamSynchronize(s->stream));
        s->pool_grows++;
    }
    return ABCORE_OK;
}

static int ensure_loop(abcore_ctx *ctx, ServeState *s) {
    if (s->next_seq > min_progress(s) && !loop_running(s)) {
        ABC_TRY(check_device_error(ctx, s));
        if (s->loop_launched) ABC_TRY(grow_pools(ctx, s));
        ABC_TRY(launch_loop(ctx, s));
    }
    return ABCORE_OK;
}

static void release_serve(abcore_ctx *ctx, ServeState *s) {
    if (s->loop_launched) {
        __atomic_store_n(ctl_stop_ptr(s->h_ctl), (int64_t)1, __ATOMIC_RELEASE);
        cudaStreamSynchronize(s->stream);
    }
    for (void *p : s->bufs) ctx->release(p);
    s->bufs.clear();
    ctx->release(s->d_targets);
    ctx->release(s->d_progress);
    ctx->release(s->d_exit_at);
    ctx->release(s->d_err);
    ctx->release(s->d_grow);
    ctx->release(s->d_comp);
    ctx->release(s->d_comp_stale);
    if (s->h_req) cudaFreeHost(s->h_req);
    if (s->h_resp) cudaFreeHost(s->h_resp);
    if (s->h_resp_seq) cudaFreeHost(s->h_resp_seq);
    if (s->h_ctl) cudaFreeHost(s->h_ctl);
    s->h_req = nullptr;
    s->h_resp = nullptr;
    s->h_resp_seq = nullptr;
    s->h_ctl = nullptr;
    if (s->loop_done) cudaEventDestroy(s->loop_done);
    s->loop_done = nullptr;
    if (s->stream) cudaStreamDestroy(s->stream);
    s->stream = nullptr;
    s->loop_launched = false;
}

// State of on-the-fly queries with the component scope (query_scope = 1): one view of the updates
// (the TargetDev fields tomb, ins, pool, pool_top, pool_cap and deg; the rest unused), the
// component forest of the current graph, and the re-peel's counts, flags and frontiers.
struct GfqState {
    TargetDev V{};
    int32_t *parent = nullptr;   // [n] union-find forest over the current graph
    int32_t *cnt = nullptr;      // [n] re-peel counts
    uint8_t *alive = nullptr;    // [n] re-peel membership (0 outside the scope)
    uint8_t *keep = nullptr;     // [n] the component a delete cuts
    int32_t *front = nullptr;    // [2n] two frontiers
    unsigned *nfront = nullptr;  // [2]
    int32_t *ids = nullptr;      // [2] the update's internal endpoint ids
    int *status = nullptr;
    unsigned long long *scope = nullptr;  // vertices re-peeled (accumulated)
    std::vector<void *> bufs;
    bool dirty = false;
};

// Rebuild the CSR from a view of the updated graph, after `drop` has released the state that
// owns the view (the view's buffers stay valid until the edges are collected), so static calls
// and new targets see the updated graph.
static int rebuild_from_view(abcore_ctx *ctx, const TargetDev &view, void (*drop)(abcore_ctx *)) {
    const Graph &g = ctx->g;
    const int64_t cap = g.m + view.pool_cap / 2 + 16;  // an inserted edge holds two pool entries
    int32_t *eu = nullptr, *ev = nullptr;
    unsigned long long *cnt = nullptr;
    ABC_TRY(ctx->alloc(&eu, (size_t)cap, "rebuild edges"));
    int rc = ctx->alloc(&ev, (size_t)cap, "rebuild edges");
    if (!rc) rc = ctx->alloc(&cnt, 1, "rebuild count");
    unsigned long long m2 = 0;
    if (!rc) {
        cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), ctx->stream);
        k_collect_edges<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(g.off, g.adj, g.new2old, g.nU, view, eu, ev, cnt);
        cudaMemcpyAsync(&m2, cnt, sizeof(m2), cudaMemcpyDeviceToHost, ctx->stream);
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = ctx->cuda_fail(e, "rebuild");
    }
    const int32_t nU = g.nU, nV = g.nV;
    if (!rc) {
        drop(ctx);
        free_batch(ctx);
        free_peel(ctx);
        rc = build_graph_from_device_edges(ctx, nU, nV, (int64_t)m2, eu, ev);
    }
    ctx->release(eu);
    ctx->release(ev);
    ctx->release(cnt);
    return rc;
}

static void drop_serve(abcore_ctx *ctx) {
    release_serve(ctx, ctx->serve);
    delete ctx->serve;
    ctx->serve = nullptr;
}

int serve_materialize(abcore_ctx *ctx) {
    if (ctx->serve && ctx->serve->loop_launched) ABC_TRY(serve_stop(ctx));  // finish outstanding requests
    if (ctx->serve && ctx->serve->dirty && !ctx->serve->tdev.empty())
        ABC_TRY(rebuild_from_view(ctx, ctx->serve->tdev[0], drop_serve));
    if (ctx->gfq && ctx->gfq->dirty) ABC_TRY(rebuild_from_view(ctx, ctx->gfq->V, free_gfq));
    return ABCORE_OK;
}

void free_gfq(abcore_ctx *ctx) {
    GfqState *q = ctx->gfq;
    if (!q) return;
    cudaStreamSynchronize(ctx->stream);
    for (void *p : q->bufs) ctx->release(p);
    delete q;
    ctx->gfq = nullptr;
}

void free_serve(abcore_ctx *ctx) {
    if (!ctx->serve) return;
    release_serve(ctx, ctx->serve);
    delete ctx->serve;
    ctx->serve = nullptr;
}

template <class T>
static int serve_alloc(abcore_ctx *ctx, ServeState *s, T **p, size_t n, const char *what) {
    ABC_TRY(ctx->alloc(p, n, what));
    s->bufs.push_back((void *)*p);
    return ABCORE_OK;
}

int serve_start(abcore_ctx *ctx, const int32_t *ta, const int32_t *tb, int32_t nt, int32_t slots) {
    ABC_TRY(serve_materialize(ctx));  // served or queried updates become the CSR
    free_serve(ctx);
    free_gfq(ctx);
    const Graph &g = ctx->g;
    const int64_t n = g.n();
    ServeState *s = new ServeState();
    ctx->serve = s;
    s->alphas.assign(ta, ta + nt);
    s->betas.assign(tb, tb + nt);
    s->slots = slots;
    // inserted-neighbour pool per target: an inserted edge takes one entry in each endpoint's
    // segment, and segments that fill up move to twice the room, so 8 entries (32 bytes) per
    // insert cover even one insert per vertex
    s->pool_cap = std::min<int64_t>(8 * std::max<int64_t>(slots, ctx->prm.serve_inserts) + 1024, INT32_MAX);
    ABC_CU(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    ABC_CU(cudaEventCreateWithFlags(&s->loop_done, cudaEventDisableTiming));
    ABC_CU(cudaHostAlloc(&s->h_req, sizeof(abcore_req) * slots, cudaHostAllocMapped));
    ABC_CU(cudaHostAlloc(&s->h_resp, sizeof(abcore_resp) * slots, cudaHostAllocMapped));
    ABC_CU(cudaHostAlloc(&s->h_resp_seq, sizeof(unsigned long long) * slots, cudaHostAllocMapped));
    ABC_CU(cudaHostAlloc(&s->h_ctl, sizeof(unsigned long long) * (16 + nt), cudaHostAllocMapped));
    memset(s->h_resp_seq, 0, sizeof(unsigned long long) * slots);
    memset(s->h_ctl, 0, sizeof(unsigned long long) * (16 + nt));
    ABC_CU(cudaHostGetDevicePointer((void **)&s->d_req, s->h_req, 0));
    ABC_CU(cudaHostGetDevicePointer((void **)&s->d_resp, s->h_resp, 0));
    ABC_CU(cudaHostGetDevicePointer((void **)&s->d_resp_seq, s->h_resp_seq, 0));
    ABC_CU(cudaHostGetDevicePointer((void **)&s->d_ctl, s->h_ctl, 0));
    ABC_TRY(ctx->alloc(&s->d_progress, nt, "serve progress"));
    ABC_TRY(ctx->alloc(&s->d_err, 1, "serve error"));
    ABC_TRY(ctx->alloc(&s->d_grow, nt, "serve pool growth"));
    ABC_CU(cudaMemsetAsync(s->d_grow, 0, sizeof(int) * nt, ctx->stream));
    ABC_TRY(ctx->alloc(&s->d_exit_at, 1, "serve exit"));
    ABC_CU(cudaMemsetAsync(s->d_progress, 0, sizeof(unsigned long long) * nt, ctx->stream));
    ABC_CU(cudaMemsetAsync(s->d_err, 0, sizeof(int), ctx->stream));
    // component labels of the graph as loaded; the serving loop keeps them current
    ABC_TRY(ctx->alloc(&s->d_comp, (size_t)std::max<int64_t>(n, 1), "serve components"));
    ABC_TRY(ctx->alloc(&s->d_comp_stale, 1, "serve components"));
    ABC_CU(cudaMemsetAsync(s->d_comp_stale, 0, sizeof(int), ctx->stream));
    ABC_TRY(cc_hook_base(ctx, s->d_comp, nullptr, ctx->stream));
    const int64_t tomb_words = (2 * g.m + 31) / 32 + 1;
    for (int32_t t = 0; t < nt; ++t) {
        TargetDev T{};
        T.alpha = ta[t];
        T.beta = tb[t];
        ABC_TRY(serve_alloc(ctx, s, &T.M, (size_t)std::max<int64_t>(n, 1), "serve mask"));
        ABC_TRY(serve_alloc(ctx, s, &T.cnt, (size_t)std::max<int64_t>(n, 1), "serve counts"));
        ABC_TRY(serve_alloc(ctx, s, &T.deg, (size_t)std::max<int64_t>(n, 1), "serve degrees"));
        ABC_TRY(serve_alloc(ctx, s, &T.tomb, (size_t)tomb_words, "serve tombstones"));
        ABC_TRY(serve_alloc(ctx, s, &T.ins, (size_t)std::max<int64_t>(n, 1), "serve inserted segments"));
        ABC_TRY(serve_alloc(ctx, s, &T.pool, (size_t)s->pool_cap, "serve inserted pool"));
        ABC_TRY(serve_alloc(ctx, s, &T.pool_top, 1, "serve inserted pool"));
        ABC_TRY(serve_alloc(ctx, s, &T.mark, (size_t)std::max<int64_t>(n, 1), "serve marks"));
        ABC_TRY(serve_alloc(ctx, s, &T.q, (size_t)std::max<int64_t>(2 * n, 1), "serve queue"));
        ABC_TRY(serve_alloc(ctx, s, &T.epoch, 1, "serve epoch"));
        ABC_TRY(serve_alloc(ctx, s, &T.rho, (size_t)std::max<int64_t>(n, 1), "serve certificate"));
        ABC_TRY(serve_alloc(ctx, s, &T.base, 1, "serve certificate"));
        ABC_TRY(serve_alloc(ctx, s, &T.st, 4, "serve stats"));
        ABC_CU(cudaMemsetAsync(T.st, 0, 4 * sizeof(unsigned long long), ctx->stream));
        T.pool_cap = (int32_t)s->pool_cap;
        ABC_CU(cudaMemsetAsync(T.tomb, 0, sizeof(uint32_t) * tomb_words, ctx->stream));
        ABC_CU(cudaMemsetAsync(T.pool_top, 0, sizeof(int32_t), ctx->stream));
        ABC_CU(cudaMemsetAsync(T.epoch, 0, sizeof(int32_t), ctx->stream));
        // the target's core and certificate on the current graph, by a level-synchronous peel
        {
            int32_t *fa = T.q, *fb = T.q + std::max<int64_t>(n, 1);  // the scratch queue holds both frontiers
            unsigned *cnts = nullptr;
            ABC_TRY(serve_alloc(ctx, s, &cnts, 2, "serve init"));
            unsigned h[2] = {0, 0};
            ABC_CU(cudaMemsetAsync(cnts, 0, 2 * sizeof(unsigned), ctx->stream));
            k_lv_init<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(g.off, g.nU, g.nV, T, fa, cnts);
            ctx->stats.launches++;
            ABC_CU(cudaMemcpyAsync(&h[0], cnts, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
            ABC_CU(cudaStreamSynchronize(ctx->stream));
            int32_t round = 0;
            while (h[0] > 0) {
                ABC_CU(cudaMemsetAsync(cnts + 1, 0, sizeof(unsigned), ctx->stream));
                const unsigned blocks = (unsigned)std::min<int64_t>(((int64_t)h[0] * 32 + 255) / 256, (int64_t)ctx->num_sms * 16);
                k_lv_round<<<std::max(blocks, 1u), 256, 0, ctx->stream>>>(g.off, g.adj, g.nU, T, fa, h[0], fb, cnts + 1, round);
                ctx->stats.launches++;
                ABC_CU(cudaMemcpyAsync(&h[1], cnts + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
                ABC_CU(cudaStreamSynchronize(ctx->stream));
                std::swap(fa, fb);
                h[0] = h[1];
                ++round;
            }
            const int64_t base0 = (int64_t)round + 2;
            ABC_CU(cudaMemcpyAsync(T.base, &base0, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
            ABC_CU(cudaStreamSynchronize(ctx->stream));
        }
        ABC_CU(cudaGetLastError());
        s->tdev.push_back(T);
    }
    ABC_TRY(ctx->alloc(&s->d_targets, nt, "serve targets"));
    ABC_CU(cudaMemcpyAsync(s->d_targets, s->tdev.data(), sizeof(TargetDev) * nt, cudaMemcpyHostToDevice, ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    return ABCORE_OK;
}

int serve_submit(abcore_ctx *ctx, const abcore_req *reqs, int32_t n, uint64_t *seq_out) {
    ServeState *s = ctx->serve;
    if (!s) return ctx->fail(ABCORE_EINVAL, "serve: not started");
    const Graph &g = ctx->g;
    for (int32_t i = 0; i < n; ++i) {
        const abcore_req &r = reqs[i];
        if (r.u < 0 || r.u >= g.nU || r.v < 0 || r.v >= g.nV) return ctx->fail(ABCORE_EINVAL, "request %d: vertex id out of range", i);
        if (r.op != ABCORE_INSERT && r.op != ABCORE_DELETE) return ctx->fail(ABCORE_EINVAL, "request %d: bad op", i);
        if (r.target < 0 || r.target >= (int32_t)s->alphas.size()) return ctx->fail(ABCORE_EINVAL, "request %d: bad target", i);
    }
    const unsigned long long low = std::min(min_progress(s), s->consumed);
    if (s->next_seq + (unsigned long long)n - low > (unsigned long long)s->slots) {
        ABC_TRY(ensure_loop(ctx, s));
        return ctx->fail(ABCORE_EBUSY, "serve: request ring full");
    }
    for (int32_t i = 0; i < n; ++i) {
        const unsigned long long k = s->next_seq + i;
        s->h_req[k % s->slots] = reqs[i];
        if (seq_out) seq_out[i] = k;
    }
    s->next_seq += n;
    __atomic_store_n(&s->h_ctl[0], s->next_seq, __ATOMIC_SEQ_CST);
    if (n > 0) s->dirty = true;
    return ensure_loop(ctx, s);
}

int serve_poll(abcore_ctx *ctx, abcore_resp *out, int32_t max, int32_t *n_out) {
    ServeState *s = ctx->serve;
    *n_out = 0;
    if (!s) return ctx->fail(ABCORE_EINVAL, "serve: not started");
    int32_t got = 0;
    while (got < max && s->consumed < s->next_seq) {
        const unsigned long long k = s->consumed;
        const unsigned long long mark = __atomic_load_n(&s->h_resp_seq[k % s->slots], __ATOMIC_ACQUIRE);
        if (mark != k + 1) break;
        out[got++] = s->h_resp[k % s->slots];
        s->consumed++;
    }
    *n_out = got;
    ABC_TRY(check_device_error(ctx, s));
    return ensure_loop(ctx, s);
}

int serve_stop(abcore_ctx *ctx) {
    ServeState *s = ctx->serve;
    if (!s) return ABCORE_OK;
    const auto t0 = std::chrono::steady_clock::now();
    while (min_progress(s) < s->next_seq) {
        ABC_TRY(check_device_error(ctx, s));
        ABC_TRY(ensure_loop(ctx, s));
        if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(ctx->prm.timeout_ms * 4))
            return ctx->fail(ABCORE_ETIMEDOUT, "serve: requests did not finish");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    __atomic_store_n(ctl_stop_ptr(s->h_ctl), (int64_t)1, __ATOMIC_SEQ_CST);
    ABC_CU(cudaStreamSynchronize(s->stream));
    __atomic_store_n(ctl_stop_ptr(s->h_ctl), (int64_t)0, __ATOMIC_SEQ_CST);
    s->loop_launched = false;
    return check_device_error(ctx, s);
}

template <class T>
static int gfq_alloc(abcore_ctx *ctx, GfqState *q, T **p, size_t n, const char *what) {
    ABC_TRY(ctx->alloc(p, n, what));
    q->bufs.push_back((void *)*p);
    return ABCORE_OK;
}

// The component-scoped query state on the current CSR: an empty view and the component forest
// (GFQ's preprocessing).
static int gfq_prepare(abcore_ctx *ctx) {
    if (ctx->gfq) return ABCORE_OK;
    ABC_TRY(serve_materialize(ctx));
    free_serve(ctx);
    const Graph &g = ctx->g;
    const int64_t n = std::max<int64_t>(g.n(), 1);
    GfqState *q = new GfqState();
    ctx->gfq = q;
    TargetDev &V = q->V;
    const int64_t tomb_words = (2 * g.m + 31) / 32 + 1;
    V.pool_cap = (int32_t)std::min<int64_t>(8 * ctx->prm.serve_inserts + 1024, INT32_MAX);
    ABC_TRY(gfq_alloc(ctx, q, &V.tomb, (size_t)tomb_words, "query tombstones"));
    ABC_TRY(gfq_alloc(ctx, q, &V.ins, (size_t)n, "query inserted segments"));
    ABC_TRY(gfq_alloc(ctx, q, &V.pool, (size_t)V.pool_cap, "query inserted pool"));
    ABC_TRY(gfq_alloc(ctx, q, &V.pool_top, 1, "query inserted pool"));
    ABC_TRY(gfq_alloc(ctx, q, &V.deg, (size_t)n, "query degrees"));
    ABC_TRY(gfq_alloc(ctx, q, &q->parent, (size_t)n, "query components"));
    ABC_TRY(gfq_alloc(ctx, q, &q->cnt, (size_t)n, "query counts"));
    ABC_TRY(gfq_alloc(ctx, q, &q->alive, (size_t)n, "query membership"));
    ABC_TRY(gfq_alloc(ctx, q, &q->keep, (size_t)n, "query cut component"));
    ABC_TRY(gfq_alloc(ctx, q, &q->front, (size_t)(2 * n), "query frontiers"));
    ABC_TRY(gfq_alloc(ctx, q, &q->nfront, 2, "query frontier sizes"));
    ABC_TRY(gfq_alloc(ctx, q, &q->ids, 2, "query endpoints"));
    ABC_TRY(gfq_alloc(ctx, q, &q->status, 1, "query status"));
    ABC_TRY(gfq_alloc(ctx, q, &q->scope, 1, "query scope size"));
    ABC_CU(cudaMemsetAsync(V.tomb, 0, sizeof(uint32_t) * tomb_words, ctx->stream));
    ABC_CU(cudaMemsetAsync(V.pool_top, 0, sizeof(int32_t), ctx->stream));
    const unsigned gi = (unsigned)std::max<int64_t>(1, std::min<int64_t>((g.n() + 255) / 256, (int64_t)ctx->num_sms * 16));
    if (g.n() > 0) k_gfq_deg<<<gi, 256, 0, ctx->stream>>>(g.off, g.n(), V.deg, V.ins);
    ctx->stats.launches++;
    ABC_TRY(cc_hook_base(ctx, q->parent, nullptr, ctx->stream));
    ABC_CU(cudaGetLastError());
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    return ABCORE_OK;
}

// Double the view's inserted-edge pool (its used prefix copied over).
static int gfq_grow(abcore_ctx *ctx, GfqState *q) {
    TargetDev &V = q->V;
    int32_t top = 0;
    ABC_CU(cudaMemcpyAsync(&top, V.pool_top, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    const int64_t ncap = std::min<int64_t>(2 * (int64_t)V.pool_cap, INT32_MAX);
    if (ncap <= V.pool_cap) return ctx->fail(ABCORE_ENOMEM, "query: the inserted-edge pool is at its 2^31-entry limit");
    int32_t *np = nullptr;
    ABC_TRY(ctx->alloc(&np, (size_t)ncap, "query inserted pool"));
    ABC_CU(cudaMemcpyAsync(np, V.pool, sizeof(int32_t) * (size_t)std::max(top, 0), cudaMemcpyDeviceToDevice,
                           ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    for (auto &b : q->bufs)
        if (b == (void *)V.pool) b = (void *)np;
    ctx->release(V.pool);
    V.pool = np;
    V.pool_cap = (int32_t)ncap;
    return ABCORE_OK;
}

// GFQ (Section 5) with the paper's scope: apply the update, keep the component forest current
// (an insert unites; a delete re-runs the affected component's components), then re-peel the
// endpoints' components from scratch with a level-synchronous peel over the current graph.
static int gfq_query(abcore_ctx *ctx, int32_t u, int32_t v, int op, int32_t alpha, int32_t beta, uint8_t *in_core) {
    ABC_TRY(gfq_prepare(ctx));
    GfqState *q = ctx->gfq;
    const Graph &g = ctx->g;
    const int64_t n = g.n();
    ServeArgs A{};
    A.off = g.off;
    A.adj = g.adj;
    A.old2new = g.old2new;
    A.nU = g.nU;
    A.nV = g.nV;
    A.err = q->status;  // (apply_update reports a pool fault here; pool_room rules it out)
    int st = POOL_FULL;
    while (st == POOL_FULL) {
        k_gfq_apply<<<1, SERVE_THREADS, 0, ctx->stream>>>(A, q->V, op, u, v, q->ids, q->status);
        ctx->stats.launches++;
        ABC_CU(cudaGetLastError());
        ABC_CU(cudaMemcpyAsync(&st, q->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        ABC_CU(cudaStreamSynchronize(ctx->stream));
        if (st == POOL_FULL) ABC_TRY(gfq_grow(ctx, q));
    }
    if (st != ABCORE_OK && st != ABCORE_EEXIST && st != ABCORE_ENOENT)
        return ctx->fail(st, "query: device reported error %d", st);
    const unsigned gi = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 16));
    if (st == ABCORE_OK) {
        q->dirty = true;
        if (op == ABCORE_INSERT) {
            k_gfq_unite<<<1, 1, 0, ctx->stream>>>(q->parent, q->ids);
            ctx->stats.launches++;
        } else {
            k_gfq_mark<<<gi, 256, 0, ctx->stream>>>(q->parent, n, q->ids, q->keep);
            k_gfq_reset<<<gi, 256, 0, ctx->stream>>>(q->parent, n, q->keep);
            ctx->stats.launches += 2;
            ABC_TRY(cc_hook_rows(ctx, q->parent, q->V.tomb, ctx->stream, q->keep));
            if (g.nU > 0) k_gfq_hook_inserted<<<gi, 256, 0, ctx->stream>>>(g.nU, q->V, q->parent, q->keep);
            ctx->stats.launches++;
        }
    }
    // the re-peel of the endpoints' components
    unsigned h[2] = {0, 0};
    unsigned long long before = 0, after = 0;
    ABC_CU(cudaMemcpyAsync(&before, q->scope, sizeof(before), cudaMemcpyDeviceToHost, ctx->stream));
    ABC_CU(cudaMemsetAsync(q->nfront, 0, 2 * sizeof(unsigned), ctx->stream));
    int32_t *fa = q->front, *fb = q->front + std::max<int64_t>(n, 1);
    k_gfq_init<<<gi, 256, 0, ctx->stream>>>(q->parent, n, g.nU, q->ids, alpha, beta, q->V.deg, q->cnt, q->alive, fa,
                                            q->nfront, q->scope);
    ctx->stats.launches++;
    ABC_CU(cudaGetLastError());
    ABC_CU(cudaMemcpyAsync(&h[0], q->nfront, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    ABC_CU(cudaMemcpyAsync(&after, q->scope, sizeof(after), cudaMemcpyDeviceToHost, ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    while (h[0] > 0) {
        ABC_CU(cudaMemsetAsync(q->nfront + 1, 0, sizeof(unsigned), ctx->stream));
        const unsigned blocks = (unsigned)std::min<int64_t>(((int64_t)h[0] * 32 + 255) / 256, (int64_t)ctx->num_sms * 16);
        k_gfq_round<<<std::max(blocks, 1u), 256, 0, ctx->stream>>>(A, q->V, alpha, beta, q->cnt, q->alive, fa, h[0], fb,
                                                                    q->nfront + 1);
        ctx->stats.launches++;
        ABC_CU(cudaGetLastError());
        ABC_CU(cudaMemcpyAsync(&h[1], q->nfront + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        ABC_CU(cudaStreamSynchronize(ctx->stream));
        std::swap(fa, fb);
        h[0] = h[1];
    }
    int32_t ids[2] = {0, 0};
    uint8_t a2[2] = {0, 0};
    ABC_CU(cudaMemcpyAsync(ids, q->ids, sizeof(ids), cudaMemcpyDeviceToHost, ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    ABC_CU(cudaMemcpyAsync(&a2[0], q->alive + ids[0], 1, cudaMemcpyDeviceToHost, ctx->stream));
    ABC_CU(cudaMemcpyAsync(&a2[1], q->alive + ids[1], 1, cudaMemcpyDeviceToHost, ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    *in_core = (a2[0] && a2[1]) ? 1 : 0;
    ctx->stats.scope_queries++;
    ctx->stats.scope_vertices += (int64_t)(after - before);
    if (st != ABCORE_OK)
        return ctx->fail(st, st == ABCORE_EEXIST ? "insert: edge already present" : "delete: edge not present");
    return ABCORE_OK;
}

void serve_counters(abcore_ctx *ctx, int64_t out[4]) {
    for (int i = 0; i < 4; ++i) out[i] = 0;
    ServeState *s = ctx->serve;
    if (!s) return;
    for (const TargetDev &T : s->tdev) {
        unsigned long long h[4] = {0, 0, 0, 0};
        if (cudaMemcpy(h, T.st, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        for (int i = 0; i < 4; ++i) out[i] += (int64_t)h[i];
    }
}

int query_edge(abcore_ctx *ctx, int32_t u, int32_t v, int op, int32_t alpha, int32_t beta, uint8_t *in_core) {
    if (ctx->prm.query_scope == 1) return gfq_query(ctx, u, v, op, alpha, beta, in_core);
    if (ctx->gfq) {
        // updates queried with the component scope become the CSR the serving loop starts from
        ABC_TRY(serve_materialize(ctx));
        free_gfq(ctx);
    }
    ServeState *s = ctx->serve;
    int32_t t = -1;
    if (s)
        for (size_t i = 0; i < s->alphas.size(); ++i)
            if (s->alphas[i] == alpha && s->betas[i] == beta) t = (int32_t)i;
    if (s && s->consumed < s->next_seq)
        return ctx->fail(ABCORE_EBUSY, "query_edge: poll the outstanding served responses first");
    if (t < 0) {
        std::vector<int32_t> a = s ? s->alphas : std::vector<int32_t>(), b = s ? s->betas : std::vector<int32_t>();
        a.push_back(alpha);
        b.push_back(beta);
        ABC_TRY(serve_start(ctx, a.data(), b.data(), (int32_t)a.size(), 1024));
        s = ctx->serve;
        t = (int32_t)a.size() - 1;
    }
    abcore_req r{op, u, v, t, 0};
    uint64_t seq = 0;
    ABC_TRY(serve_submit(ctx, &r, 1, &seq));
    const auto t0 = std::chrono::steady_clock::now();
    abcore_resp resp{};
    for (;;) {
        int32_t got = 0;
        ABC_TRY(serve_poll(ctx, &resp, 1, &got));
        if (got == 1) break;
        if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(ctx->prm.timeout_ms * 4))
            return ctx->fail(ABCORE_ETIMEDOUT, "query_edge: no response");
    }
    *in_core = resp.in_core;
    if (resp.status != ABCORE_OK)
        return ctx->fail(resp.status, resp.status == ABCORE_EEXIST ? "insert: edge already present"
                                                                   : "delete: edge not present");
    return ABCORE_OK;
}

// Component labels of the current graph while serving: wait until every submitted update has
// been applied, recompute the forest from the current graph if a delete may have split a
// component (the paper re-runs the components of the affected component; this re-runs them
// over the graph, on demand), then name the components.
int serve_components(abcore_ctx *ctx, int32_t *d_lab_u, int32_t *d_lab_v, int64_t *ncomp) {
    ServeState *s = ctx->serve;
    const auto t0 = std::chrono::steady_clock::now();
    while (min_progress(s) < s->next_seq) {
        ABC_TRY(check_device_error(ctx, s));
        ABC_TRY(ensure_loop(ctx, s));
        if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(ctx->prm.timeout_ms * 4))
            return ctx->fail(ABCORE_ETIMEDOUT, "components: served updates did not finish");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    ABC_TRY(check_device_error(ctx, s));
    int stale = 0;
    ABC_CU(cudaMemcpyAsync(&stale, s->d_comp_stale, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    if (stale) {
        ABC_TRY(cc_hook_base(ctx, s->d_comp, s->tdev[0].tomb, ctx->stream));
        k_cc_inserted<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(ctx->g.nU, s->tdev[0], s->d_comp);
        ctx->stats.launches++;
        ABC_CU(cudaGetLastError());
        ABC_CU(cudaMemsetAsync(s->d_comp_stale, 0, sizeof(int), ctx->stream));
    }
    return cc_emit(ctx, s->d_comp, d_lab_u, d_lab_v, ncomp, ctx->stream);
}
