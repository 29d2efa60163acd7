// Single (alpha, beta)-core peel (Definition 1; Algorithm 1, GCC).
//
// Layout fact used throughout: each layer is numbered by non-increasing degree, so the
// vertices that meet their bound on full degree -- the only ones that can be in the core --
// are the prefixes P_U = [0, pU) and P_V = [nU, nU + pV). Every other vertex violates at once
// (the scan phase of Algorithm 1) and is never looked at individually.
//
// Up to four launches:
//  1. k_init: for each candidate x, its count of live candidate neighbours. Per layer, either
//     (search) the position of the other layer's candidate boundary in x's sorted row -- the
//     count left after removing all initial violators -- found from where the layer's share of
//     candidate entries predicts it (peel_core.cuh: row_prefix); or (stream) the full degree,
//     corrected by step 2. Candidates already below their bound are queued (or, with round0,
//     listed for step 2).
//  2. the first peel round, when some count needs it: k_stream (layers counted by full degree:
//     the rows of the other layer's initial violators form one contiguous slice of adj, streamed
//     with 16-byte loads) and/or k_round0 (round0: the listed violators' rows); every entry that
//     hits a candidate decrements it with an atomic that returns nothing. Then k_scan queues the
//     candidates those decrements took below their bound.
//  3. k_cascade: the work-queue cascade (peel_core.cuh), then each warp writes its share of
//     the masks in the caller's ids (old2new plus a bitmap of the removed candidates, or a
//     scatter of the survivors when the candidates are few).
// The launches after k_init are programmatic dependents of the one before them.
//
// With core numbers prepared (coredecomp.cu), the same launches run pruned (Algorithm 2) on the
// core-ordered copy of the graph: a prefix of each layer is certain to be in the core and is
// never counted, decremented or removed (PeelArgs cU, cV), and the candidates are the vertices
// with core number >= min(alpha, beta).
#include <algorithm>
#include <cmath>

#include "device.cuh"
#include "internal.h"
#include "peel_core.cuh"

namespace {

using abc::LaneStats;
using abc::WarpSmem;

constexpr int INIT_THREADS = 256;
constexpr int STREAM_THREADS = 256;

__global__ void __launch_bounds__(INIT_THREADS, 5) k_init(PeelArgs a) {
    __shared__ abc::PushBuf<64> pbuf[INIT_THREADS / 32];
    abc::grid_dep_launch();
    LaneStats ls;
    unsigned long long probes = 0, inits = 0;
    abc::init_range(a, pbuf[threadIdx.x >> 5], (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, ls,
                    probes, inits);
    const unsigned long long v[3] = {inits, probes, ls.pushes};
    unsigned long long *const d[3] = {&a.ctl->st[ST_INIT], &a.ctl->st[ST_PROBES], &a.ctl->st[ST_PUSHES]};
    abc::block_add<3>(v, d);
}

__global__ void __launch_bounds__(STREAM_THREADS) k_stream(PeelArgs a, int64_t sa, int64_t ea, int64_t sb,
                                                           int64_t eb) {
    abc::grid_dep_launch();
    abc::grid_dep_wait();
    LaneStats ls;
    unsigned long long ents = 0;
    abc::stream_range(a, sa, ea, sb, eb, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                      (int64_t)gridDim.x * blockDim.x, ls, ents);
    const unsigned long long v[3] = {ents, ls.decs, ls.pushes};
    unsigned long long *const d[3] = {&a.ctl->st[ST_STREAM], &a.ctl->st[ST_SDECS], &a.ctl->st[ST_PUSHES]};
    abc::block_add<3>(v, d);
}

__global__ void __launch_bounds__(256) k_scan(PeelArgs a) {
    __shared__ abc::PushBuf<64> pbuf[256 / 32];
    abc::grid_dep_launch();
    abc::grid_dep_wait();
    LaneStats ls;
    unsigned long long scanned = 0;
    abc::scan_range<64, true>(a, pbuf[threadIdx.x >> 5], (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                              (int64_t)gridDim.x * blockDim.x, ls, scanned);
    const unsigned long long v[2] = {scanned, ls.pushes};
    unsigned long long *const d[2] = {&a.ctl->st[ST_SCAN], &a.ctl->st[ST_PUSHES]};
    abc::block_add<2>(v, d);
}

// round0: the rows of the candidates the count init found below their bound (listed in l0 with
// their first adjacency index and length) -- the first peel round of Algorithm 1 for them --
// walked with decrements that return nothing, as the violator stream does; no crossing is looked
// for here, k_scan finds every candidate the round took below its bound. Lane l of a warp takes
// list entry base + l and the warp balances their rows' entries over its lanes; the next group's
// entries are loaded while this group's rows are walked.
// Entries per lane per step (R0_ILP) and the blocks an SM must hold (R0_MINB, which caps the
// registers) are compiled in a few combinations (k_round0_variant picks one; the autotuner
// decides): nothing waits on the atomics, so only the adjacency loads' latency has to be covered,
// by entries in flight per lane or by warps per SM.
template <int R0_ILP, int R0_MINB>
__global__ void __launch_bounds__(256, R0_MINB) k_round0(PeelArgs a) {
    __shared__ long long s_start[256 / 32][32];
    __shared__ int s_excl[256 / 32][32];
    __shared__ int s_upper[256 / 32][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    abc::grid_dep_launch();
    abc::grid_dep_wait();
    const int64_t nl0 = (int64_t)a.ctl->l0n;  // written by k_init, earlier on the stream
    unsigned long long ents = 0, decs = 0;
    longlong2 nxt = make_longlong2(0, 0);
    if (gw * 32 + lane < nl0) nxt = __ldg(&a.l0[gw * 32 + lane]);
    for (int64_t g0 = gw * 32; g0 < nl0; g0 += nw * 32) {
        const longlong2 cur = nxt;  // {0, 0} past the end: an empty row
        const int64_t g1 = g0 + nw * 32 + lane;
        nxt = g1 < nl0 ? __ldg(&a.l0[g1]) : make_longlong2(0, 0);
        const int len = (int)(cur.y & 0x7fffffff);
        const int incl = abc::warp_incl_scan(len);
        const int L = __shfl_sync(ABC_FULL, incl, 31);
        s_start[wib][lane] = cur.x;
        s_excl[wib][lane] = incl - len;
        s_upper[wib][lane] = (cur.y & L0_UPPER) != 0;
        __syncwarp();
        int j = 0;
        for (int b = 0; b < L; b += 32 * R0_ILP) {
            int32_t y[R0_ILP];
            int up[R0_ILP];
#pragma unroll
            for (int u = 0; u < R0_ILP; ++u) {
                const int e = b + 32 * u + lane;
                y[u] = -1;
                up[u] = 0;
                if (e < L) {
                    while (j + 1 < 32 && s_excl[wib][j + 1] <= e) ++j;
                    y[u] = abc::ld_adj(&a.adj[s_start[wib][j] + (e - s_excl[wib][j])]);
                    up[u] = s_upper[wib][j];
                }
            }
#pragma unroll
            for (int u = 0; u < R0_ILP; ++u) {
                if (y[u] < 0) continue;
                ents++;
                int32_t t;
                if (abc::cand_of(a, y[u], up[u] != 0, t) && (t > 0 || !a.skip_zero)) {
                    abc::cnt_dec_noret(a, y[u]);
                    decs++;
                }
            }
        }
        __syncwarp();
    }
    const unsigned long long v[2] = {ents, decs};
    unsigned long long *const d[2] = {&a.ctl->st[ST_STREAM], &a.ctl->st[ST_SDECS]};
    abc::block_add<2>(v, d);
}

// One first-round decrement of candidate y. With a hub table (HUB), a decrement of one of the
// first hU U or hV V candidates -- the highest degrees, since ids follow degree, and so the most
// frequent targets of the walked rows -- is added to the block's shared-memory tally instead of
// being sent to L2; the tally goes to the counts once, when the block is done. No crossing is
// looked for in this round, so only the final counts matter and the order of the subtractions
// does not.
template <bool HUB>
__device__ __forceinline__ void r0_dec(const PeelArgs &a, int32_t y, int *s_hub, int hU, int hV,
                                       unsigned long long &hub) {
    if (HUB) {
        const int k = y < a.nU ? (y < hU ? y : -1) : (y - a.nU < hV ? hU + (y - a.nU) : -1);
        if (k >= 0) {
            atomicAdd(&s_hub[k], 1);
            hub++;
            return;
        }
    }
    abc::cnt_dec_noret(a, y);
}

// The same walk with the rows taken four at a time by the whole warp: lanes read consecutive
// entries of one row (coalesced), two 32-entry chunks of each of the four rows in flight, so no
// entry has to look up its row; lanes past a row's end idle (the rows are short, each below its
// bound). Rows longer than 64 entries finish in a loop. Warp-level body of k_round0_rows and
// k_round0_hub.
template <bool HUB>
__device__ __forceinline__ void round0_rows_walk(const PeelArgs &a, int *s_hub, int hU, int hV,
                                                 unsigned long long &ents, unsigned long long &decs,
                                                 unsigned long long &hub) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nl0 = (int64_t)a.ctl->l0n;  // written by k_init, earlier on the stream
    longlong2 nxt = make_longlong2(0, 0);
    if (gw * 32 + lane < nl0) nxt = __ldg(&a.l0[gw * 32 + lane]);
    for (int64_t g0 = gw * 32; g0 < nl0; g0 += nw * 32) {
        const longlong2 cur = nxt;  // {0, 0} past the end: an empty row
        const int64_t g1 = g0 + nw * 32 + lane;
        nxt = g1 < nl0 ? __ldg(&a.l0[g1]) : make_longlong2(0, 0);
        const int mylen = (int)(cur.y & 0x7fffffff);
        const int myup = (cur.y & L0_UPPER) != 0;
        for (int r0 = 0; r0 < 32; r0 += 4) {
            long long st[4];
            int len[4], up[4];
            int32_t y[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                st[k] = __shfl_sync(ABC_FULL, cur.x, r0 + k);
                len[k] = __shfl_sync(ABC_FULL, mylen, r0 + k);
                up[k] = __shfl_sync(ABC_FULL, myup, r0 + k);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                y[2 * k] = lane < len[k] ? abc::ld_adj(&a.adj[st[k] + lane]) : -1;
                y[2 * k + 1] = lane + 32 < len[k] ? abc::ld_adj(&a.adj[st[k] + lane + 32]) : -1;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (y[u] < 0) continue;
                ents++;
                int32_t t;
                if (abc::cand_of(a, y[u], up[u >> 1] != 0, t) && (t > 0 || !a.skip_zero)) {
                    r0_dec<HUB>(a, y[u], s_hub, hU, hV, hub);
                    decs++;
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                for (int e = 64 + lane; e < len[k]; e += 32) {
                    const int32_t z = abc::ld_adj(&a.adj[st[k] + e]);
                    ents++;
                    int32_t t;
                    if (abc::cand_of(a, z, up[k] != 0, t) && (t > 0 || !a.skip_zero)) {
                        r0_dec<HUB>(a, z, s_hub, hU, hV, hub);
                        decs++;
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ void round0_stats(const PeelArgs &a, unsigned long long ents, unsigned long long decs,
                                             unsigned long long hub, unsigned long long flushed) {
    const unsigned long long v[4] = {ents, decs, hub, flushed};
    unsigned long long *const d[4] = {&a.ctl->st[ST_STREAM], &a.ctl->st[ST_SDECS], &a.ctl->st[ST_HUBDECS],
                                      &a.ctl->st[ST_HUBFLUSH]};
    abc::block_add<4>(v, d);
}

__global__ void __launch_bounds__(256) k_round0_rows(PeelArgs a) {
    abc::grid_dep_launch();
    abc::grid_dep_wait();
    unsigned long long ents = 0, decs = 0, hub = 0;
    round0_rows_walk<false>(a, nullptr, 0, 0, ents, decs, hub);
    round0_stats(a, ents, decs, 0, 0);
}

// k_round0_rows with a hub table of hU + hV ints in dynamic shared memory, one 1024-thread block
// per SM (each block's table costs up to hU + hV atomics when it is written back, so the grid
// holds as few blocks as keep the SMs full). In degree order a row's first entries are its hub
// neighbours, and on power-law graphs a few thousand hubs per layer draw a large share of all
// decrements, which then cost a shared-memory atomic instead of an L2 one.
__global__ void __launch_bounds__(1024, 1) k_round0_hub(PeelArgs a, int hU, int hV) {
    extern __shared__ int s_hub[];
    abc::grid_dep_launch();
    for (int i = threadIdx.x; i < hU + hV; i += blockDim.x) s_hub[i] = 0;
    __syncthreads();
    abc::grid_dep_wait();
    unsigned long long ents = 0, decs = 0, hub = 0, flushed = 0;
    round0_rows_walk<true>(a, s_hub, hU, hV, ents, decs, hub);
    __syncthreads();
    for (int i = threadIdx.x; i < hU + hV; i += blockDim.x) {
        const int v = s_hub[i];
        if (v != 0) {
            abc::cnt_sub_noret(a, i < hU ? i : a.nU + (i - hU), v);
            flushed++;
        }
    }
    round0_stats(a, ents, decs, hub, flushed);
}

__device__ __forceinline__ bool alive_of(const PeelArgs &a, int32_t x) {
    if (x < a.nU) return x < a.pU && (x < a.cU || abc::cnt_load(a, x) >= a.thrU);
    return x < a.nU + a.pV && (x < a.nU + a.cV || abc::cnt_load(a, x) >= a.thrV);
}

__device__ __forceinline__ void k_cascade_emit(const PeelArgs &a, int ok, int64_t gw, int64_t nw, int lane);

__global__ void __launch_bounds__(256, 4) k_cascade(PeelArgs a) {
    __shared__ WarpSmem smem[256 / 32];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    abc::grid_dep_wait();
    if (a.phases && blockIdx.x == 0 && threadIdx.x == 0) a.ctl->ph[0] = abc::now_ns();
    LaneStats ls;
    const int ok = abc::cascade_loop(a, smem[wib], ls, a.grab_div, blockIdx.x == 0 && wib == 0);
    abc::flush_stats_block(a, ls);
    if (a.phases && threadIdx.x == 0) {
        const unsigned long long t = abc::now_ns();
        atomicMax(&a.ctl->ph[1], t);
        if (a.trace && blockIdx.x < abc::TRACE_BLOCKS) a.trace[4 + 4 * abc::TRACE_SAMPLES + 2 * blockIdx.x] = t;
    }
    if (a.emit == 2) k_cascade_emit(a, ok, gw, nw, lane);  // the gather is k_gather's
    if (a.phases) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long t = abc::now_ns();
            atomicMax(&a.ctl->ph[2], t);
            if (a.trace && blockIdx.x < abc::TRACE_BLOCKS) a.trace[4 + 4 * abc::TRACE_SAMPLES + 2 * blockIdx.x + 1] = t;
        }
    }
}

// The mask emission after the cascade (k_cascade's second phase).
__device__ __forceinline__ void k_cascade_emit(const PeelArgs &a, int ok, int64_t gw, int64_t nw, int lane) {
    if (!ok || a.emit == 0) return;
    const int64_t n = (int64_t)a.nU + a.nV;
    if (a.emit == 1) {
        // gather in the caller's order, once the queue has closed: caller id i is in the core
        // iff its internal id y = old2new[i] is a candidate that the peel did not remove. With
        // the bitmap (a.fallen), removal is bit i, set when the vertex fell; every load is then
        // coalesced, and the warp that reads a word clears it for the next peel (a word's ids
        // always fall to one warp). Without it, removal is read from y's count (one random
        // read per candidate). Lanes take four consecutive caller ids each (16-byte id loads,
        // 4-byte mask stores) when the masks' alignment allows, else one.
        const bool vec = ((reinterpret_cast<uintptr_t>(a.mask_u) | reinterpret_cast<uintptr_t>(a.mask_v)) & 3) == 0 &&
                         (a.nU & 3) == 0;
        const int64_t stride = nw * 32;
        if (vec) {
            constexpr int QILP = 4;  // quads in flight per lane
            const int64_t nq = (n + 3) >> 2;
            const int4 *o4 = reinterpret_cast<const int4 *>(a.old2new);
            for (int64_t q0 = gw * 32 + lane; q0 - lane < nq; q0 += stride * QILP) {
                int4 xv[QILP];
                uint32_t f[QILP];
#pragma unroll
                for (int k = 0; k < QILP; ++k) {
                    const int64_t q = q0 + k * stride;
                    xv[k] = make_int4(0, 0, 0, 0);
                    if (4 * q + 3 < n) {
                        xv[k] = __ldg(&o4[q]);
                    } else if (4 * q < n) {  // the last, partial quad
                        xv[k].x = __ldg(&a.old2new[4 * q]);
                        if (4 * q + 1 < n) xv[k].y = __ldg(&a.old2new[4 * q + 1]);
                        if (4 * q + 2 < n) xv[k].z = __ldg(&a.old2new[4 * q + 2]);
                    }
                    f[k] = (a.fallen != nullptr && q < nq) ? __ldcg(&a.fallen[q >> 3]) : 0u;
                }
#pragma unroll
                for (int k = 0; k < QILP; ++k) {
                    const int64_t q = q0 + k * stride;
                    if (q >= nq) continue;
                    const int32_t ys[4] = {xv[k].x, xv[k].y, xv[k].z, xv[k].w};
                    uint32_t bytes = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        bool in;
                        if (a.fallen != nullptr) {
                            const int32_t y = ys[j];
                            in = (y < a.nU ? y < a.pU : y - a.nU < a.pV) &&
                                 ((f[k] >> (((unsigned)q & 7u) * 4u + (unsigned)j)) & 1u) == 0;
                        } else {
                            in = 4 * q + j < n && alive_of(a, ys[j]);
                        }
                        bytes |= (in ? 1u : 0u) << (8 * j);
                    }
                    const int64_t i = q * 4;
                    uint8_t *dst = i < a.nU ? a.mask_u + i : a.mask_v + (i - a.nU);
                    if (i + 3 < n) {
                        *reinterpret_cast<uint32_t *>(dst) = bytes;
                    } else {
                        for (int j = 0; i + j < n; ++j) dst[j] = (uint8_t)(bytes >> (8 * j));
                    }
                }
                if (a.fallen != nullptr) {
                    // the eight lanes sharing a bitmap word have read it: the first one clears it
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < QILP; ++k) {
                        const int64_t q = q0 + k * stride;
                        if (q < nq && (q & 7) == 0 && f[k] != 0u) a.fallen[q >> 3] = 0u;
                    }
                }
            }
        } else {
            for (int64_t i0 = gw * 32 + lane; i0 - lane < n; i0 += stride) {
                const int64_t i = i0;
                const int32_t y = i < n ? __ldg(&a.old2new[i]) : 0;
                const uint32_t word = (a.fallen != nullptr && i < n) ? __ldcg(&a.fallen[i >> 5]) : 0u;
                if (i < n) {
                    bool in;
                    if (a.fallen != nullptr)
                        in = (y < a.nU ? y < a.pU : y - a.nU < a.pV) && ((word >> (i & 31)) & 1u) == 0;
                    else
                        in = alive_of(a, y);
                    if (i < a.nU) a.mask_u[i] = in ? 1 : 0;
                    else a.mask_v[i - a.nU] = in ? 1 : 0;
                }
                if (a.fallen != nullptr) {
                    __syncwarp();
                    if (lane == 0 && i < n && word != 0u) a.fallen[i >> 5] = 0u;
                }
            }
        }
    } else {
        // scatter: each lane tests SILP candidates at once (their count loads in flight
        // together), then looks up the survivors' caller ids and sets their bits
        constexpr int SILP = 8;
        const int64_t P = (int64_t)a.pU + a.pV;
        const int64_t stride = nw * 32;
        for (int64_t b = gw * 32; b < P; b += stride * SILP) {
            int32_t x[SILP];
            bool in[SILP];
#pragma unroll
            for (int k = 0; k < SILP; ++k) {
                const int64_t p = b + k * stride + lane;
                x[k] = p < a.pU ? (int32_t)p : (int32_t)(a.nU + (p - a.pU));
                in[k] = p < P && alive_of(a, x[k]);
            }
            int32_t o[SILP];
#pragma unroll
            for (int k = 0; k < SILP; ++k) o[k] = in[k] ? __ldg(&a.new2old[x[k]]) : 0;
#pragma unroll
            for (int k = 0; k < SILP; ++k) {
                if (!in[k]) continue;
                // the survivor's bit in the caller-order bitmap (k_expand writes the masks)
                const uint32_t u = (uint32_t)(x[k] < a.nU ? o[k] : a.nU + o[k]);
                atomicOr(&a.sbits[u >> 5], 1u << (u & 31));
            }
        }
    }
}

// The caller-order gather (emission 1) as a launch of its own after the cascade: its loads are
// all coalesced, so a full-occupancy grid moves them faster than the cascade's. Skipped when the
// cascade failed (the next peel then clears the removal bitmap).
__global__ void __launch_bounds__(256) k_gather(PeelArgs a) {
    abc::grid_dep_wait();
    if (abc::ld_relaxed_i32(&a.ctl->err) != 0) return;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    k_cascade_emit(a, 1, gw, nw, threadIdx.x & 31);
}

// After a scatter: both masks from the survivor bitmap, 32 caller ids (one word) per thread
// and iteration, written as two 16-byte stores where the word's ids lie in one layer and the
// destination is aligned (else byte by byte); every word is cleared for the next peel. Streaming
// stores of all n mask bytes replace a memset of the masks and random byte stores.
__global__ void __launch_bounds__(256) k_expand(PeelArgs a) {
    abc::grid_dep_launch();
    abc::grid_dep_wait();
    const int64_t n = (int64_t)a.nU + a.nV, nw = (n + 31) / 32;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    constexpr int EILP = 4;  // words per thread per pass, their loads in flight together
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w0 < nw; w0 += stride * EILP) {
        uint32_t wb[EILP];
#pragma unroll
        for (int e = 0; e < EILP; ++e) wb[e] = w0 + e * stride < nw ? __ldcg(&a.sbits[w0 + e * stride]) : 0u;
#pragma unroll
        for (int e = 0; e < EILP; ++e) {
            const int64_t w = w0 + e * stride;
            if (w >= nw) break;
            const uint32_t bits = wb[e];
            if (bits != 0u) a.sbits[w] = 0u;
            const int64_t i0 = w * 32;
            // 4 bits -> 4 bytes of 0/1: the multiplier moves bit t to bit 8t, and nothing else
            // lands on those four positions
            uint32_t q[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) q[k] = (((bits >> (4 * k)) & 0xfu) * 0x00204081u) & 0x01010101u;
            uint8_t *dst = nullptr;
            if (i0 + 32 <= a.nU) dst = a.mask_u + i0;
            else if (i0 >= a.nU && i0 + 32 <= n) dst = a.mask_v + (i0 - a.nU);
            if (dst != nullptr && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
                uint4 *d4 = reinterpret_cast<uint4 *>(dst);
                __stcs(&d4[0], make_uint4(q[0], q[1], q[2], q[3]));
                __stcs(&d4[1], make_uint4(q[4], q[5], q[6], q[7]));
            } else {
                for (int jj = 0; jj < 32 && i0 + jj < n; ++jj) {
                    const uint8_t v = (uint8_t)((bits >> jj) & 1u);
                    if (i0 + jj < a.nU) a.mask_u[i0 + jj] = v;
                    else a.mask_v[i0 + jj - a.nU] = v;
                }
            }
        }
    }
}

// Test hook: reserve queue slots that nothing will fill, so the consumers' bounded wait expires.
__global__ void k_stall(PeelCtl *ctl, long long qcap, int n) {
    if (ctl->tail + (unsigned long long)n <= (unsigned long long)qcap) atomicAdd(&ctl->tail, (unsigned long long)n);
}

}  // namespace

int cascade_grid(abcore_ctx *ctx) {
    if (ctx->cascade_blocks > 0) return ctx->cascade_blocks;
    int per_sm = ctx->prm.blocks_per_sm;
    if (per_sm <= 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cascade, 256, 0);
        if (per_sm <= 0) per_sm = 1;
    }
    ctx->cascade_blocks = per_sm * ctx->num_sms;
    return ctx->cascade_blocks;
}

int peel_prepare(abcore_ctx *ctx) {
    PeelWork &w = ctx->w;
    const Graph &g = ctx->g;
    const int64_t n = g.n();
    // every vertex is queued at most once, as ceil(row / chunk) items; idle warps may also hold
    // one ticket batch each beyond the last item
    const int64_t qcap = n + (2 * g.m) / std::max(ctx->prm.chunk, 1) + 1024 + (int64_t)ctx->num_sms * 64 * 32;
    uint32_t mu = 0, mv = 0;
    int64_t bv = 0;
    const int64_t slots = std::max(n, swz_layout(g.nU, g.nV, &mu, &mv, &bv));
    if (w.n == n && w.qcap >= qcap && w.cnt && w.cnt_slots >= slots && w.flag_blocks >= cascade_grid(ctx)) {
        // the round0 list (16 bytes a vertex) is only made once round0 is asked for
        if (ctx->prm.round0 && !w.l0) ABC_TRY(ctx->alloc(&w.l0, (size_t)std::max<int64_t>(n, 1), "initial violators"));
        return ABCORE_OK;
    }
    free_peel(ctx);
    // counts in the swizzled layout need each layer's power-of-two range
    ABC_TRY(ctx->alloc(&w.cnt, (size_t)std::max<int64_t>(slots, 1), "peel counts"));
    w.cnt_slots = slots;
    ABC_TRY(ctx->alloc(&w.plen, (size_t)std::max<int64_t>(n, 1), "peel prefixes"));
    if (ctx->prm.round0) ABC_TRY(ctx->alloc(&w.l0, (size_t)std::max<int64_t>(n, 1), "initial violators"));
    ABC_TRY(ctx->alloc(&w.q, (size_t)qcap, "peel queue"));
    ABC_TRY(ctx->alloc(&w.ctl, CTL_RING, "peel control"));
    ABC_TRY(ctx->alloc(&w.stage, (size_t)std::max<int64_t>(n, 1), "mask staging"));
    ABC_TRY(ctx->alloc(&w.fallen, (size_t)((n + 31) / 32 + 1), "removed-candidate bitmap"));
    ABC_CU(cudaMemsetAsync(w.fallen, 0, sizeof(uint32_t) * (size_t)((n + 31) / 32 + 1), ctx->stream));
    w.fallen_dirty = false;
    w.flag_blocks = cascade_grid(ctx);
    ABC_TRY(ctx->alloc(&w.flags, (size_t)w.flag_blocks * 32, "queue close flags"));
    ABC_CU(cudaMemsetAsync(w.flags, 0, sizeof(uint32_t) * (size_t)w.flag_blocks * 32, ctx->stream));
    w.epoch = 0;
    ABC_CU(cudaMallocHost(&w.ctl_host, sizeof(PeelCtl) * CTL_RING));
    for (int i = 0; i < CTL_RING; ++i) w.pending[i] = false;
    w.next = 0;
    w.last = -1;
    ABC_CU(cudaMemsetAsync(w.q, 0xff, sizeof(unsigned long long) * (size_t)qcap, ctx->stream));
    w.n = n;
    w.qcap = qcap;
    w.q_dirty = false;
    return ABCORE_OK;
}

void free_peel(abcore_ctx *ctx) {
    PeelWork &w = ctx->w;
    ctx->release(w.cnt);
    ctx->release(w.plen);
    ctx->release(w.l0);
    ctx->release(w.q);
    ctx->release(w.ctl);
    ctx->release(w.stage);
    ctx->release(w.fallen);
    ctx->release(w.flags);
    ctx->release(w.trace);
    w.flag_blocks = 0;
    if (w.ctl_host) cudaFreeHost(w.ctl_host);
    w.ctl_host = nullptr;
    for (int i = 0; i < CTL_RING; ++i) {
        w.pending[i] = false;
        for (int k = 0; k < 4; ++k)
            if (w.ev[i][k]) {
                cudaEventDestroy(w.ev[i][k]);
                w.ev[i][k] = nullptr;
            }
    }
    w.last = -1;
    w.n = w.qcap = 0;
    w.cnt_slots = 0;
}

// Launch k on the context's stream with `smem` bytes of dynamic shared memory; with `pdl`, as a programmatic dependent of the kernel before
// it on the stream (k calls grid_dep_wait before it touches memory).
template <typename... P, typename... A>
cudaError_t launch_k(bool pdl, void (*k)(P...), int64_t grid, int block, cudaStream_t st, size_t smem, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max<int64_t>(grid, 1));
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Cost model: per layer, count by searching the candidates' rows, or by streaming the rows of
// the other layer's initial violators? Both reach the same counts. Costs are in units of one
// random 32-byte sector read (a search probe), calibrated by measurement on this GPU: a streamed
// adjacency entry ~0.08, a stream decrement (atomic without return, L2-resident) ~0.8, a
// candidate's count init ~0.5. Hubs (degree >= hub_degree) count by search in both cases. A row
// search starts where the layer's share f of candidate entries puts the boundary; with the
// binomial spread sigma = sqrt(L f (1 - f)) of a row of length L about that guess, it reads
// about 1 + 2 log2(1 + sigma / 8) sectors (one, then a gallop and a bisection over the spread).
int pick_mode(const abcore_ctx *ctx, int32_t alpha, int32_t beta, int32_t pU, int32_t pV) {
    const Graph &g = ctx->g;
    if (ctx->prm.mode >= 0) return ctx->prm.mode & 3;
    const double m = (double)std::max<int64_t>(g.m, 1);
    const double pb = ctx->prm.probe_bytes / 32.0;  // relative probe cost (default 1)
    const int hd = ctx->prm.hub_degree > 0 ? ctx->prm.hub_degree : INT32_MAX;
    auto layer = [&](int64_t p, int32_t thr, const std::vector<int64_t> &cnt, const std::vector<int64_t> &edges,
                     double other_violator_entries, double f) {
        // non-hub candidates: degree in [thr, hd)
        const int32_t top = std::max(thr, hd);
        const double pn = (double)(p - std::min<int64_t>(p, cnt_ge(cnt, top)));
        const double en = (double)(cnt_ge(edges, thr) - cnt_ge(edges, top));
        const double avg = pn > 0 ? en / pn : 1.0;
        const double sigma = std::sqrt(std::max(avg, 1.0) * f * (1.0 - f));
        const double search = pn * (0.5 + pb * (1.0 + 2.0 * std::log2(1.0 + sigma / 8.0)));
        // stream: every violator entry is read; the share landing on non-hub candidates decrements
        const double stream = pn * 0.7 + other_violator_entries * (0.08 + 0.8 * (en / m));
        return search <= stream;
    };
    const double eU = (double)cnt_ge(g.edgesU_ge, alpha), eV = (double)cnt_ge(g.edgesV_ge, beta);
    // a U row's entries are V ids: the share below the bound is the V candidates' degree over m
    const bool sU = layer(pU, alpha, g.cntU_ge, g.edgesU_ge, m - eV, eV / m);
    const bool sV = layer(pV, beta, g.cntV_ge, g.edgesV_ge, m - eU, eU / m);
    return (sU ? 1 : 0) | (sV ? 2 : 0);
}

// With core numbers prepared, is the pruned peel (GCC+) the cheaper one? GCC+ initialises and
// peels the vertices with core in [min(alpha, beta), max(alpha, beta)); the plain peel those
// meeting their bound on full degree. Each side's vertex count stands for its cost: equal
// bounds leave GCC+ nothing to peel, while far-apart bounds can leave it far more vertices than
// the degree prefixes hold.
bool prefer_pruned(const abcore_ctx *ctx, int32_t alpha, int32_t beta) {
    if (!ctx->pr.ready || ctx->prm.algo == 1) return false;
    if (ctx->prm.algo == 2) return true;
    const Pruning &p = ctx->pr;
    const Graph &g = ctx->g;
    const int32_t dl = std::min(alpha, beta), dq = std::max(alpha, beta);
    const int64_t unc = (cnt_ge(p.coreU_ge, dl) - cnt_ge(p.coreU_ge, dq)) + (cnt_ge(p.coreV_ge, dl) - cnt_ge(p.coreV_ge, dq));
    const int64_t plain = cnt_ge(g.cntU_ge, alpha) + cnt_ge(g.cntV_ge, beta);
    return unc <= plain;
}

int peel_compute(abcore_ctx *ctx, int32_t alpha, int32_t beta, uint8_t *d_mask_u, uint8_t *d_mask_v,
                 bool sync_and_check, bool pruned) {
    // pruned (Algorithm 2, GCC+): the core-ordered graph; with dl = min(alpha, beta) and
    // dq = max(alpha, beta), vertices with core < dl cannot be members (Lemma 1(1)) and those
    // with core >= dq are members (Lemma 1(2)); only core in [dl, dq) is peeled, counting
    // neighbours with core >= dl, and only those vertices are ever decremented.
    const Graph &g = pruned ? ctx->pr.gc : ctx->g;
    PeelWork &w = ctx->w;
    ABC_TRY(peel_prepare(ctx));
    const int32_t nU = g.nU, nV = g.nV;
    const int64_t n = g.n();
    const int32_t dl = std::min(alpha, beta), dq = std::max(alpha, beta);
    const int32_t pU = (int32_t)(pruned ? cnt_ge(ctx->pr.coreU_ge, dl) : cnt_ge(g.cntU_ge, alpha));
    const int32_t pV = (int32_t)(pruned ? cnt_ge(ctx->pr.coreV_ge, dl) : cnt_ge(g.cntV_ge, beta));
    const int32_t cU = pruned ? (int32_t)cnt_ge(ctx->pr.coreU_ge, dq) : 0;
    const int32_t cV = pruned ? (int32_t)cnt_ge(ctx->pr.coreV_ge, dq) : 0;
    const int64_t P = (int64_t)pU + pV, Pu = (int64_t)(pU - cU) + (pV - cV);
    const int mode = pruned ? 3 : pick_mode(ctx, alpha, beta, pU, pV);

    const int slot = w.next;
    if (w.pending[slot]) ABC_TRY(peel_finish(ctx));  // ring wrapped: wait for the oldest peels
    w.next = (w.next + 1) % CTL_RING;
    PeelCtl *ctl = w.ctl + slot;

    PeelArgs a{};
    a.off = g.off;
    a.adj = g.adj;
    a.cnt = w.cnt;
    set_count_layout(a, pU, pV, ctx->prm.count_swizzle != 0);
    a.plen = w.plen;
    a.q = w.q;
    a.qcap = w.qcap;
    a.ctl = ctl;
    a.nU = nU;
    a.nV = nV;
    a.pU = pU;
    a.pV = pV;
    a.cU = cU;
    a.cV = cV;
    a.thrU = alpha;
    a.thrV = beta;
    a.chunk = std::max(ctx->prm.chunk, 32);
    a.batch_entries = ctx->prm.batch_entries;
    a.flush_steps = ctx->prm.flush_steps;
    a.local_rounds = ctx->prm.local_rounds;
    a.batch_entries_small = ctx->prm.batch_entries_small;
    a.phases = ctx->prm.log_level >= 2 ? 1 : 0;
    if (ctx->prm.log_level >= 2) {
        if (!w.trace) ABC_TRY(ctx->alloc(&w.trace, (size_t)CTL_RING * abc::TRACE_WORDS, "queue trace"));
        a.trace = w.trace + (size_t)slot * abc::TRACE_WORDS;
        ABC_CU(cudaMemsetAsync(a.trace, 0, abc::TRACE_WORDS * sizeof(unsigned long long), ctx->stream));
    }
    const int blocks = cascade_grid(ctx);
    a.grab_div = ctx->prm.grab_div > 0 ? ctx->prm.grab_div : std::max(1, blocks * (256 / 32) / 8);
    a.searchU = mode & 1;
    a.searchV = (mode >> 1) & 1;
    const bool hubs = ctx->prm.hub_degree > 0 && !pruned;
    a.hubcutU = hubs ? (int32_t)std::min<int64_t>(cnt_ge(g.cntU_ge, ctx->prm.hub_degree), pU) : 0;
    a.hubcutV = hubs ? (int32_t)std::min<int64_t>(cnt_ge(g.cntV_ge, ctx->prm.hub_degree), pV) : 0;
    a.timeout_ns = (unsigned long long)ctx->prm.timeout_ms * 1000000ull;
    a.old2new = g.old2new;
    a.new2old = g.new2old;
    a.mask_u = d_mask_u;
    a.mask_v = d_mask_v;
    const bool scatter = P * 100 <= (int64_t)ctx->prm.emit_scatter_max_pct * n;
    a.emit = (d_mask_u == nullptr && d_mask_v == nullptr) ? 0 : (scatter ? 2 : 1);
    a.skip_zero = 1;
    a.fallen = (a.emit == 1 && P * 100 >= (int64_t)ctx->prm.emit_bitmap_min_pct * n) ? w.fallen : nullptr;
    a.sbits = a.emit == 2 ? w.fallen : nullptr;  // the gather's bitmap is free in a scatter
    a.round0 = (ctx->prm.round0 && w.l0 && (a.searchU || a.searchV)) ? 1 : 0;
    a.l0 = w.l0;
    a.flags = w.flags;
    a.flag_first = 0;
    a.flag_count = blocks;
    if (++w.epoch == 0) w.epoch = 1;  // (a wrap could only meet flags 2^32 peels old)
    a.epoch = w.epoch;

    SlotInfo &si = w.info[slot];
    si = SlotInfo{};
    si.cands = pruned ? Pu : P;
    si.n = n;
    si.emit = a.emit;
    si.alpha = alpha;
    si.beta = beta;
    si.kinds = (unsigned)ctx->prm.timing_kinds & ((1u << ABCORE_K_INIT) | (1u << ABCORE_K_STREAM) | (1u << ABCORE_K_CASCADE));
    si.timed = ctx->prm.timing != 0 && si.kinds != 0;
    // events: 0 before the count init, 1 after it, 2 before the cascade, 3 after it; only those
    // bounding a timed kind are recorded
    const bool t_init = si.timed && (si.kinds & (1u << ABCORE_K_INIT));
    const bool t_first = si.timed && (si.kinds & (1u << ABCORE_K_STREAM));
    const bool t_casc = si.timed && (si.kinds & (1u << ABCORE_K_CASCADE));
    if (si.timed)
        for (int k = 0; k < 4; ++k)
            if (!w.ev[slot][k]) ABC_CU(cudaEventCreate(&w.ev[slot][k]));
    if (w.q_dirty) {
        ABC_CU(cudaMemsetAsync(w.q, 0xff, sizeof(unsigned long long) * (size_t)w.qcap, ctx->stream));
        w.q_dirty = false;
    }
    ABC_CU(cudaMemsetAsync(ctl, 0, sizeof(PeelCtl), ctx->stream));
    if ((a.fallen != nullptr || a.sbits != nullptr) && w.fallen_dirty) {
        ABC_CU(cudaMemsetAsync(w.fallen, 0, sizeof(uint32_t) * (size_t)((n + 31) / 32 + 1), ctx->stream));
        w.fallen_dirty = false;
    }
    if (t_init) ABC_CU(cudaEventRecord(w.ev[slot][0], ctx->stream));
    // the kernels after the count init follow it as programmatic dependents, except right after
    // a timing event (which must see the kernel before it end)
    const bool pdl = ctx->prm.pdl != 0;
    bool prev_k = false;  // the last operation on the stream is one of these kernels
    if (Pu > 0) {
        // at most the blocks that fit at once: each lane then walks several candidates
        if (ctx->init_blocks <= 0) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_init, INIT_THREADS, 0);
            ctx->init_blocks = std::max(per_sm, 1) * ctx->num_sms;
        }
        const int64_t gi = std::min<int64_t>((Pu + INIT_THREADS - 1) / INIT_THREADS, ctx->init_blocks);
        k_init<<<(unsigned)std::max<int64_t>(gi, 1), INIT_THREADS, 0, ctx->stream>>>(a);
        prev_k = true;
        si.has_init = true;
        ctx->stats.launches++;
        if (t_init || t_first) {
            ABC_CU(cudaEventRecord(w.ev[slot][1], ctx->stream));
            prev_k = false;
        }
        // Rows of the initial violators are contiguous: U violators [pU, nU) own
        // adj[off[pU], off[nU]) = [edgesU_ge(alpha), m), V violators [nU+pV, n) own
        // adj[m + edgesV_ge(beta), 2m). Slice A (V rows) feeds U counts, slice B (U rows) V counts.
        int64_t sa = 0, ea = 0, sb = 0, eb = 0;
        if (!a.searchU && pU > 0) {
            sa = g.m + cnt_ge(g.edgesV_ge, beta);
            ea = 2 * g.m;
        }
        if (!a.searchV && pV > 0) {
            sb = cnt_ge(g.edgesU_ge, alpha);
            eb = g.m;
        }
        const bool stream = ea > sa || eb > sb;
        if (stream) {
            const int64_t work = ((ea - sa) + (eb - sb)) / 4 + 1;
            const int64_t gs = std::min<int64_t>((work + STREAM_THREADS - 1) / STREAM_THREADS,
                                                 (int64_t)ctx->num_sms * 16);
            ABC_CU(launch_k(pdl && prev_k, k_stream, gs, STREAM_THREADS, ctx->stream, (size_t)0, a, sa, ea, sb, eb));
            si.has_stream = true;
            ctx->stats.launches++;
        }
        if (a.round0) {
            // the initial candidate violators' rows (their count is below the bound, so each row
            // is shorter than the bound)
            const int64_t gr = std::min<int64_t>((Pu + 255) / 256, (int64_t)ctx->num_sms * 16);
            switch (ctx->prm.round0_variant) {
                case 1: ABC_CU(launch_k(pdl && prev_k, k_round0<4, 8>, gr, 256, ctx->stream, (size_t)0, a)); break;
                case 2: ABC_CU(launch_k(pdl && prev_k, k_round0<16, 4>, gr, 256, ctx->stream, (size_t)0, a)); break;
                case 3: ABC_CU(launch_k(pdl && prev_k, k_round0<8, 8>, gr, 256, ctx->stream, (size_t)0, a)); break;
                case 4: ABC_CU(launch_k(pdl && prev_k, k_round0_rows, gr, 256, ctx->stream, (size_t)0, a)); break;
                case 5: {
                    const int hU = (int)std::min<int64_t>(pU, ctx->prm.round0_hub);
                    const int hV = (int)std::min<int64_t>(pV, ctx->prm.round0_hub);
                    const size_t smem = (size_t)(hU + hV) * sizeof(int);
                    if (ctx->hub_smem < smem) {
                        ABC_CU(cudaFuncSetAttribute(k_round0_hub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                        ctx->hub_smem = smem;
                    }
                    ABC_CU(launch_k(pdl && prev_k, k_round0_hub, std::min<int64_t>(gr, ctx->num_sms), 1024,
                                    ctx->stream, smem, a, hU, hV));
                    break;
                }
                default: ABC_CU(launch_k(pdl && prev_k, k_round0<8, 1>, gr, 256, ctx->stream, (size_t)0, a)); break;
            }
            si.has_stream = true;
            ctx->stats.launches++;
        }
        if (stream || a.round0) {
            // the candidates these first-round decrements took below their bound
            const int64_t ns = a.round0 ? Pu
                                        : (a.searchU ? 0 : (int64_t)pU - a.hubcutU) + (a.searchV ? 0 : (int64_t)pV - a.hubcutV);
            // at most the blocks that fit at once: fewer blocks, fewer reservations on the queue
            if (ctx->scan_blocks <= 0) {
                int per_sm = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan, 256, 0);
                ctx->scan_blocks = std::max(per_sm, 1) * ctx->num_sms;
            }
            const int64_t gsc = std::min<int64_t>((ns + 255) / 256, ctx->scan_blocks);
            ABC_CU(launch_k(pdl && prev_k, k_scan, gsc, 256, ctx->stream, (size_t)0, a));
            ctx->stats.launches++;
        }
    }
    if (ctx->prm.debug_stall_slots > 0) {
        k_stall<<<1, 1, 0, ctx->stream>>>(ctl, w.qcap, ctx->prm.debug_stall_slots);
        prev_k = false;
    }
    if (t_first || t_casc) {
        ABC_CU(cudaEventRecord(w.ev[slot][2], ctx->stream));
        prev_k = false;
    }
    ABC_CU(launch_k(pdl && prev_k, k_cascade, blocks, 256, ctx->stream, (size_t)0, a));
    ctx->stats.launches++;
    if (a.emit == 1) {
        if (ctx->gather_blocks <= 0) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gather, 256, 0);
            ctx->gather_blocks = std::max(per_sm, 1) * ctx->num_sms;
        }
        ABC_CU(launch_k(pdl, k_gather, ctx->gather_blocks, 256, ctx->stream, (size_t)0, a));
        ctx->stats.launches++;
    }
    if (a.emit == 2) {
        if (ctx->expand_blocks <= 0) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand, 256, 0);
            ctx->expand_blocks = std::max(per_sm, 1) * ctx->num_sms;
        }
        const int64_t ge = std::min<int64_t>(((n + 31) / 32 + 255) / 256, ctx->expand_blocks);
        ABC_CU(launch_k(pdl, k_expand, ge, 256, ctx->stream, (size_t)0, a));
        ctx->stats.launches++;
    }
    if (t_casc) ABC_CU(cudaEventRecord(w.ev[slot][3], ctx->stream));
    ABC_CU(cudaGetLastError());
    ABC_CU(cudaMemcpyAsync(w.ctl_host + slot, ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, ctx->stream));
    w.pending[slot] = true;
    w.last = slot;
    ctx->stats.mode = mode;
    ctx->stats.grid_blocks = blocks;
    ctx->pending_async = true;
    if (sync_and_check) return peel_finish(ctx);
    return ABCORE_OK;
}

// Wait for every peel in flight and turn their device status into a return code; the stats
// describe the most recent one.
// Log level 2: the cascade's queue over time, from the watcher's samples (time, done, tail,
// head), about 24 points.
static void log_queue_trace(abcore_ctx *ctx, const unsigned long long *dev) {
    std::vector<unsigned long long> h(abc::TRACE_WORDS);
    if (cudaMemcpy(h.data(), dev, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess) return;
    const unsigned long long k = std::min<unsigned long long>(h[0], abc::TRACE_SAMPLES);
    if (k == 0) return;
    std::string line;
    const unsigned long long step = std::max<unsigned long long>(1, k / 24);
    for (unsigned long long i = 0; i < k; i += step) {
        const unsigned long long *smp = h.data() + 4 + 4 * i;
        char b[96];
        snprintf(b, sizeof b, " %.0fus:%llu/%llu/%llu", smp[0] / 1e3, smp[1], smp[2], smp[3]);
        line += b;
    }
    const unsigned long long *last = h.data() + 4 + 4 * (k - 1);
    char b[96];
    snprintf(b, sizeof b, " end %.0fus:%llu/%llu", last[0] / 1e3, last[1], last[2]);
    line += b;
    ctx->log(2, "cascade queue (time:done/tail/head):%s", line.c_str());
    // blocks' cascade exit and emission end, from the watcher's start: quantiles
    std::vector<double> ex, em;
    const unsigned long long *blk = h.data() + 4 + 4 * abc::TRACE_SAMPLES;
    for (int i = 0; i < abc::TRACE_BLOCKS; ++i) {
        if (blk[2 * i] >= h[1] && h[1] != 0) ex.push_back((blk[2 * i] - h[1]) / 1e3);
        if (blk[2 * i + 1] >= h[1] && h[1] != 0) em.push_back((blk[2 * i + 1] - h[1]) / 1e3);
    }
    auto q = [](std::vector<double> &v, double f) {
        if (v.empty()) return 0.0;
        std::sort(v.begin(), v.end());
        return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1)))];
    };
    if (!ex.empty())
        ctx->log(2, "cascade blocks (%zu): exit us min %.0f med %.0f p90 %.0f max %.0f; emission end min %.0f med %.0f p90 %.0f max %.0f",
                 ex.size(), q(ex, 0), q(ex, 0.5), q(ex, 0.9), q(ex, 1), q(em, 0), q(em, 0.5), q(em, 0.9), q(em, 1));
}

int peel_finish(abcore_ctx *ctx) {
    if (!ctx->pending_async) return ABCORE_OK;
    ctx->pending_async = false;
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    PeelWork &w = ctx->w;
    abcore_stats &s = ctx->stats;
    int first_err = 0;
    for (int i = 0; i < CTL_RING; ++i) {
        if (!w.pending[i]) continue;
        w.pending[i] = false;
        const PeelCtl &c = w.ctl_host[i];
        const SlotInfo &si = w.info[i];
        if (c.err != 0 && first_err == 0) first_err = c.err;
        s.peels++;
        s.candidates += si.cands;
        s.init_vertices += (int64_t)c.st[ST_INIT];
        s.search_probes += (int64_t)c.st[ST_PROBES];
        s.stream_entries += (int64_t)c.st[ST_STREAM];
        s.entries += (int64_t)c.st[ST_ENTRIES];
        s.decrements += (int64_t)c.st[ST_DECS] + (int64_t)c.st[ST_SDECS];
        s.stream_decrements += (int64_t)c.st[ST_SDECS];
        s.scanned += (int64_t)c.st[ST_SCAN];
        s.pushes += (int64_t)c.st[ST_PUSHES];
        s.items += (int64_t)c.st[ST_ITEMS];
        s.round0_rows += (int64_t)c.l0n;
        if (c.ph[0] != 0 && c.ph[2] >= c.ph[1] && c.ph[1] >= c.ph[0])
            ctx->log(2, "peel (%d,%d): cascade queue drained after %.1f us, mask emission %.1f us", si.alpha, si.beta,
                     (c.ph[1] - c.ph[0]) / 1e3, (c.ph[2] - c.ph[1]) / 1e3);
        if (ctx->prm.log_level >= 2 && w.trace) log_queue_trace(ctx, w.trace + (size_t)i * abc::TRACE_WORDS);
        s.hub_decrements += (int64_t)c.st[ST_HUBDECS];
        s.hub_flushes += (int64_t)c.st[ST_HUBFLUSH];
        if (si.emit == 1) s.emit_gathered += si.n;
        if (si.emit == 2) {
            s.emit_scattered += si.cands;
            s.mask_zeroed += si.n;
        }
        if (si.timed) {
            float ms = 0.f;
            if (si.has_init && (si.kinds & (1u << ABCORE_K_INIT)) &&
                cudaEventElapsedTime(&ms, w.ev[i][0], w.ev[i][1]) == cudaSuccess) {
                s.kernel_ms[ABCORE_K_INIT] += ms;
                s.kernel_launches[ABCORE_K_INIT]++;
            }
            if (si.has_stream && (si.kinds & (1u << ABCORE_K_STREAM)) &&
                cudaEventElapsedTime(&ms, w.ev[i][1], w.ev[i][2]) == cudaSuccess) {
                s.kernel_ms[ABCORE_K_STREAM] += ms;
                s.kernel_launches[ABCORE_K_STREAM]++;
            }
            if ((si.kinds & (1u << ABCORE_K_CASCADE)) && cudaEventElapsedTime(&ms, w.ev[i][2], w.ev[i][3]) == cudaSuccess) {
                s.kernel_ms[ABCORE_K_CASCADE] += ms;
                s.kernel_launches[ABCORE_K_CASCADE]++;
            }
        }
    }
    if (first_err != 0) {
        w.q_dirty = true;
        w.fallen_dirty = true;
        if (first_err == ABCORE_ETIMEDOUT)
            return ctx->fail(ABCORE_ETIMEDOUT, "peel: a bounded device wait expired (limit %lld ms)",
                             (long long)ctx->prm.timeout_ms);
        return ctx->fail(first_err, "peel: device reported error %d", first_err);
    }
    return ABCORE_OK;
}
