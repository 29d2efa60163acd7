// An (alpha, beta)-core entry point that allocates nothing, for callers that cannot call
// cudaMalloc: code running where the allocator belongs to someone else (a host framework with a
// locked memory pool, a plugin inside another application's process) or where device memory is
// fully reserved ahead of time. The paper has no counterpart; this is an interface convenience
// around the same peel.
//
// The caller passes its graph and output masks as device pointers. The working memory -- one
// count per vertex, the removal queue and a control block -- is a file-scope __device__ array of
// fixed size, so graphs are limited to ABCORE_STATIC_MAX_VERTICES vertices and
// ABCORE_STATIC_MAX_ITEMS queue items. Every GPU that loads this library holds the array
// (about 13 MiB) until the process exits. Host code cannot use the array's name as a device
// address (in host code it names a host-side stand-in); the entry point asks the runtime for the
// device address with cudaGetSymbolAddress, once per device, on the first call made while that
// device is current. Every call shares the array and finds the previous call's contents in it,
// so each call clears the parts that must start empty, and calls that overlap on the GPU race.
// Each call reads two small values back to the host (the graph's queue need, then the error
// word), so it waits for its stream twice before returning.
//
// The peel itself is the plain one: counts start at the full degree, vertices below their
// bound are queued, and a ticket-queue cascade removes the rest, one exact crossing per vertex.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "device.cuh"
#include "../../include/abcore.h"

namespace {

constexpr int64_t MAXV = ABCORE_STATIC_MAX_VERTICES;
constexpr int64_t MAXQ = ABCORE_STATIC_MAX_ITEMS;
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_DEVICES = 64;
constexpr unsigned long long NA_EMPTY = ~0ull;

struct NaCtl {
    unsigned long long head;
    unsigned long long pad0[15];
    unsigned long long tail;
    unsigned long long pad1[15];
    unsigned long long done;
    unsigned long long pad2[15];
    int err;
    int pad3[31];
    unsigned long long chunks;  // queue items the graph needs: sum over rows of ceil(len / chunk)
    unsigned long long bad;     // rows with a negative length (offsets that decrease)
    long long m2;               // off[n]: adjacency entries
    unsigned long long pad4[13];
};

struct NaScratch {
    NaCtl ctl;
    int32_t cnt[MAXV];                // live-neighbour count per vertex
    unsigned long long q[MAXQ];       // queue items: vertex << 32 | chunk index
};

// The working memory shared by every call on this device (see the header comment).
static __device__ __align__(256) NaScratch g_na_scratch;

constexpr int NA_CHUNK = 1024;

struct NaArgs {
    const int64_t *off;
    const int32_t *adj;
    int32_t nU, nV, alpha, beta;
    uint8_t *mask_u, *mask_v;
    NaScratch *s;
    unsigned long long timeout_ns;
};

__device__ __forceinline__ int32_t na_thr(const NaArgs &a, int32_t x) { return x < a.nU ? a.alpha : a.beta; }

// Lanes with `want` queue x as one item per chunk of its row.
__device__ __forceinline__ void na_push(const NaArgs &a, bool want, int32_t x) {
    const unsigned pm = __ballot_sync(ABC_FULL, want);
    if (!pm) return;
    const int lane = threadIdx.x & 31;
    int nch = 0;
    if (want) nch = (int)((a.off[x + 1] - a.off[x] + NA_CHUNK - 1) / NA_CHUNK);
    const int incl = abc::warp_incl_scan(nch);
    const int total = __shfl_sync(ABC_FULL, incl, 31);
    if (total == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.s->ctl.tail, (unsigned long long)total);
    base = __shfl_sync(ABC_FULL, base, 0);
    if (base + total > (unsigned long long)MAXQ) {
        if (lane == 0) abc::set_error(&a.s->ctl.err, ABCORE_ENOMEM);
        return;
    }
    for (int i = 0; i < nch; ++i)
        abc::st_relaxed(&a.s->q[base + incl - nch + i], ((unsigned long long)(uint32_t)x << 32) | (unsigned)i);
}

// Checks before anything is queued: the queue items every vertex would need if it fell
// (ceil(row length / chunk) each; a vertex is queued at most once), off[n], and the offset faults
// that would send the cascade outside adj -- a negative off[0] or offsets that decrease.
// (Adjacency ids are checked where the cascade reads them.)
__global__ void __launch_bounds__(NA_THREADS) k_na_size(const int64_t *off, int64_t n, NaCtl *c) {
    unsigned long long ch = 0, bad = 0;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = t0; x < n; x += nt) {
        const int64_t d = off[x + 1] - off[x];
        if (d < 0) bad++;
        else ch += (unsigned long long)((d + NA_CHUNK - 1) / NA_CHUNK);
    }
    if (t0 == 0 && off[0] < 0) bad++;
    ch = (unsigned long long)abc::warp_sum64((long long)ch);
    bad = (unsigned long long)abc::warp_sum64((long long)bad);
    if ((threadIdx.x & 31) == 0) {
        if (ch) atomicAdd(&c->chunks, ch);
        if (bad) atomicAdd(&c->bad, bad);
    }
    if (t0 == 0) c->m2 = off[n];
}

// Counts start at the full degree; vertices below their bound are queued.
__global__ void __launch_bounds__(NA_THREADS) k_na_init(NaArgs a) {
    const int64_t n = (int64_t)a.nU + a.nV;
    const int lane = threadIdx.x & 31;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = t0 - lane; b < n; b += nt) {
        const int64_t x = b + lane;
        bool viol = false;
        if (x < n) {
            const int d = (int)(a.off[x + 1] - a.off[x]);
            a.s->cnt[x] = d;
            viol = d < na_thr(a, (int32_t)x);
        }
        na_push(a, viol, (int32_t)x);
    }
}

// Ticket-queue cascade (one item per warp at a time), then the masks. A warp takes a ticket
// (a queue slot number) and waits for its slot to be filled; when done == tail (read in that
// order) nothing is in flight and nothing can be queued any more, so every warp leaves.
__global__ void __launch_bounds__(NA_THREADS) k_na_cascade(NaArgs a) {
    const int lane = threadIdx.x & 31;
    NaCtl *c = &a.s->ctl;
    unsigned long long idle_since = abc::now_ns(), last_done = ~0ull, my = 0;
    bool holding = false;
    for (;;) {
        if (!holding) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(&c->head, 1ull);
            my = __shfl_sync(ABC_FULL, t, 0);
            holding = my < (unsigned long long)MAXQ;  // past the array: wait for the drain only
        }
        const unsigned long long it = holding ? abc::ld_relaxed(&a.s->q[my]) : NA_EMPTY;
        if (it != NA_EMPTY) {
            holding = false;
            __syncwarp();
            if (lane == 0) abc::st_relaxed(&a.s->q[my], NA_EMPTY);
            const int32_t x = (int32_t)(it >> 32);
            const int ch = (int)(it & 0xffffffffu);
            const int64_t s = a.off[x] + (int64_t)ch * NA_CHUNK;
            const int64_t e = min(a.off[x + 1], s + NA_CHUNK);
            for (int64_t p0 = s; p0 < e; p0 += 32) {
                const int64_t p = p0 + lane;
                bool push = false;
                int32_t y = 0;
                if (p < e) {
                    y = a.adj[p];
                    if (y < 0 || y >= a.nU + a.nV) {  // not a vertex: report it, touch nothing
                        abc::set_error(&a.s->ctl.err, ABCORE_EINVAL);
                    } else {
                        const int old = atomicSub(&a.s->cnt[y], 1);
                        push = old == na_thr(a, y);  // the one decrement that crosses below the bound
                    }
                }
                na_push(a, push, y);
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicAdd(&c->done, 1ull);
            idle_since = abc::now_ns();
            continue;
        }
        int verdict = 0;  // 0 keep waiting, 1 drained, 2 error
        if (lane == 0) {
            const unsigned long long d = abc::ld_acquire(&c->done);
            const unsigned long long tl = abc::ld_acquire(&c->tail);
            if (d == tl) verdict = 1;
            else if (abc::ld_relaxed_i32(&c->err)) verdict = 2;
            else if (d != last_done) {
                last_done = d;
                idle_since = abc::now_ns();
            } else if (abc::now_ns() - idle_since > a.timeout_ns) {
                abc::set_error(&c->err, ABCORE_ETIMEDOUT);
                verdict = 2;
            }
        }
        verdict = __shfl_sync(ABC_FULL, verdict, 0);
        if (verdict == 2) return;
        if (verdict == 1) break;
        __nanosleep(128);
    }
    const int64_t n = (int64_t)a.nU + a.nV;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = gw * 32 + lane; x < n; x += nw * 32) {
        const uint8_t v = __ldcg(&a.s->cnt[x]) >= na_thr(a, (int32_t)x) ? 1 : 0;
        if (x < a.nU) a.mask_u[x] = v;
        else a.mask_v[x - a.nU] = v;
    }
}

// Device address of g_na_scratch, looked up once per device.
void *g_na_addr[NA_MAX_DEVICES];

}  // namespace

extern "C" int abcore_compute_static(int32_t nU, int32_t nV, const int64_t *off, const int32_t *adj,
                                     int32_t alpha, int32_t beta, uint8_t *mask_u, uint8_t *mask_v,
                                     void *cuda_stream) {
    if (nU < 0 || nV < 0 || alpha < 0 || beta < 0) return ABCORE_EINVAL;
    const int64_t n = (int64_t)nU + nV;
    if (n > MAXV) return ABCORE_EINVAL;
    if (n == 0) return ABCORE_OK;
    if (!off || (nU > 0 && !mask_u) || (nV > 0 && !mask_v)) return ABCORE_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return ABCORE_ECUDA;
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return ABCORE_ECUDA;
        }
        g_na_addr[dev] = p;
    }
    NaScratch *s = (NaScratch *)g_na_addr[dev];
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the array keeps the previous call's contents: clear the control block, then measure the
    // graph's queue need (every vertex is queued at most once, as ceil(row / chunk) items)
    NaCtl size{};
    if (cudaMemsetAsync(&s->ctl, 0, sizeof(NaCtl), st) != cudaSuccess) return ABCORE_ECUDA;
    k_na_size<<<(unsigned)std::min<int64_t>((n + NA_THREADS - 1) / NA_THREADS, (int64_t)std::max(sms, 1) * 8),
                NA_THREADS, 0, st>>>(off, n, &s->ctl);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&size, &s->ctl, sizeof(NaCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ABCORE_ECUDA;
    if (size.bad != 0 || size.m2 < 0 || size.chunks > (unsigned long long)MAXQ) return ABCORE_EINVAL;
    if (size.m2 > 0 && !adj) return ABCORE_EINVAL;
    if (cudaMemsetAsync(s->q, 0xff, sizeof(unsigned long long) * MAXQ, st) != cudaSuccess) return ABCORE_ECUDA;
    NaArgs a{off, adj, nU, nV, alpha, beta, mask_u, mask_v, s, 4000ull * 1000000ull};
    const unsigned gi = (unsigned)std::min<int64_t>((n + NA_THREADS - 1) / NA_THREADS, (int64_t)sms * 8);
    k_na_init<<<gi, NA_THREADS, 0, st>>>(a);
    k_na_cascade<<<(unsigned)sms * 4, NA_THREADS, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return ABCORE_ECUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, &s->ctl.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ABCORE_ECUDA;
    return err ? err : ABCORE_OK;
}
