// Device CSR builder for both layers (Section 3: CSR storage; Section 4.1: flat continuous ids).
//
// From m distinct edges (u, v) it builds, entirely on the GPU:
//   * a renumbering of each layer by non-increasing degree (ties by caller id), so that for any
//     threshold t the vertices of a layer with degree >= t form a prefix of its id range;
//   * unified internal ids: U vertex i is i, V vertex j is nU + j;
//   * off[n+1] (int64) and adj[2m] (int32, unified ids): rows 0..nU-1 list V neighbours, rows
//     nU..n-1 list U neighbours, every row ascending (so also by non-increasing degree);
//   * new2old / old2new permutations, and host tables of vertex and edge counts per threshold.
// Sorting is a stable least-significant-digit radix sort over 64-bit keys written for this
// library: 8-bit digits, a fixed grid whose blocks own contiguous key ranges, per-block digit
// histograms, one exclusive scan, and a scatter whose in-warp ranks come from match.any.
#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "internal.h"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_IPT = 16;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
constexpr int RS_RADIX = 256;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t *__restrict__ keys, int64_t N,
                                                        int shift, int64_t tiles_per_block,
                                                        unsigned *__restrict__ hist, int G) {
    __shared__ unsigned h[RS_WARPS][RS_RADIX];
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    int64_t start = (int64_t)blockIdx.x * tiles_per_block * RS_TILE;
    int64_t end = min(start + tiles_per_block * RS_TILE, N);
    for (int64_t i = start + threadIdx.x; i < end; i += RS_THREADS) {
        unsigned d = (unsigned)(keys[i] >> shift) & 255u;
        atomicAdd(&h[w][d], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_RADIX; d += RS_THREADS) {
        unsigned s = 0;
        for (int k = 0; k < RS_WARPS; ++k) s += h[k][d];
        hist[(int64_t)d * G + blockIdx.x] = s;
    }
}

// Exclusive scan of `count` unsigned values (digit-major) into 64-bit offsets, one block.
__global__ void __launch_bounds__(1024) k_rs_scan(const unsigned *__restrict__ hist, int count,
                                                  unsigned long long *__restrict__ offs) {
    __shared__ unsigned long long part[1024];
    const int t = threadIdx.x;
    const int per = (count + 1023) / 1024;
    const int b = t * per, e = min(b + per, count);
    unsigned long long s = 0;
    for (int i = b; i < e; ++i) s += hist[i];
    part[t] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        unsigned long long v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned long long run = part[t] - s;
    for (int i = b; i < e; ++i) {
        offs[i] = run;
        run += hist[i];
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t *__restrict__ in,
                                                           uint64_t *__restrict__ out, int64_t N,
                                                           int shift, int64_t tiles_per_block,
                                                           const unsigned long long *__restrict__ offs,
                                                           int G) {
    __shared__ unsigned long long base[RS_RADIX];
    __shared__ unsigned wcnt[RS_WARPS][RS_RADIX];
    __shared__ unsigned woff[RS_WARPS][RS_RADIX];
    __shared__ unsigned tcnt[RS_RADIX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * G + blockIdx.x];
    const int64_t t0 = (int64_t)blockIdx.x * tiles_per_block;
    const int64_t total_tiles = (N + RS_TILE - 1) / RS_TILE;
    const int64_t t1 = min(t0 + tiles_per_block, total_tiles);
    const unsigned lt = abc::lanemask_lt();
    for (int64_t tile = t0; tile < t1; ++tile) {
        for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const int64_t seg = tile * RS_TILE + (int64_t)w * 32 * RS_IPT;
        uint64_t k[RS_IPT];
        unsigned r[RS_IPT];
#pragma unroll
        for (int it = 0; it < RS_IPT; ++it) {
            const int64_t idx = seg + it * 32 + lane;
            const bool valid = idx < N;
            k[it] = valid ? in[idx] : 0ull;
        }
#pragma unroll
        for (int it = 0; it < RS_IPT; ++it) {
            const int64_t idx = seg + it * 32 + lane;
            const bool valid = idx < N;
            const unsigned act = __ballot_sync(ABC_FULL, valid);
            r[it] = 0;
            if (valid) {
                const unsigned d = (unsigned)(k[it] >> shift) & 255u;
                const unsigned peers = __match_any_sync(act, d);
                const unsigned before = __popc(peers & lt);
                const unsigned prev = wcnt[w][d];
                __syncwarp(act);
                if (before == 0) wcnt[w][d] = prev + __popc(peers);
                __syncwarp(act);
                r[it] = prev + before;
            }
        }
        __syncthreads();
        {
            const int d = threadIdx.x;
            unsigned s = 0;
#pragma unroll
            for (int q = 0; q < RS_WARPS; ++q) {
                woff[q][d] = s;
                s += wcnt[q][d];
            }
            tcnt[d] = s;
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < RS_IPT; ++it) {
            const int64_t idx = seg + it * 32 + lane;
            if (idx < N) {
                const unsigned d = (unsigned)(k[it] >> shift) & 255u;
                out[base[d] + woff[w][d] + r[it]] = k[it];
            }
        }
        __syncthreads();
        base[threadIdx.x] += tcnt[threadIdx.x];
        __syncthreads();
    }
}

// Sort N keys on bits [bit_lo, bit_hi); bits outside that range ride along. *result is a or b.
int radix_sort_u64(abcore_ctx *ctx, uint64_t *a, uint64_t *b, int64_t N, int bit_lo, int bit_hi,
                   uint64_t **result) {
    *result = a;
    if (N <= 1 || bit_hi <= bit_lo) return ABCORE_OK;
    const int64_t tiles = (N + RS_TILE - 1) / RS_TILE;
    int G = (int)std::min<int64_t>(tiles, (int64_t)ctx->num_sms * 4);
    const int64_t tpb = (tiles + G - 1) / G;
    G = (int)((tiles + tpb - 1) / tpb);
    unsigned *hist = nullptr;
    unsigned long long *offs = nullptr;
    ABC_TRY(ctx->alloc(&hist, (size_t)RS_RADIX * G, "radix histogram"));
    int rc = ctx->alloc(&offs, (size_t)RS_RADIX * G, "radix offsets");
    if (rc) { ctx->release(hist); return rc; }
    uint64_t *src = a, *dst = b;
    for (int shift = bit_lo; shift < bit_hi; shift += 8) {
        k_rs_hist<<<G, RS_THREADS, 0, ctx->stream>>>(src, N, shift, tpb, hist, G);
        k_rs_scan<<<1, 1024, 0, ctx->stream>>>(hist, RS_RADIX * G, offs);
        k_rs_scatter<<<G, RS_THREADS, 0, ctx->stream>>>(src, dst, N, shift, tpb, offs, G);
        std::swap(src, dst);
    }
    cudaError_t e = cudaGetLastError();
    ctx->release(hist);
    ctx->release(offs);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "radix sort launch");
    *result = src;
    return ABCORE_OK;
}

// ---- exclusive scan of int32 counts into int64 offsets (out[N] = total) -------------------
constexpr int SC_THREADS = 256, SC_IPT = 16, SC_TILE = SC_THREADS * SC_IPT;

__device__ long long block_excl_scan(long long v, long long *total) {
    __shared__ long long wsum[SC_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = abc::warp_incl_scan64(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long x = lane < SC_THREADS / 32 ? wsum[lane] : 0;
        long long xi = abc::warp_incl_scan64(x);
        if (lane < SC_THREADS / 32) wsum[lane] = xi - x;
        if (lane == SC_THREADS / 32 - 1) *total = xi;
    }
    __syncthreads();
    long long r = inc - v + wsum[w];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_part(const int32_t *__restrict__ in, int64_t N,
                                                          long long *__restrict__ part) {
    __shared__ long long tot;
    const int64_t b = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_IPT;
    long long s = 0;
    for (int i = 0; i < SC_IPT; ++i)
        if (b + i < N) s += in[b + i];
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(long long *part, int64_t nb, int64_t *out_total) {
    __shared__ long long sh[1024];
    const int t = threadIdx.x;
    const int64_t per = (nb + 1023) / 1024;
    const int64_t b = t * per, e = min(b + per, nb);
    long long s = 0;
    for (int64_t i = b; i < e; ++i) s += part[i];
    sh[t] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        long long v = t >= d ? sh[t - d] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    long long run = sh[t] - s;
    for (int64_t i = b; i < e; ++i) {
        long long x = part[i];
        part[i] = run;
        run += x;
    }
    if (t == 1023) *out_total = sh[1023];
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_final(const int32_t *__restrict__ in, int64_t N,
                                                           const long long *__restrict__ part,
                                                           int64_t *__restrict__ out) {
    __shared__ long long tot;
    const int64_t b = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_IPT;
    int32_t v[SC_IPT];
    long long s = 0;
    for (int i = 0; i < SC_IPT; ++i) {
        v[i] = b + i < N ? in[b + i] : 0;
        s += v[i];
    }
    long long run = block_excl_scan(s, &tot) + part[blockIdx.x];
    for (int i = 0; i < SC_IPT; ++i)
        if (b + i < N) {
            out[b + i] = run;
            run += v[i];
        }
}

int exclusive_scan_i32(abcore_ctx *ctx, const int32_t *in, int64_t N, int64_t *out) {
    if (N == 0) {
        ABC_CU(cudaMemsetAsync(out, 0, sizeof(int64_t), ctx->stream));
        return ABCORE_OK;
    }
    const int64_t nb = (N + SC_TILE - 1) / SC_TILE;
    long long *part = nullptr;
    ABC_TRY(ctx->alloc(&part, (size_t)nb, "scan partials"));
    k_scan_part<<<(unsigned)nb, SC_THREADS, 0, ctx->stream>>>(in, N, part);
    k_scan_top<<<1, 1024, 0, ctx->stream>>>(part, nb, out + N);
    k_scan_final<<<(unsigned)nb, SC_THREADS, 0, ctx->stream>>>(in, N, part, out);
    cudaError_t e = cudaGetLastError();
    ctx->release(part);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "scan launch");
    return ABCORE_OK;
}

// ---- builder kernels --------------------------------------------------------------------
__global__ void k_count_deg(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev, int64_t m,
                            int32_t nU, int32_t nV, int32_t *__restrict__ degU,
                            int32_t *__restrict__ degV, int *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = eu[i], v = ev[i];
        if (u < 0 || u >= nU || v < 0 || v >= nV) {
            abc::set_error(err, ABCORE_EINVAL);
            continue;
        }
        atomicAdd(&degU[u], 1);
        atomicAdd(&degV[v], 1);
    }
}

__global__ void k_max(const int32_t *__restrict__ a, int64_t n, int *out) {
    int mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, a[i]);
    for (int d = 16; d >= 1; d >>= 1) mx = max(mx, __shfl_xor_sync(ABC_FULL, mx, d));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

__global__ void k_relabel_keys(const int32_t *__restrict__ deg, int64_t n, int32_t maxdeg,
                               uint64_t *__restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = ((uint64_t)(uint32_t)(maxdeg - deg[i]) << 32) | (uint64_t)i;
}

__global__ void k_relabel_finish(const uint64_t *__restrict__ keys, int64_t n, int32_t base,
                                 int32_t maxdeg, int32_t *__restrict__ new2old,
                                 int32_t *__restrict__ old2new, int32_t *__restrict__ degnew) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[p];
        const int32_t old = (int32_t)(k & 0xffffffffu);
        new2old[base + p] = old;
        old2new[base + old] = base + (int32_t)p;
        degnew[base + p] = maxdeg - (int32_t)(k >> 32);
    }
}

// Row-major edge keys: (row rank << cbits) | column rank, both in internal per-layer ranks.
__global__ void k_edge_keys(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev, int64_t m,
                            const int32_t *__restrict__ old2new, int32_t nU, int upper_rows,
                            int cbits, uint64_t *__restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ru = (uint64_t)old2new[eu[i]];
        const uint64_t rv = (uint64_t)(old2new[nU + ev[i]] - nU);
        keys[i] = upper_rows ? ((ru << cbits) | rv) : ((rv << cbits) | ru);
    }
}

__global__ void k_extract(const uint64_t *__restrict__ keys, int64_t m, uint64_t cmask, int32_t add,
                          int32_t *__restrict__ adj, int *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        if (i > 0 && keys[i - 1] == k) abc::set_error(err, ABCORE_EEXIST);
        adj[i] = (int32_t)(k & cmask) + add;
    }
}

// Second ordering pass (build with a rank): position p of the degree order gets the key
// (maxrank - rank) << 32 | p, so a stable sort orders by non-increasing rank, ties by degree
// order.
__global__ void k_rank_keys(const uint64_t *__restrict__ by_degree, int64_t n, int32_t base,
                            const int32_t *__restrict__ rank, int32_t maxrank, uint64_t *__restrict__ keys) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t old = (int32_t)(by_degree[p] & 0xffffffffu);
        keys[p] = ((uint64_t)(uint32_t)(maxrank - rank[base + old]) << 32) | (uint64_t)p;
    }
}

__global__ void k_rank_finish(const uint64_t *__restrict__ by_rank, const uint64_t *__restrict__ by_degree,
                              int64_t n, int32_t base, int32_t maxdeg, int32_t *__restrict__ new2old,
                              int32_t *__restrict__ old2new, int32_t *__restrict__ degnew) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = (int64_t)(by_rank[q] & 0xffffffffu);
        const uint64_t k = by_degree[p];
        const int32_t old = (int32_t)(k & 0xffffffffu);
        new2old[base + q] = old;
        old2new[base + old] = base + (int32_t)q;
        degnew[base + q] = maxdeg - (int32_t)(k >> 32);
    }
}

// Caller-id edges of a CSR's U rows: (new2old[row], new2old[column]).
__global__ void k_edges_of(const int32_t *__restrict__ rowid, const int32_t *__restrict__ adj, int64_t m,
                           const int32_t *__restrict__ new2old, int32_t *__restrict__ eu, int32_t *__restrict__ ev) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        eu[i] = new2old[rowid[i]];
        ev[i] = new2old[adj[i]];
    }
}

// cnt_ge[t] for t in [0, maxdeg+1] from a layer's degrees sorted non-increasing.
__global__ void k_cnt_ge(const int32_t *__restrict__ deg, int64_t nl, int32_t maxdeg,
                         int64_t *__restrict__ cnt_ge) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nl;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = deg[p];
        const int32_t dn = p + 1 < nl ? deg[p + 1] : -1;
        for (int32_t t = dn + 1; t <= d; ++t) cnt_ge[t] = p + 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cnt_ge[maxdeg + 1] = 0;
        if (nl == 0) cnt_ge[0] = 0;
    }
}

__global__ void k_edges_ge(const int64_t *__restrict__ cnt_ge, int32_t maxdeg,
                           const int64_t *__restrict__ off, int64_t base,
                           int64_t *__restrict__ edges_ge) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= maxdeg + 1;
         t += (int64_t)gridDim.x * blockDim.x)
        edges_ge[t] = off[base + cnt_ge[t]] - off[base];
}

// Expand a CSR into the row id of every entry: one warp per row.
__global__ void k_expand_rows(const int64_t *__restrict__ off, int32_t nrows, int32_t *__restrict__ rowid) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t s = off[r], e = off[r + 1];
        for (int64_t j = s + lane; j < e; j += 32) rowid[j] = (int32_t)r;
    }
}

__global__ void k_check_off(const int64_t *__restrict__ off, int32_t nrows, int64_t m, int *err) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (off[r + 1] < off[r]) abc::set_error(err, ABCORE_EINVAL);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[nrows] != m))
        abc::set_error(err, ABCORE_EINVAL);
}

__global__ void k_pair_keys(const int32_t *__restrict__ a, const int32_t *__restrict__ b, int64_t m,
                            int32_t nb, uint64_t *__restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint64_t)a[i] * (uint64_t)nb + (uint64_t)b[i];
}

__global__ void k_diff(const uint64_t *__restrict__ a, const uint64_t *__restrict__ b, int64_t m, int *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        if (a[i] != b[i]) abc::set_error(err, ABCORE_EINVAL);
}

int bits_for(int64_t n) {  // bits needed to hold values 0..n-1 (at least 1)
    int b = 1;
    while (b < 63 && ((int64_t)1 << b) < n) ++b;
    return b;
}

unsigned grid_for(abcore_ctx *ctx, int64_t n, int threads = 256) {
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)ctx->num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

int read_err(abcore_ctx *ctx, int *d_err, int *h_err) {
    ABC_CU(cudaMemcpyAsync(h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    return ABCORE_OK;
}

}  // namespace

void free_graph_of(abcore_ctx *ctx, Graph &g) {
    ctx->release(g.off);
    ctx->release(g.adj);
    ctx->release(g.new2old);
    ctx->release(g.old2new);
    g.cntU_ge.clear(); g.edgesU_ge.clear(); g.cntV_ge.clear(); g.edgesV_ge.clear();
    g.loaded = false;
    g.nU = g.nV = 0;
    g.m = 0;
}

void free_graph(abcore_ctx *ctx) {
    free_pruning(ctx);
    free_graph_of(ctx, ctx->g);
}

int check_csr_offsets(abcore_ctx *ctx, int32_t nrows, const int64_t *d_off, int64_t m) {
    int *d_err = nullptr;
    ABC_TRY(ctx->alloc(&d_err, 1, "error word"));
    int h_err = 0;
    cudaMemsetAsync(d_err, 0, sizeof(int), ctx->stream);
    k_check_off<<<grid_for(ctx, nrows), 256, 0, ctx->stream>>>(d_off, nrows, m, d_err);
    int rc = read_err(ctx, d_err, &h_err);
    ctx->release(d_err);
    if (rc) return rc;
    if (h_err) return ctx->fail(ABCORE_EINVAL, "CSR offsets must start at 0, be non-decreasing and end at m");
    return ABCORE_OK;
}

int expand_csr_to_edges(abcore_ctx *ctx, int32_t nrows, const int64_t *d_off, const int32_t *d_adj,
                        int64_t m, int32_t *d_rowid) {
    (void)d_adj;
    (void)m;
    if (nrows > 0)
        k_expand_rows<<<grid_for(ctx, (int64_t)nrows * 32), 256, 0, ctx->stream>>>(d_off, nrows, d_rowid);
    ABC_CU(cudaGetLastError());
    return ABCORE_OK;
}

// Compare two edge lists as sets (both distinct): EINVAL if they differ.
int compare_edge_sets(abcore_ctx *ctx, int32_t nV, int64_t m, const int32_t *eu1, const int32_t *ev1,
                      const int32_t *eu2, const int32_t *ev2) {
    uint64_t *a = nullptr, *b = nullptr, *c = nullptr, *d = nullptr;
    int *d_err = nullptr;
    int rc = ctx->alloc(&a, (size_t)m, "validate keys");
    if (!rc) rc = ctx->alloc(&b, (size_t)m, "validate keys");
    if (!rc) rc = ctx->alloc(&c, (size_t)m, "validate keys");
    if (!rc) rc = ctx->alloc(&d, (size_t)m, "validate keys");
    if (!rc) rc = ctx->alloc(&d_err, 1, "error word");
    int h_err = 0;
    if (!rc) {
        cudaMemsetAsync(d_err, 0, sizeof(int), ctx->stream);
        k_pair_keys<<<grid_for(ctx, m), 256, 0, ctx->stream>>>(eu1, ev1, m, nV, a);
        k_pair_keys<<<grid_for(ctx, m), 256, 0, ctx->stream>>>(eu2, ev2, m, nV, c);
        int64_t maxkey = (int64_t)ctx->g.nU * nV;
        int bits = bits_for(maxkey > 1 ? maxkey : 2);
        uint64_t *r1, *r2;
        rc = radix_sort_u64(ctx, a, b, m, 0, bits, &r1);
        if (!rc) rc = radix_sort_u64(ctx, c, d, m, 0, bits, &r2);
        if (!rc) {
            k_diff<<<grid_for(ctx, m), 256, 0, ctx->stream>>>(r1, r2, m, d_err);
            rc = read_err(ctx, d_err, &h_err);
        }
    }
    ctx->release(a); ctx->release(b); ctx->release(c); ctx->release(d); ctx->release(d_err);
    if (rc) return rc;
    if (h_err) return ctx->fail(ABCORE_EINVAL, "the two CSR layers describe different edge sets");
    return ABCORE_OK;
}

int build_graph_from_device_edges(abcore_ctx *ctx, int32_t nU, int32_t nV, int64_t m,
                                  const int32_t *d_eu, const int32_t *d_ev) {
    free_graph(ctx);
    return build_graph(ctx, ctx->g, nU, nV, m, d_eu, d_ev, nullptr, 0);
}

int csr_edges(abcore_ctx *ctx, const Graph &g, int32_t *d_eu, int32_t *d_ev) {
    int32_t *rowid = nullptr;
    ABC_TRY(ctx->alloc(&rowid, (size_t)std::max<int64_t>(g.m, 1), "edge rows"));
    int rc = expand_csr_to_edges(ctx, g.nU, g.off, g.adj, g.m, rowid);
    if (!rc && g.m > 0) {
        k_edges_of<<<grid_for(ctx, g.m), 256, 0, ctx->stream>>>(rowid, g.adj, g.m, g.new2old, d_eu, d_ev);
        const cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = ctx->cuda_fail(e, "edge list");
    }
    ctx->release(rowid);
    return rc;
}

int build_graph(abcore_ctx *ctx, Graph &g, int32_t nU, int32_t nV, int64_t m, const int32_t *d_eu,
                const int32_t *d_ev, const int32_t *d_rank, int32_t maxrank) {
    const int64_t n = (int64_t)nU + nV;
    int32_t *deg = nullptr, *degnew = nullptr;
    int *d_err = nullptr, *d_max = nullptr;
    uint64_t *ka = nullptr, *kb = nullptr, *rk = nullptr;
    int64_t *cnt_ge = nullptr, *edges_ge = nullptr;
    int h_err = 0, h_max[2] = {0, 0};
    int rc = ABCORE_OK;

#define STEP(x)            \
    do {                   \
        rc = (x);          \
        if (rc) goto fail; \
    } while (0)

    STEP(ctx->alloc(&deg, (size_t)n, "degrees"));
    STEP(ctx->alloc(&degnew, (size_t)n, "sorted degrees"));
    STEP(ctx->alloc(&d_err, 1, "error word"));
    STEP(ctx->alloc(&d_max, 2, "max degree"));
    STEP(ctx->alloc(&g.off, (size_t)n + 1, "row offsets"));
    STEP(ctx->alloc(&g.adj, (size_t)(2 * m), "adjacency"));
    STEP(ctx->alloc(&g.new2old, (size_t)n, "new2old"));
    STEP(ctx->alloc(&g.old2new, (size_t)n, "old2new"));
    cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)(n ? n : 1), ctx->stream);
    cudaMemsetAsync(d_err, 0, sizeof(int), ctx->stream);
    cudaMemsetAsync(d_max, 0, 2 * sizeof(int), ctx->stream);
    if (m > 0)
        k_count_deg<<<grid_for(ctx, m), 256, 0, ctx->stream>>>(d_eu, d_ev, m, nU, nV, deg, deg + nU, d_err);
    STEP(read_err(ctx, d_err, &h_err));
    if (h_err) {
        rc = ctx->fail(ABCORE_EINVAL, "edge endpoint out of range (u must be < nU, v < nV)");
        goto fail;
    }
    if (nU > 0) k_max<<<grid_for(ctx, nU), 256, 0, ctx->stream>>>(deg, nU, d_max);
    if (nV > 0) k_max<<<grid_for(ctx, nV), 256, 0, ctx->stream>>>(deg + nU, nV, d_max + 1);
    ABC_CU(cudaMemcpyAsync(h_max, d_max, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    ABC_CU(cudaStreamSynchronize(ctx->stream));
    g.maxdegU = h_max[0];
    g.maxdegV = h_max[1];

    {
        const int64_t kcap = std::max<int64_t>(std::max<int64_t>(m, n), 1);
        STEP(ctx->alloc(&ka, (size_t)kcap, "sort keys"));
        STEP(ctx->alloc(&kb, (size_t)kcap, "sort keys"));
        // renumber each layer by non-increasing degree; ties keep caller-id order (stable)
        for (int layer = 0; layer < 2; ++layer) {
            const int64_t nl = layer == 0 ? nU : nV;
            const int32_t base = layer == 0 ? 0 : nU;
            const int32_t md = layer == 0 ? g.maxdegU : g.maxdegV;
            if (nl == 0) continue;
            k_relabel_keys<<<grid_for(ctx, nl), 256, 0, ctx->stream>>>(deg + base, nl, md, ka);
            uint64_t *sorted;
            STEP(radix_sort_u64(ctx, ka, kb, nl, 32, 32 + bits_for((int64_t)md + 1), &sorted));
            if (!d_rank) {
                k_relabel_finish<<<grid_for(ctx, nl), 256, 0, ctx->stream>>>(sorted, nl, base, md, g.new2old,
                                                                             g.old2new, degnew);
            } else {
                // then by non-increasing rank, ties keeping the degree order
                if (!rk) STEP(ctx->alloc(&rk, (size_t)std::max<int64_t>(std::max<int64_t>(nU, nV), 1) * 2, "rank keys"));
                uint64_t *ra = rk, *rb = rk + std::max<int64_t>(nU, nV);
                k_rank_keys<<<grid_for(ctx, nl), 256, 0, ctx->stream>>>(sorted, nl, base, d_rank, maxrank, ra);
                uint64_t *sorted2;
                STEP(radix_sort_u64(ctx, ra, rb, nl, 32, 32 + bits_for((int64_t)maxrank + 1), &sorted2));
                k_rank_finish<<<grid_for(ctx, nl), 256, 0, ctx->stream>>>(sorted2, sorted, nl, base, md, g.new2old,
                                                                          g.old2new, degnew);
            }
        }
        STEP(exclusive_scan_i32(ctx, degnew, n, g.off));
        // rows of both layers, sorted by (row, column) in internal ranks
        const int ubits = bits_for(std::max<int32_t>(nU, 1)), vbits = bits_for(std::max<int32_t>(nV, 1));
        for (int layer = 0; layer < 2 && m > 0; ++layer) {
            const int cbits = layer == 0 ? vbits : ubits;
            const int rbits = layer == 0 ? ubits : vbits;
            k_edge_keys<<<grid_for(ctx, m), 256, 0, ctx->stream>>>(d_eu, d_ev, m, g.old2new, nU, layer == 0,
                                                                   cbits, ka);
            uint64_t *sorted;
            STEP(radix_sort_u64(ctx, ka, kb, m, 0, cbits + rbits, &sorted));
            k_extract<<<grid_for(ctx, m), 256, 0, ctx->stream>>>(sorted, m, ((uint64_t)1 << cbits) - 1,
                                                                 layer == 0 ? nU : 0, g.adj + layer * m, d_err);
        }
        STEP(read_err(ctx, d_err, &h_err));
        if (h_err) {
            rc = ctx->fail(ABCORE_EEXIST, "an edge appears more than once in the input");
            goto fail;
        }
    }
    // host tables: vertices and edges at or above each degree threshold, per layer (a graph
    // ordered by rank is not in degree order, and gets none)
    for (int layer = 0; layer < 2 && !d_rank; ++layer) {
        const int64_t nl = layer == 0 ? nU : nV;
        const int32_t md = layer == 0 ? g.maxdegU : g.maxdegV;
        const int64_t base = layer == 0 ? 0 : nU;
        std::vector<int64_t> &cg = layer == 0 ? g.cntU_ge : g.cntV_ge;
        std::vector<int64_t> &eg = layer == 0 ? g.edgesU_ge : g.edgesV_ge;
        cg.assign((size_t)md + 2, 0);
        eg.assign((size_t)md + 2, 0);
        STEP(ctx->alloc(&cnt_ge, (size_t)md + 2, "degree table"));
        STEP(ctx->alloc(&edges_ge, (size_t)md + 2, "degree table"));
        k_cnt_ge<<<grid_for(ctx, std::max<int64_t>(nl, 1)), 256, 0, ctx->stream>>>(degnew + base, nl, md, cnt_ge);
        k_edges_ge<<<grid_for(ctx, md + 2), 256, 0, ctx->stream>>>(cnt_ge, md, g.off, base, edges_ge);
        ABC_CU(cudaMemcpyAsync(cg.data(), cnt_ge, sizeof(int64_t) * (md + 2), cudaMemcpyDeviceToHost, ctx->stream));
        ABC_CU(cudaMemcpyAsync(eg.data(), edges_ge, sizeof(int64_t) * (md + 2), cudaMemcpyDeviceToHost, ctx->stream));
        ABC_CU(cudaStreamSynchronize(ctx->stream));
        ctx->release(cnt_ge);
        ctx->release(edges_ge);
    }
    ABC_CU(cudaGetLastError());
    ctx->release(deg); ctx->release(degnew); ctx->release(d_err); ctx->release(d_max);
    ctx->release(ka); ctx->release(kb); ctx->release(rk);
    g.nU = nU;
    g.nV = nV;
    g.m = m;
    g.loaded = true;
    return ABCORE_OK;

fail:
    cudaStreamSynchronize(ctx->stream);
    ctx->release(deg); ctx->release(degnew); ctx->release(d_err); ctx->release(d_max);
    ctx->release(ka); ctx->release(kb); ctx->release(rk); ctx->release(cnt_ge); ctx->release(edges_ge);
    free_graph_of(ctx, g);
    return rc;
#undef STEP
}
