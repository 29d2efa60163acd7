// Device throughput probe for random 32-bit atomics: the rate that bounds a cascade whose counts
// sit in L2. Random indices come from the lowbias32 integer hash (a public-domain finisher by
// C. Wellons) of the thread's element number.
#include <algorithm>

#include "internal.h"

namespace {

__device__ __forceinline__ unsigned hash32(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void k_atomics_ret(int *a, unsigned mask, long long n, int *sink) {
    int acc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += atomicSub(&a[hash32((unsigned)i) & mask], 1);
    if (acc == 0x7fffffff) *sink = acc;  // keeps the returned values live
}

__global__ void k_atomics_noret(int *a, unsigned mask, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        atomicSub(&a[hash32((unsigned)i) & mask], 1);
}

}  // namespace

int measure_atomics(abcore_ctx *ctx, int64_t array_bytes, double *with_return, double *without_return) {
    int bits = 10;
    while (bits < 30 && ((int64_t)4 << (bits + 1)) <= array_bytes) ++bits;  // 2^bits ints fit
    const unsigned mask = (1u << bits) - 1;
    int *a = nullptr, *sink = nullptr;
    ABC_TRY(ctx->alloc(&a, (size_t)1 << bits, "atomic probe array"));
    int rc = ctx->alloc(&sink, 1, "atomic probe sink");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = ctx->fail(ABCORE_ECUDA, "atomic probe: events");
    const long long n = 1LL << 26;
    const unsigned grid = (unsigned)ctx->num_sms * 8;
    float best[2] = {1e30f, 1e30f};
    for (int rep = 0; rep < 4 && !rc; ++rep) {
        cudaMemsetAsync(a, 0, sizeof(int) << bits, ctx->stream);
        for (int kind = 0; kind < 2; ++kind) {
            cudaEventRecord(e0, ctx->stream);
            if (kind == 0) k_atomics_ret<<<grid, 256, 0, ctx->stream>>>(a, mask, n, sink);
            else k_atomics_noret<<<grid, 256, 0, ctx->stream>>>(a, mask, n);
            cudaEventRecord(e1, ctx->stream);
            const cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = ctx->cuda_fail(e, "atomic probe");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best[kind] = std::min(best[kind], ms);  // the first round warms up
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ctx->release(a);
    ctx->release(sink);
    if (!rc) {
        *with_return = (double)n / (best[0] * 1e-3);
        *without_return = (double)n / (best[1] * 1e-3);
    }
    return rc;
}
