// Device-side helpers shared by the library's kernels: warp primitives, memory-order loads and
// stores, and the bounded-wait clock. Every spin in this library reads globaltimer and gives
// up after a limit, recording ABCORE_ETIMEDOUT instead of hanging the GPU.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define ABC_FULL 0xffffffffu

namespace abc {

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Programmatic dependent launch. A kernel launched with programmatic stream serialization may be
// scheduled while the kernel before it on the stream is still running; grid_dep_wait blocks until
// that grid has completed and its memory operations are visible, so a kernel calls it before it
// touches global memory. grid_dep_launch lets the next such kernel start launching blocks (they
// then wait in grid_dep_wait). Both do nothing for a normally serialized launch.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_i32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Inclusive warp scan of a 32-bit value.
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int t = __shfl_up_sync(ABC_FULL, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__device__ __forceinline__ long long warp_incl_scan64(long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long t = __shfl_up_sync(ABC_FULL, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(ABC_FULL, v, d);
    return v;
}

// Block-collective: add every thread's v[i] to *dst[i], with one global atomic per counter per
// block. A launch's thousands of warps finishing at once would otherwise queue on the same few
// words (same-address atomics are served one at a time).
template <int N>
__device__ __forceinline__ void block_add(const unsigned long long (&v)[N], unsigned long long *const (&dst)[N]) {
    __shared__ unsigned long long s_acc[N];
    if (threadIdx.x < N) s_acc[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const unsigned long long x = (unsigned long long)warp_sum64((long long)v[i]);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_acc[i], x);
    }
    __syncthreads();
    if (threadIdx.x < N && s_acc[threadIdx.x]) atomicAdd(dst[threadIdx.x], s_acc[threadIdx.x]);
}

// Record the first error code seen by any thread (0 = none).
__device__ __forceinline__ void set_error(int *err, int code) { atomicCAS(err, 0, code); }

}  // namespace abc
