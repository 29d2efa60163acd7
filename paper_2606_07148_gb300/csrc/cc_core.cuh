// Union-find on the device for connected components (the component labels GFQ keeps, Section 5).
//
// parent[x] <= x always: a union hooks the larger of two roots under the smaller with one
// atomicCAS, so every tree's root is the smallest id in it and a parent pointer only ever moves
// to an ancestor. find() halves paths as it goes; a racing halving store can only replace one
// ancestor by another, so every pointer stays valid without locks.
#pragma once

#include <cstdint>

namespace abc {

__device__ __forceinline__ int32_t cc_find(int32_t *parent, int32_t x) {
    for (;;) {
        const int32_t p = __ldcg(&parent[x]);
        if (p == x) return x;
        const int32_t gp = __ldcg(&parent[p]);
        if (gp == p) return p;
        parent[x] = gp;  // path halving
        x = gp;
    }
}

__device__ __forceinline__ void cc_unite(int32_t *parent, int32_t a, int32_t b) {
    for (;;) {
        a = cc_find(parent, a);
        b = cc_find(parent, b);
        if (a == b) return;
        const int32_t lo = a < b ? a : b, hi = a < b ? b : a;
        if (atomicCAS(&parent[hi], hi, lo) == hi) return;
        // hi was hooked by someone else meanwhile: retry from the new roots
    }
}

}  // namespace abc
