// Device helpers for sorted-set work on degree-ranked adjacency lists.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pg_internal.h"

#define PG_FULL 0xffffffffu

struct Slice {
    const int *p;
    int len;
    int owner; // vertex whose adjacency list this is, -1 for scratch
};

__device__ __forceinline__ const int *adj_of(const DevGraph &g, int4 vi) {
    return g.adj + ((size_t)(unsigned)vi.x << 2);
}

// first index i in a[0, len) with a[i] >= x
__device__ __forceinline__ int lower_bound_g(const int *__restrict__ a, int len, int x) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool contains_g(const int *__restrict__ a, int len, int x) {
    // branch-reduced search: halve while len > 1
    const int *base = a;
    int n = len;
    if (n <= 0) return false;
    while (n > 1) {
        const int half = n >> 1;
        base = (__ldg(base + half - 1) < x) ? base + half : base;
        n -= half;
    }
    return __ldg(base) == x;
}

// Same searches on scratch written earlier in this kernel (coherent loads,
// never the read-only path).
__device__ __forceinline__ int lower_bound_s(const int *a, int len, int x) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool contains_s(const int *a, int len, int x) {
    const int i = lower_bound_s(a, len, x);
    return i < len && a[i] == x;
}

// Restrict a sorted list to values in the open interval (lo, hi).
__device__ __forceinline__ Slice bound_slice(const int *p, int len, int lo, int hi, int owner = -1) {
    const int b = lo < 0 ? 0 : lower_bound_g(p, len, lo + 1);
    const int e = hi == 0x7fffffff ? len : lower_bound_g(p, len, hi);
    Slice s;
    s.p = p + b;
    s.len = e > b ? e - b : 0;
    s.owner = owner;
    return s;
}

// x in the slice, for x known to lie inside the slice's value bounds: a bit
// test when the slice belongs to a hub, else a binary search.
__device__ __forceinline__ bool in_slice(const DevGraph &g, const Slice &s, int x) {
    if (s.owner >= 0 && s.owner < g.n_hubs)
        return (__ldg(g.hubbits + (size_t)s.owner * g.hub_stride + (x >> 5)) >> (x & 31)) & 1u;
    return contains_g(s.p, s.len, x);
}

// 128-bit exact accumulation into two 64-bit words (low, high).
__device__ __forceinline__ void atomic_add_u128(unsigned long long *c, unsigned __int128 x) {
    const unsigned long long lo = (unsigned long long)x;
    unsigned long long hi = (unsigned long long)(x >> 64);
    if (lo) {
        const unsigned long long old = atomicAdd(c, lo);
        if (old + lo < old) hi += 1;
    }
    if (hi) atomicAdd(c + 1, hi);
}

// C(s, g) exactly, g <= 8, in 128 bits.
__device__ __forceinline__ unsigned __int128 choose_u128(unsigned long long s, int g) {
    if (g == 1) return s;
    if ((long long)s < g) return 0;
    unsigned __int128 r = 1;
    for (int i = 0; i < g; ++i) r = r * (unsigned __int128)(s - i) / (unsigned __int128)(i + 1);
    return r;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(PG_FULL, x, o);
    return x;
}

// Exact warp sum of 64-bit lane values as a 128-bit integer (every lane
// gets the total).
__device__ __forceinline__ unsigned __int128 warp_sum_u128(unsigned long long x) {
    unsigned long long lo = x, hi = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l2 = __shfl_xor_sync(PG_FULL, lo, o), h2 = __shfl_xor_sync(PG_FULL, hi, o);
        const unsigned long long s = lo + l2;
        hi += h2 + (s < lo ? 1ull : 0ull);
        lo = s;
    }
    return ((unsigned __int128)hi << 64) | lo;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Run control (PgRunCtl).  ctl_begin: the first warp of the launch to call
// it stores the launch's start time; call from one lane.  ctl_poll: true
// when the launch must stop; raises the stop and timed-out flags when the
// budget has run out.  Call from one lane and broadcast the answer.
__device__ __forceinline__ void ctl_begin(const PgRunCtl &c) {
    if (c.words && c.budget_ns) atomicCAS(c.words + 2, 0ull, globaltimer_ns());
}

__device__ __forceinline__ bool ctl_poll(const PgRunCtl &c) {
    if (!c.words) return false;
    if (*(volatile unsigned long long *)c.words) return true;
    if (c.budget_ns && globaltimer_ns() - *(volatile unsigned long long *)(c.words + 2) > c.budget_ns) {
        atomicExch(c.words + 1, 1ull);
        atomicExch(c.words, 1ull);
        return true;
    }
    return false;
}

// Warp-uniform stop decision (lane 0 polls).
__device__ __forceinline__ bool ctl_stop(const PgRunCtl &c, int lane) {
    int f = 0;
    if (lane == 0) f = ctl_poll(c) ? 1 : 0;
    return __shfl_sync(PG_FULL, f, 0) != 0;
}

// Existence mode: add a warp's 128-bit partial count to the launch total
// (counts, (low, high)) and raise the stop flag once the total reaches the
// target.  Call from one lane.
__device__ __forceinline__ void ctl_publish(const PgRunCtl &c, unsigned long long *counts, unsigned __int128 x) {
    if (!x) return;
    atomic_add_u128(counts, x);
    // high word first: a torn read can only under-estimate
    const unsigned long long hi = *(volatile unsigned long long *)(counts + 1);
    const unsigned long long lo = *(volatile unsigned long long *)counts;
    if (hi || lo >= c.target) atomicExch(c.words, 1ull);
}
