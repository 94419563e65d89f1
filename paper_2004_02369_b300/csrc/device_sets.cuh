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

// Four membership tests against one slice at once (x[j] in the slice,
// ANDed into ok[j], negated for set differences).  The four branch-free
// binary searches run over the same length, so each step issues four
// independent loads: four times the memory-level parallelism of one search
// per lane.  Hub slices answer from their membership bitmap for the keys
// still in play (ok[j]); the searches' loads stay inside the slice whatever
// the keys are.
__device__ __forceinline__ void in_slice4(const DevGraph &g, const Slice &s, const int (&x)[4], bool (&ok)[4],
                                          bool negate) {
    bool f[4];
    if (s.owner >= 0 && s.owner < g.n_hubs) {
        const unsigned *row = g.hubbits + (size_t)s.owner * g.hub_stride;
        // only keys still in play are looked up: the others may be padding
#pragma unroll
        for (int j = 0; j < 4; ++j) f[j] = ok[j] && ((__ldg(row + ((unsigned)x[j] >> 5)) >> (x[j] & 31)) & 1u);
    } else if (s.len <= 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) f[j] = false;
    } else {
        const int *p = s.p;
        int b0 = 0, b1 = 0, b2 = 0, b3 = 0;
        int n = s.len;
        while (n > 1) {
            const int half = n >> 1;
            const int v0 = __ldg(p + b0 + half - 1), v1 = __ldg(p + b1 + half - 1), v2 = __ldg(p + b2 + half - 1),
                      v3 = __ldg(p + b3 + half - 1);
            b0 += v0 < x[0] ? half : 0;
            b1 += v1 < x[1] ? half : 0;
            b2 += v2 < x[2] ? half : 0;
            b3 += v3 < x[3] ? half : 0;
            n -= half;
        }
        f[0] = __ldg(p + b0) == x[0];
        f[1] = __ldg(p + b1) == x[1];
        f[2] = __ldg(p + b2) == x[2];
        f[3] = __ldg(p + b3) == x[3];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) ok[j] = ok[j] && (f[j] != negate);
}

// Four lower bounds at once: pos[j] = first index i of a[0, len) with
// a[i] >= x[j] (len for none).  Branch-free searches over the same length,
// so each step issues four independent loads.  RO: read-only path (lists);
// else coherent loads (scratch written earlier by this warp).  Every load
// stays inside a[0, len).
template <bool RO>
__device__ __forceinline__ void lower_bound4(const int *a, int len, const int (&x)[4], int (&pos)[4]) {
    if (len <= 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) pos[j] = 0;
        return;
    }
    int b[4] = {0, 0, 0, 0};
    int n = len;
    while (n > 1) {
        const int half = n >> 1;
        int v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = RO ? __ldg(a + b[j] + half - 1) : a[b[j] + half - 1];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] += v[j] < x[j] ? half : 0;
        n -= half;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) pos[j] = b[j] + ((RO ? __ldg(a + b[j]) : a[b[j]]) < x[j] ? 1 : 0);
}

// The driver slice d of a level, read four elements per lane with one
// aligned 16-byte load: lists start 16-byte aligned and are padded to 4
// entries, so the groups covering d stay inside its list.  Group g of a
// warp step holds elements d.p[-off + 4 * (base/4 + lane) + j].
struct Driver4 {
    const int4 *v;
    int off, total; // elements before d.p in its group; off + d.len
};

__device__ __forceinline__ Driver4 driver4(const Slice &d) {
    Driver4 r;
    r.off = (int)(((uintptr_t)d.p >> 2) & 3u);
    r.v = (const int4 *)(d.p - r.off);
    r.total = d.len + r.off;
    return r;
}

// Lane's four elements at warp step `base` (a multiple of 128) and which of
// them lie inside the slice.
__device__ __forceinline__ void driver4_load(const Driver4 &dv, int base, int lane, int (&x)[4], bool (&ok)[4]) {
    const int q = base + 4 * lane;
    int4 t = make_int4(0x7fffffff, 0x7fffffff, 0x7fffffff, 0x7fffffff);
    if (q < dv.total) t = __ldg(dv.v + (q >> 2));
    x[0] = t.x;
    x[1] = t.y;
    x[2] = t.z;
    x[3] = t.w;
#pragma unroll
    for (int j = 0; j < 4; ++j) ok[j] = q + j >= dv.off && q + j < dv.total;
}

// Warp-wide exclusive prefix of c (lane order); *total gets the sum.
__device__ __forceinline__ int warp_excl_scan(int c, int lane, int *total) {
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(PG_FULL, incl, o);
        if (lane >= o) incl += y;
    }
    *total = __shfl_sync(PG_FULL, incl, 31);
    return incl - c;
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
