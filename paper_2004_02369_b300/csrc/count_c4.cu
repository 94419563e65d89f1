// Edge-induced 4-cycles by co-degree accumulation.
//
// The 4-cycle's exploration plan (Section 4.1) binds a path of three core
// vertices and completes the fourth, non-core vertex by a set intersection
// per matched path (Section 5.1).  On a GPU that is one intersection of two
// adjacency lists per out-neighbour pair of the start vertex, which is the
// dominant term of 4-vertex motif counting (Section 6, non-core completion
// dominating the time).  This kernel counts the same number with the
// non-core completion done by cardinality over a whole neighbourhood at once:
//
//   every 4-cycle has a unique vertex w of smallest degree rank (highest
//   degree, Section 5.2 order); its opposite vertex x and its two cycle
//   neighbours a, b all rank after w.  With c_w(x) = |{a in adj(w) : a > w,
//   x in adj(a), x > w}| (x != a, b holds since the graph has no loops), the
//   cycles anchored at w are sum over x of C(c_w(x), 2).
//
// Raising c_w(x) from k to k+1 adds k new pairs, so the count is the sum of
// the counters' old values over all increments, and no pass over the
// counters is needed.  The increments of w are the suffixes of adj(a) above
// w for a in adj(w) above w; their total T_w is bounded by sum over a of
// deg(a) * out-degree(a) (the Chiba-Nishizeki bound), so hubs are anchors of
// few cycles' worth of work each.
//
// B300 mapping (two persistent launches):
//  * light pass (4-warp CTAs): anchors one per warp in rank order; counters
//    live in a per-warp open-addressing hash table in shared memory sized
//    for T_w.  An anchor of degree above kLightDeg, or with more than kLightT
//    increments, is appended to a deferred list instead;
//  * tiled pass (16-warp CTAs, two per SM): deferred anchors one per CTA.
//    The counters of x in (w, n) are kept in shared memory one x-range tile
//    at a time (96 KB: 49,152 16-bit counters when the anchor has fewer than
//    2^16 neighbours above it, else 24,576 32-bit ones); each tile takes,
//    from every neighbour's suffix, the elements inside the tile (a per
//    neighbour cursor in global memory, advanced by a galloping search), so
//    every suffix element is read once and every increment is a shared-memory
//    atomic; the tile is cleared before the next.  No counter lives in
//    global memory.
//  Both walk the suffixes 32 neighbours a at a time: lanes search their a's
//  suffix start, a warp prefix sum flattens the 32 suffixes, and lanes read
//  the flattened increments with coalesced loads.
#include <mutex>

#include "device_sets.cuh"

namespace {

constexpr int kWarps = 4;
constexpr int kBlock = kWarps * 32;   // light pass
constexpr int kTileBlock = 512;       // tiled pass
constexpr int kTileWords = 24576;     // 96 KB of counters per tiled CTA
constexpr size_t kTileSmem = (size_t)kTileWords * sizeof(unsigned);
constexpr int kLightDeg = 256;        // light anchors: degree <= kLightDeg
constexpr int kHashCap = 1024;        // per-warp hash slots (power of two)
constexpr int kLightT = kHashCap / 2; // light anchors: at most this many increments
constexpr int kEmpty = -1;

struct C4Args {
    DevGraph g;
    int n;
    unsigned *cursors;      // per tiled CTA: cur_stride suffix cursors (absolute adj indices)
    long long cur_stride;
    int *deferred;          // anchors left to the CTAs
    unsigned long long *q;  // [0] warp cursor, [1] deferred count, [2] deferred cursor
    unsigned long long *count; // (low, high)
    long long stride, offset; // anchor selection: offset, offset + stride, ... (samples, partition)
    PgRunCtl ctl;
};

// Per-warp shared memory of the light path.
struct WarpSmem {
    int keys[kHashCap];
    unsigned vals[kHashCap];
    unsigned start[kLightDeg]; // suffix start in adj(a) (absolute adj index)
    int len[kLightDeg];        // suffix length
};

__device__ __forceinline__ int upper_bound_g(const int *__restrict__ a, int len, int x) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(a + mid) <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Suffix of adj(a) above w (lane-local): absolute start index and length.
__device__ __forceinline__ void suffix_of(const DevGraph &g, int a, int w, unsigned *start, int *len) {
    const int4 ai = __ldg(&g.vinfo[a]);
    const int *aa = adj_of(g, ai);
    const int q = upper_bound_g(aa, ai.y, w);
    *start = ((unsigned)ai.x << 2) + (unsigned)q;
    *len = ai.y - q;
}

// Walks the flattened suffixes of a chunk of up to 32 neighbours (lane j
// holds neighbour j's suffix start and length) and calls f(x) for every
// element, lanes reading consecutive elements.
template <class F>
__device__ __forceinline__ void walk_chunk(const DevGraph &g, unsigned my_start, int my_len, int lane, F &&f) {
    int incl = my_len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(PG_FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(PG_FULL, incl, 31);
    const int excl = incl - my_len;
    for (int base = 0; base < total; base += 32) {
        const int e = base + lane;
        // owner: the last lane j with excl_j <= e (binary search over lanes)
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int ex = __shfl_sync(PG_FULL, excl, lo + step);
            if (ex <= e) lo += step;
        }
        const unsigned st = __shfl_sync(PG_FULL, my_start, lo);
        const int ex = __shfl_sync(PG_FULL, excl, lo);
        if (e < total) f(__ldg(g.adj + (size_t)st + (unsigned)(e - ex)));
    }
}

// First index i in [p, end) with adj[i] >= v (end if none), galloping from
// p: cheap when few elements precede v.
__device__ __forceinline__ unsigned gallop_lb(const int *__restrict__ adj, unsigned p, unsigned end, int v) {
    if (p >= end || __ldg(adj + p) >= v) return p;
    unsigned lo = p, step = 1, hi = p + 1; // adj[lo] < v
    while (hi < end && __ldg(adj + hi) < v) {
        lo = hi;
        step <<= 1;
        hi = lo + step;
    }
    if (hi > end) hi = end; // the answer lies in (lo, hi]
    ++lo;
    while (lo < hi) {
        const unsigned mid = (lo + hi) >> 1;
        if (__ldg(adj + mid) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Heavy anchor w by the whole CTA, x-range tile by x-range tile, on the
// shared counters T; cur: this CTA's cursors.  Returns this thread's share
// of the anchored count; stops early (partial) when the run control says so
// (*s_stop set).
__device__ unsigned long long tiled_anchor(const C4Args &a, int w, unsigned *T, unsigned *cur, int *s_next,
                                           int *s_p, int *s_stop) {
    const DevGraph &g = a.g;
    const int lane = threadIdx.x & 31;
    const int4 wi = __ldg(&g.vinfo[w]);
    const int *aw = adj_of(g, wi);
    if (threadIdx.x == 0) {
        *s_p = upper_bound_g(aw, wi.y, w);
        *s_next = 0;
    }
    __syncthreads();
    const int p = *s_p, na = wi.y - p;
    if (na < 2) return 0; // uniform across the CTA
    const bool packed = na < 65536; // a counter never exceeds na
    const int R = packed ? 2 * kTileWords : kTileWords;
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
        const int4 ai = __ldg(&g.vinfo[__ldg(aw + p + i)]);
        cur[i] = ((unsigned)ai.x << 2) + (unsigned)upper_bound_g(adj_of(g, ai), ai.y, w);
    }
    for (int i = threadIdx.x; i < kTileWords; i += blockDim.x) T[i] = 0u;
    __syncthreads();
    unsigned long long cnt = 0;
    for (long long t0 = (long long)w + 1; t0 < a.n; t0 += R) {
        const int lo = (int)t0;
        const int hi = (int)min((long long)a.n, t0 + R);
        for (;;) {
            int c = 0;
            if (lane == 0) c = atomicAdd(s_next, 32);
            c = __shfl_sync(PG_FULL, c, 0);
            if (c >= na) break;
            unsigned st = 0;
            int ln = 0;
            if (c + lane < na) {
                const int4 ai = __ldg(&g.vinfo[__ldg(aw + p + c + lane)]);
                st = cur[c + lane];
                const unsigned e = gallop_lb(g.adj, st, ((unsigned)ai.x << 2) + (unsigned)ai.y, hi);
                ln = (int)(e - st);
                cur[c + lane] = e;
            }
            // every element lies in [lo, hi): the previous tile ended at lo
            if (packed)
                walk_chunk(g, st, ln, lane, [&](int x) {
                    const unsigned i = (unsigned)(x - lo), sh = (i & 1u) << 4;
                    cnt += (atomicAdd(T + (i >> 1), 1u << sh) >> sh) & 0xFFFFu;
                });
            else
                walk_chunk(g, st, ln, lane, [&](int x) { cnt += atomicAdd(T + (x - lo), 1u); });
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *s_next = 0;
            *s_stop = a.ctl.words && ctl_poll(a.ctl) ? 1 : 0;
        }
        if (hi < a.n)
            for (int i = threadIdx.x; i < kTileWords; i += blockDim.x) T[i] = 0u;
        __syncthreads();
        if (*s_stop) break;
    }
    return cnt;
}

__device__ __forceinline__ unsigned hash_inc(int *keys, unsigned *vals, unsigned mask, int x) {
    unsigned s = ((unsigned)x * 0x9E3779B1u) >> 7;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        s &= mask;
        const int k = keys[s];
        if (k == x) return atomicAdd(vals + s, 1u);
        if (k == kEmpty) {
            const int prev = atomicCAS(keys + s, kEmpty, x);
            if (prev == kEmpty || prev == x) return atomicAdd(vals + s, 1u);
        }
        ++s;
    }
    return 0u; // unreachable: the table is sized at twice the increments
}

// Light anchor w by one warp with a shared-memory hash table.  Returns
// false (nothing counted) when its degree exceeds kLightDeg or its
// increments exceed kLightT.
__device__ bool light_anchor(const C4Args &a, int w, WarpSmem &sm, int lane, unsigned long long &cnt) {
    const DevGraph &g = a.g;
    const int4 wi = __ldg(&g.vinfo[w]);
    if (wi.y > kLightDeg) return false;
    const int *aw = adj_of(g, wi);
    int p = 0;
    if (lane == 0) p = upper_bound_g(aw, wi.y, w);
    p = __shfl_sync(PG_FULL, p, 0);
    const int na = wi.y - p;
    if (na < 2) return true;
    int total = 0;
    for (int c = lane; c < na; c += 32) {
        unsigned st;
        int ln;
        suffix_of(g, __ldg(aw + p + c), w, &st, &ln);
        sm.start[c] = st;
        sm.len[c] = ln;
        total += ln;
    }
    total = __reduce_add_sync(PG_FULL, total);
    if (total > kLightT) return false;
    if (total < 2) return true;
    unsigned cap = 64;
    while (cap < 2u * (unsigned)total) cap <<= 1;
    for (unsigned i = lane; i < cap; i += 32) {
        sm.keys[i] = kEmpty;
        sm.vals[i] = 0u;
    }
    __syncwarp();
    const unsigned mask = cap - 1;
    for (int c = 0; c < na; c += 32) {
        unsigned st = 0;
        int ln = 0;
        if (c + lane < na) {
            st = sm.start[c + lane];
            ln = sm.len[c + lane];
        }
        walk_chunk(g, st, ln, lane, [&](int x) { cnt += hash_inc(sm.keys, sm.vals, mask, x); });
    }
    __syncwarp();
    return true;
}

// Light pass: one warp per anchor, rank order; heavy anchors deferred.
__global__ void __launch_bounds__(kBlock) k_c4_light(C4Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const bool polled = a.ctl.words != nullptr;
    if (polled && lane == 0) ctl_begin(a.ctl);
    unsigned long long cnt = 0;
    WarpSmem &sm = ((WarpSmem *)smem_raw)[warp];
    const long long n_tasks = a.n > a.offset ? ((long long)a.n - a.offset + a.stride - 1) / a.stride : 0;
    for (;;) {
        if (polled && ctl_stop(a.ctl, lane)) break;
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.q, 1ull);
        t = __shfl_sync(PG_FULL, t, 0);
        if ((long long)t >= n_tasks) break;
        const int w = (int)((unsigned long long)a.offset + t * (unsigned long long)a.stride);
        if (!light_anchor(a, w, sm, lane, cnt) && lane == 0) a.deferred[atomicAdd(a.q + 1, 1ull)] = w;
    }
    const unsigned __int128 tot = warp_sum_u128(cnt);
    if (lane == 0 && tot) atomic_add_u128(a.count, tot);
}

// Tiled pass: one CTA per deferred anchor, counters in shared memory.
__global__ void __launch_bounds__(kTileBlock) k_c4_tiled(C4Args a) {
    extern __shared__ __align__(16) unsigned tile[];
    __shared__ int s_task, s_next, s_p, s_stop;
    const int lane = threadIdx.x & 31;
    const bool polled = a.ctl.words != nullptr;
    if (polled && threadIdx.x == 0) ctl_begin(a.ctl);
    unsigned long long cnt = 0;
    unsigned *cur = a.cursors + (size_t)blockIdx.x * (size_t)a.cur_stride;
    const unsigned long long n_def = *(volatile unsigned long long *)(a.q + 1);
    for (;;) {
        if (threadIdx.x == 0) {
            int w = -1;
            if (!polled || !ctl_poll(a.ctl)) {
                const unsigned long long t = atomicAdd(a.q + 2, 1ull);
                if (t < n_def) w = a.deferred[t];
            }
            s_task = w;
            s_stop = 0;
        }
        __syncthreads();
        const int w = s_task;
        __syncthreads();
        if (w < 0) break;
        cnt += tiled_anchor(a, w, tile, cur, &s_next, &s_p, &s_stop);
        if (s_stop) break;
    }
    const unsigned __int128 tot = warp_sum_u128(cnt);
    if (lane == 0 && tot) atomic_add_u128(a.count, tot);
}

constexpr size_t kLightSmem = (size_t)kWarps * sizeof(WarpSmem);

// Grids per device, computed once (the shared-memory attribute is a
// per-device setting): launches then only enqueue work, as stream capture
// requires.
constexpr int kMaxDevices = 64;
std::once_flag g_once[kMaxDevices];
cudaError_t g_err[kMaxDevices];
int g_light_per_sm[kMaxDevices], g_tiled_per_sm[kMaxDevices];

int c4_grids(const pg_graph *g, int *light, int *tiled) {
    const int dev = g->device;
    if (dev < 0 || dev >= kMaxDevices) return pg_set_error(PG_EINVAL, "device index out of range");
    std::call_once(g_once[dev], [dev] {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaError_t e = cudaSetDevice(dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_c4_light, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLightSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_light_per_sm[dev], k_c4_light, kBlock, kLightSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_c4_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_tiled_per_sm[dev], k_c4_tiled, kTileBlock, kTileSmem);
        cudaSetDevice(prev);
        g_err[dev] = e;
    });
    if (g_err[dev] != cudaSuccess) return pg_cuda_error(g_err[dev], "4-cycle kernel set-up");
    *light = std::max(1, g_light_per_sm[dev]) * g->num_sms;
    *tiled = std::max(1, g_tiled_per_sm[dev]) * g->num_sms;
    return PG_OK;
}

}  // namespace

size_t pg_c4_scratch_bytes(const pg_graph *g) {
    int light = 0, tiled = 0;
    if (c4_grids(g, &light, &tiled) != PG_OK) tiled = 2 * g->num_sms;
    const size_t cur = (size_t)tiled * (size_t)((g->max_deg + 31) & ~31ll) * sizeof(unsigned);
    return cur + (size_t)(g->n + 1) * sizeof(int) + 256;
}

// Adds the number of edge-induced 4-cycles of g into count_dev (128-bit,
// low / high).  Uses the graph's scratch arena (pg_c4_scratch_bytes) and
// queue words queue_slot .. queue_slot + 3.
int pg_launch_c4(pg_graph *g, unsigned long long *count_dev, int queue_slot, cudaStream_t s, const PgRunCtl *ctl) {
    if (g->n < 4) return PG_OK;
    if (queue_slot + 3 > PG_CTL_WORDS_SLOT) return pg_set_error(PG_EINVAL, "queue slot out of range");
    if (g->adj_entries >= (1ll << 32)) return pg_set_error(PG_EUNSUPPORTED, "4-cycle kernel: adjacency above 2^32 entries");
    int light = 0, tiled = 0;
    int rc = c4_grids(g, &light, &tiled);
    if (rc) return rc;
    if (pg_c4_scratch_bytes(g) > g->ex->scratch_bytes) return pg_set_error(PG_ENOMEM, "scratch smaller than the 4-cycle kernel needs");
    C4Args a;
    a.g = g->d;
    a.n = (int)g->n;
    a.cur_stride = (g->max_deg + 31) & ~31ll;
    a.cursors = (unsigned *)g->ex->scratch;
    a.deferred = (int *)((unsigned char *)g->ex->scratch + (size_t)tiled * (size_t)a.cur_stride * sizeof(unsigned));
    a.q = g->ex->queues + queue_slot;
    a.count = count_dev;
    const PgTaskSel sel = pg_task_sel(g);
    a.stride = sel.stride;
    a.offset = sel.offset;
    a.ctl = ctl ? *ctl : PgRunCtl{};
    PG_CUDA(cudaMemsetAsync(a.q, 0, 3 * sizeof(unsigned long long), s));
    k_c4_light<<<light, kBlock, kLightSmem, s>>>(a);
    PG_CUDA(cudaGetLastError());
    k_c4_tiled<<<tiled, kTileBlock, kTileSmem, s>>>(a);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}
