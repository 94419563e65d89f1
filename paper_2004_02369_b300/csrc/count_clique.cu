// K2: k-clique counting, persistent, bitmap sub-graph per start vertex.
//
// The k-clique plan (Section 4.1) has a total partial order u1 < ... < uk,
// core {u2..uk} and one counted non-core vertex u1; with the degree ranking
// of Section 5.2 and the high-to-low matching order, the start vertex binds
// uk and every other vertex is drawn from its out-neighbourhood
// N+(v) = adj(v) restricted to smaller ranks.  Every later level intersects
// N+(v) with the out-lists of already bound vertices, restricted by the
// order bounds, and the last level is counted by cardinality (Section 5.1).
//
// B300 mapping.  For a start vertex v with d = |N+(v)| the kernel builds the
// bitmap rows R[i] = { j < i : N+(v)[j] in N+(N+(v)[i]) } (the level-1
// intersections, each out-list read once from L2/HBM) and then runs every
// deeper level as word-wise ANDs of rows; a prefix of p sub-graph vertices
// with candidate set C leaves popc(C) cliques of size p + 2, so one traversal
// counts every clique size kmin..kmax (several clique patterns share one
// launch).
//  * Heavy vertices (d > PG_CLIQUE_LIGHT_D, sorted by d, largest first) are
//    processed by a whole CTA: 8 warps share one tile in shared memory (or a
//    per-CTA global slab when the tile does not fit), take rows from a CTA
//    counter for the row build and the traversal.
//  * Light vertices are processed by single warps on per-warp tiles, taken in
//    rank order (highest degree first, Section 5.2) from a device counter.
//  * Traversal: warp-uniform loops over all levels but the last; the last
//    level is lane-parallel over a compacted candidate list, so every lane
//    does one popcount-of-AND row product per candidate.
//  * Sizes: KMAX = 8 (the tuned variant) or 16 (large cliques, e.g. the
//    14-clique existence query of the paper's evaluation).  A branch whose
//    candidate set is too small to reach kmin is cut (cardinality pruning).
//  * Exact counts: lane counters are 64-bit and are moved into the 128-bit
//    totals after any start vertex that leaves them at 2^62 or more (see
//    bump); the final warp sums are 128-bit.
//  * Run control (PgRunCtl): existence mode publishes counts after every
//    row and stops all warps once the target is reached; a device work
//    budget stops the launch and flags it as timed out.
#include <mutex>

#include "device_sets.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kBlock = kWarps * 32;
constexpr int kLightD = PG_CLIQUE_LIGHT_D;
constexpr int kLightWs = (kLightD / 32) | 1;
// per-warp light tile: list, rows, row start / length / element prefix
constexpr int kLightTile = kLightD + kLightD * kLightWs + 3 * kLightD + 1;
constexpr int kItems = 256; // queued (candidate set, vertex) products per warp
constexpr int kCtl = 8;
constexpr size_t kSmemBudget = 96 * 1024;

struct CliqueArgs {
    DevGraph g;
    int kmin, kmax;
    const int *heavy;
    int n_heavy;
    int n;
    int dpad, hws;           // heavy tile: list entries (padded), row stride in words
    int heavy_in_smem;       // 1: heavy tile in shared memory, else in the CTA slab
    int cws;                 // candidate bitmap stride (words)
    int nslots;              // candidate bitmaps kept per warp between flushes
    int region_words;        // shared union of the heavy tile and the light tiles
    int warp_words;          // per-warp scratch: level bitmaps, slot ring, items
    unsigned *slabs;         // per-CTA global slabs (may be null)
    long long slab_words;
    unsigned long long *queue; // [0] light cursor, [1] heavy cursor
    unsigned long long *counts;
    int chunk;                 // light start vertices per queue grab
    int heavy_min;             // light vertices have out-degree <= heavy_min (<= kLightD)
    int stride;                // task selection: offset, offset + stride, ... (samples, partition)
    int offset;
    long long n_light_tasks;   // selected start vertices
    long long n_heavy_tasks;   // selected entries of the heavy list
    PgRunCtl ctl;              // early termination / work budget (words null: none)
    int plain;                 // extended variant only: 0 persistent; 1 one CTA per heavy start
                               // vertex (blockIdx); 2 one warp per light start vertex (global warp)
};

// cnt[S] = lane counter of (S+3)-cliques.  A lane adds at most 2^16 per
// row product and a product takes at least one issue slot, so a counter
// below 2^62 needs more than 2^63 / 2^16 products (over 19 hours of one
// lane at 2 GHz) to wrap: checking after every start vertex and moving
// counters of 2^62 or more into the 128-bit totals keeps the counts exact.
template <int S>
__device__ __forceinline__ void bump(unsigned long long *cnt, unsigned long long x) {
    cnt[S] += x;
}

// (run-time indexed loops keep the counters in local memory, off the
// register budget of the traversal)
template <int KMAX>
__device__ __forceinline__ void guard_counts(unsigned long long *cnt, const CliqueArgs &a) {
#pragma unroll 1
    for (int s = 0; s < KMAX; ++s)
        if (cnt[s] >> 62) {
            if (s + 3 >= a.kmin && s + 3 <= a.kmax) atomic_add_u128(a.counts + 2 * (s + 3 - a.kmin), cnt[s]);
            cnt[s] = 0;
        }
}

// Sub-graph tile of one start vertex: list = N+(v) (d entries), rows[i] =
// bitmap of j < i adjacent to i, and per-row build bookkeeping.
struct Tile {
    int *list;
    unsigned *rows;
    int ws;
    int *rstart; // list start of N+(list[i]) in 16-byte units
    int *rlen;   // |N+(list[i])|
    int *pre;    // exclusive prefix of per-row work elements (d + 1 entries)
};

// Per-warp traversal scratch.
struct Walker {
    unsigned *cbuf; // KMAX level bitmaps of cws words
    unsigned *ring; // nslots candidate bitmaps
    int *items;     // kItems packed (slot << 16 | l)
    unsigned *bsh;  // 32 re-indexed rows of compressed_row
    int cws, nslots;
    int m;          // queued items
    int used;       // ring slots in use
    int kmin;       // smallest size counted (cardinality pruning)
};

// Run control of the extended variant, copied to shared memory once per CTA
// so the traversal can poll it without carrying it in registers (with the
// count words that existence mode publishes to).
__shared__ PgRunCtl s_run_ctl;
__shared__ unsigned long long *s_counts;

// Existence mode inside a traversal: publish the warp's kmax-clique count so
// far (products still queued are published later), so that the first match
// stops the launch without waiting for the end of its row.  Warp-uniform.
__device__ __forceinline__ void publish_walk(unsigned long long *cnt, int kmax, int lane) {
    const unsigned long long mine = cnt[kmax - 3];
    if (!__any_sync(PG_FULL, mine != 0)) return;
    cnt[kmax - 3] = 0;
    const unsigned __int128 tot = warp_sum_u128(mine);
    if (lane == 0) ctl_publish(s_run_ctl, s_counts, tot);
}

// Group-wide barrier: the CTA for heavy vertices, the warp for light ones.
template <bool CTA>
__device__ __forceinline__ void group_sync() {
    if constexpr (CTA) __syncthreads(); else __syncwarp();
}

// Level-1 intersections of the tile (Section 5.1 candidate sets restricted to
// N+(v)): rows[i] = { j < i : list[j] in N+(list[i]) }.  Work is flattened
// over the group: row i costs |N+(list[i])| lookups of its elements in
// list[0, i) (shared memory) or, when that list is much longer than i, i
// lookups of list[j] in N+(list[i]) (global binary search).
template <bool CTA>
__device__ void build_rows(const DevGraph &g, const Tile &t, int d, int tid, int nthreads,
                           unsigned long long &tri) {
    const int lane = threadIdx.x & 31;
    for (int i = tid; i < d; i += nthreads) {
        const int4 ui = __ldg(&g.vinfo[t.list[i]]);
        t.rstart[i] = ui.x;
        t.rlen[i] = ui.z;
    }
    for (int w = tid; w < d * t.ws; w += nthreads) t.rows[w] = 0u;
    group_sync<CTA>();
    // exclusive prefix of per-row elements (first warp of the group)
    if (tid < 32) {
        int carry = 0;
        for (int base = 0; base < d; base += 32) {
            const int i = base + lane;
            int e = 0;
            if (i > 0 && i < d) {
                const int du = t.rlen[i];
                e = du <= 4 * i + 32 ? du : i;
            }
            int incl = e;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(PG_FULL, incl, o);
                if (lane >= o) incl += y;
            }
            if (i < d) t.pre[i] = carry + incl - e;
            carry += __shfl_sync(PG_FULL, incl, 31);
        }
        if (lane == 0) t.pre[d] = carry;
    }
    group_sync<CTA>();
    const int total = t.pre[d];
    for (int e = tid; e < total; e += nthreads) {
        // row of element e: last i with pre[i] <= e
        int lo = 1, hi = d - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (t.pre[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const int i = lo;
        const int k = e - t.pre[i];
        const int du = t.rlen[i];
        const int *nu = g.adj + ((size_t)(unsigned)t.rstart[i] << 2);
        if (du <= 4 * i + 32) {
            const int x = __ldg(nu + k);
            int a = 0, b = i;
            while (a < b) {
                const int mid = (a + b) >> 1;
                if (t.list[mid] < x) a = mid + 1; else b = mid;
            }
            if (a < i && t.list[a] == x) atomicOr(&t.rows[(size_t)i * t.ws + (a >> 5)], 1u << (a & 31));
        } else if (in_slice(g, Slice{nu, du, t.list[i]}, t.list[k])) {
            atomicOr(&t.rows[(size_t)i * t.ws + (k >> 5)], 1u << (k & 31));
        }
    }
    group_sync<CTA>();
    unsigned long long c = 0;
    for (int w = tid; w < d * t.ws; w += nthreads) c += __popc(t.rows[w]);
    tri += c;
}

// Run the queued products: item (s, l) adds popc(ring[s] & rows[l]).
__device__ __forceinline__ unsigned long long flush(const Tile &t, Walker &wk, int lane) {
    __syncwarp();
    unsigned long long acc = 0;
    for (int e = lane; e < wk.m; e += 32) {
        const int it = wk.items[e];
        const unsigned *C = wk.ring + (size_t)(it >> 16) * wk.cws;
        const int l = it & 0xffff;
        const unsigned *rl = t.rows + (size_t)l * t.ws;
        const int nl = (l + 31) >> 5;
        unsigned s = 0;
        for (int w = 0; w < nl; ++w) s += __popc(C[w] & rl[w]);
        acc += s;
    }
    __syncwarp();
    wk.m = 0;
    return acc;
}

// Queue one product per candidate l of C (bits below `limit`) for the last
// level; the result counts into cnt[P].
template <int P>
__device__ __forceinline__ void emit(const Tile &t, Walker &wk, const unsigned *C, int limit, int lane,
                                     unsigned long long *cnt) {
    const int nw = (limit + 31) >> 5;
    if (wk.used == wk.nslots) {
        bump<P>(cnt, flush(t, wk, lane));
        wk.used = 0;
    }
    const int slot = wk.used++;
    unsigned *S = wk.ring + (size_t)slot * wk.cws;
    for (int w = lane; w < nw; w += 32) S[w] = C[w];
    __syncwarp();
    for (int w = 0; w < nw; ++w) {
        const unsigned x = S[w];
        const int c = __popc(x);
        if (wk.m + c > kItems) bump<P>(cnt, flush(t, wk, lane));
        if ((x >> lane) & 1u) wk.items[wk.m + __popc(x & ((1u << lane) - 1))] = (slot << 16) | (w * 32 + lane);
        wk.m += c;
    }
}

// Candidate set C after a prefix of P sub-graph vertices (bits below
// `limit`): popc(C) has been counted as (P + 2)-cliques by the caller; count
// every larger size up to kmax.  All levels but the last are warp-uniform
// loops; the last level is queued as lane-parallel products.  A candidate
// whose extension N has fewer than kmin - P - 2 bits cannot lie in a
// kmin-clique, and neither can any branch below it: skipped.
template <int P, int KMAX, bool XT>
__device__ void walk(const Tile &t, Walker &wk, const unsigned *C, int limit, int kmax, int lane,
                     unsigned long long *cnt) {
    if constexpr (P >= KMAX - 2) {
        return;
    } else {
        if (P + 3 > kmax) return;
        if (P + 3 == kmax) {
            emit<P>(t, wk, C, limit, lane, cnt);
            return;
        }
        const bool prune = XT && wk.kmin > P + 3;
        const int nw = (limit + 31) >> 5;
        unsigned *N = wk.cbuf + (size_t)P * wk.cws;
        for (int w = 0; w < nw; ++w) {
            unsigned x = C[w];
            while (x) {
                if constexpr (XT && P <= 2) {
                    // long traversals (large k in dense regions) stop soon
                    // after the launch's stop flag or work budget says so
                    if (s_run_ctl.words) {
                        if (s_run_ctl.target) publish_walk(cnt, kmax, lane);
                        if (ctl_stop(s_run_ctl, lane)) return;
                    }
                }
                const int l = w * 32 + __ffs(x) - 1;
                x &= x - 1;
                const unsigned *rl = t.rows + (size_t)l * t.ws;
                const int nl = (l + 31) >> 5;
                unsigned c = 0;
                for (int v = lane; v < nl; v += 32) {
                    const unsigned y = C[v] & rl[v];
                    N[v] = y;
                    c += __popc(y);
                }
                bump<P>(cnt, c);
                __syncwarp();
                if (!prune || (int)__reduce_add_sync(PG_FULL, c) >= wk.kmin - P - 2)
                    walk<P + 1, KMAX, XT>(t, wk, N, l, kmax, lane, cnt);
                __syncwarp();
            }
        }
    }
}

// Rows with at most 32 bits: re-index the sub-graph induced on R_i (the
// common out-neighbours of v and list[i]) onto those bits, so that every
// candidate set of the deeper levels is one 32-bit word.  Lane a holds
// B_a = {b < a : p_b in R_{p_a}} for the a-th set bit p_a of R_i:
//   4-cliques through (v, list[i]):  sum_a popc(B_a)
//   5-cliques:  sum_a sum_{b in B_a} popc(B_a & B_b)
//   6-cliques:  sum_a sum_{b in B_a} sum_{q in B_a & B_b} popc(B_a & B_b & B_q)
// Returns false (nothing counted) when R_i has more than 32 bits.
// Position of the set bit of x with k set bits below it (0 <= k < popc(x)):
// a binary search on the bit counts of halves, quarters, ... (five fixed
// steps, the same for every lane).
__device__ __forceinline__ int nth_set_bit(unsigned x, int k) {
    int pos = 0;
#pragma unroll
    for (int width = 16; width > 0; width >>= 1) {
        const int low = __popc(x & ((1u << width) - 1u));
        const bool up = k >= low;
        k -= up ? low : 0;
        x = up ? x >> width : x;
        pos += up ? width : 0;
    }
    return pos;
}

__device__ __forceinline__ bool compressed_row(const Tile &t, int i, int kmax, unsigned *bsh, int lane,
                                               unsigned long long *cnt) {
    const unsigned *Ri = t.rows + (size_t)i * t.ws;
    const int nw = (i + 31) >> 5;
    int c = 0;
    for (int w = 0; w < nw; ++w) c += __popc(Ri[w]);
    if (c > 32) return false;
    if (c < 2) return true; // no edge inside R_i
    // position p_a of the a-th bit, and the word prefix of bit counts
    int pa = -1, prefix = 0;
    for (int w = 0; w < nw; ++w) {
        const unsigned x = Ri[w];
        const int pc = __popc(x);
        if (lane >= prefix && lane < prefix + pc) pa = w * 32 + nth_set_bit(x, lane - prefix);
        prefix += pc;
    }
    unsigned B = 0;
    if (lane < c) {
        const unsigned *Rp = t.rows + (size_t)pa * t.ws;
        int pre = 0;
        for (int w = 0; w <= ((pa - 1) >> 5) && pa > 0; ++w) {
            const unsigned riw = Ri[w];
            unsigned x = Rp[w] & riw;
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1;
                B |= 1u << (pre + __popc(riw & ((1u << b) - 1)));
            }
            pre += __popc(riw);
        }
    }
    bump<1>(cnt, __popc(B));
    if (kmax >= 5) {
        bsh[lane] = B;
        __syncwarp();
        unsigned long long s5 = 0, s6 = 0;
        unsigned y = B;
        while (y) {
            const int b = __ffs(y) - 1;
            y &= y - 1;
            const unsigned z = B & bsh[b];
            s5 += __popc(z);
            if (kmax >= 6) {
                unsigned zz = z;
                while (zz) {
                    const int q = __ffs(zz) - 1;
                    zz &= zz - 1;
                    s6 += __popc(z & bsh[q]);
                }
            }
        }
        bump<2>(cnt, s5);
        bump<3>(cnt, s6);
        __syncwarp();
    }
    return true;
}

// Pending products of the last level belong to size kmax: cnt[kmax - 3]
// (a switch over constant indices).
template <int KMAX>
__device__ __forceinline__ void drain(const Tile &t, Walker &wk, int kmax, int lane, unsigned long long *cnt) {
    if (wk.m == 0) {
        wk.used = 0;
        return;
    }
    const unsigned long long s = flush(t, wk, lane);
    switch (kmax) {
        case 4: cnt[1] += s; break;
        case 5: cnt[2] += s; break;
        case 6: cnt[3] += s; break;
        case 7: cnt[4] += s; break;
        case 8: cnt[5] += s; break;
        default:
            if constexpr (KMAX > 8) {
#pragma unroll
                for (int k = 9; k <= KMAX; ++k)
                    if (k == kmax) cnt[k - 3] += s;
            }
            break;
    }
    wk.used = 0;
}

// Traversal of one row i of a tile (the cliques through v and list[i]).
template <int KMAX, bool XT>
__device__ __forceinline__ void run_row(const Tile &t, Walker &wk, int i, int kmax, int lane,
                                        unsigned long long *cnt) {
    if (KMAX <= 8 && kmax <= 6 && compressed_row(t, i, kmax, wk.bsh, lane, cnt)) return;
    walk<1, KMAX, XT>(t, wk, t.rows + (size_t)i * t.ws, i, kmax, lane, cnt);
}

// Existence mode: publish the warp's kmax count after a row (kmin == kmax).
template <int KMAX>
__device__ __forceinline__ void publish_row(const Tile &t, Walker &wk, int lane, unsigned long long *cnt,
                                            const CliqueArgs &a) {
    drain<KMAX>(t, wk, a.kmax, lane, cnt);
    const unsigned long long mine = cnt[a.kmax - 3];
    cnt[a.kmax - 3] = 0;
    const unsigned __int128 tot = warp_sum_u128(mine);
    if (lane == 0) ctl_publish(a.ctl, a.counts, tot);
}

// MINB CTAs per SM: 3 (80 registers) or 4 (64 registers, some spilling;
// more resident warps against the fixed-latency dependency stalls).  KMAX:
// largest clique size the traversal can reach (8 or 16).  XT: the extended
// variant with cardinality pruning and run control (large kmin, existence
// queries, work budgets); the plain variants keep their registers for the
// traversal.
template <int MINB, int KMAX, bool XT>
__global__ void __launch_bounds__(kBlock, MINB) k_count_clique(CliqueArgs a) {
    extern __shared__ __align__(16) unsigned smem[];
    int *ctl = (int *)smem;
    unsigned *region = smem + kCtl;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const DevGraph &g = a.g;
    unsigned *slab = a.slabs ? a.slabs + (size_t)blockIdx.x * a.slab_words : nullptr;
    const bool polled = XT && a.ctl.words != nullptr;
    const bool exist = XT && a.ctl.target > 0;
    if (polled && lane == 0) ctl_begin(a.ctl);

    Walker wk;
    wk.cws = a.cws;
    wk.nslots = a.nslots;
    wk.cbuf = smem + kCtl + a.region_words + (size_t)warp * a.warp_words;
    wk.ring = wk.cbuf + (size_t)KMAX * a.cws;
    wk.items = (int *)(wk.ring + (size_t)a.nslots * a.cws);
    wk.bsh = (unsigned *)(wk.items + kItems);
    wk.m = 0;
    wk.used = 0;
    wk.kmin = a.kmin;
    if constexpr (XT) {
        if (threadIdx.x == 0) {
            s_run_ctl = a.ctl;
            s_counts = a.counts;
        }
        __syncthreads();
    }

    unsigned long long cnt[KMAX];
#pragma unroll 1
    for (int s = 0; s < KMAX; ++s) cnt[s] = 0;

    // ---- heavy vertices: one CTA each --------------------------------------
    Tile ht;
    {
        unsigned *base = a.heavy_in_smem ? region : slab;
        ht.list = (int *)base;
        ht.rstart = ht.list + a.dpad;
        ht.rlen = ht.rstart + a.dpad;
        ht.pre = ht.rlen + a.dpad;
        ht.rows = (unsigned *)(ht.pre + a.dpad + 4);
        ht.ws = a.hws;
    }
    for (int iter = 0;; ++iter) {
        if (threadIdx.x == 0) {
            int v = -1;
            if (XT && a.plain) {
                // non-persistent: this block's own heavy start vertex, once
                if (a.plain == 1 && iter == 0 && blockIdx.x < a.n_heavy_tasks)
                    v = a.heavy[(unsigned long long)a.offset + blockIdx.x * (unsigned long long)a.stride];
            } else if (!polled || !ctl_poll(a.ctl)) {
                const unsigned long long h = atomicAdd(a.queue + 1, 1ull);
                if (h < (unsigned long long)a.n_heavy_tasks)
                    v = a.heavy[(unsigned long long)a.offset + h * (unsigned long long)a.stride];
            }
            ctl[0] = v;
            ctl[1] = 0; // rows traversed
        }
        __syncthreads();
        const int v = ctl[0];
        if (v < 0) break;
        const int4 vi = __ldg(&g.vinfo[v]);
        const int d = vi.z;
        const int *nv = adj_of(g, vi);
        for (int i = threadIdx.x; i < d; i += kBlock) ht.list[i] = __ldg(nv + i);
        __syncthreads();
        build_rows<true>(g, ht, d, threadIdx.x, kBlock, cnt[0]);
        if (a.kmax >= 4) {
            for (;;) {
                int r = 0;
                if (lane == 0) r = atomicAdd(&ctl[1], 1);
                r = __shfl_sync(PG_FULL, r, 0);
                const int i = d - 1 - r; // longest rows first
                if (i < 2) break;
                if (polled && ctl_stop(a.ctl, lane)) break;
                run_row<KMAX, XT>(ht, wk, i, a.kmax, lane, cnt);
                if (exist) publish_row<KMAX>(ht, wk, lane, cnt, a);
            }
            drain<KMAX>(ht, wk, a.kmax, lane, cnt);
        }
        guard_counts<KMAX>(cnt, a);
        __syncthreads();
    }

    // ---- light vertices: one warp each, rank order -------------------------
    Tile lt;
    {
        unsigned *base = region + (size_t)warp * kLightTile;
        lt.list = (int *)base;
        lt.rstart = lt.list + kLightD;
        lt.rlen = lt.rstart + kLightD;
        lt.pre = lt.rlen + kLightD;
        lt.rows = (unsigned *)(lt.pre + kLightD + 1);
        lt.ws = kLightWs;
    }
    for (int iter = 0;; ++iter) {
        if (polled && ctl_stop(a.ctl, lane)) break;
        unsigned long long base = 0;
        int chunk = a.chunk;
        if (XT && a.plain) {
            // non-persistent: this warp's own light start vertex, once
            if (a.plain != 2 || iter > 0) break;
            base = (unsigned long long)blockIdx.x * kWarps + warp;
            chunk = 1;
        } else {
            if (lane == 0) base = atomicAdd(a.queue, (unsigned long long)a.chunk);
            base = __shfl_sync(PG_FULL, base, 0);
        }
        if (base >= (unsigned long long)a.n_light_tasks) break;
        for (int q = 0; q < chunk; ++q) {
            const unsigned long long t = base + (unsigned long long)q;
            if (t >= (unsigned long long)a.n_light_tasks) break;
            const int v = (int)((unsigned long long)a.offset + t * (unsigned long long)a.stride);
            const int4 vi = __ldg(&g.vinfo[v]);
            const int d = vi.z;
            if (d < a.kmin - 1 || d > a.heavy_min) continue;
            const int *nv = adj_of(g, vi);
            for (int i = lane; i < d; i += 32) lt.list[i] = __ldg(nv + i);
            __syncwarp();
            build_rows<false>(g, lt, d, lane, 32, cnt[0]);
            if (a.kmax >= 4) {
                for (int i = d - 1; i >= 2; --i) {
                    if (polled && ctl_stop(a.ctl, lane)) break;
                    run_row<KMAX, XT>(lt, wk, i, a.kmax, lane, cnt);
                    if (exist) publish_row<KMAX>(lt, wk, lane, cnt, a);
                }
                drain<KMAX>(lt, wk, a.kmax, lane, cnt);
            }
            guard_counts<KMAX>(cnt, a);
            __syncwarp();
        }
    }

#pragma unroll 1
    for (int s = a.kmin - 3; s <= a.kmax - 3; ++s) {
        const unsigned __int128 tot = warp_sum_u128(cnt[s]);
        if (lane == 0 && tot) atomic_add_u128(a.counts + 2 * (s + 3 - a.kmin), tot);
    }
}

// ---------------------------------------------------------------- host ----

struct Layout {
    CliqueArgs a;
    size_t smem_bytes;
};

int kmax_variant(int kmax) { return kmax <= 8 ? 8 : 16; }

// the extended variant: run control, or pruning worth its registers
bool extended_variant(int kmin, int kmax, const PgRunCtl *ctl) {
    return (ctl && ctl->words) || kmin >= 6 || kmax > 8;
}

Layout layout_for(const pg_graph *g, int kvar) {
    Layout L{};
    CliqueArgs &a = L.a;
    const long long D = std::max<long long>(g->max_out, 1);
    a.dpad = (int)((D + 3) & ~3ll);
    a.hws = (int)(((D + 31) / 32) | 1);
    a.cws = std::max(a.hws, kLightWs);
    a.nslots = (int)std::min<long long>(32, std::max<long long>(2, 1024 / a.cws));
    a.warp_words = (int)(((size_t)kvar * a.cws + (size_t)a.nslots * a.cws + kItems + 32 + 3) & ~3ull);
    const size_t heavy_words = (size_t)4 * a.dpad + 4 + (size_t)D * a.hws;
    const size_t light_words = (size_t)kWarps * kLightTile;
    const size_t warps_words = (size_t)kWarps * a.warp_words;
    a.heavy_in_smem = (kCtl + std::max(heavy_words, light_words) + warps_words) * 4 <= kSmemBudget;
    a.region_words = (int)(((a.heavy_in_smem ? std::max(heavy_words, light_words) : light_words) + 3) & ~3ull);
    a.slab_words = a.heavy_in_smem ? 0 : (long long)((heavy_words + 3) & ~3ull);
    L.smem_bytes = (kCtl + (size_t)a.region_words + warps_words) * 4;
    return L;
}

void *clique_fn(const pg_graph *g, int kvar, bool xt) {
    if (kvar > 8) return (void *)k_count_clique<3, 16, true>;
    if (xt) return (void *)k_count_clique<3, 8, true>;
    return g->tune.clique_min_blocks == 4 ? (void *)k_count_clique<4, 8, false> : (void *)k_count_clique<3, 8, false>;
}

// The dynamic shared-memory limit is a per-device function attribute: set
// once per device (thread-safe), checked.
constexpr int kMaxDevices = 64;
std::once_flag g_attr_once[kMaxDevices];
cudaError_t g_attr_err[kMaxDevices];

int ensure_attributes(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return pg_set_error(PG_EINVAL, "device index out of range");
    std::call_once(g_attr_once[dev], [dev] {
        const int bytes = 200 * 1024;
        void *fns[] = {(void *)k_count_clique<3, 8, false>, (void *)k_count_clique<4, 8, false>,
                       (void *)k_count_clique<3, 8, true>, (void *)k_count_clique<3, 16, true>};
        cudaError_t e = cudaSuccess;
        for (void *f : fns)
            if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        g_attr_err[dev] = e;
    });
    if (g_attr_err[dev] != cudaSuccess) return pg_cuda_error(g_attr_err[dev], "cudaFuncSetAttribute(k_count_clique)");
    return PG_OK;
}

int clique_grid(const pg_graph *g, size_t smem, int kvar, bool xt, int *grid) {
    int rc = ensure_attributes(g->device);
    if (rc) return rc;
    int per_sm = 0;
    PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, clique_fn(g, kvar, xt), kBlock, smem));
    if (per_sm < 1) per_sm = 1;
    if (g->tune.clique_blocks_per_sm > 0) per_sm = std::min(per_sm, g->tune.clique_blocks_per_sm);
    *grid = per_sm * g->num_sms;
    return PG_OK;
}

int launch(pg_graph *g, int kmin, int kmax, unsigned long long *counts_dev, unsigned long long *queue,
           void *slabs, long long max_slabs, cudaStream_t s, const PgRunCtl *rctl) {
    if (kmin < 3 || kmax > PG_MAX_CLIQUE || kmin > kmax)
        return pg_set_error(PG_EINVAL, "clique sizes must satisfy 3 <= kmin <= kmax <= 16");
    if (kmax > 8 && kmax - kmin > 7) return pg_set_error(PG_EINVAL, "at most 8 clique sizes per launch");
    if (g->n == 0) return PG_OK;
    if (g->max_out >= 65536) return pg_set_error(PG_EUNSUPPORTED, "clique kernel needs out-degrees below 65536");
    const int kvar = kmax_variant(kmax);
    Layout L = layout_for(g, kvar);
    CliqueArgs a = L.a;
    a.g = g->d;
    a.kmin = kmin;
    a.kmax = kmax;
    a.heavy = g->heavy;
    a.n_heavy = (int)g->n_heavy;
    a.n = (int)g->n;
    a.slabs = a.slab_words ? (unsigned *)slabs : nullptr;
    a.queue = queue;
    a.counts = counts_dev;
    a.chunk = g->tune.clique_chunk;
    a.heavy_min = g->heavy_min_built; // the threshold the heavy list was built with
    const PgTaskSel sel = pg_task_sel(g);
    a.stride = (int)sel.stride;
    a.offset = (int)sel.offset;
    a.n_light_tasks = sel.count(g->n);
    a.n_heavy_tasks = sel.count(g->n_heavy);
    a.ctl = rctl ? *rctl : PgRunCtl{};
    a.plain = 0;
    if (a.ctl.target > 0 && (kmin != kmax || !a.ctl.words))
        return pg_set_error(PG_EINVAL, "internal: existence mode needs one clique size and control words");
    const bool xt = extended_variant(kmin, kmax, rctl);
    int blocks = 0;
    int rc = clique_grid(g, L.smem_bytes, kvar, xt, &blocks);
    if (rc) return rc;
    if (a.slab_words && blocks > max_slabs) blocks = (int)max_slabs;
    if (blocks < 1) return pg_set_error(PG_EINVAL, "scratch holds no slab for a single block");
    PG_CUDA(cudaMemsetAsync(queue, 0, 2 * sizeof(unsigned long long), s));
    void *args[] = {&a};
    PG_CUDA(cudaLaunchKernel(clique_fn(g, kvar, xt), dim3((unsigned)blocks), dim3(kBlock), args, L.smem_bytes, s));
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

}  // namespace

size_t pg_clique_slab_bytes(const pg_graph *g, int kmax) {
    return (size_t)layout_for(g, kmax_variant(kmax)).a.slab_words * sizeof(unsigned);
}

size_t pg_clique_scratch_bytes(const pg_graph *g, int kmax) {
    const int kvar = kmax_variant(kmax);
    const Layout L = layout_for(g, kvar);
    int blocks = 0;
    if (clique_grid(g, L.smem_bytes, kvar, kvar > 8, &blocks) != PG_OK) blocks = 4 * g->num_sms;
    return (size_t)blocks * (size_t)L.a.slab_words * sizeof(unsigned);
}

int pg_launch_clique(pg_graph *g, int kmin, int kmax, unsigned long long *counts_dev, int queue_slot,
                     cudaStream_t s, const PgRunCtl *ctl) {
    if (queue_slot + 1 >= PG_CTL_WORDS_SLOT) return pg_set_error(PG_EINVAL, "queue slot out of range");
    return launch(g, kmin, kmax, counts_dev, g->ex->queues + queue_slot, g->ex->scratch,
                  (long long)(g->ex->scratch_bytes / std::max<size_t>(pg_clique_slab_bytes(g, kmax), 1)), s, ctl);
}

// The plain form of the same traversal: no persistence and no shared
// traversal of several sizes.  One launch of one CTA per heavy start vertex
// and one launch of one warp per light start vertex, for a single clique
// size k; adds into counts_dev (low, high).  Heavy tiles must fit shared
// memory.
int pg_launch_clique_plain(pg_graph *g, int k, unsigned long long *counts_dev, cudaStream_t s) {
    if (k < 3 || k > PG_MAX_CLIQUE) return pg_set_error(PG_EINVAL, "clique size must be 3..16");
    if (g->n == 0) return PG_OK;
    if (g->max_out >= 65536) return pg_set_error(PG_EUNSUPPORTED, "clique kernel needs out-degrees below 65536");
    const int kvar = kmax_variant(k);
    Layout L = layout_for(g, kvar);
    if (!L.a.heavy_in_smem)
        return pg_set_error(PG_EUNSUPPORTED, "plain clique launches need the heavy tiles in shared memory");
    int rc = ensure_attributes(g->device);
    if (rc) return rc;
    CliqueArgs a = L.a;
    a.g = g->d;
    a.kmin = a.kmax = k;
    a.heavy = g->heavy;
    a.n_heavy = (int)g->n_heavy;
    a.n = (int)g->n;
    a.slabs = nullptr;
    a.queue = nullptr;
    a.counts = counts_dev;
    a.chunk = 1;
    a.heavy_min = g->heavy_min_built;
    const PgTaskSel sel = pg_task_sel(g);
    a.stride = (int)sel.stride;
    a.offset = (int)sel.offset;
    a.n_light_tasks = sel.count(g->n);
    a.n_heavy_tasks = sel.count(g->n_heavy);
    a.ctl = PgRunCtl{};
    void *fn = kvar > 8 ? (void *)k_count_clique<3, 16, true> : (void *)k_count_clique<3, 8, true>;
    void *args[] = {&a};
    if (a.n_heavy_tasks > 0) {
        a.plain = 1;
        PG_CUDA(cudaLaunchKernel(fn, dim3((unsigned)a.n_heavy_tasks), dim3(kBlock), args, L.smem_bytes, s));
        PG_CUDA(cudaGetLastError());
    }
    if (a.n_light_tasks > 0) {
        a.plain = 2;
        const long long blocks = (a.n_light_tasks + kWarps - 1) / kWarps;
        PG_CUDA(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(kBlock), args, L.smem_bytes, s));
        PG_CUDA(cudaGetLastError());
    }
    return PG_OK;
}

// Same kernel on caller-supplied scratch: `queue` = two 64-bit counters
// (zeroed here on the stream), `slabs` = room for `max_slabs` per-CTA slabs of
// pg_clique_slab_bytes() bytes; the grid is cut to max_slabs CTAs.
int pg_launch_clique_on(pg_graph *g, int kmin, int kmax, unsigned long long *counts_dev,
                        unsigned long long *queue, void *slabs, long long max_slabs, cudaStream_t s) {
    return launch(g, kmin, kmax, counts_dev, queue, slabs, max_slabs, s, nullptr);
}
