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
// B300 mapping: one warp per start vertex v, handed out by a device atomic
// counter in rank order (highest degree first, Section 5.2).  The warp loads
// N+(v) (d entries) and builds the bitmap rows R[i] = { j < i : N+(v)[j] in
// N+(N+(v)[i]) } -- the level-1 intersections, each read once from L2/HBM --
// in shared memory (or a per-warp global scratch slab when d exceeds the
// shared-memory tile).  All deeper levels are word-wise ANDs of rows with
// __popc for the counted level: a depth-D prefix (i, j, ...) leaves the
// candidate set AND_s R[r_s], and its popcount is the number of
// (D+2)-cliques through that prefix, so one traversal yields the counts of
// every clique size up to kmax (several clique patterns share one launch).
// Pairs (i, j in R[i]) are compacted through a per-warp queue so that all 32
// lanes do work.
#include "device_sets.cuh"

namespace {

constexpr int kWarps = 4;
constexpr int kBlock = kWarps * 32;
constexpr int kSmemD = 256;                 // out-degree handled in shared memory
constexpr int kSmemWs = (kSmemD / 32) | 1;  // odd row stride (bank spread)
constexpr int kQueue = 64;
constexpr int kMaxK = 8;

struct WarpSmem {
    int list[kSmemD];
    unsigned rows[kSmemD * kSmemWs];
    int qi[kQueue], qj[kQueue];
};

struct CliqueArgs {
    DevGraph g;
    int kmin, kmax;       // counted clique sizes kmin..kmax (3 <= kmin <= kmax <= 8)
    unsigned *gscratch;   // per-warp slab for out-degree > kSmemD
    long long slab_words; // words per warp slab
    int gws;              // row stride of the global slab
    unsigned long long *queue;
    int n;
    unsigned long long *counts; // 2 words per size kmin..kmax
};

// Depth-first count below a prefix whose candidate set is AND of rows r[0..D).
// Adds popc(candidates) to cnt[D] (the (D+2)-cliques in the full graph) and
// recurses while D + 2 < kmax.
// cnt[s] accumulates (s + 3)-cliques; dfs<D> adds to cnt[D - 1].
template <int D>
__device__ __forceinline__ void dfs(const unsigned *rows, int ws, int *r, int limit_bits, int kmax,
                                    unsigned long long *cnt) {
    if constexpr (D >= kMaxK - 1) {
        return;
    } else {
        const int nwords = (limit_bits + 31) >> 5;
        for (int t = 0; t < nwords; ++t) {
            unsigned x = rows[r[0] * ws + t];
#pragma unroll
            for (int s = 1; s < D; ++s) x &= rows[r[s] * ws + t];
            if (!x) continue;
            cnt[D - 1] += __popc(x);
            if (D + 2 < kmax) {
                while (x) {
                    const int b = __ffs(x) - 1;
                    x &= x - 1;
                    r[D] = t * 32 + b;
                    dfs<D + 1>(rows, ws, r, r[D], kmax, cnt);
                }
            }
        }
    }
}

__device__ void process_vertex(const CliqueArgs &a, int v, WarpSmem &sm, unsigned *slab, int lane,
                               unsigned long long *cnt) {
    const DevGraph &g = a.g;
    const int4 vi = __ldg(&g.vinfo[v]);
    const int d = vi.z; // out-degree
    if (d < a.kmin - 1) return;
    const bool in_smem = d <= kSmemD;
    int *list = in_smem ? sm.list : (int *)slab;
    unsigned *rows = in_smem ? sm.rows : slab + ((d + 3) & ~3);
    const int ws = in_smem ? kSmemWs : a.gws;
    const int *nv = adj_of(g, vi);
    for (int i = lane; i < d; i += 32) list[i] = __ldg(nv + i);
    __syncwarp();
    // ---- level-1 intersections into bitmap rows -------------------------
    for (int i = 1; i < d; ++i) {
        const int nw = (i + 31) >> 5;
        for (int t = lane; t < nw; t += 32) rows[i * ws + t] = 0u;
        __syncwarp();
        const int u = list[i];
        const int4 ui = __ldg(&g.vinfo[u]);
        const int du = ui.z;
        const int *nu = adj_of(g, ui);
        if (du <= 4 * i + 32) {
            // scan N+(u), look each element up in list[0, i)
            for (int c = lane; c < du; c += 32) {
                const int x = __ldg(nu + c);
                int lo = 0, hi = i;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (list[mid] < x) lo = mid + 1; else hi = mid;
                }
                if (lo < i && list[lo] == x) atomicOr(&rows[i * ws + (lo >> 5)], 1u << (lo & 31));
            }
        } else {
            // look each list[j], j < i, up in N+(u)
            for (int j = lane; j < i; j += 32)
                if (contains_g(nu, du, list[j])) atomicOr(&rows[i * ws + (j >> 5)], 1u << (j & 31));
        }
        __syncwarp();
    }
    // ---- 3-cliques: edges of the sub-graph ------------------------------
    {
        unsigned long long c = 0;
        for (int i = 1 + lane; i < d; i += 32) {
            const int nw = (i + 31) >> 5;
            for (int t = 0; t < nw; ++t) c += __popc(rows[i * ws + t]);
        }
        cnt[0] += c;
    }
    if (a.kmax < 4) return;
    // ---- pairs (i, j in R[i]) through a warp queue ---------------------
    int qn = 0;
    int r[kMaxK];
    auto drain = [&](int count) {
        if (lane < count) {
            r[0] = sm.qi[lane];
            r[1] = sm.qj[lane];
            dfs<2>(rows, ws, r, r[1], a.kmax, cnt);
        }
    };
    for (int i = 2; i < d; ++i) {
        const int nw = (i + 31) >> 5;
        for (int t = 0; t < nw; ++t) {
            const unsigned w = rows[i * ws + t];
            if (!w) continue;
            const bool mine = (w >> lane) & 1u;
            const unsigned bal = __ballot_sync(PG_FULL, mine);
            const int pos = qn + __popc(bal & ((1u << lane) - 1));
            if (mine) {
                sm.qi[pos] = i;
                sm.qj[pos] = t * 32 + lane;
            }
            qn += __popc(bal);
            __syncwarp();
            if (qn >= 32) {
                drain(32);
                __syncwarp();
                // move the overflow to the queue front
                const int rest = qn - 32;
                if (lane < rest) {
                    sm.qi[lane] = sm.qi[32 + lane];
                    sm.qj[lane] = sm.qj[32 + lane];
                }
                __syncwarp();
                qn = rest;
            }
        }
    }
    drain(qn);
    __syncwarp();
}

__global__ void __launch_bounds__(kBlock) k_count_clique(CliqueArgs a) {
    __shared__ WarpSmem smem[kWarps];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    unsigned *slab = a.gscratch ? a.gscratch + gw * a.slab_words : nullptr;
    unsigned long long cnt[kMaxK];
    for (int s = 0; s < kMaxK; ++s) cnt[s] = 0;
    for (;;) {
        int v = 0;
        if (lane == 0) v = (int)atomicAdd(a.queue, 1ull);
        v = __shfl_sync(PG_FULL, v, 0);
        if (v >= a.n) break;
        process_vertex(a, v, smem[wib], slab, lane, cnt);
    }
    for (int k = a.kmin; k <= a.kmax; ++k) {
        const int s = k - 3;
        const unsigned long long tot = warp_sum_u64(cnt[s]);
        if (lane == 0 && tot) atomic_add_u128(a.counts + 2 * (k - a.kmin), tot);
    }
}

int clique_grid(const pg_graph *g) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_clique, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * g->num_sms;
}

long long slab_words(const pg_graph *g, int *gws) {
    const long long D = g->max_out;
    *gws = (int)(((D + 31) / 32) | 1);
    if (D <= kSmemD) return 0;
    return ((D + 3) & ~3ll) + D * (*gws);
}

}  // namespace

size_t pg_clique_scratch_bytes(const pg_graph *g) {
    int gws;
    return (size_t)clique_grid(g) * kWarps * (size_t)slab_words(g, &gws) * sizeof(unsigned);
}

int pg_launch_clique(pg_graph *g, int kmin, int kmax, unsigned long long *counts_dev, int queue_slot,
                     cudaStream_t s) {
    if (kmin < 3 || kmax > kMaxK || kmin > kmax) return pg_set_error(PG_EINVAL, "clique sizes must be 3..8");
    if (g->n == 0) return PG_OK;
    CliqueArgs a;
    a.g = g->d;
    a.kmin = kmin;
    a.kmax = kmax;
    a.slab_words = slab_words(g, &a.gws);
    a.gscratch = a.slab_words ? (unsigned *)g->scratch : nullptr;
    a.queue = g->queues + queue_slot;
    a.n = (int)g->n;
    a.counts = counts_dev;
    PG_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s));
    k_count_clique<<<clique_grid(g), kBlock, 0, s>>>(a);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

// Launch of the same kernel on caller-supplied scratch: `queue` is one zeroed
// 64-bit counter and `slabs` holds `max_warps` per-warp slabs of
// pg_clique_slab_bytes() bytes; the grid is cut so that no warp indexes a
// slab beyond max_warps.  Used by the entry point that allocates nothing.
size_t pg_clique_slab_bytes(const pg_graph *g) {
    int gws;
    return (size_t)slab_words(g, &gws) * sizeof(unsigned);
}

int pg_launch_clique_on(pg_graph *g, int kmin, int kmax, unsigned long long *counts_dev,
                        unsigned long long *queue, void *slabs, long long max_warps, cudaStream_t s) {
    if (kmin < 3 || kmax > kMaxK || kmin > kmax) return pg_set_error(PG_EINVAL, "clique sizes must be 3..8");
    if (g->n == 0) return PG_OK;
    CliqueArgs a;
    a.g = g->d;
    a.kmin = kmin;
    a.kmax = kmax;
    a.slab_words = slab_words(g, &a.gws);
    a.gscratch = a.slab_words ? (unsigned *)slabs : nullptr;
    a.queue = queue;
    a.n = (int)g->n;
    a.counts = counts_dev;
    long long blocks = clique_grid(g);
    if (a.slab_words && blocks * kWarps > max_warps) blocks = max_warps / kWarps;
    if (blocks < 1) return pg_set_error(PG_EINVAL, "scratch holds fewer slabs than one block needs");
    k_count_clique<<<(unsigned)blocks, kBlock, 0, s>>>(a);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}
