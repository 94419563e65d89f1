// K6: match listing (the match(G, p, f) call of the paper's API, Section 3.2;
// the user callback becomes an output array of matches).
//
// Runs the plan's listing program: the same matching orders and partial
// order as counting (Section 4.1), but every vertex, non-core ones included,
// is bound on its own level, so each canonical match (one per automorphism
// class, Section 5.2) is reached exactly once as a full assignment.  The last
// level's candidate set is materialised like any other level and every
// element becomes one output row.
//
// GPU mapping: one warp per (start vertex, matching order) task from a
// device work queue, as in the counting interpreter.  A warp that completes
// a last-level set of n candidates reserves n consecutive output rows with
// one atomicAdd on the match counter; lanes then write one row each.  Rows
// past `capacity` are counted but not written, so the caller learns the full
// total and can retry with a larger buffer or list start-vertex ranges page
// by page.
#include "level_ops.cuh"

namespace {

using namespace pgk;

constexpr int kWarpsPerBlock = 8;
constexpr int kBlock = kWarpsPerBlock * 32;

struct MatchArgs {
    DevGraph g;
    const PgOrder *orders;
    int n_orders;
    int k;
    unsigned anti_mask;          // pattern vertices that are anti-vertices
    const int *orig;             // rank -> original id
    int *scratch;
    long long warp_stride;
    long long lvl_off[PGP_MAXK];
    unsigned long long *queue;
    unsigned long long task_begin, task_end;
    int *out;                    // capacity rows of k ints
    unsigned long long capacity;
    unsigned long long *n_total;
    PgRunCtl ctl; // work budget (polled between tasks and first-level candidates)
};

// Rows for the candidates buf[0, n) of the last level l (lanes stride rows).
__device__ void emit(const MatchArgs &a, const PgOrder &ord, int l, const int *m, const int *buf, int n, int lane) {
    if (n <= 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.n_total, (unsigned long long)n);
    base = __shfl_sync(PG_FULL, base, 0);
    for (int i = lane; i < n; i += 32) {
        const unsigned long long slot = base + (unsigned long long)i;
        if (slot >= a.capacity) break;
        int *row = a.out + slot * (unsigned long long)a.k;
        for (int j = 0; j < l; ++j) row[ord.lv[j].pattern_vertex] = __ldg(a.orig + m[j]);
        row[ord.lv[l].pattern_vertex] = __ldg(a.orig + buf[i]);
        for (int u = 0; u < a.k; ++u)
            if (a.anti_mask >> u & 1) row[u] = -1;
    }
}

__device__ void list_task(const MatchArgs &a, int v, const PgOrder &ord, int *wbuf, int lane) {
    const DevGraph &g = a.g;
    const int L = ord.n_levels;
    const int4 v0 = __ldg(&g.vinfo[v]);
    if (ord.lv[0].label >= 0 && v0.w != ord.lv[0].label) return;
    int m[PGP_MAXK];
    int sz[PGP_MAXK], idx[PGP_MAXK];
    m[0] = v;
    if (ord.lv[0].n_anti && !checks_ok(g, ord, 0, m, lane)) return;
    if (L == 1) {
        emit(a, ord, 0, m, m, 1, lane);
        return;
    }
    int l = 1;
    for (;;) {
        const PgLevel &lv = ord.lv[l];
        int *buf = wbuf + a.lvl_off[l];
        sz[l] = fill_level(g, lv, m, buf, lane);
        if (lv.n_anti) sz[l] = filter_anti(g, ord, l, m, buf, sz[l], lane);
        idx[l] = 0;
        if (l == L - 1) emit(a, ord, l, m, buf, sz[l], lane);
        while (l >= 1 && (l == L - 1 || idx[l] >= sz[l])) --l;
        if (l < 1) break;
        if (l <= 3 && a.ctl.words && ctl_stop(a.ctl, lane)) break;
        m[l] = wbuf[a.lvl_off[l] + idx[l]];
        ++idx[l];
        ++l;
    }
}

__global__ void __launch_bounds__(kBlock) k_match_list(MatchArgs a) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    int *wbuf = a.scratch + gw * a.warp_stride;
    if (a.ctl.words && lane == 0) ctl_begin(a.ctl);
    for (;;) {
        if (a.ctl.words && ctl_stop(a.ctl, lane)) break;
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.queue, 1ull);
        t = __shfl_sync(PG_FULL, t, 0) + a.task_begin;
        if (t >= a.task_end) break;
        const int v = (int)(t / (unsigned long long)a.n_orders);
        const int o = (int)(t % (unsigned long long)a.n_orders);
        list_task(a, v, a.orders[o], wbuf, lane);
    }
}

int match_grid(const pg_graph *g) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match_list, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * g->num_sms;
}

}  // namespace

size_t pg_match_scratch_bytes(const pg_graph *g, const pg_plan *p) {
    long long off[PGP_MAXK];
    const long long per_warp = pg_level_layout(g, p->h.list_orders, true, off);
    return (size_t)match_grid(g) * kWarpsPerBlock * (size_t)per_warp * sizeof(int);
}

int pg_launch_match(pg_graph *g, const pg_plan *p, int64_t rank_begin, int64_t rank_end, int32_t *out,
                    unsigned long long capacity, unsigned long long *n_total_dev, cudaStream_t s,
                    const PgRunCtl *ctl) {
    if (p->h.big_clique) return pg_set_error(PG_EUNSUPPORTED, "cliques above 8 vertices run on the k-clique kernel only");
    PG_CUDA(cudaMemsetAsync(n_total_dev, 0, sizeof(unsigned long long), s));
    if (rank_end <= rank_begin || p->h.list_orders.empty()) return PG_OK;
    MatchArgs a;
    a.g = g->d;
    a.orders = p->d_list_orders;
    a.n_orders = (int)p->h.list_orders.size();
    a.k = p->h.pat.k;
    a.anti_mask = 0;
    for (int u = 0; u < a.k; ++u)
        if (p->h.pat.anti_vertex[u]) a.anti_mask |= 1u << u;
    a.orig = g->orig;
    a.warp_stride = pg_level_layout(g, p->h.list_orders, true, a.lvl_off);
    a.scratch = (int *)g->ex->scratch;
    a.queue = g->ex->queues;
    a.task_begin = (unsigned long long)rank_begin * (unsigned long long)a.n_orders;
    a.task_end = (unsigned long long)rank_end * (unsigned long long)a.n_orders;
    a.out = out;
    a.capacity = capacity;
    a.n_total = n_total_dev;
    a.ctl = ctl ? *ctl : PgRunCtl{};
    PG_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s));
    k_match_list<<<match_grid(g), kBlock, 0, s>>>(a);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}
