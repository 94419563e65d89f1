// K1: plan-interpreter counting kernel (any pattern the compiler accepts).
//
// Section 5.1 "Pattern-Aware Processing Model" figure: every task is one
// (start vertex, matching order) pair; the start vertex binds the highest
// core position and the remaining core vertices are bound level by level
// (matchFrom), candidates being intersections / differences of sorted
// adjacency lists cut to the id range that the partial order allows (the
// "PO" stage, found by binary search on the sorted lists).  Non-core vertices
// other than the counted group are bound the same way; the counted group is
// never enumerated: its candidate set's cardinality |S| gives C(|S|, g)
// matches (Section 5.1, completing a core match by set operations).
//
// GPU mapping: one warp per task, tasks handed out through a device atomic
// counter in start-vertex rank order, i.e. highest degree first (Section
// 5.2, Section 5.5).  A warp binds levels depth first with an explicit stack;
// each level's candidate set is built cooperatively (lanes take driver
// elements, check membership in the other lists by binary search, compact
// with __ballot_sync/__popc) into a per-warp scratch buffer.  The last level
// is counted, by inclusion-exclusion over its difference lists when that
// touches fewer elements than filtering the driver list.  Levels that carry
// anti-vertex checks (Section 4.3) are filtered candidate by candidate; a
// checked last level is enumerated instead of counted.
#include "level_ops.cuh"

namespace {

using namespace pgk;

constexpr int kWarpsPerBlock = 8;
constexpr int kBlock = kWarpsPerBlock * 32;

struct GenericArgs {
    DevGraph g;
    const PgOrder *orders;
    int n_orders;
    int *scratch;
    long long warp_stride;      // ints per warp
    long long lvl_off[PGP_MAXK]; // offset of level l's buffer inside a warp's region
    unsigned long long *queue;  // dynamic task counter (persistent mode)
    unsigned long long n_tasks; // selected tasks: offset + t * stride over (start vertex, order) pairs
    unsigned long long offset, stride;
    int persistent;             // 0: one task per warp, no queue
    unsigned long long *counts; // (low, high)
    // run control: existence mode (ctl.target > 0) publishes counts after
    // every task and the warp that sees the total reach the target raises
    // the stop flag; with a work budget the launch stops once it is spent.
    // Warps poll between tasks and between first-level candidates (Section
    // 5.4, early termination).
    PgRunCtl ctl;
};

__device__ unsigned __int128 run_task(const GenericArgs &a, int v, const PgOrder &ord, int *wbuf, int lane) {
    const DevGraph &g = a.g;
    const int L = ord.n_levels;
    const int4 v0 = __ldg(&g.vinfo[v]);
    if (ord.lv[0].label >= 0 && v0.w != ord.lv[0].label) return 0;
    int m[PGP_MAXK];
    int sz[PGP_MAXK], idx[PGP_MAXK];
    m[0] = v;
    if (ord.lv[0].n_anti && !checks_ok(g, ord, 0, m, lane)) return 0;
    if (L == 1) return 1;
    unsigned __int128 total = 0;
    int l = 1;
    for (;;) {
        const PgLevel &lv = ord.lv[l];
        if (l == L - 1 && !lv.n_anti) {
            const unsigned long long c = count_last(g, lv, m, lane);
            total += choose_u128(c, lv.group);
        } else {
            int *buf = wbuf + a.lvl_off[l];
            sz[l] = fill_level(g, lv, m, buf, lane);
            if (lv.n_anti) sz[l] = filter_anti(g, ord, l, m, buf, sz[l], lane);
            idx[l] = 0;
            if (l == L - 1) total += (unsigned)sz[l]; // checked vertices are never grouped
        }
        // advance to the next unexplored candidate
        while (l >= 1 && (l == L - 1 || idx[l] >= sz[l])) --l;
        if (l < 1) break;
        if (l <= 3 && a.ctl.words && ctl_stop(a.ctl, lane)) break;
        m[l] = wbuf[a.lvl_off[l] + idx[l]];
        ++idx[l];
        ++l;
    }
    return total;
}

__global__ void __launch_bounds__(kBlock) k_count_generic(GenericArgs a) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    int *wbuf = a.scratch + gw * a.warp_stride;
    unsigned __int128 acc = 0;
    if (a.ctl.words && lane == 0) ctl_begin(a.ctl);
    for (;;) {
        if (a.ctl.words && ctl_stop(a.ctl, lane)) break;
        unsigned long long t = (unsigned long long)gw;
        if (a.persistent) {
            if (lane == 0) t = atomicAdd(a.queue, 1ull);
            t = __shfl_sync(PG_FULL, t, 0);
        }
        if (t >= a.n_tasks) break;
        const unsigned long long tt = a.offset + t * a.stride;
        const int v = (int)(tt / (unsigned long long)a.n_orders);
        const int o = (int)(tt % (unsigned long long)a.n_orders);
        acc += run_task(a, v, a.orders[o], wbuf, lane);
        if (a.ctl.target && acc) {
            if (lane == 0) ctl_publish(a.ctl, a.counts, acc);
            acc = 0;
        }
        if (!a.persistent) break;
    }
    if (lane == 0 && acc) atomic_add_u128(a.counts, acc);
}

// ---- algorithmic operand bytes (measurement) --------------------------------
//
// The plan's set operations read, per level and bound prefix m, every
// intersected and every subtracted list cut to the level's partial-order
// range (lo, hi).  level_operand_elems gives the total length of those
// slices; the walk below visits the same prefixes as run_task (every level
// but the last materialised and enumerated) and sums it over every set
// operation, the last level's for all candidates of the level before it in
// parallel across lanes.

__device__ __forceinline__ unsigned long long level_operand_elems(const DevGraph &g, const PgLevel &L, const int *m) {
    const LevelRange r = level_range(L, m);
    if (r.lo + 1 >= r.hi) return 0;
    unsigned long long e = 0;
    for (int i = 0; i < L.n_int + L.n_diff; ++i) {
        const int w = m[i < L.n_int ? L.int_src[i] : L.diff_src[i - L.n_int]];
        const int4 vi = __ldg(&g.vinfo[w]);
        e += (unsigned long long)bound_slice(adj_of(g, vi), vi.y, r.lo, r.hi).len;
    }
    return e;
}

__device__ void operand_walk(const GenericArgs &a, int v, const PgOrder &ord, int *wbuf, int lane,
                             unsigned long long &elems, unsigned long long &ops) {
    const DevGraph &g = a.g;
    const int L = ord.n_levels;
    const int4 v0 = __ldg(&g.vinfo[v]);
    if (ord.lv[0].label >= 0 && v0.w != ord.lv[0].label) return;
    int m[PGP_MAXK];
    int sz[PGP_MAXK], idx[PGP_MAXK];
    m[0] = v;
    if (ord.lv[0].n_anti && !checks_ok(g, ord, 0, m, lane)) return;
    if (L == 1) return;
    if (L == 2) {
        if (lane == 0) {
            elems += level_operand_elems(g, ord.lv[1], m);
            ++ops;
        }
        return;
    }
    int l = 1;
    for (;;) {
        const PgLevel &lv = ord.lv[l];
        if (lane == 0) {
            elems += level_operand_elems(g, lv, m);
            ++ops;
        }
        int *buf = wbuf + a.lvl_off[l];
        sz[l] = fill_level(g, lv, m, buf, lane);
        if (lv.n_anti) sz[l] = filter_anti(g, ord, l, m, buf, sz[l], lane);
        idx[l] = 0;
        if (l == L - 2) {
            // the last level's operation for every candidate of this one
            int mm[PGP_MAXK];
            for (int i = 0; i < l; ++i) mm[i] = m[i];
            for (int c = lane; c < sz[l]; c += 32) {
                mm[l] = buf[c];
                elems += level_operand_elems(g, ord.lv[L - 1], mm);
                ++ops;
            }
            idx[l] = sz[l];
        }
        while (l >= 1 && idx[l] >= sz[l]) --l;
        if (l < 1) break;
        m[l] = wbuf[a.lvl_off[l] + idx[l]];
        ++idx[l];
        ++l;
    }
}

__global__ void __launch_bounds__(kBlock) k_operand_bytes(GenericArgs a, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    int *wbuf = a.scratch + gw * a.warp_stride;
    unsigned long long elems = 0, ops = 0;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.queue, 1ull);
        t = __shfl_sync(PG_FULL, t, 0);
        if (t >= a.n_tasks) break;
        const unsigned long long tt = a.offset + t * a.stride;
        operand_walk(a, (int)(tt / (unsigned long long)a.n_orders), a.orders[tt % (unsigned long long)a.n_orders],
                     wbuf, lane, elems, ops);
    }
    for (int o = 16; o; o >>= 1) {
        elems += __shfl_down_sync(PG_FULL, elems, o);
        ops += __shfl_down_sync(PG_FULL, ops, o);
    }
    if (lane == 0) {
        atomicAdd(out, elems);
        atomicAdd(out + 1, ops);
    }
}

int generic_grid(const pg_graph *g) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_generic, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * g->num_sms;
}

}  // namespace

// Per-warp buffer layout: every materialised level l >= 1 (all but a counted
// last level) gets max out-degree ints when its candidates lie in a bound
// vertex's out-neighbourhood, else max degree ints (each rounded to 32).
long long pg_level_layout(const pg_graph *g, const std::vector<PgOrder> &orders, bool listing, long long *off) {
    const long long cap_out = (g->max_out + 31) & ~31ll, cap_all = (g->max_deg + 31) & ~31ll;
    long long total = 0;
    for (int l = 0; l < PGP_MAXK; ++l) {
        off[l] = total;
        bool any = false, all_out = true;
        for (auto &o : orders)
            if (l >= 1 && (l < o.n_levels - 1 || (l == o.n_levels - 1 && (listing || o.lv[l].n_anti)))) {
                any = true;
                all_out &= o.lv[l].out_bounded != 0;
            }
        if (any) total += all_out ? cap_out : cap_all;
    }
    return total;
}

namespace {

long long level_layout(const pg_graph *g, const pg_plan *p, long long *off) {
    return pg_level_layout(g, p->h.orders, false, off);
}

unsigned long long n_tasks_of(const pg_graph *g, const pg_plan *p) {
    return (unsigned long long)pg_task_sel(g).count((long long)g->n * (long long)p->h.orders.size());
}

int grid_of(const pg_graph *g, const pg_plan *p, bool persistent) {
    if (persistent) return generic_grid(g);
    const unsigned long long w = n_tasks_of(g, p);
    return (int)((w + kWarpsPerBlock - 1) / kWarpsPerBlock);
}

}  // namespace

size_t pg_generic_scratch_bytes(const pg_graph *g, const pg_plan *p, bool persistent) {
    long long off[PGP_MAXK];
    const long long per_warp = level_layout(g, p, off);
    return (size_t)grid_of(g, p, persistent) * kWarpsPerBlock * (size_t)per_warp * sizeof(int);
}

int pg_launch_generic(pg_graph *g, const pg_plan *p, unsigned long long *counts_dev, int queue_slot,
                      bool persistent, cudaStream_t s, const PgRunCtl *ctl) {
    if (p->h.big_clique) return pg_set_error(PG_EUNSUPPORTED, "cliques above 8 vertices run on the k-clique kernel only");
    if (g->n == 0 || p->h.orders.empty()) return PG_OK;
    GenericArgs a;
    a.g = g->d;
    a.orders = p->d_orders;
    a.n_orders = (int)p->h.orders.size();
    a.warp_stride = level_layout(g, p, a.lvl_off);
    a.scratch = (int *)g->ex->scratch;
    a.queue = g->ex->queues + queue_slot;
    a.n_tasks = n_tasks_of(g, p);
    const PgTaskSel sel = pg_task_sel(g);
    a.offset = (unsigned long long)sel.offset;
    a.stride = (unsigned long long)sel.stride;
    a.persistent = persistent ? 1 : 0;
    a.counts = counts_dev;
    a.ctl = ctl ? *ctl : PgRunCtl{};
    if (persistent) PG_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s));
    k_count_generic<<<grid_of(g, p, persistent), kBlock, 0, s>>>(a);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

int pg_launch_operand_bytes(pg_graph *g, const pg_plan *p, unsigned long long *out_dev, cudaStream_t s) {
    PG_CUDA(cudaMemsetAsync(out_dev, 0, 2 * sizeof(unsigned long long), s));
    if (p->h.big_clique) return pg_set_error(PG_EUNSUPPORTED, "cliques above 8 vertices have no level program");
    if (g->n == 0 || p->h.orders.empty()) return PG_OK;
    GenericArgs a;
    a.g = g->d;
    a.orders = p->d_orders;
    a.n_orders = (int)p->h.orders.size();
    a.warp_stride = level_layout(g, p, a.lvl_off);
    a.scratch = (int *)g->ex->scratch;
    a.queue = g->ex->queues;
    a.n_tasks = n_tasks_of(g, p);
    const PgTaskSel sel = pg_task_sel(g);
    a.offset = (unsigned long long)sel.offset;
    a.stride = (unsigned long long)sel.stride;
    a.persistent = 1;
    a.counts = nullptr;
    a.ctl = PgRunCtl{};
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_operand_bytes, kBlock, 0);
    const int grid = std::max(1, per_sm) * g->num_sms;
    const int rc = pg_ensure_scratch(g, (size_t)grid * kWarpsPerBlock * (size_t)a.warp_stride * sizeof(int), s);
    if (rc) return rc;
    a.scratch = (int *)g->ex->scratch; // the arena may have moved
    PG_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s));
    k_operand_bytes<<<grid, kBlock, 0, s>>>(a, out_dev);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}
