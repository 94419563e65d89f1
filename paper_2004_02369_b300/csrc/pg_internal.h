// Internal types shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pg.h"
#include "plan.h"

// Device view of a resident graph.  Vertices are degree-ranked ids (rank 0 =
// highest degree; ties by original id).  vinfo[v] = {start / 4, degree,
// out-degree, label}: the list of v is adj[4*start4 .. 4*start4 + degree),
// sorted ascending and padded with PG_PAD up to a multiple of 4 entries (16
// bytes); out-degree counts the neighbours with smaller rank (higher degree).
struct DevGraph {
    const int4 *vinfo;
    const int *adj;
    int n;
    int max_deg;
    int max_out;
    int labeled;
    // Membership bitmaps of the n_hubs highest-degree vertices (ranks
    // 0..n_hubs-1): bit x of row r is set iff x is in adj(r).  Lets set
    // operations test "x in adj(hub)" with one load instead of a binary search.
    const unsigned *hubbits;
    int n_hubs;
    int hub_stride; // words per row = ceil(n / 32)
};

#define PG_HUB_MIN_DEGREE 1024
#define PG_MAX_HUBS 512

#define PG_PAD 0x7fffffff

#define PG_MAX_QUEUES 64

// Run control of one persistent launch: early termination (existence
// queries, Section 5.4) and a device work budget.  `words` (device, zeroed
// before the launch): [0] stop flag, [1] set when the budget ran out, [2]
// start time of the launch in %globaltimer nanoseconds (first warp to poll).
// A warp polls between tasks and between first-level candidates, so a
// launch ends soon after the stop flag is raised.
struct PgRunCtl {
    unsigned long long *words = nullptr; // null: no polling at all
    unsigned long long target = 0;       // > 0: stop once the count reaches target
    unsigned long long budget_ns = 0;    // > 0: stop after this much device time
};
// queue words of an execution context reserved for run control
#define PG_CTL_WORDS_SLOT (PG_MAX_QUEUES - 4)

// Per-launch-stream device state: the scratch arena (grown on demand), the
// work-queue counters and small count buffers.  Launches that may overlap on
// the device use different contexts.
struct pg_exec {
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    unsigned long long *queues = nullptr;     // PG_MAX_QUEUES counters
    unsigned long long *tmp_counts = nullptr; // 2 * PG_MAX_QUEUES words
};
int pg_exec_init(pg_exec *x);
void pg_exec_release(pg_exec *x);
#define PG_CLIQUE_LIGHT_D 64 // out-degree up to which one warp handles a clique start vertex

// Defaults of the launch parameters (pg_tuning in pg.h).
inline pg_tuning pg_default_tuning() {
    pg_tuning t;
    t.clique_chunk = 4;
    t.clique_blocks_per_sm = 0;
    t.clique_heavy_min = PG_CLIQUE_LIGHT_D;
    t.batched_warps = 4;
    t.batched_chunk = 1;
    t.batched_blocks_per_sm = 0;
    t.hub_min_degree = PG_HUB_MIN_DEGREE;
    t.hub_max = PG_MAX_HUBS;
    t.batched_split_grain = 512;
    t.batched_regcap = 0;
    t.clique_min_blocks = 3;
    t.pad = 0;
    return t;
}

struct pg_graph {
    DevGraph d{};
    int4 *vinfo = nullptr;
    int *adj = nullptr;
    int *rank = nullptr; // original id -> rank
    int *orig = nullptr; // rank -> original id
    unsigned *hubbits = nullptr;
    int64_t n = 0, m = 0, adj_entries = 0;
    int64_t max_deg = 0, max_out = 0;
    int n_hubs = 0, hub_stride = 0;
    int32_t labeled = 0, n_labels = 0;
    int device = 0;
    int num_sms = 0;
    // execution context used by launches on this graph: the graph's own one,
    // or (in server stream views) one per stream
    pg_exec exec0;
    pg_exec *ex = &exec0;
    bool is_view = false;
    // vertices with out-degree > heavy_min_built, by out-degree descending
    int *heavy = nullptr;
    int64_t n_heavy = 0;
    int heavy_min_built = PG_CLIQUE_LIGHT_D; // out-degree threshold of the heavy list
    // batched-kernel task split of the highest-degree ranks (see count_batched.cu)
    long long *split_prefix = nullptr;
    int n_split = 0;
    long long n_split_tasks = 0;
    int split_grain_built = 0;
    int servers = 0;                         // running servers holding views of this graph
    // last batch built by pg_count_ex for a plan list (keyed by plan serials)
    pg_batch *batch_cache = nullptr;
    std::vector<uint64_t> batch_key;
    int64_t bytes_device = 0;  // vinfo, adj, rank maps (hubs and heavy list: pg_graph_bytes)
    pg_tuning tune = pg_default_tuning();
    // launches take every sample_stride-th start vertex (timing samples of
    // pg_autotune only; 1 otherwise)
    int sample_stride = 1;
    // device work budget of the synchronous calls (pg_set_time_budget), ns; 0 = none
    unsigned long long budget_ns = 0;
    // task partition (pg_set_partition): launches take the tasks t with
    // t mod n_parts == part (one GPU's share of a multi-GPU count)
    int part = 0, n_parts = 1;
};

// Task selection of a launch: tasks offset, offset + stride, ... below n
// (timing samples and the task partition combined).
struct PgTaskSel {
    long long offset, stride;
    long long count(long long n) const { return n > offset ? (n - offset + stride - 1) / stride : 0; }
};
inline PgTaskSel pg_task_sel(const pg_graph *g) {
    PgTaskSel t;
    t.stride = (long long)(g->sample_stride > 1 ? g->sample_stride : 1) * (g->n_parts > 1 ? g->n_parts : 1);
    t.offset = g->n_parts > 1 ? g->part : 0;
    return t;
}

// Run control of a synchronous call on g: the graph's work budget (if any)
// and, for existence queries, a target.  Zeroes the control words on s.
// force: control words even without a target or budget (launches that may be
// stopped from the host)
int pg_run_ctl(pg_graph *g, unsigned long long target, cudaStream_t s, PgRunCtl *out, bool force = false);
// PG_ETIMEOUT if the launch behind ctl ran out of budget (synchronises s).
int pg_run_ctl_check(const PgRunCtl &ctl, cudaStream_t s);

#define PG_STATIC_SCRATCH_BYTES (32u << 20) // fixed scratch of pg_count_cliques_noalloc

struct pg_batch;

// pattern vertices of a plan (cliques above PGP_MAXK keep no pattern matrix)
inline int pg_plan_size(const PgPlanHost &h) { return h.big_clique ? h.clique_k : h.pat.k; }

struct pg_plan {
    PgPlanHost h;
    uint64_t serial = 0;         // unique per compiled plan (batch cache key)
    PgOrder *d_orders = nullptr; // device copy of h.orders
    PgOrder *d_list_orders = nullptr; // device copy of h.list_orders
    int kernel_auto = PG_KERNEL_GENERIC;
};

// error reporting (thread-local message)
int pg_set_error(int code, const std::string &msg);
int pg_cuda_error(cudaError_t e, const char *what);

#define PG_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return pg_cuda_error(_e, #call);        \
    } while (0)

#define PG_TRY(call)                                                   \
    do {                                                               \
        const int _rc = (call);                                        \
        if (_rc != PG_OK) return _rc;                                  \
    } while (0)

// Device memory of graphs, their load temporaries and execution arenas
// comes from a library memory pool per device (stream-ordered; freed memory
// stays with the pool up to 8 GiB, so repeated graph loads and arena growth
// reuse mapped memory).  pg_dalloc: *p on the current device, usable on
// stream s (and on other streams after s is synchronised).  pg_dfree:
// stream-ordered free on s; callers that may still have work on other
// streams synchronise first.  Memory from pg_dalloc is freed only by
// pg_dfree.
int pg_dalloc(void **p, size_t bytes, cudaStream_t s);
void pg_dfree(void *p, cudaStream_t s);

// graph.cu
int pg_graph_build(pg_graph *g, const int64_t *d_off, const int32_t *d_adj, int64_t nnz,
                   const int32_t *d_labels, cudaStream_t s);
int pg_graph_build_hubs(pg_graph *g, int min_degree, int max_hubs, cudaStream_t s);
int pg_graph_build_heavy(pg_graph *g, int heavy_min, cudaStream_t s);
int pg_graph_build_split(pg_graph *g, int grain, cudaStream_t s);
int64_t pg_graph_bytes(const pg_graph *g);

// scratch management (api.cu)
int pg_ensure_scratch(pg_graph *g, size_t bytes, cudaStream_t s);
int pg_plan_upload(pg_plan *p);

// count_generic.cu (persistent = dynamic task queue over a resident grid;
// otherwise one warp per task, one launch per pattern)
// ctl (may be null): existence mode (target) and work budget
int pg_launch_generic(pg_graph *g, const pg_plan *p, unsigned long long *counts_dev,
                      int queue_slot, bool persistent, cudaStream_t s, const PgRunCtl *ctl = nullptr);
size_t pg_generic_scratch_bytes(const pg_graph *g, const pg_plan *p, bool persistent);
// algorithmic operand elements of the plan's set operations and their number
// into out_dev[0], out_dev[1] (reserves its own scratch)
int pg_launch_operand_bytes(pg_graph *g, const pg_plan *p, unsigned long long *out_dev, cudaStream_t s);
// per-warp level buffers of a level program (offsets per level, total ints)
long long pg_level_layout(const pg_graph *g, const std::vector<PgOrder> &orders, bool listing, long long *off);

// match_list.cu: listing of the matches whose start vertex has rank in
// [rank_begin, rank_end); rows of k original ids (-1 at anti-vertices)
int pg_launch_match(pg_graph *g, const pg_plan *p, int64_t rank_begin, int64_t rank_end, int32_t *out,
                    unsigned long long capacity, unsigned long long *n_total_dev, cudaStream_t s,
                    const PgRunCtl *ctl = nullptr);
size_t pg_match_scratch_bytes(const pg_graph *g, const pg_plan *p);

// count_clique.cu: sizes kmin..kmax in one launch, counts_dev[2*(k-kmin)]
// (sizes up to PG_MAX_CLIQUE; ctl: existence mode / work budget, may be null)
int pg_launch_clique(pg_graph *g, int kmin, int kmax, unsigned long long *counts_dev,
                     int queue_slot, cudaStream_t s, const PgRunCtl *ctl = nullptr);
size_t pg_clique_scratch_bytes(const pg_graph *g, int kmax);
// non-persistent form, one size per launch pair (PG_KERNEL_CLIQUE_NONPERSISTENT)
int pg_launch_clique_plain(pg_graph *g, int k, unsigned long long *counts_dev, cudaStream_t s);
size_t pg_clique_slab_bytes(const pg_graph *g, int kmax);

// fsm.cu
int pg_fsm_run(pg_graph *g, int max_edges, unsigned long long threshold, pg_fsm_pattern *out, int64_t capacity,
               int64_t *n_frequent, cudaStream_t s);

// fsm_general.cu
int pg_fsm_general_run(pg_graph *g, int max_edges, unsigned long long threshold, pg_fsm_general_pattern *out,
                       int64_t capacity, int64_t *n_frequent, cudaStream_t s);

// labeled_motifs.cu
int pg_labeled_motif3_run(pg_graph *g, pg_labeled_count *out, int64_t capacity, int64_t *n_out, cudaStream_t s);
// labeled_motifs4.cpp
int pg_labeled_motif4_run(pg_graph *g, pg_labeled_count4 *out, int64_t capacity, int64_t *n_out, cudaStream_t s);

// count_batched.cu: many plans in one launch (prefix trees, task groups)
int pg_batch_build(pg_plan *const *plans, int n_plans, int flags, pg_batch **out);
int pg_batch_build_trie(pg_batch *b);
#define PG_BATCH_HOST_ONLY 0x100 // internal flag: build the tree only, stage later
int pg_batch_upload(pg_batch *b);
int pg_batch_stage(pg_batch *b, void *dev_area, void *host_area, size_t area_bytes, cudaStream_t s);
void pg_batch_free(pg_batch *b);
void pg_batch_stats(const pg_batch *b, int *nodes, int *programs, int *levels_total);
int pg_batch_slots(const pg_batch *b);
bool pg_batch_labeled(const pg_batch *b);
size_t pg_batch_scratch_bytes(const pg_graph *g, const pg_batch *b);
int pg_launch_batched(pg_graph *g, const pg_batch *b, unsigned long long *counts_dev, int queue_slot,
                      cudaStream_t s, const PgRunCtl *ctl = nullptr);
// count_c4.cu: edge-induced 4-cycles by co-degree accumulation (adds into
// the 128-bit count_dev; queue words queue_slot .. queue_slot + 2)
int pg_launch_c4(pg_graph *g, unsigned long long *count_dev, int queue_slot, cudaStream_t s, const PgRunCtl *ctl);
size_t pg_c4_scratch_bytes(const pg_graph *g);
int pg_launch_clique_on(pg_graph *g, int kmin, int kmax, unsigned long long *counts_dev,
                        unsigned long long *queue, void *slabs, long long max_warps, cudaStream_t s);
