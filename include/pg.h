/*
 * pg.h - C-ABI of the pattern-aware subgraph matching library (libpg.so).
 *
 * The library implements the matching engine of Peregrine (Jamshidi, Mahadasa,
 * Vora, "Peregrine: A Pattern-Aware Graph Mining System", EuroSys 2020) on one
 * CUDA device: a host plan compiler turns a pattern into an exploration plan
 * (Section 4.1, "Computing exploration plan" figure) and CUDA kernels extend
 * every start vertex of a device-resident graph along that plan (Section 5.1,
 * "Pattern-Aware Processing Model" figure), counting matches exactly
 * (128-bit counters returned as two uint64 words).
 *
 * Conventions for every entry point:
 *  - Return value: PG_OK (0) on success, otherwise one of the PG_E* codes.
 *    pg_last_error() then gives a human-readable message for the calling
 *    host thread.  No entry point aborts the process.
 *  - Pointers documented as "host" must be readable by the CPU; "device"
 *    pointers must be CUDA device (or managed) memory of the current device.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Functions documented as asynchronous only enqueue work on it.
 *  - Objects returned through `**out` are owned by the caller and released
 *    with the matching pg_free_* function.
 *  - Vertex ids are int32 (n < 2^31); adjacency offsets are int64.
 *  - The library allocates its own device memory with cudaMalloc for graphs,
 *    plans and scratch, and frees it in the pg_free_* calls.
 *  - One graph handle holds one scratch arena and one set of work-queue and
 *    count words: calls on the same graph must be ordered (one stream, or
 *    synchronised between streams).  For concurrent queries on one resident
 *    graph use the server (pg_server_*), which gives each of its streams its
 *    own arena, or load the graph once per stream.
 */
#ifndef PG_H
#define PG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define PG_OK 0
#define PG_EINVAL 1    /* malformed argument: bad CSR, bad pattern, size limit */
#define PG_ENOMEM 2    /* host or device allocation failed */
#define PG_ETRUNC 3    /* output buffer too small (match listing); totals still valid */
#define PG_ETIMEOUT 4  /* a kernel's work budget ran out; partial results discarded */
#define PG_EDEVICE 5   /* CUDA runtime error (launch failure, no device, ...) */
#define PG_EUNSUPPORTED 6 /* valid request that this build does not implement */
#define PG_ECANCELED 7 /* the query was cancelled (pg_server_cancel) */

#define PG_MAX_PATTERN 8 /* pattern vertices, regular plus anti-vertices */
#define PG_MAX_CLIQUE 16 /* k-cliques (unlabeled complete patterns) up to this size */

typedef struct pg_graph pg_graph; /* device-resident data graph (opaque) */
typedef struct pg_plan pg_plan;   /* compiled exploration plan (opaque, host) */
typedef struct pg_batch pg_batch; /* several plans merged for one launch (opaque) */

/*
 * Pattern description (Section 3.1, "Pattern Interface" figure; anti-edges
 * Section 3.1.1; anti-vertices Section 3.1.2; vertex-induced matching
 * Section 3.1.3).  Pattern vertices are 0..k-1.
 *   edges        n_edges pairs (u, v), u != v.
 *   anti_edges   n_anti pairs (u, v): m(u) and m(v) must not be adjacent.
 *   labels       k labels, -1 = any label; NULL = unlabeled pattern.
 *   anti_vertex  k flags (1 = anti-vertex: never matched, only its anti-edges
 *                constrain the match); NULL = none.  For an anti-vertex a
 *                with regular neighbours N(a) (the vertices it has
 *                anti-edges to) a match is valid only if no data vertex lies
 *                in adj(m(u)) for every u in N(a) apart from the images of
 *                the pattern neighbours of N(a) (Section 3.1.2).  An
 *                anti-vertex has anti-edges only, to regular vertices only,
 *                and no label (PG_EINVAL otherwise).  Anti-vertex patterns
 *                run on PG_KERNEL_GENERIC (batches refuse them with
 *                PG_EUNSUPPORTED).
 *   vertex_induced  1: every non-adjacent pair of regular vertices becomes
 *                an anti-edge (the Theorem of Section 3.1.3).
 * All arrays are host memory, read during pg_compile_pattern only.
 */
typedef struct {
    int32_t k;
    int32_t n_edges;
    const int32_t *edges;
    int32_t n_anti;
    const int32_t *anti_edges;
    const int32_t *labels;
    const uint8_t *anti_vertex;
    int32_t vertex_induced;
} pg_pattern_desc;

/* Pattern-set construction from descriptions and element access (see the
 * pattern generators below). */
typedef struct pg_pattern_set pg_pattern_set;
int pg_patterns_from(const pg_pattern_desc *descs, int64_t n, pg_pattern_set **out);
int pg_patterns_get(const pg_pattern_set *s, int64_t i, int32_t *k, int32_t *n_edges, int32_t *edges,
                    int32_t *vertex_induced);

/*
 * Pattern generators (Section 3.1, "Pattern Interface" figure:
 * generateAllVertexInduced, generateAllEdgeInduced, extendByVertex,
 * extendByEdge).  A pattern set is a host object holding unlabeled patterns
 * without anti-edges or anti-vertices, one per isomorphism class.
 *   pg_patterns_all     vertex_induced = 1: every connected pattern on
 *                       `size` vertices (1..7), flagged vertex-induced;
 *                       0: every connected pattern with `size` edges (1..7),
 *                       edge-induced.
 *   pg_patterns_from    a set from n descriptions (isomorphic ones merged).
 *   pg_patterns_extend  by_vertex = 1: add one vertex joined to any
 *                       non-empty subset of a pattern's vertices; 0: add one
 *                       edge between two non-adjacent vertices or to a new
 *                       vertex.  Results over all input patterns, merged by
 *                       isomorphism; patterns already at 8 vertices only get
 *                       edges.  The vertex-induced flag is kept.
 *   pg_patterns_get     pattern i: k, its edges as pairs u < v into `edges`
 *                       (room for 2 * 28 ints), and the flag.
 * Host only.  Errors: PG_EINVAL (size out of range, labeled or anti-edged
 * input, index out of range), PG_ENOMEM.
 */
int pg_patterns_all(int32_t size, int32_t vertex_induced, pg_pattern_set **out);
int pg_patterns_extend(const pg_pattern_set *in, int32_t by_vertex, pg_pattern_set **out);
int pg_patterns_size(const pg_pattern_set *s, int64_t *n);
void pg_free_patterns(pg_pattern_set *s);

/* Graph facts after loading (all counts of the undirected simple graph). */
typedef struct {
    int64_t n;           /* vertices */
    int64_t m;           /* undirected edges */
    int64_t max_degree;
    int64_t max_out_degree; /* neighbours of higher degree rank (Section 5.2 order) */
    int64_t device_bytes;   /* device memory held by the graph */
    int32_t labeled;
    int32_t n_labels;       /* 1 + largest label, 0 if unlabeled */
} pg_graph_info;

/* Plan facts for inspection and tests. */
typedef struct {
    int32_t k;               /* pattern vertices (regular + anti) */
    int32_t n_regular;
    uint64_t automorphisms;  /* |Aut| restricted to regular vertices */
    int32_t n_po;            /* symmetry-breaking pairs, po[i] = (a, b) means m(a) < m(b) */
    int32_t po[2 * 28];
    uint32_t core_mask;      /* bit u set: pattern vertex u is in the core p_C */
    int32_t n_orders;        /* matching orders (valid core vertex sequences) */
    int32_t n_levels;        /* levels per order: core + enumerated non-core + counted */
    int32_t counted_group;   /* size of the non-core group counted by C(|S|, g) */
    int32_t kernel;          /* PG_KERNEL_* the automatic dispatch would choose */
    double compile_ms;       /* host time spent in pg_compile_pattern */
} pg_plan_info;

/* Kernel families for pg_count_ex. */
#define PG_KERNEL_AUTO 0
#define PG_KERNEL_GENERIC 1       /* plan interpreter, any pattern */
#define PG_KERNEL_CLIQUE_PLAIN 2  /* plan interpreter, one warp per task, one launch per pattern */
#define PG_KERNEL_CLIQUE 3        /* k-clique, persistent, bitmap sub-graph */
#define PG_KERNEL_BATCHED 4       /* all plans in one launch (pg_compile_batch) */
#define PG_KERNEL_CLIQUE_NONPERSISTENT 5 /* k-clique bitmap kernel without persistence: one warp per
                                            start vertex (one CTA per heavy one), one launch pair
                                            per pattern -- the plain form of PG_KERNEL_CLIQUE */

/*
 * pg_load_graph - make a data graph resident on the current device.
 * Section 5.5 (adjacency lists) and Section 5.2 (degree ordering).
 *   offsets  int64[n+1], adj int32[nnz]: an undirected simple graph in CSR
 *            form, every list sorted strictly ascending, no self loops, every
 *            edge present in both directions (nnz = 2m).
 *   labels   int32[n] vertex labels >= 0, or NULL.
 *   inputs_on_device  0: offsets/adj/labels are host memory (copied in);
 *            1: they are device memory (read, not kept).
 *   stream   stream for the copies and the relabelling kernels; the call
 *            synchronises it before returning.
 * The library relabels vertices by (degree descending, id ascending), so that
 * lower ids mean higher degree, rewrites and re-sorts every list in the new
 * ids and pads each list to 16 bytes.  Results never expose the new ids
 * except through pg_graph_rank.
 * Errors: PG_EINVAL (n < 0, nnz mismatch, unsorted list, self loop,
 * asymmetric edge, vertex id out of range, negative label), PG_ENOMEM,
 * PG_EDEVICE.
 */
int pg_load_graph(const int64_t *offsets, int64_t n, const int32_t *adj, int64_t nnz,
                  const int32_t *labels, int32_t inputs_on_device, void *stream,
                  pg_graph **out);

/* pg_graph_get_info - facts about a loaded graph (host struct out). */
int pg_graph_get_info(const pg_graph *g, pg_graph_info *out);

/* pg_graph_rank - copy the relabelling to host: rank_out[v] = new id of
 * original vertex v (int32[n], host).  Synchronous. */
int pg_graph_rank(const pg_graph *g, int32_t *rank_out);

/* pg_free_graph - release the graph's device memory (NULL is a no-op). */
void pg_free_graph(pg_graph *g);

/*
 * pg_compile_pattern - build the exploration plan of a pattern (Section 4.1
 * "Computing exploration plan" figure; anti-edges Section 4.2; anti-vertices
 * Section 4.3): automorphisms, symmetry-breaking partial order, minimum
 * connected vertex cover as the core, matching orders, and the per-level set
 * operations of the core and of the non-core completion.  Host only; touches
 * no graph.
 * A pattern of 9..PG_MAX_CLIQUE vertices is accepted only as an unlabeled
 * clique (every pair an edge; no anti-edges, labels or anti-vertices): its
 * plan is the clique's total order u0 < ... < u(k-1) and it runs on the
 * k-clique kernel only (pg_count, pg_count_ex with PG_KERNEL_AUTO or
 * PG_KERNEL_CLIQUE, pg_count_until, pg_autotune); every other call refuses
 * it with PG_EUNSUPPORTED.
 * Errors: PG_EINVAL (k outside 1..8 for non-cliques or above PG_MAX_CLIQUE,
 * self loop, pair both edge and anti-edge, regular vertices not connected by
 * edges, anti-vertex with a true edge or with no anti-edge), PG_ENOMEM.
 */
int pg_compile_pattern(const pg_pattern_desc *desc, pg_plan **out);

/* pg_plan_get_info - inspect a plan (host struct out). */
int pg_plan_get_info(const pg_plan *p, pg_plan_info *out);

/* pg_plan_describe - the plan as text: automorphism count, partial order,
 * core, and per matching order the level program (for every level: bound
 * pattern vertex, intersected / subtracted / bounding / excluded earlier
 * levels, label, counted group size).  Writes at most `size` bytes including
 * the terminating NUL into host buffer `buf`; PG_ETRUNC if it did not fit. */
int pg_plan_describe(const pg_plan *p, char *buf, int64_t size);

/* pg_free_plan - release a plan and its device copies (NULL is a no-op). */
void pg_free_plan(pg_plan *p);

/*
 * pg_count - number of distinct matches of each plan's pattern in the graph
 * (Section 3.2: count() is match() with an incrementing callback).
 *   plans       n_plans compiled plans (host array of handles), n_plans <= 64.
 *   counts_out  uint64[2 * n_plans], host: count i is the 128-bit integer
 *               counts_out[2i] + 2^64 * counts_out[2i+1] (exact; star counts
 *               on hub-heavy graphs exceed 2^64).
 * Synchronous: returns after the counts are on the host.  Kernel choice is
 * automatic (PG_KERNEL_AUTO).  With a work budget on the graph
 * (pg_set_time_budget) the kernels stop once it is spent and the call returns
 * PG_ETIMEOUT without counts.  Errors: PG_EINVAL, PG_ENOMEM, PG_EDEVICE,
 * PG_ETIMEOUT, PG_EUNSUPPORTED (a clique above 8 vertices on a graph with
 * out-degrees of 65536 or more).
 */
int pg_count(pg_graph *g, pg_plan *const *plans, int32_t n_plans, uint64_t *counts_out,
             void *stream);

/*
 * pg_count_ex - asynchronous counting with an explicit kernel family.
 *   counts_dev  uint64[2 * n_plans], device, same (low, high) layout as
 *               pg_count; the call zeroes it on `stream` and the kernels add
 *               into it.
 *   kernel      PG_KERNEL_*; PG_EINVAL if the family cannot run these plans
 *               (e.g. PG_KERNEL_CLIQUE for a non-clique).
 * Only enqueues work (no host synchronisation, no allocation once the
 * graph's scratch has been sized by a first call with the same plans), so a
 * sequence of calls can be captured in a CUDA graph after one warm-up call.
 * The graph's work budget does not apply (the call cannot report it).
 */
int pg_count_ex(pg_graph *g, pg_plan *const *plans, int32_t n_plans, uint64_t *counts_dev,
                int32_t kernel, void *stream);

/*
 * pg_count_until - count one plan's matches until `target` of them are found
 * (existence queries, Section 3.2.3, with early termination, Section 5.4).
 * Warps add their counts to a device total after every task; the first that
 * sees the total reach `target` raises a device stop flag, which the others
 * poll between tasks and between first-level candidates, so exploration ends
 * soon after the target is met.
 *   target     >= 1 (1 = "does a match exist?").
 *   count_out  host uint64[2], (low, high): the number of matches found
 *              before exploration stopped.  Exact when *reached is 0 (the
 *              whole graph was explored); otherwise a partial count >= target.
 *   reached    host: 1 if at least `target` matches exist, else 0.
 * Unlabeled cliques (3..PG_MAX_CLIQUE vertices, e.g. the 14-clique existence
 * query of the paper's evaluation) run on the k-clique kernel, which
 * publishes its count after every first-level row of the start vertex's
 * sub-graph and, inside a row, at every candidate of the traversal's first
 * three levels, and cuts branches too small to reach k; other patterns run on
 * the plan interpreter (PG_KERNEL_GENERIC).  Honours the graph's work budget
 * (PG_ETIMEOUT).  Synchronous.  Errors: PG_EINVAL (target 0, NULL argument,
 * labeled pattern on an unlabeled graph), PG_ENOMEM, PG_EDEVICE, PG_ETIMEOUT.
 */
int pg_count_until(pg_graph *g, pg_plan *p, uint64_t target, uint64_t *count_out, int32_t *reached,
                   void *stream);

/*
 * pg_plan_operand_bytes - measurement aid: the algorithmic bytes of plan p
 * on graph g, i.e. 4 bytes times the length of every operand of every set
 * operation the plan's level program performs, each operand being an
 * adjacency list cut to the level's partial-order range (Section 4.1
 * bounds; Section 4.2 differences touch their lists too), summed over every
 * (start vertex, matching order) task, every bound prefix and every level,
 * the counted last level included (Section 5.1 processing model).  This is
 * the work a sorted-list implementation of the plan must read, whatever a
 * kernel does instead; a roofline divides it by a kernel's time.  Computed
 * by a dedicated device walk over the same prefixes as the interpreter
 * kernel (it counts no matches).  Honours pg_set_partition.
 *   bytes_out  host uint64: the algorithmic bytes.
 *   ops_out    host uint64: the number of set operations.
 * Synchronous.  Errors: PG_EINVAL (NULL argument, labeled pattern on an
 * unlabeled graph), PG_EUNSUPPORTED (cliques above 8 vertices), PG_ENOMEM,
 * PG_EDEVICE.
 */
int pg_plan_operand_bytes(pg_graph *g, pg_plan *p, uint64_t *bytes_out, uint64_t *ops_out, void *stream);

/*
 * pg_clustering_coefficient_above - the clustering-coefficient program of
 * Section 3.2.3: whether the global clustering coefficient 3T / W of g
 * exceeds `bound`, with W = connected triples (3-vertex star matches,
 * counted exactly) and T = triangles, counted only until 3T > bound * W is
 * established (pg_count_until).  Outputs (host): *answer 1 or 0;
 * triangles_out[2] = (low, high) triangles counted before the stop (exact
 * when *answer is 0); wedges_out[2] = (low, high) W.  The paper counts
 * "triplets" as twice the star matches; this call uses the standard 3T / W
 * (1 on a complete graph).  Synchronous.  Errors: PG_EINVAL (NULL argument,
 * negative or non-finite bound), PG_ENOMEM, PG_EDEVICE, PG_ETIMEOUT.
 */
int pg_clustering_coefficient_above(pg_graph *g, double bound, int32_t *answer, uint64_t *triangles_out,
                                    uint64_t *wedges_out, void *stream);

/*
 * pg_set_partition - count only this GPU's share of the tasks: the counting
 * kernels (pg_count, pg_count_ex, pg_count_batch, pg_count_until, the
 * k-clique no-allocation entry point) take the tasks t with
 * t mod n_parts == part, where tasks are start vertices in degree-rank order
 * (Section 5.1 tasks; hub start vertices split into several tasks, and
 * (start vertex, matching order) pairs on the interpreter).  Every match
 * belongs to exactly one task, so the counts of parts 0..n_parts-1 on
 * copies of the same graph sum to the full count (the multi-GPU split: one
 * sum all-reduce of the counters).  Interleaving by rank deals hubs evenly.
 * (0, 1) restores the whole graph.  Listing (pg_match), FSM and labeled
 * motifs ignore the partition.  Host only.  Errors: PG_EINVAL (NULL graph,
 * part outside 0..n_parts-1, a server running on the graph).
 */
int pg_set_partition(pg_graph *g, int32_t part, int32_t n_parts);

/*
 * pg_set_time_budget - device work budget of the synchronous calls on g
 * (pg_count, pg_count_until, pg_match, pg_match_range): budget_ms > 0 limits
 * each call's kernels to about that much device time, 0 removes the limit.
 * The persistent kernels read %globaltimer between tasks and between
 * first-level candidates, so a launch ends within one such step of the
 * budget; the call then returns PG_ETIMEOUT and its partial results are
 * discarded.  The paper has no counterpart (its runtime runs a program to
 * completion); this bounds a query on a resident graph without killing the
 * process or the device context.  Host only.  Errors: PG_EINVAL (NULL graph,
 * negative or non-finite budget).
 * pg_get_time_budget - the current budget in milliseconds (host double out).
 */
int pg_set_time_budget(pg_graph *g, double budget_ms);
int pg_get_time_budget(const pg_graph *g, double *budget_ms);

/*
 * pg_match - list the distinct matches of one plan's pattern (Section 3.2,
 * match(G, p, f): the callback f becomes an output array).
 *   out_dev   int32[capacity * k], device, caller-owned: row r holds one
 *             match, column u the ORIGINAL id of the data vertex matched to
 *             pattern vertex u (-1 in anti-vertex columns).  One row per
 *             match (one representative per automorphism class, the one the
 *             symmetry-breaking partial order of Section 4.1 keeps); row
 *             order is unspecified.
 *   capacity  rows available in out_dev (0 with out_dev NULL only counts).
 *   n_total   host uint64: the number of matches, whatever the capacity.
 * Synchronous (returns after *n_total is on the host).  If n_total exceeds
 * capacity the first `capacity` rows are valid, distinct matches and the call
 * returns PG_ETRUNC.  Honours the graph's work budget (PG_ETIMEOUT; rows
 * written before the stop are valid matches, the total is not).  Errors:
 * PG_EINVAL (NULL argument, labeled pattern on an unlabeled graph),
 * PG_ETRUNC, PG_ENOMEM, PG_EDEVICE, PG_ETIMEOUT.
 */
int pg_match(pg_graph *g, pg_plan *p, int32_t *out_dev, uint64_t capacity, uint64_t *n_total,
             void *stream);

/*
 * pg_match_range - pg_match restricted to the matches whose start vertex (the
 * data vertex of the first matching-order position, Section 5.1 task) has
 * degree rank in [rank_begin, rank_end), 0 <= rank_begin <= rank_end <= n.
 * Disjoint ranges list disjoint sets of matches whose union over a partition
 * of [0, n) is the full listing, so a result larger than one buffer can be
 * paged range by range.  Same output and errors as pg_match, plus PG_EINVAL
 * for a range outside [0, n].
 */
int pg_match_range(pg_graph *g, pg_plan *p, int64_t rank_begin, int64_t rank_end, int32_t *out_dev,
                   uint64_t capacity, uint64_t *n_total, void *stream);

/*
 * pg_count_cliques_noalloc - k-clique counts for every k in kmin..kmax
 * (3 <= kmin <= kmax <= 8), computed by the same kernel as PG_KERNEL_CLIQUE,
 * without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate while they count,
 * e.g. a process whose device memory is reserved up front by another
 * allocator (where a cudaMalloc at query time can fail or fragment the pool)
 * or a latency-bound caller that cannot take the implicit synchronisation of
 * cudaMalloc / cudaFree.
 *   g           a graph loaded earlier (its memory was allocated at load).
 *   counts_dev  uint64[2 * (kmax - kmin + 1)], device, caller-owned: the
 *               (low, high) words of the count of k-cliques at index
 *               2 * (k - kmin); zeroed by the call on `stream`.
 * Scratch comes from a fixed 32 MiB array compiled into the library (every
 * device that loads libpg holds it until the process exits).  The first call
 * on a device looks the array's device address up (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * With the CUDA runtime's lazy module loading (its default) that first call
 * is also when the array's 32 MiB (and the kernel's code) are reserved on
 * the device: a caller that hands the rest of device memory to a pool
 * should make one call at start-up, before filling the pool.  The address
 * is kept for the life of the process; after cudaDeviceReset the library's
 * state on that device (graphs, this address) is invalid.
 * All calls share the array and each call clears what must start at zero, so
 * calls that overlap on the GPU (other streams, other host threads) race:
 * serialise them.  Asynchronous: only enqueues work on `stream`.
 * Errors: PG_EINVAL (NULL argument, bad sizes, graph on another device, or a
 * graph whose maximum out-degree needs per-block slabs that do not fit the
 * array for at least one block per SM: roughly out-degree above 1300 on a
 * 148-SM B300), PG_EDEVICE.  Never calls cudaMalloc or cudaFree.
 */
int pg_count_cliques_noalloc(pg_graph *g, int32_t kmin, int32_t kmax, uint64_t *counts_dev,
                             void *stream);

/*
 * pg_compile_batch - the matching-order programs of n_plans plans (1..64)
 * for a single launch (Section 5.1 processing model applied to several
 * patterns at once).  The programs of one counted pattern form a prefix
 * tree (shared candidate sets of identical level prefixes); by default each
 * counted pattern is a task group of its own, the launch's warps taking the
 * (pattern, start vertex) tasks pattern by pattern, so that the warps on an
 * SM mostly run one pattern's code at a time.  Host object with a device
 * copy on the current device; plans may be freed afterwards.
 *   flags  PG_BATCH_EXPAND_ANTI: count a plan with anti-edges (no
 *          anti-vertices, at most 6 anti-edges) as the signed sum over its
 *          edge-induced supergraphs, maps(E, A) = sum over T in A of
 *          (-1)^|T| maps(E + T) (inclusion-exclusion over anti-edges, the
 *          pattern-level form of Section 4.2's set differences; with the
 *          Theorem of Section 3.1.3 it covers vertex-induced patterns);
 *          isomorphic terms of all plans are counted once.  0: anti-edges
 *          are applied as set differences inside each plan.
 *          PG_BATCH_SHARE_PREFIXES: merge the programs of all counted
 *          patterns into one prefix tree walked once per start vertex
 *          (candidate sets of identical prefixes computed once for all).
 * At most 64 distinct counted patterns per batch after expansion.
 * Errors: PG_EINVAL, PG_EUNSUPPORTED (too many counted patterns),
 * PG_ENOMEM, PG_EDEVICE.
 */
#define PG_BATCH_EXPAND_ANTI 1
#define PG_BATCH_SHARE_PREFIXES 2
int pg_compile_batch(pg_plan *const *plans, int32_t n_plans, int32_t flags, pg_batch **out);

/* pg_batch_get_info - tree nodes, merged programs, and the total number of
 * levels of the programs before merging (host ints out). */
int pg_batch_get_info(const pg_batch *b, int32_t *n_nodes, int32_t *n_programs, int32_t *n_levels_total);

/*
 * pg_count_batch - counts of every plan of the batch in one persistent
 * launch.  counts_dev: uint64[2 * n_plans] device, (low, high) words in the
 * plans' order; zeroed on `stream`.  Asynchronous; allocates only when the
 * graph's scratch arena must grow (first call for this batch size).
 * Errors: PG_EINVAL (labeled plan on unlabeled graph), PG_ENOMEM, PG_EDEVICE.
 */
int pg_count_batch(pg_graph *g, const pg_batch *b, uint64_t *counts_dev, void *stream);

/* pg_free_batch - release a batch (NULL is a no-op). */
void pg_free_batch(pg_batch *b);

/*
 * Launch parameters of the persistent kernels, held per graph.  The paper
 * fixes its runtime's task granularity by hand (Section 5.5); this library
 * exposes the equivalent knobs and tunes them on the graph at hand.
 *   clique_chunk          start vertices a warp takes per work-queue grab in
 *                         the k-clique kernel (1..64; default 4).
 *   clique_blocks_per_sm  CTAs per SM of the k-clique kernel (0 = as many as
 *                         fit; larger values are clamped to that).
 *   clique_heavy_min      start vertices with out-degree above this get a
 *                         whole CTA, the rest one warp (8..64; default 64).
 *   batched_warps         warps per CTA of the batched kernel (2, 4 or 8;
 *                         default 4).
 *   batched_chunk         start vertices per work-queue grab (1..64; default 1).
 *   batched_blocks_per_sm CTAs per SM (0 = as many as fit).
 *   hub_min_degree        vertices of at least this degree get a membership
 *   hub_max               bitmap row, at most hub_max of them (highest degree
 *                         first; defaults 1024 and 512; hub_max 0 = none).
 *   batched_split_grain   a start vertex of degree d > grain becomes
 *                         ceil(d / grain) batched-kernel tasks (at most 1024)
 *                         that share its first-level candidates, so that hub
 *                         start vertices do not serialise on one warp
 *                         (0 = no split; default 512).
 *   batched_regcap        register cap of the batched kernel: 1 = 64
 *                         registers per thread (more resident warps, some
 *                         spilling), 2 = about 100, 0 = the compiler's
 *                         choice (default).
 *   clique_min_blocks     k-clique kernel variant: 3 CTAs per SM (80
 *                         registers, default) or 4 (64 registers, some
 *                         spilling).
 *   pad                   0.
 */
typedef struct {
    int32_t clique_chunk;
    int32_t clique_blocks_per_sm;
    int32_t clique_heavy_min;
    int32_t batched_warps;
    int32_t batched_chunk;
    int32_t batched_blocks_per_sm;
    int32_t hub_min_degree;
    int32_t hub_max;
    int32_t batched_split_grain;
    int32_t batched_regcap;
    int32_t clique_min_blocks;
    int32_t pad;
} pg_tuning;

/* Outcome of pg_autotune. */
typedef struct {
    pg_tuning chosen;     /* now in effect on the graph */
    double default_ms;    /* timed launch with the parameters in effect before */
    double tuned_ms;      /* best timed launch of the search (same sample) */
    double full_default_ms; /* sample_stride > 1 and a different choice: full */
    double full_tuned_ms;   /* launches with the old and the chosen parameters; the
                               chosen ones are kept only if faster (else -1) */
    double wall_ms;       /* host time of the whole search */
    int32_t trials;       /* configurations timed */
    int32_t kernel;       /* PG_KERNEL_* family tuned (CLIQUE or BATCHED) */
    int32_t sample_stride;
    int32_t pad;
} pg_tune_report;

/* pg_get_tuning / pg_set_tuning - read or replace a graph's launch
 * parameters.  Setting rebuilds the hub bitmaps or the heavy-vertex list when
 * their knobs change (synchronous).  Counts never depend on these values.
 * Errors: PG_EINVAL (value out of range), PG_ENOMEM, PG_EDEVICE. */
int pg_get_tuning(const pg_graph *g, pg_tuning *out);
int pg_set_tuning(pg_graph *g, const pg_tuning *t, void *stream);

/*
 * pg_autotune - choose the launch parameters for counting `plans` on `g` by
 * measurement, and keep them on the graph.  The kernel family is the one
 * PG_KERNEL_AUTO picks for these plans (k-clique or batched; other families
 * have nothing to tune and return PG_EUNSUPPORTED).  Coordinate descent over
 * the family's knobs: each value is timed with CUDA events on `stream` (one
 * untimed launch, then the best of two), the best kept before the next knob.
 * sample_stride >= 1 times only every sample_stride-th task (in rank
 * order), so a workload whose full launch takes seconds is tuned in
 * proportionally less time; 1 times the full launch.  A choice made on a
 * sample is then timed against the previous parameters on the full launch
 * and kept only if faster.  Synchronous; report
 * (host) may be NULL.  Errors: PG_EINVAL, PG_EUNSUPPORTED, PG_ENOMEM,
 * PG_EDEVICE.
 */
int pg_autotune(pg_graph *g, pg_plan *const *plans, int32_t n_plans, int32_t sample_stride,
                pg_tune_report *report, void *stream);

/*
 * pg_fsm - labeled frequent subgraph mining with MNI support (Section 2.1
 * FSM and minimum node image support; Section 3.2 "FSM" program with label
 * discovery; Section 5.5 domains).  Finds every connected labeled pattern
 * with 1..max_edges edges (max_edges <= 3) whose MNI support (the smallest,
 * over pattern vertices, number of distinct data vertices that vertex maps
 * to in edge-induced matches) is >= threshold.  MNI support is
 * anti-monotone, so this is the set the paper's extend-by-edge loop returns.
 *   out        host array of `capacity` records, filled in canonical order
 *              (shape, then labels); *n_frequent = size of the frequent set.
 * Shapes and canonical label tuples (pattern vertices in tuple order):
 *   PG_FSM_EDGE     (x, y), x <= y            edge 0-1
 *   PG_FSM_WEDGE    (c, x, y), x <= y         centre 0, leaves 1, 2
 *   PG_FSM_TRIANGLE (x, y, z), sorted         triangle 0-1-2
 *   PG_FSM_PATH     (a, b, c, d) = min of the tuple and its reverse, path 0-1-2-3
 *   PG_FSM_STAR     (c, x, y, z), x <= y <= z  centre 0, leaves 1, 2, 3
 * Unused label slots are -1.  Synchronous.  Needs a labeled graph with at
 * most 32 labels.  Errors: PG_EINVAL, PG_EUNSUPPORTED (> 32 labels),
 * PG_ETRUNC (capacity too small; *n_frequent still exact), PG_ENOMEM,
 * PG_EDEVICE.
 */
#define PG_FSM_EDGE 1
#define PG_FSM_WEDGE 2
#define PG_FSM_TRIANGLE 3
#define PG_FSM_PATH 4
#define PG_FSM_STAR 5
typedef struct {
    int32_t shape;
    int32_t labels[4];
    int32_t pad;
    uint64_t support;
} pg_fsm_pattern;

int pg_fsm(pg_graph *g, int32_t max_edges, uint64_t threshold, pg_fsm_pattern *out, int64_t capacity,
           int64_t *n_frequent, void *stream);

/*
 * pg_fsm_general - labeled frequent subgraph mining for any number of edges
 * (Section 3.2 FSM program: match, keep the patterns whose MNI support
 * (Section 2.1) is >= threshold, extendByEdge the survivors with label
 * discovery (Section 3.2.1), repeat; MNI is anti-monotone, so candidates
 * with an infrequent connected sub-pattern are never matched).  Domains are
 * decided vertex by vertex on the GPU: for each candidate and each orbit of
 * its automorphism group, one warp per data vertex with the orbit's label
 * searches for one match that binds the orbit's vertex to it and stops at
 * the first (Section 5.5 domains; a candidate leaves as soon as one of its
 * domains is below the threshold).  Supports are exact.
 *   max_edges  1..PG_FSM_MAX_EDGES (patterns up to 8 vertices).
 *   out        host array of `capacity` records, sorted by edge count then
 *              canonical form: vertices 0..k-1 with their labels, edges as
 *              pairs u < v, and the MNI support.  *n_frequent = size of the
 *              frequent set (exact even when capacity is short).
 * For max_edges <= 3 the frequent set equals pg_fsm's (a second,
 * independent GPU path).  Needs a labeled graph.  Synchronous; allocates
 * its buffers.  Errors: PG_EINVAL (unlabeled graph, max_edges or threshold
 * out of range), PG_ETRUNC, PG_ENOMEM, PG_EDEVICE.
 */
#define PG_FSM_MAX_EDGES 7
typedef struct {
    int32_t k;        /* pattern vertices */
    int32_t n_edges;
    int32_t edges[2 * PG_FSM_MAX_EDGES];
    int32_t labels[PG_MAX_PATTERN]; /* -1 past k */
    uint64_t support;
} pg_fsm_general_pattern;
int pg_fsm_general(pg_graph *g, int32_t max_edges, uint64_t threshold, pg_fsm_general_pattern *out,
                   int64_t capacity, int64_t *n_frequent, void *stream);

/*
 * pg_labeled_motif3 - labeled 3-motifs with label discovery (the paper's
 * labeled motif workload, Section 6; labels discovered from the matches,
 * Section 3.2.1): the number of vertex-induced matches of every labeled
 * triangle and wedge present in the graph.
 *   out        host array of `capacity` records, filled in no particular
 *              order: shape PG_FSM_TRIANGLE with labels (a, b, c) sorted, or
 *              PG_FSM_WEDGE with labels (centre, x, y), x <= y; count as a
 *              128-bit (low, high) pair.  Only nonzero counts are listed.
 *   n_out      host: number of records (exact even when capacity is short).
 * Needs a labeled graph with labels 0..31.  Synchronous; allocates its
 * tables.  Errors: PG_EINVAL (unlabeled graph), PG_EUNSUPPORTED (a label
 * above 31), PG_ETRUNC (capacity too small), PG_ENOMEM, PG_EDEVICE.
 */
typedef struct {
    int32_t shape;
    int32_t labels[3];
    uint64_t count_lo, count_hi;
} pg_labeled_count;
int pg_labeled_motif3(pg_graph *g, pg_labeled_count *out, int64_t capacity, int64_t *n_out, void *stream);

/*
 * pg_labeled_motif4 - labeled 4-motifs with label discovery (Section 6
 * labeled motifs; Section 3.2.1 label discovery): the number of
 * vertex-induced matches of every labeled connected 4-vertex pattern present
 * in the graph.  The labeled 3-motifs present (pg_labeled_motif3) discover the
 * candidates: a labeled 4-motif is counted only if each of its connected
 * induced 3-vertex sub-patterns, with its labels, occurs (it cannot occur
 * otherwise); candidates are counted exactly in fused batches of
 * vertex-induced labeled plans.
 *   out    host array of `capacity` records: shape PG_MOTIF4_*, labels of
 *          pattern vertices 0..3 (the smallest tuple over the shape's
 *          automorphisms), count as a 128-bit (low, high) pair; only
 *          nonzero counts, in no particular order.
 *   n_out  host: number of records (exact even when capacity is short).
 * Shapes and vertex numbering:
 *   PG_MOTIF4_PATH     path 0-1-2-3
 *   PG_MOTIF4_STAR     centre 0, leaves 1, 2, 3
 *   PG_MOTIF4_CYCLE    0-1-2-3-0
 *   PG_MOTIF4_TAILED   triangle 0-1-2, tail 3 at 0
 *   PG_MOTIF4_DIAMOND  cycle 0-1-2-3-0 with chord 1-3
 *   PG_MOTIF4_CLIQUE   all six pairs
 * Needs a labeled graph with labels 0..31.  Synchronous; allocates its
 * tables.  Errors: PG_EINVAL (unlabeled graph), PG_EUNSUPPORTED (a label
 * above 31), PG_ETRUNC, PG_ENOMEM, PG_EDEVICE.
 */
#define PG_MOTIF4_PATH 1
#define PG_MOTIF4_STAR 2
#define PG_MOTIF4_CYCLE 3
#define PG_MOTIF4_TAILED 4
#define PG_MOTIF4_DIAMOND 5
#define PG_MOTIF4_CLIQUE 6
typedef struct {
    int32_t shape;
    int32_t labels[4];
    int32_t pad;
    uint64_t count_lo, count_hi;
} pg_labeled_count4;
int pg_labeled_motif4(pg_graph *g, pg_labeled_count4 *out, int64_t capacity, int64_t *n_out, void *stream);

/*
 * Serving: a request loop over a resident graph.  Queries are submitted at
 * any time from any host thread; a worker thread admits waiting queries into
 * batches whenever one of n_streams streams is free and the batch's scratch
 * requirement fits that stream's preallocated share of memory_budget (a
 * batch that does not fit is split; a query that does not fit alone fails
 * with PG_ENOMEM in its result), counts each batch in one launch (the batch
 * kernel, one task group per pattern; cliques by the clique kernel), and
 * publishes per-query results with submit / start / completion times.
 * Batches on different streams overlap on the device, and queries arriving
 * while others run are admitted as soon as a stream frees up.  Plans are
 * compiled once per distinct pattern and kept, with the pattern's measured
 * service time: the first query of a pattern runs alone, and a pattern that
 * took longer than batch_limit_ms alone keeps running alone (with the
 * waiting queries of the same pattern), on at most n_streams - 1 streams
 * (one under a query time limit: a persistent launch keeps its SMs until it
 * ends, so a second long launch would start only past its deadlines),
 * so batches gather the short queries (which overtake long ones waiting in
 * the queue) and a long query never holds a batch of short ones.  An
 * anti-vertex query is launched alone on the plan interpreter
 * (PG_KERNEL_GENERIC), since batches do not take anti-vertex plans.  The paper runs one mining
 * program at a time (Section 5.1); this loop applies its processing model to
 * a stream of patterns.
 *   n_streams      concurrent batches (1..16); memory_budget: device bytes
 *                  for scratch (0: 40% of free memory, at most 64 GiB);
 *   max_batch      queries per batch (1..64); serial = 1: one query per
 *                  launch and one launch at a time (the baseline).
 * Times are seconds since pg_server_create (host steady clock); t_done is
 * when the worker observed the batch's completion.
 */
typedef struct pg_server pg_server;
typedef struct {
    int32_t n_streams;
    int32_t max_batch;
    int64_t memory_budget;
    int32_t serial;
    int32_t pad;
    double query_timeout_s; /* > 0: a query not done this long after its
                               submission fails with PG_ETIMEOUT.  Enforced
                               as the device work budget of its launch (see
                               pg_set_time_budget) and on the host clock (a
                               launch past its deadline gets its stop word
                               raised): a launch of one pattern gets the
                               least time left among its queries, a batch of
                               several patterns half of it.  When a batch
                               runs out its queries are launched again one
                               by one, so only the slow one fails; when a
                               one-pattern launch runs out, its queries with
                               more time left than it ran go to the back of
                               the queue.  The first (measuring) run of a
                               pattern, and the first rerun after a batch
                               ran out, get at most a quarter of the time
                               left.  Waiting queries fail as soon as their
                               limit passes.  0: no limit */
    double batch_limit_ms;  /* > 0: a pattern whose query took longer than
                               this alone is not batched again; 0: 20 ms;
                               < 0: no measuring, any query may be batched */
    double alone_sm_fraction; /* with n_streams > 1, launches of queries
                               that run alone (long, unmeasured, isolated;
                               with the waiting queries of the same pattern)
                               hold at most n_streams - 1 streams (1 with a
                               query time limit) and use this
                               fraction of the SMs (a smaller persistent
                               grid), leaving the rest to batches of short
                               queries; (0, 1], 0: 1 (all SMs) */
} pg_server_config;

typedef struct {
    uint64_t ticket;
    int32_t status;     /* PG_OK or the error that failed the query */
    int32_t batch_size; /* queries in the launch that counted it */
    uint64_t count_lo, count_hi; /* 128-bit count */
    double t_submit, t_start, t_done;
} pg_query_result;

typedef struct {
    int32_t n_streams;
    int32_t pad;
    int64_t batches, launched_queries, outstanding, cached_plans;
    int64_t scratch_bytes_per_stream;
    double now;
} pg_server_stats;

/* pg_server_create - start the worker on the current device.  The graph
 * must outlive the server.  Errors: PG_EINVAL, PG_ENOMEM, PG_EDEVICE. */
int pg_server_create(pg_graph *g, const pg_server_config *cfg, pg_server **out);
/* pg_server_submit - enqueue one count query; *ticket identifies its result.
 * Compiles the pattern on first sight (errors as pg_compile_pattern). */
int pg_server_submit(pg_server *s, const pg_pattern_desc *q, uint64_t *ticket);
/* pg_server_poll - move up to max_results finished results into out (host). */
int pg_server_poll(pg_server *s, pg_query_result *out, int32_t max_results, int32_t *n_out);
/* pg_server_cancel - withdraw a query.  A query still waiting gets a
 * PG_ECANCELED result at once.  A query being counted stops its launch: the
 * launch's stop flag is raised from a separate stream, the kernels leave at
 * their next poll (between tasks and between first-level candidates), the
 * query gets PG_ECANCELED and the other queries of that launch go back to
 * the front of the queue (they are counted again, results unchanged).  A
 * query that already has a result is left alone.  Errors: PG_EINVAL (NULL
 * server, ticket never issued or already finished). */
int pg_server_cancel(pg_server *s, uint64_t ticket);
/* pg_server_drain - wait until every submitted query has a result, or
 * PG_ETIMEOUT after timeout_s seconds. */
int pg_server_drain(pg_server *s, double timeout_s);
/* pg_server_get_stats - counters of the server (host struct out). */
int pg_server_get_stats(pg_server *s, pg_server_stats *out);
/* pg_server_free - stop the worker, wait for launches, release everything. */
void pg_server_free(pg_server *s);

/* pg_last_error - message of the last failed call on this host thread. */
const char *pg_last_error(void);

/* pg_version - library version (major * 10000 + minor * 100 + patch). */
int pg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PG_H */
