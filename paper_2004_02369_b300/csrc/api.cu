// C-ABI entry points (include/pg.h): argument checking, ownership, kernel
// dispatch.  No compute happens here; every step of the path runs in the
// library's kernels.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "pg_internal.h"

namespace {
thread_local std::string g_last_error;

// A temporary from the library pool, freed on its stream at scope exit.
struct DevTmp {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    int alloc(size_t bytes, cudaStream_t st) {
        s = st;
        return pg_dalloc(&p, bytes, st);
    }
    ~DevTmp() { if (p) pg_dfree(p, s); }
};

constexpr int kMaxPoolDevices = 64;
std::once_flag g_pool_once[kMaxPoolDevices];
cudaMemPool_t g_pool[kMaxPoolDevices];
cudaError_t g_pool_err[kMaxPoolDevices];
}  // namespace

int pg_dalloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    int dev = 0;
    PG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxPoolDevices) return pg_set_error(PG_EINVAL, "device index out of range");
    std::call_once(g_pool_once[dev], [dev] {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&g_pool[dev], &props);
        if (e == cudaSuccess) {
            uint64_t keep = 8ull << 30; // freed memory the pool keeps mapped
            e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        g_pool_err[dev] = e;
    });
    if (g_pool_err[dev] != cudaSuccess) return pg_cuda_error(g_pool_err[dev], "library memory pool");
    const cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, g_pool[dev], s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return pg_cuda_error(e, "pool allocation");
    }
    return PG_OK;
}

void pg_dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int pg_set_error(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int pg_cuda_error(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PG_ENOMEM : PG_EDEVICE;
}

extern "C" const char *pg_last_error(void) { return g_last_error.c_str(); }

extern "C" int pg_version(void) { return 100; }

// ---------------------------------------------------------------- graph ----

extern "C" int pg_load_graph(const int64_t *offsets, int64_t n, const int32_t *adj, int64_t nnz,
                             const int32_t *labels, int32_t inputs_on_device, void *stream, pg_graph **out) {
    if (!out) return pg_set_error(PG_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 0 || nnz < 0 || !offsets || (nnz > 0 && !adj))
        return pg_set_error(PG_EINVAL, "bad graph arguments");
    if (n >= 0x7fffffff) return pg_set_error(PG_EINVAL, "more than 2^31-1 vertices");
    cudaStream_t s = (cudaStream_t)stream;
    pg_graph *g = new (std::nothrow) pg_graph();
    if (!g) return pg_set_error(PG_ENOMEM, "host allocation failed");
    g->n = n;
    g->m = nnz / 2;
    g->labeled = labels ? 1 : 0;
    int rc = PG_OK;
    do {
        cudaError_t e = cudaGetDevice(&g->device);
        if (e != cudaSuccess) { rc = pg_cuda_error(e, "cudaGetDevice"); break; }
        e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
        if (e != cudaSuccess) { rc = pg_cuda_error(e, "cudaDeviceGetAttribute"); break; }
        DevTmp toff, tadj, tlab;
        const int64_t *d_off = offsets;
        const int32_t *d_adj = adj;
        const int32_t *d_lab = labels;
        if (!inputs_on_device) {
            if (offsets[0] != 0 || offsets[n] != nnz) { rc = pg_set_error(PG_EINVAL, "offsets[0] must be 0 and offsets[n] == nnz"); break; }
            if ((rc = toff.alloc((n + 1) * sizeof(int64_t), s)) != PG_OK) break;
            if ((rc = tadj.alloc((nnz > 0 ? nnz : 1) * sizeof(int32_t), s)) != PG_OK) break;
            if ((e = cudaMemcpyAsync(toff.p, offsets, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s)) != cudaSuccess) { rc = pg_cuda_error(e, "cudaMemcpyAsync"); break; }
            if (nnz > 0 && (e = cudaMemcpyAsync(tadj.p, adj, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s)) != cudaSuccess) { rc = pg_cuda_error(e, "cudaMemcpyAsync"); break; }
            if (labels) {
                if ((rc = tlab.alloc((n > 0 ? n : 1) * sizeof(int32_t), s)) != PG_OK) break;
                if (n > 0 && (e = cudaMemcpyAsync(tlab.p, labels, n * sizeof(int32_t), cudaMemcpyHostToDevice, s)) != cudaSuccess) { rc = pg_cuda_error(e, "cudaMemcpyAsync"); break; }
            }
            d_off = (const int64_t *)toff.p;
            d_adj = (const int32_t *)tadj.p;
            d_lab = labels ? (const int32_t *)tlab.p : nullptr;
        }
        rc = pg_graph_build(g, d_off, d_adj, nnz, d_lab, s);
        if (rc) break;
        if ((rc = pg_exec_init(&g->exec0)) != PG_OK) break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { rc = pg_cuda_error(e, "cudaStreamSynchronize"); break; }
    } while (0);
    if (rc) {
        pg_free_graph(g);
        return rc;
    }
    g->d.vinfo = g->vinfo;
    g->d.adj = g->adj;
    g->d.n = (int)g->n;
    g->d.max_deg = (int)g->max_deg;
    g->d.max_out = (int)g->max_out;
    g->d.labeled = g->labeled;
    g->d.hubbits = g->hubbits;
    g->d.n_hubs = g->n_hubs;
    g->d.hub_stride = g->hub_stride;
    *out = g;
    return PG_OK;
}

extern "C" int pg_graph_get_info(const pg_graph *g, pg_graph_info *out) {
    if (!g || !out) return pg_set_error(PG_EINVAL, "NULL argument");
    out->n = g->n;
    out->m = g->m;
    out->max_degree = g->max_deg;
    out->max_out_degree = g->max_out;
    out->device_bytes = pg_graph_bytes(g) + (int64_t)g->ex->scratch_bytes;
    out->labeled = g->labeled;
    out->n_labels = g->n_labels;
    return PG_OK;
}

extern "C" int pg_graph_rank(const pg_graph *g, int32_t *rank_out) {
    if (!g || (!rank_out && g->n > 0)) return pg_set_error(PG_EINVAL, "NULL argument");
    if (g->n > 0) PG_CUDA(cudaMemcpy(rank_out, g->rank, g->n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return PG_OK;
}

extern "C" void pg_free_graph(pg_graph *g) {
    if (!g) return;
    int prev = 0;
    const bool switched = cudaGetDevice(&prev) == cudaSuccess && prev != g->device &&
                          cudaSetDevice(g->device) == cudaSuccess;
    // launches on any stream may still read the graph
    cudaDeviceSynchronize();
    pg_dfree(g->vinfo, nullptr);
    pg_dfree(g->adj, nullptr);
    pg_dfree(g->rank, nullptr);
    pg_dfree(g->orig, nullptr);
    pg_dfree(g->hubbits, nullptr);
    pg_exec_release(&g->exec0);
    pg_dfree(g->heavy, nullptr);
    pg_dfree(g->split_prefix, nullptr);
    if (g->batch_cache) pg_batch_free(g->batch_cache);
    delete g;
    if (switched) cudaSetDevice(prev);
}

int pg_exec_init(pg_exec *x) {
    PG_CUDA(cudaMalloc(&x->queues, PG_MAX_QUEUES * sizeof(unsigned long long)));
    PG_CUDA(cudaMalloc(&x->tmp_counts, 2 * PG_MAX_QUEUES * sizeof(unsigned long long)));
    return PG_OK;
}

void pg_exec_release(pg_exec *x) {
    if (x->scratch) {
        cudaDeviceSynchronize(); // launches on any stream may still use the arena
        pg_dfree(x->scratch, nullptr);
    }
    if (x->queues) cudaFree(x->queues);
    if (x->tmp_counts) cudaFree(x->tmp_counts);
    x->scratch = nullptr;
    x->queues = x->tmp_counts = nullptr;
    x->scratch_bytes = 0;
}

int pg_ensure_scratch(pg_graph *g, size_t bytes, cudaStream_t s) {
    if (bytes <= g->ex->scratch_bytes) return PG_OK;
    if (g->ex->scratch) {
        // earlier launches on any stream may still read the old arena
        PG_CUDA(cudaDeviceSynchronize());
        pg_dfree(g->ex->scratch, s);
        g->ex->scratch = nullptr;
        g->ex->scratch_bytes = 0;
    }
    PG_TRY(pg_dalloc(&g->ex->scratch, bytes, s));
    g->ex->scratch_bytes = bytes;
    return PG_OK;
}

// ---------------------------------------------------------------- plans ----

namespace {

std::atomic<uint64_t> g_next_serial{1};

// A pattern above PGP_MAXK vertices is accepted only as an unlabeled clique
// (every pair an edge, no anti-edges or anti-vertices): its plan is the total
// order u0 < ... < u(k-1) of Section 4.1 for a clique, run by the k-clique
// kernel, with no level program for the interpreters.
int compile_big_clique(const pg_pattern_desc *d, pg_plan **out) {
    const int k = d->k;
    if (k > PG_MAX_CLIQUE)
        return pg_set_error(PG_EINVAL, "pattern size must be 1..8 (unlabeled cliques: up to 16)");
    const char *why = "patterns above 8 vertices must be unlabeled cliques (up to 16 vertices)";
    if (d->n_anti > 0 || d->n_edges < 0 || (d->n_edges > 0 && !d->edges)) return pg_set_error(PG_EINVAL, why);
    for (int u = 0; u < k; ++u) {
        if (d->labels && d->labels[u] != -1) return pg_set_error(PG_EINVAL, why);
        if (d->anti_vertex && d->anti_vertex[u]) return pg_set_error(PG_EINVAL, why);
    }
    uint32_t adj[PG_MAX_CLIQUE] = {};
    for (int i = 0; i < d->n_edges; ++i) {
        const int u = d->edges[2 * i], w = d->edges[2 * i + 1];
        if (u < 0 || w < 0 || u >= k || w >= k) return pg_set_error(PG_EINVAL, "pattern vertex out of range");
        if (u == w) return pg_set_error(PG_EINVAL, "self loop in pattern");
        adj[u] |= 1u << w;
        adj[w] |= 1u << u;
    }
    const uint32_t all = (1u << k) - 1;
    for (int u = 0; u < k; ++u)
        if ((adj[u] | (1u << u)) != all) return pg_set_error(PG_EINVAL, why);
    pg_plan *pl = new (std::nothrow) pg_plan();
    if (!pl) return pg_set_error(PG_ENOMEM, "host allocation failed");
    PgPlanHost &h = pl->h;
    h.pat = PgPattern{};
    h.big_clique = true;
    h.is_clique = true;
    h.clique_k = k;
    h.n_regular = k;
    h.aut = 1;
    for (int i = 2; i <= k; ++i) h.aut *= (uint64_t)i;
    for (int i = 0; i + 1 < k; ++i) h.po.push_back({i, i + 1});
    h.core_mask = all & ~1u;
    h.counted_group = 1;
    pl->serial = g_next_serial++;
    pl->kernel_auto = PG_KERNEL_CLIQUE;
    *out = pl;
    return PG_OK;
}

}  // namespace

extern "C" int pg_compile_pattern(const pg_pattern_desc *d, pg_plan **out) {
    if (!d || !out) return pg_set_error(PG_EINVAL, "NULL argument");
    *out = nullptr;
    if (d->k > PG_MAX_PATTERN) return compile_big_clique(d, out);
    if (d->k < 1) return pg_set_error(PG_EINVAL, "pattern size must be 1..8 (unlabeled cliques: up to 16)");
    PgPattern p;
    p.k = d->k;
    auto add = [&](const int32_t *pairs, int32_t np, uint8_t val) -> int {
        if (np < 0 || (np > 0 && !pairs)) return pg_set_error(PG_EINVAL, "bad edge array");
        for (int i = 0; i < np; ++i) {
            int u = pairs[2 * i], w = pairs[2 * i + 1];
            if (u < 0 || w < 0 || u >= d->k || w >= d->k) return pg_set_error(PG_EINVAL, "pattern vertex out of range");
            if (u == w) return pg_set_error(PG_EINVAL, "self loop in pattern");
            if (p.rel[u][w] && p.rel[u][w] != val) return pg_set_error(PG_EINVAL, "pair is both edge and anti-edge");
            p.rel[u][w] = p.rel[w][u] = val;
        }
        return PG_OK;
    };
    int rc = add(d->edges, d->n_edges, 1);
    if (rc) return rc;
    rc = add(d->anti_edges, d->n_anti, 2);
    if (rc) return rc;
    for (int u = 0; u < d->k; ++u) {
        p.label[u] = d->labels ? d->labels[u] : -1;
        p.anti_vertex[u] = d->anti_vertex ? (d->anti_vertex[u] ? 1 : 0) : 0;
    }
    pg_plan *pl = new (std::nothrow) pg_plan();
    if (!pl) return pg_set_error(PG_ENOMEM, "host allocation failed");
    std::string err;
    rc = pg_plan_compile(p, d->vertex_induced != 0, pl->h, err);
    if (rc) {
        delete pl;
        return pg_set_error(rc, err);
    }
    pl->serial = g_next_serial++;
    pl->kernel_auto = (pl->h.is_clique && pl->h.pat.k >= 3) ? PG_KERNEL_CLIQUE
                      : pl->h.anti_vertices                  ? PG_KERNEL_GENERIC
                                                             : PG_KERNEL_BATCHED;
    *out = pl;
    return PG_OK;
}

extern "C" int pg_plan_get_info(const pg_plan *pl, pg_plan_info *out) {
    if (!pl || !out) return pg_set_error(PG_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    const PgPlanHost &h = pl->h;
    out->k = pg_plan_size(h);
    out->n_regular = h.n_regular;
    out->automorphisms = h.aut;
    out->n_po = (int32_t)h.po.size();
    for (int i = 0; i < out->n_po && i < 28; ++i) {
        out->po[2 * i] = h.po[i].first;
        out->po[2 * i + 1] = h.po[i].second;
    }
    out->core_mask = h.core_mask;
    out->n_orders = (int32_t)h.orders.size();
    out->n_levels = h.orders.empty() ? 0 : h.orders[0].n_levels;
    out->counted_group = h.counted_group;
    out->kernel = pl->kernel_auto;
    out->compile_ms = h.compile_ms;
    return PG_OK;
}

extern "C" int pg_plan_describe(const pg_plan *pl, char *buf, int64_t size) {
    if (!pl || (!buf && size > 0) || size < 0) return pg_set_error(PG_EINVAL, "bad argument");
    const PgPlanHost &h = pl->h;
    std::string out;
    auto vlist = [](const int8_t *src, int n) {
        std::string s = "[";
        for (int i = 0; i < n; ++i) s += (i ? "," : "") + std::to_string(src[i]);
        return s + "]";
    };
    out += "k=" + std::to_string(pg_plan_size(h)) + " aut=" + std::to_string(h.aut) + " core_mask=" +
           std::to_string(h.core_mask) + " orders=" + std::to_string(h.orders.size()) + " po=";
    for (auto &e : h.po) out += "(" + std::to_string(e.first) + "<" + std::to_string(e.second) + ")";
    out += "\n";
    if (h.big_clique) out += "k-clique above 8 vertices: counted by the k-clique kernel (no level program)\n";
    for (size_t o = 0; o < h.orders.size(); ++o) {
        const PgOrder &ord = h.orders[o];
        out += "order " + std::to_string(o) + ":\n";
        for (int l = 0; l < ord.n_levels; ++l) {
            const PgLevel &L = ord.lv[l];
            out += "  L" + std::to_string(l) + " u" + std::to_string(L.pattern_vertex) + (L.is_core ? " core" : " noncore") +
                   " int=" + vlist(L.int_src, L.n_int) + " diff=" + vlist(L.diff_src, L.n_diff) + " lo=" +
                   vlist(L.lo_src, L.n_lo) + " hi=" + vlist(L.hi_src, L.n_hi) + " excl=" + vlist(L.excl_src, L.n_excl) +
                   " label=" + std::to_string(L.label) + " group=" + std::to_string(L.group) +
                   (L.out_bounded ? " out" : "") + (L.joint ? " joint" : "") + "\n";
        }
    }
    if (size > 0) {
        const size_t n = std::min<size_t>(out.size(), (size_t)size - 1);
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return out.size() + 1 <= (size_t)size ? PG_OK : pg_set_error(PG_ETRUNC, "buffer too small for the plan text");
}

extern "C" void pg_free_plan(pg_plan *pl) {
    if (!pl) return;
    if (pl->d_orders) cudaFree(pl->d_orders);
    if (pl->d_list_orders) cudaFree(pl->d_list_orders);
    delete pl;
}

int pg_plan_upload(pg_plan *pl) {
    if (pl->d_orders || pl->h.orders.empty()) return PG_OK;
    const size_t bytes = pl->h.orders.size() * sizeof(PgOrder);
    const size_t lbytes = pl->h.list_orders.size() * sizeof(PgOrder);
    PG_CUDA(cudaMalloc(&pl->d_orders, bytes));
    PG_CUDA(cudaMemcpy(pl->d_orders, pl->h.orders.data(), bytes, cudaMemcpyHostToDevice));
    PG_CUDA(cudaMalloc(&pl->d_list_orders, lbytes));
    PG_CUDA(cudaMemcpy(pl->d_list_orders, pl->h.list_orders.data(), lbytes, cudaMemcpyHostToDevice));
    return PG_OK;
}

// ---------------------------------------------------------------- count ----

int pg_run_ctl(pg_graph *g, unsigned long long target, cudaStream_t s, PgRunCtl *out, bool force) {
    *out = PgRunCtl{};
    if (!target && !g->budget_ns && !force) return PG_OK;
    out->words = g->ex->queues + PG_CTL_WORDS_SLOT;
    out->target = target;
    out->budget_ns = g->budget_ns;
    PG_CUDA(cudaMemsetAsync(out->words, 0, 3 * sizeof(unsigned long long), s));
    return PG_OK;
}

int pg_run_ctl_check(const PgRunCtl &ctl, cudaStream_t s) {
    if (!ctl.words || !ctl.budget_ns) return PG_OK;
    unsigned long long timed_out = 0;
    PG_CUDA(cudaMemcpyAsync(&timed_out, ctl.words + 1, sizeof(timed_out), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    if (timed_out) return pg_set_error(PG_ETIMEOUT, "the graph's device work budget ran out; partial results discarded");
    return PG_OK;
}

namespace {

// Counting of n_plans plans with one kernel family (see pg_count_ex);
// ctl: run control of a synchronous caller, or null.
int count_dispatch(pg_graph *g, pg_plan *const *plans, int32_t n_plans, uint64_t *counts_dev, int32_t kernel,
                   cudaStream_t s, const PgRunCtl *ctl) {
    bool all_clique = true, any_anti_vertex = false, any_big = false;
    int kmin = PG_MAX_CLIQUE + 1, kmax = 0;
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i]) return pg_set_error(PG_EINVAL, "NULL plan");
        const PgPlanHost &h = plans[i]->h;
        if (h.labeled && !g->labeled) return pg_set_error(PG_EINVAL, "labeled pattern on an unlabeled graph");
        const int k = pg_plan_size(h);
        all_clique &= h.is_clique && k >= 3;
        any_anti_vertex |= h.anti_vertices;
        any_big |= h.big_clique;
        kmin = std::min(kmin, k);
        kmax = std::max(kmax, k);
    }
    if (all_clique && g->max_out >= 65536) {
        if (any_big) return pg_set_error(PG_EUNSUPPORTED, "the k-clique kernel needs out-degrees below 65536");
        all_clique = false;
    }
    if (kernel == PG_KERNEL_AUTO)
        kernel = all_clique ? PG_KERNEL_CLIQUE : any_anti_vertex ? PG_KERNEL_GENERIC : PG_KERNEL_BATCHED;
    if (any_big && kernel != PG_KERNEL_CLIQUE && kernel != PG_KERNEL_CLIQUE_NONPERSISTENT)
        return pg_set_error(PG_EUNSUPPORTED, "cliques above 8 vertices run on the k-clique kernel only");
    if (any_anti_vertex && kernel != PG_KERNEL_GENERIC && kernel != PG_KERNEL_CLIQUE_PLAIN)
        return pg_set_error(PG_EUNSUPPORTED, "anti-vertex patterns run on the plan interpreter (PG_KERNEL_GENERIC)");
    if ((kernel == PG_KERNEL_CLIQUE || kernel == PG_KERNEL_CLIQUE_NONPERSISTENT) && !all_clique)
        return pg_set_error(PG_EINVAL, "the k-clique kernels need unlabeled k-clique patterns, k >= 3");
    if (kernel != PG_KERNEL_GENERIC && kernel != PG_KERNEL_CLIQUE_PLAIN && kernel != PG_KERNEL_CLIQUE &&
        kernel != PG_KERNEL_BATCHED && kernel != PG_KERNEL_CLIQUE_NONPERSISTENT)
        return pg_set_error(PG_EINVAL, "unknown kernel family");
    if (kernel == PG_KERNEL_CLIQUE_NONPERSISTENT) {
        PG_CUDA(cudaMemsetAsync(counts_dev, 0, 2 * sizeof(uint64_t) * n_plans, s));
        for (int i = 0; i < n_plans; ++i) {
            int rc = pg_launch_clique_plain(g, pg_plan_size(plans[i]->h), (unsigned long long *)counts_dev + 2 * i, s);
            if (rc) return rc;
        }
        return PG_OK;
    }
    if (kernel == PG_KERNEL_BATCHED) {
        std::vector<uint64_t> key;
        for (int i = 0; i < n_plans; ++i) key.push_back(plans[i]->serial);
        if (!g->batch_cache || g->batch_key != key) {
            pg_batch *b = nullptr;
            int rc = pg_batch_build(plans, n_plans, PG_BATCH_EXPAND_ANTI, &b);
            if (rc) return rc;
            if (g->batch_cache) {
                PG_CUDA(cudaDeviceSynchronize()); // earlier launches may still read it
                pg_batch_free(g->batch_cache);
            }
            g->batch_cache = b;
            g->batch_key = key;
        }
        const pg_batch *b = g->batch_cache;
        int rc = pg_ensure_scratch(g, pg_batch_scratch_bytes(g, b), s);
        if (rc) return rc;
        PG_CUDA(cudaMemsetAsync(counts_dev, 0, 2 * sizeof(uint64_t) * pg_batch_slots(b), s));
        return pg_launch_batched(g, b, (unsigned long long *)counts_dev, 0, s, ctl);
    }
    size_t need = 0;
    for (int i = 0; i < n_plans; ++i) {
        int rc = pg_plan_upload(plans[i]);
        if (rc) return rc;
        if (kernel == PG_KERNEL_GENERIC) need = std::max(need, pg_generic_scratch_bytes(g, plans[i], true));
        if (kernel == PG_KERNEL_CLIQUE_PLAIN) need = std::max(need, pg_generic_scratch_bytes(g, plans[i], false));
    }
    if (kernel == PG_KERNEL_CLIQUE) need = pg_clique_scratch_bytes(g, kmax);
    int rc = pg_ensure_scratch(g, need, s);
    if (rc) return rc;
    PG_CUDA(cudaMemsetAsync(counts_dev, 0, 2 * sizeof(uint64_t) * n_plans, s));
    if (kernel == PG_KERNEL_CLIQUE) {
        // one launch counts every size kmin..kmax; copy each plan's size out
        PG_CUDA(cudaMemsetAsync(g->ex->tmp_counts, 0, 2 * sizeof(uint64_t) * (kmax - kmin + 1), s));
        rc = pg_launch_clique(g, kmin, kmax, g->ex->tmp_counts, 0, s, ctl);
        if (rc) return rc;
        for (int i = 0; i < n_plans; ++i)
            PG_CUDA(cudaMemcpyAsync(counts_dev + 2 * i, g->ex->tmp_counts + 2 * (pg_plan_size(plans[i]->h) - kmin),
                                    2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        return PG_OK;
    }
    // one launch per plan, in stream order (each launch resets its queue word)
    for (int i = 0; i < n_plans; ++i) {
        rc = pg_launch_generic(g, plans[i], (unsigned long long *)counts_dev + 2 * i, i % 8,
                               kernel == PG_KERNEL_GENERIC, s, ctl);
        if (rc) return rc;
    }
    return PG_OK;
}

}  // namespace

extern "C" int pg_count_ex(pg_graph *g, pg_plan *const *plans, int32_t n_plans, uint64_t *counts_dev,
                           int32_t kernel, void *stream) {
    if (!g || (n_plans > 0 && (!plans || !counts_dev)) || n_plans < 0)
        return pg_set_error(PG_EINVAL, "NULL argument");
    if (n_plans > PG_MAX_QUEUES) return pg_set_error(PG_EINVAL, "at most 64 plans per call");
    if (n_plans == 0) return PG_OK;
    return count_dispatch(g, plans, n_plans, counts_dev, kernel, (cudaStream_t)stream, nullptr);
}

extern "C" int pg_set_partition(pg_graph *g, int32_t part, int32_t n_parts) {
    if (!g || n_parts < 1 || part < 0 || part >= n_parts) return pg_set_error(PG_EINVAL, "need 0 <= part < n_parts");
    if (g->servers > 0) return pg_set_error(PG_EINVAL, "a server is running on this graph");
    g->part = part;
    g->n_parts = n_parts;
    return PG_OK;
}

extern "C" int pg_set_time_budget(pg_graph *g, double budget_ms) {
    if (!g || !(budget_ms >= 0.0) || budget_ms > 1e12) return pg_set_error(PG_EINVAL, "bad argument");
    g->budget_ns = (unsigned long long)(budget_ms * 1e6);
    return PG_OK;
}

extern "C" int pg_get_time_budget(const pg_graph *g, double *budget_ms) {
    if (!g || !budget_ms) return pg_set_error(PG_EINVAL, "NULL argument");
    *budget_ms = (double)g->budget_ns / 1e6;
    return PG_OK;
}

extern "C" int pg_compile_batch(pg_plan *const *plans, int32_t n_plans, int32_t flags, pg_batch **out) {
    if (!plans || !out) return pg_set_error(PG_EINVAL, "NULL argument");
    *out = nullptr;
    for (int i = 0; i < n_plans; ++i)
        if (!plans[i]) return pg_set_error(PG_EINVAL, "NULL plan");
    return pg_batch_build(plans, n_plans, flags, out);
}

extern "C" int pg_batch_get_info(const pg_batch *b, int32_t *n_nodes, int32_t *n_programs, int32_t *n_levels_total) {
    if (!b || !n_nodes || !n_programs || !n_levels_total) return pg_set_error(PG_EINVAL, "NULL argument");
    int a, p, l;
    pg_batch_stats(b, &a, &p, &l);
    *n_nodes = a;
    *n_programs = p;
    *n_levels_total = l;
    return PG_OK;
}

extern "C" void pg_free_batch(pg_batch *b) { pg_batch_free(b); }

extern "C" int pg_count_batch(pg_graph *g, const pg_batch *b, uint64_t *counts_dev, void *stream) {
    if (!g || !b || !counts_dev) return pg_set_error(PG_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = pg_ensure_scratch(g, pg_batch_scratch_bytes(g, b), s);
    if (rc) return rc;
    if (pg_batch_labeled(b) && !g->labeled) return pg_set_error(PG_EINVAL, "labeled pattern on an unlabeled graph");
    const int n_slots = pg_batch_slots(b);
    PG_CUDA(cudaMemsetAsync(counts_dev, 0, 2 * sizeof(uint64_t) * n_slots, s));
    return pg_launch_batched(g, b, (unsigned long long *)counts_dev, 0, s);
}

extern "C" int pg_count(pg_graph *g, pg_plan *const *plans, int32_t n_plans, uint64_t *counts_out, void *stream) {
    if (!g || (n_plans > 0 && (!plans || !counts_out)) || n_plans < 0) return pg_set_error(PG_EINVAL, "NULL argument");
    if (n_plans > PG_MAX_QUEUES) return pg_set_error(PG_EINVAL, "at most 64 plans per call");
    if (n_plans == 0) return PG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevTmp c;
    PG_TRY(c.alloc(2 * sizeof(uint64_t) * n_plans, s));
    PgRunCtl ctl;
    int rc = pg_run_ctl(g, 0, s, &ctl);
    if (rc) return rc;
    rc = count_dispatch(g, plans, n_plans, (uint64_t *)c.p, PG_KERNEL_AUTO, s, &ctl);
    if (rc) return rc;
    if ((rc = pg_run_ctl_check(ctl, s)) != PG_OK) return rc;
    PG_CUDA(cudaMemcpyAsync(counts_out, c.p, 2 * sizeof(uint64_t) * n_plans, cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    return PG_OK;
}

// ------------------------------------------------------------ existence ----

extern "C" int pg_count_until(pg_graph *g, pg_plan *pl, uint64_t target, uint64_t *count_out, int32_t *reached,
                              void *stream) {
    if (!g || !pl || !count_out || !reached) return pg_set_error(PG_EINVAL, "NULL argument");
    if (target < 1) return pg_set_error(PG_EINVAL, "target must be >= 1");
    if (pl->h.labeled && !g->labeled) return pg_set_error(PG_EINVAL, "labeled pattern on an unlabeled graph");
    cudaStream_t s = (cudaStream_t)stream;
    const int k = pg_plan_size(pl->h);
    const bool clique = pl->h.is_clique && k >= 3 && g->max_out < 65536;
    if (pl->h.big_clique && !clique)
        return pg_set_error(PG_EUNSUPPORTED, "the k-clique kernel needs out-degrees below 65536");
    int rc = pg_plan_upload(pl);
    if (rc) return rc;
    rc = pg_ensure_scratch(g, clique ? pg_clique_scratch_bytes(g, k) : pg_generic_scratch_bytes(g, pl, true), s);
    if (rc) return rc;
    unsigned long long *counts = g->ex->tmp_counts; // (low, high)
    PG_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s));
    PgRunCtl ctl;
    if ((rc = pg_run_ctl(g, target, s, &ctl)) != PG_OK) return rc;
    // cliques: the bitmap kernel, publishing its count during traversals
    rc = clique ? pg_launch_clique(g, k, k, counts, 0, s, &ctl) : pg_launch_generic(g, pl, counts, 0, true, s, &ctl);
    if (rc) return rc;
    if ((rc = pg_run_ctl_check(ctl, s)) != PG_OK) return rc;
    unsigned long long host[2];
    PG_CUDA(cudaMemcpyAsync(host, counts, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    count_out[0] = host[0];
    count_out[1] = host[1];
    *reached = (host[1] != 0 || host[0] >= target) ? 1 : 0;
    return PG_OK;
}

extern "C" int pg_plan_operand_bytes(pg_graph *g, pg_plan *pl, uint64_t *bytes_out, uint64_t *ops_out, void *stream) {
    if (!g || !pl || !bytes_out || !ops_out) return pg_set_error(PG_EINVAL, "NULL argument");
    if (pl->h.labeled && !g->labeled) return pg_set_error(PG_EINVAL, "labeled pattern on an unlabeled graph");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = pg_plan_upload(pl);
    if (rc) return rc;
    unsigned long long *d = g->ex->tmp_counts;
    if ((rc = pg_launch_operand_bytes(g, pl, d, s)) != PG_OK) return rc;
    unsigned long long h[2];
    PG_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    *bytes_out = 4ull * h[0];
    *ops_out = h[1];
    return PG_OK;
}

// The clustering-coefficient program of Section 3.2.3: W = matches of the
// 3-vertex star (connected triples), counted exactly; triangles T are then
// counted only until 3T > bound * W is established (existence with a target).
extern "C" int pg_clustering_coefficient_above(pg_graph *g, double bound, int32_t *answer, uint64_t *triangles_out,
                                               uint64_t *wedges_out, void *stream) {
    if (!g || !answer || !triangles_out || !wedges_out) return pg_set_error(PG_EINVAL, "NULL argument");
    if (!(bound >= 0.0) || bound > 1e300) return pg_set_error(PG_EINVAL, "bound must be finite and >= 0");
    const int32_t star[4] = {0, 1, 0, 2}, tri[6] = {0, 1, 1, 2, 0, 2};
    pg_pattern_desc ds{3, 2, star, 0, nullptr, nullptr, nullptr, 0};
    pg_pattern_desc dt{3, 3, tri, 0, nullptr, nullptr, nullptr, 0};
    pg_plan *ps = nullptr, *pt = nullptr;
    int rc = pg_compile_pattern(&ds, &ps);
    if (rc == PG_OK) rc = pg_compile_pattern(&dt, &pt);
    uint64_t w[2] = {0, 0}, t[2] = {0, 0};
    if (rc == PG_OK) rc = pg_count(g, &ps, 1, w, stream);
    int32_t reached = 0;
    if (rc == PG_OK) {
        const long double W = (long double)w[0] + 18446744073709551616.0L * (long double)w[1];
        // smallest T with 3T > bound * W
        const long double x = (long double)bound * W / 3.0L;
        const long double need = floorl(x) + 1.0L;
        const uint64_t target = need >= 18446744073709551615.0L ? UINT64_MAX : (uint64_t)need;
        rc = pg_count_until(g, pt, target, t, &reached, stream);
        if (rc == PG_OK) {
            const long double T = (long double)t[0] + 18446744073709551616.0L * (long double)t[1];
            *answer = (reached && 3.0L * T > (long double)bound * W) ? 1 : 0;
            triangles_out[0] = t[0];
            triangles_out[1] = t[1];
            wedges_out[0] = w[0];
            wedges_out[1] = w[1];
        }
    }
    pg_free_plan(ps);
    pg_free_plan(pt);
    return rc;
}

// ---------------------------------------------------------------- match ----

extern "C" int pg_match_range(pg_graph *g, pg_plan *pl, int64_t rank_begin, int64_t rank_end, int32_t *out_dev,
                              uint64_t capacity, uint64_t *n_total, void *stream) {
    if (!g || !pl || !n_total || (capacity > 0 && !out_dev)) return pg_set_error(PG_EINVAL, "NULL argument");
    if (rank_begin < 0 || rank_end < rank_begin || rank_end > g->n)
        return pg_set_error(PG_EINVAL, "start-vertex rank range out of bounds");
    if (pl->h.labeled && !g->labeled) return pg_set_error(PG_EINVAL, "labeled pattern on an unlabeled graph");
    if (pl->h.big_clique) return pg_set_error(PG_EUNSUPPORTED, "cliques above 8 vertices are counted, not listed");
    if (capacity > (uint64_t)INT64_MAX / (uint64_t)pl->h.pat.k) return pg_set_error(PG_EINVAL, "capacity too large");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = pg_plan_upload(pl);
    if (rc) return rc;
    rc = pg_ensure_scratch(g, pg_match_scratch_bytes(g, pl), s);
    if (rc) return rc;
    unsigned long long *counter = g->ex->tmp_counts;
    PgRunCtl ctl;
    if ((rc = pg_run_ctl(g, 0, s, &ctl)) != PG_OK) return rc;
    rc = pg_launch_match(g, pl, rank_begin, rank_end, out_dev, capacity, counter, s, &ctl);
    if (rc) return rc;
    if ((rc = pg_run_ctl_check(ctl, s)) != PG_OK) return rc;
    unsigned long long total = 0;
    PG_CUDA(cudaMemcpyAsync(&total, counter, sizeof(total), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    *n_total = total;
    if (total > capacity)
        return pg_set_error(PG_ETRUNC, "more matches than capacity: the first `capacity` rows were written");
    return PG_OK;
}

extern "C" int pg_match(pg_graph *g, pg_plan *pl, int32_t *out_dev, uint64_t capacity, uint64_t *n_total,
                        void *stream) {
    if (!g) return pg_set_error(PG_EINVAL, "NULL argument");
    return pg_match_range(g, pl, 0, g->n, out_dev, capacity, n_total, stream);
}

extern "C" int pg_labeled_motif3(pg_graph *g, pg_labeled_count *out, int64_t capacity, int64_t *n_out,
                                 void *stream) {
    if (!g || !n_out || (capacity > 0 && !out) || capacity < 0) return pg_set_error(PG_EINVAL, "bad argument");
    return pg_labeled_motif3_run(g, out, capacity, n_out, (cudaStream_t)stream);
}

extern "C" int pg_labeled_motif4(pg_graph *g, pg_labeled_count4 *out, int64_t capacity, int64_t *n_out,
                                 void *stream) {
    if (!g || !n_out || (capacity > 0 && !out) || capacity < 0) return pg_set_error(PG_EINVAL, "bad argument");
    return pg_labeled_motif4_run(g, out, capacity, n_out, (cudaStream_t)stream);
}

extern "C" int pg_fsm_general(pg_graph *g, int32_t max_edges, uint64_t threshold, pg_fsm_general_pattern *out,
                              int64_t capacity, int64_t *n_frequent, void *stream) {
    if (!g || !n_frequent || (capacity > 0 && !out) || capacity < 0) return pg_set_error(PG_EINVAL, "bad argument");
    return pg_fsm_general_run(g, max_edges, threshold, out, capacity, n_frequent, (cudaStream_t)stream);
}

extern "C" int pg_fsm(pg_graph *g, int32_t max_edges, uint64_t threshold, pg_fsm_pattern *out, int64_t capacity,
                      int64_t *n_frequent, void *stream) {
    if (!g || !n_frequent || (capacity > 0 && !out) || capacity < 0) return pg_set_error(PG_EINVAL, "bad argument");
    return pg_fsm_run(g, max_edges, threshold, out, capacity, n_frequent, (cudaStream_t)stream);
}
