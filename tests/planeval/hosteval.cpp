// Test aid: a sequential CPU interpreter of the compiled level program.
//
// It links the library's host plan compiler (plan.cpp) and walks every
// (start vertex, matching order) task with plain std::vector set operations,
// so that the plan compiler can be checked against the oracle on machines
// without a GPU.  It is not part of the library and never runs on its path.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/pg.h"
#include "../../paper_2004_02369_b300/csrc/plan.h"

namespace {

struct RankedGraph {
    int n = 0;
    std::vector<int64_t> off;
    std::vector<int32_t> adj, label;
};

RankedGraph rank_graph(const int64_t *off, int64_t n, const int32_t *adj, const int32_t *labels) {
    std::vector<int> order(n), rank(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (off[a + 1] - off[a]) > (off[b + 1] - off[b]);
    });
    for (int r = 0; r < n; ++r) rank[order[r]] = r;
    RankedGraph g;
    g.n = (int)n;
    g.off.assign(n + 1, 0);
    g.label.assign(n, 0);
    for (int r = 0; r < n; ++r) {
        int v = order[r];
        g.off[r + 1] = g.off[r] + (off[v + 1] - off[v]);
        if (labels) g.label[r] = labels[v];
    }
    g.adj.resize(g.off[n]);
    for (int r = 0; r < n; ++r) {
        int v = order[r];
        int64_t w = g.off[r];
        for (int64_t e = off[v]; e < off[v + 1]; ++e) g.adj[w++] = rank[adj[e]];
        std::sort(g.adj.begin() + g.off[r], g.adj.begin() + g.off[r + 1]);
    }
    return g;
}

bool has(const RankedGraph &g, int v, int x) {
    return std::binary_search(g.adj.begin() + g.off[v], g.adj.begin() + g.off[v + 1], x);
}

std::vector<int> level_set(const RankedGraph &g, const PgLevel &L, const int *m) {
    int lo = -1, hi = 0x7fffffff;
    for (int i = 0; i < L.n_lo; ++i) lo = std::max(lo, m[L.lo_src[i]]);
    for (int i = 0; i < L.n_hi; ++i) hi = std::min(hi, m[L.hi_src[i]]);
    std::vector<int> out;
    const int a = m[L.int_src[0]];
    for (int64_t e = g.off[a]; e < g.off[a + 1]; ++e) {
        int x = g.adj[e];
        if (x <= lo || x >= hi) continue;
        bool ok = true;
        for (int i = 1; i < L.n_int && ok; ++i) ok = has(g, m[L.int_src[i]], x);
        for (int i = 0; i < L.n_diff && ok; ++i) ok = !has(g, m[L.diff_src[i]], x);
        for (int i = 0; i < L.n_excl && ok; ++i) ok = x != m[L.excl_src[i]];
        if (ok && L.label >= 0) ok = g.label[x] == L.label;
        if (ok) out.push_back(x);
    }
    return out;
}

unsigned __int128 choose(uint64_t s, int k) {
    if ((int64_t)s < k) return 0;
    unsigned __int128 r = 1;
    for (int i = 0; i < k; ++i) r = r * (s - i) / (i + 1);
    return r;
}

// Anti-vertex check: no data vertex lies in every adj(m[int_src]) other than
// the images m[excl_src].
bool anti_ok(const RankedGraph &g, const PgAntiCheck &C, const int *m) {
    const int a = m[C.int_src[0]];
    for (int64_t e = g.off[a]; e < g.off[a + 1]; ++e) {
        const int x = g.adj[e];
        bool in = true;
        for (int i = 1; i < C.n_int && in; ++i) in = has(g, m[C.int_src[i]], x);
        for (int i = 0; i < C.n_excl && in; ++i) in = x != m[C.excl_src[i]];
        if (in) return false;
    }
    return true;
}

bool checks_ok(const RankedGraph &g, const PgOrder &o, int l, const int *m) {
    for (int c = 0; c < o.n_checks; ++c)
        if (o.chk[c].level == l && !anti_ok(g, o.chk[c], m)) return false;
    return true;
}

unsigned __int128 walk(const RankedGraph &g, const PgOrder &o, int l, int *m) {
    const PgLevel &L = o.lv[l];
    std::vector<int> s = level_set(g, L, m);
    if (L.n_anti) {
        std::vector<int> kept;
        for (int x : s) {
            m[l] = x;
            if (checks_ok(g, o, l, m)) kept.push_back(x);
        }
        s.swap(kept);
    }
    if (l == o.n_levels - 1) return choose(s.size(), L.group);
    unsigned __int128 t = 0;
    for (int x : s) {
        m[l] = x;
        t += walk(g, o, l + 1, m);
    }
    return t;
}

// Operand elements of level L at prefix m: every intersected and subtracted
// list cut to the level's open range (lo, hi).
uint64_t operand_elems(const RankedGraph &g, const PgLevel &L, const int *m) {
    int lo = -1, hi = 0x7fffffff;
    for (int i = 0; i < L.n_lo; ++i) lo = std::max(lo, m[L.lo_src[i]]);
    for (int i = 0; i < L.n_hi; ++i) hi = std::min(hi, m[L.hi_src[i]]);
    if (lo + 1 >= hi) return 0;
    uint64_t e = 0;
    for (int i = 0; i < L.n_int + L.n_diff; ++i) {
        const int w = i < L.n_int ? m[L.int_src[i]] : m[L.diff_src[i - L.n_int]];
        for (int64_t k = g.off[w]; k < g.off[w + 1]; ++k) e += (g.adj[k] > lo && g.adj[k] < hi) ? 1 : 0;
    }
    return e;
}

void walk_ops(const RankedGraph &g, const PgOrder &o, int l, int *m, uint64_t &elems, uint64_t &ops) {
    const PgLevel &L = o.lv[l];
    elems += operand_elems(g, L, m);
    ++ops;
    if (l == o.n_levels - 1) return;
    std::vector<int> s = level_set(g, L, m);
    for (int x : s) {
        m[l] = x;
        if (L.n_anti && !checks_ok(g, o, l, m)) continue;
        walk_ops(g, o, l + 1, m, elems, ops);
    }
}

}  // namespace

// Operand elements and set operations of p's counting program on the graph
// (every level of every task, the counted last level included).
extern "C" int pe_operand_elems(const int64_t *off, int64_t n, const int32_t *adj, const int32_t *labels,
                                const pg_pattern_desc *d, uint64_t *out2) {
    PgPattern p;
    p.k = d->k;
    for (int i = 0; i < d->n_edges; ++i) {
        int u = d->edges[2 * i], w = d->edges[2 * i + 1];
        p.rel[u][w] = p.rel[w][u] = 1;
    }
    for (int i = 0; i < d->n_anti; ++i) {
        int u = d->anti_edges[2 * i], w = d->anti_edges[2 * i + 1];
        p.rel[u][w] = p.rel[w][u] = 2;
    }
    for (int u = 0; u < d->k; ++u) {
        p.label[u] = d->labels ? d->labels[u] : -1;
        p.anti_vertex[u] = d->anti_vertex ? d->anti_vertex[u] : 0;
    }
    PgPlanHost h;
    std::string err;
    int rc = pg_plan_compile(p, d->vertex_induced != 0, h, err);
    if (rc) return rc;
    RankedGraph g = rank_graph(off, n, adj, labels);
    uint64_t elems = 0, ops = 0;
    int m[PGP_MAXK];
    for (const PgOrder &o : h.orders)
        for (int v = 0; v < g.n; ++v) {
            if (o.lv[0].label >= 0 && g.label[v] != o.lv[0].label) continue;
            m[0] = v;
            if (!checks_ok(g, o, 0, m)) continue;
            if (o.n_levels > 1) walk_ops(g, o, 1, m, elems, ops);
        }
    out2[0] = elems;
    out2[1] = ops;
    return 0;
}

// Counts p on the graph by walking the compiled counting program (use_list =
// 0) or the listing program (use_list = 1, every vertex enumerated).
extern "C" int pe_count(const int64_t *off, int64_t n, const int32_t *adj, const int32_t *labels,
                        const pg_pattern_desc *d, int32_t use_list, uint64_t *out2, int32_t *info) {
    PgPattern p;
    p.k = d->k;
    for (int i = 0; i < d->n_edges; ++i) {
        int u = d->edges[2 * i], w = d->edges[2 * i + 1];
        p.rel[u][w] = p.rel[w][u] = 1;
    }
    for (int i = 0; i < d->n_anti; ++i) {
        int u = d->anti_edges[2 * i], w = d->anti_edges[2 * i + 1];
        p.rel[u][w] = p.rel[w][u] = 2;
    }
    for (int u = 0; u < d->k; ++u) {
        p.label[u] = d->labels ? d->labels[u] : -1;
        p.anti_vertex[u] = d->anti_vertex ? d->anti_vertex[u] : 0;
    }
    PgPlanHost h;
    std::string err;
    int rc = pg_plan_compile(p, d->vertex_induced != 0, h, err);
    if (rc) return rc;
    RankedGraph g = rank_graph(off, n, adj, labels);
    unsigned __int128 total = 0;
    int m[PGP_MAXK];
    for (const PgOrder &o : use_list ? h.list_orders : h.orders) {
        for (int v = 0; v < g.n; ++v) {
            if (o.lv[0].label >= 0 && g.label[v] != o.lv[0].label) continue;
            m[0] = v;
            if (!checks_ok(g, o, 0, m)) continue;
            if (o.n_levels == 1) { total += 1; continue; }
            total += walk(g, o, 1, m);
        }
    }
    out2[0] = (uint64_t)total;
    out2[1] = (uint64_t)(total >> 64);
    if (info) {
        info[0] = (int32_t)h.orders.size();
        info[1] = (int32_t)h.core_mask;
        info[2] = h.counted_group;
        info[3] = h.orders.empty() ? 0 : h.orders[0].n_levels;
    }
    return 0;
}
