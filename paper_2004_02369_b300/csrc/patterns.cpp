// Pattern generators of the pattern interface (Section 3.1, "Pattern
// Interface" figure): every connected pattern of a given size, and the
// extension of a pattern set by one vertex or by one edge, each result
// deduplicated by isomorphism.  Host only; patterns are unlabeled and have
// no anti-edges or anti-vertices (a vertex-induced flag is carried along).
//
// Isomorphism classes are keyed by a canonical code: the smallest bit string
// of the upper adjacency triangle over all vertex permutations (k <= 8, so
// at most 8! permutations of 28 bits).
#include <algorithm>
#include <cstring>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "pg_internal.h"

namespace {

struct Pat {
    int k = 0;
    uint8_t adj[PGP_MAXK] = {}; // bit w of adj[u]: edge (u, w)
    int vertex_induced = 0;
};

uint32_t code_of(const Pat &p, const int *perm) {
    uint32_t c = 0;
    for (int u = 0; u < p.k; ++u)
        for (int w = u + 1; w < p.k; ++w) c = (c << 1) | ((p.adj[perm[u]] >> perm[w]) & 1u);
    return c;
}

// (k, smallest code over all permutations): equal iff isomorphic
uint64_t canonical(const Pat &p) {
    int perm[PGP_MAXK];
    for (int i = 0; i < p.k; ++i) perm[i] = i;
    uint32_t best = 0xffffffffu;
    do best = std::min(best, code_of(p, perm));
    while (std::next_permutation(perm, perm + p.k));
    return ((uint64_t)p.k << 32) | best;
}

int n_edges(const Pat &p) {
    int e = 0;
    for (int u = 0; u < p.k; ++u) e += __builtin_popcount(p.adj[u]);
    return e / 2;
}

struct Collector {
    std::set<uint64_t> seen;
    std::vector<Pat> out;
    void add(const Pat &p) {
        if (seen.insert(canonical(p)).second) out.push_back(p);
    }
};

// one new vertex joined to every non-empty subset of the existing vertices
void extend_vertex(const std::vector<Pat> &in, Collector &c) {
    for (const Pat &p : in) {
        const int k = p.k;
        if (k < 1 || k >= PGP_MAXK) continue;
        for (uint32_t sub = 1; sub < (1u << k); ++sub) {
            Pat q = p;
            q.k = k + 1;
            q.adj[k & (PGP_MAXK - 1)] = (uint8_t)sub;
            for (int u = 0; u < k; ++u)
                if (sub >> u & 1) q.adj[u] |= (uint8_t)(1u << k);
            c.add(q);
        }
    }
}

// one new edge: between two non-adjacent vertices, or to a new vertex
void extend_edge(const std::vector<Pat> &in, Collector &c) {
    for (const Pat &p : in) {
        for (int u = 0; u < p.k; ++u)
            for (int w = u + 1; w < p.k; ++w)
                if (!(p.adj[u] >> w & 1)) {
                    Pat q = p;
                    q.adj[u] |= (uint8_t)(1u << w);
                    q.adj[w] |= (uint8_t)(1u << u);
                    c.add(q);
                }
        const int k = p.k;
        if (k < 1 || k >= PGP_MAXK) continue;
        for (int u = 0; u < k; ++u) {
            Pat q = p;
            q.k = k + 1;
            q.adj[u] |= (uint8_t)(1u << k);
            q.adj[k & (PGP_MAXK - 1)] = (uint8_t)(1u << u);
            c.add(q);
        }
    }
}

}  // namespace

struct pg_pattern_set {
    std::vector<Pat> pats;
};

namespace {

int finish(Collector &c, pg_pattern_set **out) {
    pg_pattern_set *s = new (std::nothrow) pg_pattern_set();
    if (!s) return pg_set_error(PG_ENOMEM, "host allocation failed");
    s->pats = std::move(c.out);
    *out = s;
    return PG_OK;
}

}  // namespace

extern "C" int pg_patterns_all(int32_t size, int32_t vertex_induced, pg_pattern_set **out) {
    if (!out) return pg_set_error(PG_EINVAL, "NULL argument");
    *out = nullptr;
    Collector c;
    std::vector<Pat> cur(1);
    if (vertex_induced) {
        if (size < 1 || size > 7) return pg_set_error(PG_EINVAL, "vertex-induced sizes are 1..7 vertices");
        cur[0].k = 1;
        for (int v = 1; v < size; ++v) {
            Collector step;
            extend_vertex(cur, step);
            cur = std::move(step.out);
        }
    } else {
        if (size < 1 || size > 7) return pg_set_error(PG_EINVAL, "edge-induced sizes are 1..7 edges");
        cur[0].k = 2;
        cur[0].adj[0] = 2;
        cur[0].adj[1] = 1;
        for (int e = 1; e < size; ++e) {
            Collector step;
            extend_edge(cur, step);
            cur = std::move(step.out);
        }
        // 7 edges need at most 8 vertices, so no pattern was cut off
        for (const Pat &p : cur)
            if (n_edges(p) != size) return pg_set_error(PG_EINVAL, "internal: edge count mismatch");
    }
    for (Pat &p : cur) {
        p.vertex_induced = vertex_induced ? 1 : 0;
        c.add(p);
    }
    return finish(c, out);
}

extern "C" int pg_patterns_from(const pg_pattern_desc *descs, int64_t n, pg_pattern_set **out) {
    if (!out || (n > 0 && !descs) || n < 0) return pg_set_error(PG_EINVAL, "bad argument");
    *out = nullptr;
    Collector c;
    for (int64_t i = 0; i < n; ++i) {
        const pg_pattern_desc &d = descs[i];
        if (d.k < 1 || d.k > PGP_MAXK) return pg_set_error(PG_EINVAL, "pattern size must be 1..8");
        if (d.n_edges < 0 || (d.n_edges > 0 && !d.edges)) return pg_set_error(PG_EINVAL, "bad edge array");
        if (d.n_anti || d.labels || d.anti_vertex)
            return pg_set_error(PG_EINVAL, "generators take unlabeled patterns without anti-edges or anti-vertices");
        Pat p;
        p.k = d.k;
        p.vertex_induced = d.vertex_induced ? 1 : 0;
        for (int e = 0; e < d.n_edges; ++e) {
            const int u = d.edges[2 * e], w = d.edges[2 * e + 1];
            if (u < 0 || w < 0 || u >= d.k || w >= d.k || u == w) return pg_set_error(PG_EINVAL, "bad pattern edge");
            p.adj[u] |= (uint8_t)(1u << w);
            p.adj[w] |= (uint8_t)(1u << u);
        }
        c.add(p);
    }
    return finish(c, out);
}

extern "C" int pg_patterns_extend(const pg_pattern_set *in, int32_t by_vertex, pg_pattern_set **out) {
    if (!in || !out) return pg_set_error(PG_EINVAL, "NULL argument");
    *out = nullptr;
    Collector c;
    if (by_vertex) extend_vertex(in->pats, c);
    else extend_edge(in->pats, c);
    return finish(c, out);
}

extern "C" int pg_patterns_size(const pg_pattern_set *s, int64_t *n) {
    if (!s || !n) return pg_set_error(PG_EINVAL, "NULL argument");
    *n = (int64_t)s->pats.size();
    return PG_OK;
}

extern "C" int pg_patterns_get(const pg_pattern_set *s, int64_t i, int32_t *k, int32_t *n_edges_out, int32_t *edges,
                               int32_t *vertex_induced) {
    if (!s || !k || !n_edges_out || !edges || !vertex_induced) return pg_set_error(PG_EINVAL, "NULL argument");
    if (i < 0 || i >= (int64_t)s->pats.size()) return pg_set_error(PG_EINVAL, "index out of range");
    const Pat &p = s->pats[i];
    *k = p.k;
    int e = 0;
    for (int u = 0; u < p.k; ++u)
        for (int w = u + 1; w < p.k; ++w)
            if (p.adj[u] >> w & 1) {
                edges[2 * e] = u;
                edges[2 * e + 1] = w;
                ++e;
            }
    *n_edges_out = e;
    *vertex_induced = p.vertex_induced;
    return PG_OK;
}

extern "C" void pg_free_patterns(pg_pattern_set *s) { delete s; }
