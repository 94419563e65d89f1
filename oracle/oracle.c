/*
 * Plain CPU oracle for pattern counting and MNI support.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * Every function states the definition it writes out:
 *
 *  or_count_maps     Section 2.1 (match / edge-induced / vertex-induced),
 *                    Section 3.1.1 (anti-edge constraint) and Section 3.1.2
 *                    (anti-vertex constraint): the number of injective maps
 *                    phi from the regular pattern vertices into G that keep
 *                    every edge, every anti-edge, every label and every
 *                    anti-vertex constraint.  Backtracking by neighbour
 *                    expansion (patterns are connected), no partial order.
 *  or_list_maps      the maps counted by or_count_maps themselves, one row of
 *                    k images per map (-1 at anti-vertices), for listing
 *                    (Section 3.2, match()): matches are the classes of maps
 *                    under Aut, formed by the caller.
 *  or_pattern_aut    |Aut| of a pattern by brute force over all k!
 *                    permutations (edges, anti-edges, labels and anti-vertex
 *                    status preserved), restricted to the regular vertices.
 *                    Distinct matches = maps / |Aut| (Section 2.1: automorphic
 *                    matches are one subgraph seen through several maps).
 *  or_triangles      trace(A^3)/6 written as sum over edges of common
 *                    neighbours / 3.
 *  or_kcliques       textbook oriented k-clique lister (Chiba-Nishizeki /
 *                    kClist style: orient every edge from lower to higher
 *                    (degree, id), recurse on out-neighbour intersections).
 *  or_motif4_noninduced  non-induced counts of the six connected 4-vertex
 *                    shapes by plain degree / co-degree formulas.
 *  or_mni_bruteforce MNI support (Section 2.1, minimum node image): for every
 *                    pattern vertex the set of data vertices some valid map
 *                    sends it to; support = the smallest such set.
 *  or_fsm_domains    domain sizes of every labeled pattern with 1..3 edges by
 *                    per-vertex search (see the function).
 *  or_domain_sizes   MNI domains by their plain definition, one vertex at a
 *                    time: v is in D(u) iff backtracking from u -> v finds
 *                    one valid map (first hit ends the search).  Shares no
 *                    shortcut with or_fsm_domains, so it checks it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXK 8

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_EOVERFLOW = 3 };

typedef struct {
    int64_t n;
    const int64_t *off;   /* n+1 */
    const int32_t *adj;   /* off[n], each list sorted ascending */
    const int32_t *label; /* n, or NULL */
} or_graph;

typedef struct {
    int32_t k;
    uint8_t rel[OR_MAXK * OR_MAXK]; /* 0 none, 1 edge, 2 anti-edge (symmetric) */
    int32_t label[OR_MAXK];         /* -1 = any */
    uint8_t anti_vertex[OR_MAXK];   /* 1 = anti-vertex */
    int32_t vertex_induced;         /* 1 = the image must induce exactly p's edges */
} or_pattern;

/* ------------------------------------------------------------------------ */

static int adjacent(const or_graph *g, int64_t a, int64_t b) {
    int64_t lo = g->off[a], hi = g->off[a + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        int32_t x = g->adj[mid];
        if (x == b) return 1;
        if (x < b) lo = mid + 1; else hi = mid;
    }
    return 0;
}

static int pat_rel(const or_pattern *p, int u, int w) { return p->rel[u * OR_MAXK + w]; }

/* Regular vertices in a BFS order over regular edges; parent[i] is the
 * position of an earlier regular neighbour (-1 for the root). */
typedef struct {
    int nreg;
    int order[OR_MAXK];
    int parent[OR_MAXK];
} bfs_order;

static int make_order(const or_pattern *p, bfs_order *o) {
    int k = p->k, seen[OR_MAXK] = {0}, pos_of[OR_MAXK];
    o->nreg = 0;
    int root = -1;
    for (int u = 0; u < k; ++u) if (!p->anti_vertex[u]) { root = u; break; }
    if (root < 0) return OR_EINVAL;
    o->order[0] = root; o->parent[0] = -1; seen[root] = 1; pos_of[root] = 0; o->nreg = 1;
    for (int i = 0; i < o->nreg; ++i) {
        int u = o->order[i];
        for (int w = 0; w < k; ++w) {
            if (seen[w] || p->anti_vertex[w] || pat_rel(p, u, w) != 1) continue;
            seen[w] = 1; pos_of[w] = o->nreg;
            o->order[o->nreg] = w; o->parent[o->nreg] = i; o->nreg++;
        }
    }
    int nreg_total = 0;
    for (int u = 0; u < k; ++u) nreg_total += !p->anti_vertex[u];
    if (o->nreg != nreg_total) return OR_EINVAL; /* disconnected */
    (void)pos_of;
    return OR_OK;
}

static int validate_pattern(const or_pattern *p) {
    if (p->k < 1 || p->k > OR_MAXK) return OR_EINVAL;
    for (int u = 0; u < p->k; ++u) {
        if (pat_rel(p, u, u) != 0) return OR_EINVAL;
        for (int w = 0; w < p->k; ++w) {
            if (pat_rel(p, u, w) != pat_rel(p, w, u)) return OR_EINVAL;
            if (pat_rel(p, u, w) > 2) return OR_EINVAL;
            /* anti-vertices touch other vertices through anti-edges only */
            if ((p->anti_vertex[u] || p->anti_vertex[w]) && pat_rel(p, u, w) == 1) return OR_EINVAL;
        }
        if (p->anti_vertex[u]) {
            int any = 0;
            for (int w = 0; w < p->k; ++w) any |= (pat_rel(p, u, w) == 2 && !p->anti_vertex[w]);
            if (!any) return OR_EINVAL;
        }
    }
    return OR_OK;
}

/* ---------------------------- |Aut| -------------------------------------- */

static int next_perm(int *a, int k) {
    int i = k - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) return 0;
    int j = k - 1;
    while (a[j] <= a[i]) --j;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = k - 1; l < r; ++l, --r) { t = a[l]; a[l] = a[r]; a[r] = t; }
    return 1;
}

/* Relation used for automorphisms: for a vertex-induced pattern every
 * non-adjacent pair of regular vertices is constrained to be non-adjacent,
 * which a permutation preserving edges preserves as well. */
int or_pattern_aut(const or_pattern *p, uint64_t *aut_out) {
    if (validate_pattern(p)) return OR_EINVAL;
    int k = p->k, perm[OR_MAXK];
    for (int i = 0; i < k; ++i) perm[i] = i;
    /* distinct restrictions to regular vertices, encoded base-8 */
    uint64_t *seen = NULL; size_t nseen = 0, cap = 0;
    do {
        int ok = 1;
        for (int u = 0; u < k && ok; ++u) {
            if (p->anti_vertex[u] != p->anti_vertex[perm[u]]) ok = 0;
            if (p->label[u] != p->label[perm[u]]) ok = 0;
            for (int w = 0; w < k && ok; ++w)
                if (pat_rel(p, u, w) != pat_rel(p, perm[u], perm[w])) ok = 0;
        }
        if (!ok) continue;
        uint64_t code = 0;
        for (int u = 0; u < k; ++u)
            code = code * 8 + (p->anti_vertex[u] ? 0 : (uint64_t)perm[u]);
        int dup = 0;
        for (size_t i = 0; i < nseen; ++i) if (seen[i] == code) { dup = 1; break; }
        if (dup) continue;
        if (nseen == cap) {
            cap = cap ? cap * 2 : 64;
            uint64_t *t = (uint64_t *)realloc(seen, cap * sizeof(uint64_t));
            if (!t) { free(seen); return OR_ENOMEM; }
            seen = t;
        }
        seen[nseen++] = code;
    } while (next_perm(perm, k));
    free(seen);
    *aut_out = nseen;
    return OR_OK;
}

/* ---------------------------- count maps ---------------------------------- */

typedef struct {
    const or_graph *g;
    const or_pattern *p;
    bfs_order o;
    int64_t phi[OR_MAXK]; /* indexed by pattern vertex */
} bt_ctx;

/* Anti-vertex constraint (Section 3.1.2): with S the images of the anti-vertex's
 * neighbours, no data vertex may lie in every adj(v) \ m(adj_p(m^-1(v))), v in S. */
static int anti_vertices_ok(bt_ctx *c) {
    const or_pattern *p = c->p;
    const or_graph *g = c->g;
    for (int a = 0; a < p->k; ++a) {
        if (!p->anti_vertex[a]) continue;
        int nb[OR_MAXK], nn = 0;
        for (int u = 0; u < p->k; ++u)
            if (!p->anti_vertex[u] && pat_rel(p, a, u) == 2) nb[nn++] = u;
        int64_t v0 = c->phi[nb[0]];
        for (int64_t e = g->off[v0]; e < g->off[v0 + 1]; ++e) {
            int64_t x = g->adj[e];
            int in_all = 1;
            for (int i = 0; i < nn && in_all; ++i) {
                int u = nb[i];
                int64_t v = c->phi[u];
                if (i > 0 && !adjacent(g, v, x)) { in_all = 0; break; }
                /* x must not be the image of a pattern neighbour of u */
                for (int w = 0; w < p->k; ++w)
                    if (!p->anti_vertex[w] && pat_rel(p, u, w) == 1 && c->phi[w] == x) { in_all = 0; break; }
            }
            if (in_all) return 0;
        }
    }
    return 1;
}

static int compatible(bt_ctx *c, int pos, int64_t x) {
    const or_pattern *p = c->p;
    const or_graph *g = c->g;
    int u = c->o.order[pos];
    if (p->label[u] >= 0) {
        if (!g->label || g->label[x] != p->label[u]) return 0;
    }
    for (int i = 0; i < pos; ++i) {
        int w = c->o.order[i];
        int64_t y = c->phi[w];
        if (y == x) return 0; /* injective */
        int r = pat_rel(p, u, w);
        int adjg = adjacent(g, x, y);
        if (r == 1 && !adjg) return 0;
        if (r == 2 && adjg) return 0;
        if (r == 0 && p->vertex_induced && adjg) return 0;
    }
    return 1;
}

static uint64_t bt(bt_ctx *c, int pos) {
    if (pos == c->o.nreg) return anti_vertices_ok(c) ? 1u : 0u;
    int u = c->o.order[pos];
    int64_t par = c->phi[c->o.order[c->o.parent[pos]]];
    uint64_t total = 0;
    for (int64_t e = c->g->off[par]; e < c->g->off[par + 1]; ++e) {
        int64_t x = c->g->adj[e];
        if (!compatible(c, pos, x)) continue;
        c->phi[u] = x;
        total += bt(c, pos + 1);
    }
    return total;
}

int or_count_maps(const or_graph *g, const or_pattern *p, int nthreads, uint64_t *maps_out) {
    if (validate_pattern(p)) return OR_EINVAL;
    bfs_order o;
    if (make_order(p, &o)) return OR_EINVAL;
    uint64_t total = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (int64_t v = 0; v < g->n; ++v) {
        bt_ctx c;
        c.g = g; c.p = p; c.o = o;
        if (!compatible(&c, 0, v)) continue;
        c.phi[o.order[0]] = v;
        total += bt(&c, 1);
    }
    *maps_out = total;
    return OR_OK;
}

/* ---------------------------- list maps ----------------------------------- */

typedef struct {
    bt_ctx c;
    int32_t *out;
    uint64_t capacity, n;
} list_ctx;

static void bt_list(list_ctx *L, int pos) {
    bt_ctx *c = &L->c;
    if (pos == c->o.nreg) {
        if (!anti_vertices_ok(c)) return;
        if (L->n < L->capacity) {
            int32_t *row = L->out + L->n * (uint64_t)c->p->k;
            for (int u = 0; u < c->p->k; ++u) row[u] = c->p->anti_vertex[u] ? -1 : (int32_t)c->phi[u];
        }
        L->n++;
        return;
    }
    int u = c->o.order[pos];
    int64_t par = c->phi[c->o.order[c->o.parent[pos]]];
    for (int64_t e = c->g->off[par]; e < c->g->off[par + 1]; ++e) {
        int64_t x = c->g->adj[e];
        if (!compatible(c, pos, x)) continue;
        c->phi[u] = x;
        bt_list(L, pos + 1);
    }
}

/* Every valid map as a row of k data vertices (phi(u) in column u, -1 for
 * anti-vertices), at most `capacity` rows written; *n_out = number of maps.
 * Single-threaded: meant for small graphs. */
int or_list_maps(const or_graph *g, const or_pattern *p, int32_t *out, uint64_t capacity, uint64_t *n_out) {
    if (validate_pattern(p)) return OR_EINVAL;
    list_ctx L;
    if (make_order(p, &L.c.o)) return OR_EINVAL;
    L.c.g = g; L.c.p = p;
    L.out = out; L.capacity = capacity; L.n = 0;
    for (int64_t v = 0; v < g->n; ++v) {
        if (!compatible(&L.c, 0, v)) continue;
        L.c.phi[L.c.o.order[0]] = v;
        bt_list(&L, 1);
    }
    *n_out = L.n;
    return OR_OK;
}

/* ---------------------------- MNI domains --------------------------------- */

typedef struct {
    bt_ctx c;
    uint8_t *dom; /* k * n flags */
} mni_ctx;

static void bt_mni(mni_ctx *m, int pos) {
    bt_ctx *c = &m->c;
    if (pos == c->o.nreg) {
        if (!anti_vertices_ok(c)) return;
        for (int i = 0; i < c->o.nreg; ++i) {
            int u = c->o.order[i];
            m->dom[(int64_t)u * c->g->n + c->phi[u]] = 1;
        }
        return;
    }
    int u = c->o.order[pos];
    int64_t par = c->phi[c->o.order[c->o.parent[pos]]];
    for (int64_t e = c->g->off[par]; e < c->g->off[par + 1]; ++e) {
        int64_t x = c->g->adj[e];
        if (!compatible(c, pos, x)) continue;
        c->phi[u] = x;
        bt_mni(m, pos + 1);
    }
}

/* Domain sizes |{phi(u)}| per pattern vertex u (anti-vertices get 0) over all
 * valid maps; the MNI support is the minimum over regular vertices.
 * Single-threaded: meant for small graphs. */
int or_mni_bruteforce(const or_graph *g, const or_pattern *p, uint64_t *domain_size_out) {
    if (validate_pattern(p)) return OR_EINVAL;
    mni_ctx m;
    if (make_order(p, &m.c.o)) return OR_EINVAL;
    m.c.g = g; m.c.p = p;
    m.dom = (uint8_t *)calloc((size_t)p->k * (size_t)g->n, 1);
    if (!m.dom) return OR_ENOMEM;
    for (int64_t v = 0; v < g->n; ++v) {
        if (!compatible(&m.c, 0, v)) continue;
        m.c.phi[m.c.o.order[0]] = v;
        bt_mni(&m, 1);
    }
    for (int u = 0; u < p->k; ++u) {
        uint64_t s = 0;
        for (int64_t v = 0; v < g->n; ++v) s += m.dom[(int64_t)u * g->n + v];
        domain_size_out[u] = s;
    }
    free(m.dom);
    return OR_OK;
}

/* ---------------------------- domain membership ---------------------------- */

/* BFS order of the regular vertices rooted at `root`. */
static int make_order_from(const or_pattern *p, int root, bfs_order *o) {
    int k = p->k, seen[OR_MAXK] = {0};
    if (root < 0 || root >= k || p->anti_vertex[root]) return OR_EINVAL;
    o->order[0] = root; o->parent[0] = -1; seen[root] = 1; o->nreg = 1;
    for (int i = 0; i < o->nreg; ++i) {
        int u = o->order[i];
        for (int w = 0; w < k; ++w) {
            if (seen[w] || p->anti_vertex[w] || pat_rel(p, u, w) != 1) continue;
            seen[w] = 1;
            o->order[o->nreg] = w; o->parent[o->nreg] = i; o->nreg++;
        }
    }
    int nreg_total = 0;
    for (int u = 0; u < k; ++u) nreg_total += !p->anti_vertex[u];
    return o->nreg == nreg_total ? OR_OK : OR_EINVAL;
}

/* 1 as soon as one valid completion of the positions pos.. exists. */
static int bt_exists(bt_ctx *c, int pos) {
    if (pos == c->o.nreg) return anti_vertices_ok(c);
    int u = c->o.order[pos];
    int64_t par = c->phi[c->o.order[c->o.parent[pos]]];
    for (int64_t e = c->g->off[par]; e < c->g->off[par + 1]; ++e) {
        int64_t x = c->g->adj[e];
        if (!compatible(c, pos, x)) continue;
        c->phi[u] = x;
        if (bt_exists(c, pos + 1)) return 1;
    }
    return 0;
}

/* Is data vertex v the image of pattern vertex u under some valid map? */
int or_domain_member(const or_graph *g, const or_pattern *p, int u, int64_t v, int *member) {
    if (validate_pattern(p) || v < 0 || v >= g->n) return OR_EINVAL;
    bt_ctx c;
    c.g = g; c.p = p;
    if (make_order_from(p, u, &c.o)) return OR_EINVAL;
    *member = 0;
    if (!compatible(&c, 0, v)) return OR_OK;
    c.phi[u] = v;
    *member = bt_exists(&c, 1);
    return OR_OK;
}

/* |D(u)| for every pattern vertex u (0 for anti-vertices): the number of
 * data vertices v with or_domain_member(u, v).  OpenMP over v. */
int or_domain_sizes(const or_graph *g, const or_pattern *p, int nthreads, uint64_t *size_out) {
    if (validate_pattern(p)) return OR_EINVAL;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int u = 0; u < p->k; ++u) {
        size_out[u] = 0;
        if (p->anti_vertex[u]) continue;
        bfs_order o;
        if (make_order_from(p, u, &o)) return OR_EINVAL;
        uint64_t s = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : s)
        for (int64_t v = 0; v < g->n; ++v) {
            bt_ctx c;
            c.g = g; c.p = p; c.o = o;
            if (!compatible(&c, 0, v)) continue;
            c.phi[u] = v;
            s += (uint64_t)bt_exists(&c, 1);
        }
        size_out[u] = s;
    }
    return OR_OK;
}

/* ---------------------------- triangles ----------------------------------- */

static int64_t common_count(const int32_t *a, int64_t na, const int32_t *b, int64_t nb) {
    int64_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

/* trace(A^3)/6 = (1/3) sum over undirected edges {u,v} of |N(u) & N(v)|. */
uint64_t or_triangles(const or_graph *g, int nthreads) {
    uint64_t s = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : s)
    for (int64_t u = 0; u < g->n; ++u) {
        for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e) {
            int64_t v = g->adj[e];
            if (v <= u) continue;
            s += (uint64_t)common_count(g->adj + g->off[u], g->off[u + 1] - g->off[u],
                                        g->adj + g->off[v], g->off[v + 1] - g->off[v]);
        }
    }
    return s / 3;
}

/* Per-vertex triangle counts t_v (sum over edges at v of common neighbours / 2). */
int or_triangles_per_vertex(const or_graph *g, int nthreads, uint64_t *t_out) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t u = 0; u < g->n; ++u) {
        uint64_t s = 0;
        for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e) {
            int64_t v = g->adj[e];
            s += (uint64_t)common_count(g->adj + g->off[u], g->off[u + 1] - g->off[u],
                                        g->adj + g->off[v], g->off[v + 1] - g->off[v]);
        }
        t_out[u] = s / 2;
    }
    return OR_OK;
}

/* ---------------------------- k-cliques ----------------------------------- */

/* Orientation u -> v iff (deg u, u) < (deg v, v): a total order, so every
 * k-clique is listed exactly once, from its lowest vertex in that order. */
static int build_out(const or_graph *g, int64_t **out_off, int32_t **out_adj, int64_t *maxout) {
    int64_t n = g->n;
    int64_t *oo = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!oo) return OR_ENOMEM;
    oo[0] = 0;
    *maxout = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t du = g->off[u + 1] - g->off[u], c = 0;
        for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e) {
            int64_t v = g->adj[e], dv = g->off[v + 1] - g->off[v];
            if (du < dv || (du == dv && u < v)) ++c;
        }
        oo[u + 1] = oo[u] + c;
        if (c > *maxout) *maxout = c;
    }
    int32_t *oa = (int32_t *)malloc((size_t)(oo[n] ? oo[n] : 1) * sizeof(int32_t));
    if (!oa) { free(oo); return OR_ENOMEM; }
    for (int64_t u = 0; u < n; ++u) {
        int64_t du = g->off[u + 1] - g->off[u], w = oo[u];
        for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e) {
            int64_t v = g->adj[e], dv = g->off[v + 1] - g->off[v];
            if (du < dv || (du == dv && u < v)) oa[w++] = (int32_t)v;
        }
    }
    *out_off = oo; *out_adj = oa;
    return OR_OK;
}

static int64_t intersect_into(const int32_t *a, int64_t na, const int32_t *b, int64_t nb, int32_t *out) {
    int64_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { out[c++] = a[i]; ++i; ++j; }
    }
    return c;
}

static uint64_t clique_rec(const int64_t *oo, const int32_t *oa, const int32_t *P, int64_t np,
                           int depth, int k, int32_t *buf, int64_t maxout) {
    /* P = candidates common to the depth vertices chosen so far */
    if (depth == k - 1) return (uint64_t)np;
    uint64_t s = 0;
    int32_t *next = buf;
    for (int64_t i = 0; i < np; ++i) {
        int32_t u = P[i];
        int64_t nn = intersect_into(P, np, oa + oo[u], oo[u + 1] - oo[u], next);
        if (depth + 1 == k - 1) s += (uint64_t)nn;
        else s += clique_rec(oo, oa, next, nn, depth + 1, k, buf + maxout, maxout);
    }
    return s;
}

/* Number of k-cliques whose lowest vertex (in (degree, id) order) lies in
 * sources[0..nsources) (sources == NULL: all vertices). */
int or_kcliques(const or_graph *g, int k, int nthreads, const int32_t *sources, int64_t nsources,
                uint64_t *count_out) {
    if (k < 1 || k > 16) return OR_EINVAL;
    if (k == 1) { *count_out = sources ? (uint64_t)nsources : (uint64_t)g->n; return OR_OK; }
    int64_t *oo; int32_t *oa; int64_t maxout;
    if (build_out(g, &oo, &oa, &maxout)) return OR_ENOMEM;
    int64_t ns = sources ? nsources : g->n;
    uint64_t total = 0;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel reduction(+ : total)
    {
        int32_t *buf = (int32_t *)malloc((size_t)(maxout + 1) * (size_t)(k + 1) * sizeof(int32_t));
        if (!buf) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t i = 0; i < ns; ++i) {
                int64_t v = sources ? sources[i] : i;
                total += clique_rec(oo, oa, oa + oo[v], oo[v + 1] - oo[v], 1, k, buf, maxout + 1);
            }
            free(buf);
        }
    }
    free(oo); free(oa);
    if (err) return OR_ENOMEM;
    *count_out = total;
    return OR_OK;
}

/* ---------------------------- 4-vertex shapes ----------------------------- */

/* Non-induced counts (number of subgraphs isomorphic to the shape):
 * out[0] star   = sum_v C(d_v, 3)
 * out[1] path   = sum_{edges uv} (d_u - 1)(d_v - 1) - 3 T
 * out[2] tailed = sum_v t_v (d_v - 2)
 * out[3] cycle  = 1/2 sum_{u < w} C(codeg(u, w), 2)
 * out[4] diamond= sum_{edges uv} C(codeg(u, v), 2)
 * out[5] clique = number of 4-cliques (oriented lister)
 */
int or_motif4_noninduced(const or_graph *g, int nthreads, uint64_t *out) {
    int64_t n = g->n;
    uint64_t *t = (uint64_t *)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    if (!t) return OR_ENOMEM;
    or_triangles_per_vertex(g, nthreads, t);
    unsigned __int128 star = 0, path = 0, tailed = 0, tri3 = 0, diamond = 0, cyc2 = 0;
    for (int64_t v = 0; v < n; ++v) {
        uint64_t d = (uint64_t)(g->off[v + 1] - g->off[v]);
        if (d >= 3) star += (unsigned __int128)d * (d - 1) * (d - 2) / 6;
        if (d >= 2) tailed += (unsigned __int128)t[v] * (d - 2);
        tri3 += t[v]; /* sum_v t_v = 3 T */
    }
    free(t);
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        unsigned __int128 lpath = 0, ldiamond = 0, lcyc2 = 0;
        int32_t *cnt = (int32_t *)calloc((size_t)(n ? n : 1), sizeof(int32_t));
        int32_t *touched = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
        if (!cnt || !touched) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t u = 0; u < n; ++u) {
                uint64_t du = (uint64_t)(g->off[u + 1] - g->off[u]);
                /* co-degree of u with every w > u: walk wedges u - a - w */
                int64_t nt = 0;
                for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e) {
                    int64_t a = g->adj[e];
                    for (int64_t f = g->off[a]; f < g->off[a + 1]; ++f) {
                        int64_t w = g->adj[f];
                        if (w <= u) continue;
                        if (cnt[w]++ == 0) touched[nt++] = (int32_t)w;
                    }
                }
                for (int64_t i = 0; i < nt; ++i) {
                    uint64_t c = (uint64_t)cnt[touched[i]];
                    lcyc2 += (unsigned __int128)c * (c - 1) / 2;
                }
                /* edges uv with v > u: path middle edge and diamond chord */
                for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e) {
                    int64_t v = g->adj[e];
                    if (v <= u) continue;
                    uint64_t dv = (uint64_t)(g->off[v + 1] - g->off[v]);
                    lpath += (unsigned __int128)(du - 1) * (dv - 1);
                    uint64_t c = (uint64_t)cnt[v];
                    ldiamond += (unsigned __int128)c * (c - 1) / 2;
                }
                for (int64_t i = 0; i < nt; ++i) cnt[touched[i]] = 0;
            }
#pragma omp critical
            {
                path += lpath; diamond += ldiamond; cyc2 += lcyc2;
            }
        }
        free(cnt); free(touched);
    }
    if (err) return OR_ENOMEM;
    uint64_t k4;
    if (or_kcliques(g, 4, nthreads, NULL, 0, &k4)) return OR_ENOMEM;
    unsigned __int128 vals[6];
    vals[0] = star;
    vals[1] = path - tri3; /* 3T == sum_v t_v */
    vals[2] = tailed;
    vals[3] = cyc2 / 2;
    vals[4] = diamond;
    vals[5] = k4;
    for (int i = 0; i < 6; ++i) {
        if (vals[i] > (unsigned __int128)UINT64_MAX) return OR_EOVERFLOW;
        out[i] = (uint64_t)vals[i];
    }
    return OR_OK;
}

int or_version(void) { return 1; }

/* ---------------------------- FSM (MNI, <= 3 edges) ----------------------- */

/*
 * Labeled frequent subgraph mining up to three edges (Section 2.1 FSM with the
 * MNI support; Section 3.2.1 label discovery): for every connected labeled
 * edge-induced pattern with 1..3 edges, the MNI support = min over pattern
 * vertices u of |{phi(u)}| over all valid maps phi.  A data vertex v lies in
 * the domain of position u iff some valid map sends u to v; this oracle
 * decides that per vertex by direct search over v's neighbourhood, using
 * neighbour label counts only for the last (leaf) vertex of a shape, with the
 * vertices already used subtracted explicitly.
 *
 * Output per label tuple (L = number of labels, v's own label first):
 *   E[L][L]        v has a neighbour labeled y                      (edge end)
 *   WC[L][L][L]    v has distinct neighbours labeled x, y           (wedge centre)
 *   WL[L][L][L]    v - w(c) - u(y), u != v                          (wedge leaf)
 *   T[L][L][L]     v in a triangle with neighbours labeled y, z     (triangle)
 *   SC[L][L][L][L] v has distinct neighbours labeled x, y, z        (star centre)
 *   SL[L][L][L][L] v - w(c), w has two more neighbours y, z (!= v)  (star leaf)
 *   PE[L][L][L][L] v - w(b) - u(c) - x(d), all distinct             (path end)
 *   PI[L][L][L][L] a'(a) - v - c'(c) - d'(d), all distinct          (path inner)
 * Each entry counts the vertices with label = first index satisfying it.
 * Only index combinations with the listed meaning are filled (x <= y etc. are
 * not assumed: all orderings are filled).
 */
static int has_edge(const or_graph *g, int64_t a, int64_t b) { return adjacent(g, a, b); }

int or_fsm_domains(const or_graph *g, int nl, int nthreads, uint64_t *E, uint64_t *WC, uint64_t *WL,
                   uint64_t *T, uint64_t *SC, uint64_t *SL, uint64_t *PE, uint64_t *PI) {
    if (!g->label || nl < 1 || nl > 32) return OR_EINVAL;
    const int64_t n = g->n;
    const int L = nl, L2 = nl * nl, L3 = nl * nl * nl;
    size_t sE = (size_t)L2, s3 = (size_t)L3, s4 = (size_t)L3 * L;
    memset(E, 0, sE * 8); memset(WC, 0, s3 * 8); memset(WL, 0, s3 * 8); memset(T, 0, s3 * 8);
    memset(SC, 0, s4 * 8); memset(SL, 0, s4 * 8); memset(PE, 0, s4 * 8); memset(PI, 0, s4 * 8);
    /* neighbour label counts */
    int32_t *H = (int32_t *)calloc((size_t)n * L + 1, sizeof(int32_t));
    if (!H) return OR_ENOMEM;
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e) H[v * L + g->label[g->adj[e]]]++;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        uint8_t *fWL = (uint8_t *)malloc((size_t)L2), *fT = (uint8_t *)malloc((size_t)L2);
        uint8_t *fSL = (uint8_t *)malloc((size_t)L3), *fPE = (uint8_t *)malloc((size_t)L3);
        uint8_t *fPI = (uint8_t *)malloc((size_t)L3);
        uint64_t *lE = (uint64_t *)calloc(sE, 8), *lWC = (uint64_t *)calloc(s3, 8), *lWL = (uint64_t *)calloc(s3, 8);
        uint64_t *lT = (uint64_t *)calloc(s3, 8), *lSC = (uint64_t *)calloc(s4, 8), *lSL = (uint64_t *)calloc(s4, 8);
        uint64_t *lPE = (uint64_t *)calloc(s4, 8), *lPI = (uint64_t *)calloc(s4, 8);
        if (!fWL || !fT || !fSL || !fPE || !fPI || !lE || !lWC || !lWL || !lT || !lSC || !lSL || !lPE || !lPI) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t v = 0; v < n; ++v) {
                const int lv = g->label[v];
                const int32_t *Hv = H + v * L;
                /* edge end, wedge centre, star centre: from v's own counts */
                for (int y = 0; y < L; ++y) {
                    if (Hv[y] >= 1) lE[lv * L + y]++;
                    for (int x = 0; x < L; ++x) {
                        const int ok = (x == y) ? (Hv[x] >= 2) : (Hv[x] >= 1 && Hv[y] >= 1);
                        if (ok) lWC[(size_t)lv * L2 + x * L + y]++;
                        for (int z = 0; z < L; ++z) {
                            int cnt[32] = {0};
                            cnt[x]++; cnt[y]++; cnt[z]++;
                            if (Hv[x] >= cnt[x] && Hv[y] >= cnt[y] && Hv[z] >= cnt[z])
                                lSC[(size_t)lv * L3 + (size_t)x * L2 + y * L + z]++;
                        }
                    }
                }
                memset(fWL, 0, L2); memset(fT, 0, L2); memset(fSL, 0, L3); memset(fPE, 0, L3); memset(fPI, 0, L3);
                for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e) {
                    const int64_t w = g->adj[e];
                    const int lw = g->label[w];
                    const int32_t *Hw = H + w * L;
                    /* wedge leaf and star leaf: centre w, other leaves among adj(w) \ {v} */
                    for (int y = 0; y < L; ++y) {
                        int hy = Hw[y] - (y == lv);
                        if (hy >= 1) fWL[lw * L + y] = 1;
                        for (int z = 0; z < L; ++z) {
                            int hz = Hw[z] - (z == lv);
                            int ok = (y == z) ? (hy >= 2) : (hy >= 1 && hz >= 1);
                            if (ok) fSL[(size_t)lw * L2 + y * L + z] = 1;
                        }
                    }
                    /* triangle: u in adj(v) n adj(w), by merging the two lists */
                    {
                        int64_t i = g->off[v], j = g->off[w];
                        while (i < g->off[v + 1] && j < g->off[w + 1]) {
                            if (g->adj[i] < g->adj[j]) ++i;
                            else if (g->adj[i] > g->adj[j]) ++j;
                            else { fT[lw * L + g->label[g->adj[i]]] = 1; ++i; ++j; }
                        }
                    }
                    /* path end: v - w - u - x with u != v, x not in {v, w}.
                     * Labels d with a neighbour x of u other than w: count
                     * Hu[d] - [d == lw] >= 1; when it is exactly 1 for d = lv
                     * the single candidate may be v itself (if v ~ u). */
                    for (int64_t f = g->off[w]; f < g->off[w + 1]; ++f) {
                        const int64_t u = g->adj[f];
                        if (u == v) continue;
                        const int lu = g->label[u];
                        const int32_t *Hu = H + u * L;
                        uint8_t *row = fPE + (size_t)lw * L2 + lu * L;
                        for (int d = 0; d < L; ++d) {
                            int c = Hu[d] - (d == lw);
                            if (d == lv && c == 1 && has_edge(g, v, u)) c = 0;
                            if (c >= 1) row[d] = 1;
                        }
                    }
                    /* path inner: a' - v - w(=c') - d', a' != w, d' not in {v, a'} */
                    for (int a = 0; a < L; ++a) {
                        int na = Hv[a] - (a == lw); /* a' in adj(v) \ {w} */
                        if (na < 1) continue;
                        for (int d = 0; d < L; ++d) {
                            int nd = Hw[d] - (d == lv); /* d' in adj(w) \ {v} */
                            if (nd < 1) continue;
                            int ok = 1;
                            if (a == d && na == 1 && nd == 1) {
                                /* the single a' and the single d' coincide iff
                                 * some common neighbour of v and w has label a */
                                for (int64_t f = g->off[v]; f < g->off[v + 1]; ++f) {
                                    const int64_t u = g->adj[f];
                                    if (u != w && g->label[u] == a && has_edge(g, w, u)) { ok = 0; break; }
                                }
                            }
                            if (ok) fPI[(size_t)a * L2 + lw * L + d] = 1;
                        }
                    }
                }
                for (int i = 0; i < L2; ++i) {
                    if (fWL[i]) lWL[(size_t)lv * L2 + i]++;
                    if (fT[i]) lT[(size_t)lv * L2 + i]++;
                }
                for (int i = 0; i < L3; ++i) {
                    if (fSL[i]) lSL[(size_t)lv * L3 + i]++;
                    if (fPE[i]) lPE[(size_t)lv * L3 + i]++;
                    if (fPI[i]) lPI[(size_t)lv * L3 + i]++;
                }
            }
#pragma omp critical
            {
                for (size_t i = 0; i < sE; ++i) E[i] += lE[i];
                for (size_t i = 0; i < s3; ++i) { WC[i] += lWC[i]; WL[i] += lWL[i]; T[i] += lT[i]; }
                for (size_t i = 0; i < s4; ++i) { SC[i] += lSC[i]; SL[i] += lSL[i]; PE[i] += lPE[i]; PI[i] += lPI[i]; }
            }
        }
        free(fWL); free(fT); free(fSL); free(fPE); free(fPI);
        free(lE); free(lWC); free(lWL); free(lT); free(lSC); free(lSL); free(lPE); free(lPI);
    }
    free(H);
    return err ? OR_ENOMEM : OR_OK;
}
