// Host plan compiler (Section 4.1, "Computing exploration plan" figure).
//
//   generatePlan(p):  breakSymmetries -> minConnectedVertexCover ->
//                     vertexInducedSubgraph -> computeMatchingOrders
//
// followed by the lowering of every matching order into the level program of
// plan.h.  Pattern-only: no graph is touched (Section 4.1, last paragraph).
#include "plan.h"

#include <algorithm>
#include <array>
#include <chrono>
#include <cstring>

#include "../../include/pg.h"

namespace {

using Perm = std::array<int8_t, PGP_MAXK>;

bool next_perm(int *a, int k) { return std::next_permutation(a, a + k); }

// All permutations of the k pattern vertices that keep edges, anti-edges,
// labels and anti-vertex status (anti-vertex-aware, Section 4.3).
std::vector<Perm> automorphisms(const PgPattern &p) {
    std::vector<Perm> out;
    int a[PGP_MAXK];
    for (int i = 0; i < p.k; ++i) a[i] = i;
    do {
        bool ok = true;
        for (int u = 0; u < p.k && ok; ++u) {
            if (p.label[u] != p.label[a[u]] || p.anti_vertex[u] != p.anti_vertex[a[u]]) ok = false;
            for (int w = 0; w < p.k && ok; ++w)
                if (p.rel[u][w] != p.rel[a[u]][a[w]]) ok = false;
        }
        if (ok) {
            Perm q{};
            for (int u = 0; u < p.k; ++u) q[u] = (int8_t)a[u];
            out.push_back(q);
        }
    } while (next_perm(a, p.k));
    return out;
}

int popcount(uint32_t x) { return __builtin_popcount(x); }

bool connected_by_edges(const PgPattern &p, uint32_t mask) {
    if (!mask) return false;
    int root = __builtin_ctz(mask);
    uint32_t seen = 1u << root, frontier = seen;
    while (frontier) {
        int u = __builtin_ctz(frontier);
        frontier &= frontier - 1;
        for (int w = 0; w < p.k; ++w)
            if ((mask >> w & 1) && !(seen >> w & 1) && p.rel[u][w] == 1) {
                seen |= 1u << w;
                frontier |= 1u << w;
            }
    }
    return seen == mask;
}

struct Closure {
    bool less[PGP_MAXK][PGP_MAXK] = {};
};

Closure close_po(int k, const std::vector<std::pair<int, int>> &po) {
    Closure c;
    for (auto &e : po) c.less[e.first][e.second] = true;
    for (int m = 0; m < k; ++m)
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j)
                if (c.less[i][m] && c.less[m][j]) c.less[i][j] = true;
    return c;
}

// Non-core vertices are independent (the core covers every edge and
// anti-edge).  A set G of non-core vertices is one counted chain when all of
// them carry the same label and the same relation (edge / anti-edge / none)
// to every vertex outside G, the same partial-order relation to every vertex
// outside G, and G is totally ordered by the partial order: the g members
// then share one candidate set S and have exactly C(|S|, g) increasing
// assignments.  Twin classes that fail the order conditions are split into
// single vertices.
bool twins(const PgPattern &p, int u, int w) {
    if (p.label[u] != p.label[w]) return false;
    for (int x = 0; x < p.k; ++x)
        if (x != u && x != w && p.rel[u][x] != p.rel[w][x]) return false;
    return true;
}

bool is_chain_group(const PgPattern &p, const Closure &c, const std::vector<int> &g) {
    uint32_t in = 0;
    for (int u : g) in |= 1u << u;
    for (int a : g)
        for (int b : g)
            if (a != b && !(c.less[a][b] || c.less[b][a])) return false;
    for (int x = 0; x < p.k; ++x) {
        if (in >> x & 1) continue;
        for (int u : g)
            if (c.less[u][x] != c.less[g[0]][x] || c.less[x][u] != c.less[x][g[0]]) return false;
    }
    return true;
}

std::vector<std::vector<int>> noncore_groups(const PgPattern &p, const Closure &c, uint32_t noncore,
                                             uint32_t singles = 0) {
    std::vector<std::vector<int>> classes, groups;
    for (int u = 0; u < p.k; ++u) {
        if (!(noncore >> u & 1)) continue;
        if (singles >> u & 1) {
            groups.push_back({u});
            continue;
        }
        bool placed = false;
        for (auto &g : classes)
            if (twins(p, g[0], u)) {
                g.push_back(u);
                placed = true;
                break;
            }
        if (!placed) classes.push_back({u});
    }
    for (auto &g : classes) {
        if (g.size() > 1 && is_chain_group(p, c, g)) {
            std::sort(g.begin(), g.end(), [&](int a, int b) { return c.less[a][b]; });
            groups.push_back(g);
        } else {
            for (int u : g) groups.push_back({u});
        }
    }
    return groups;
}

// Core levels, summed over all matching orders of `core`, that have no
// earlier-bound true neighbour placed above them in the order.  The start
// vertex binds the highest position, then the highest-position core vertex
// adjacent to a bound one (the exploration order used below); a level with a
// bound neighbour above it draws candidates from that neighbour's
// out-neighbourhood.
int core_scan_cost(const PgPattern &p, const Closure &cl, uint32_t core_mask) {
    std::vector<int> seq;
    for (int u = 0; u < p.k; ++u)
        if (core_mask >> u & 1) seq.push_back(u);
    const int c = (int)seq.size();
    int cost = 0;
    do {
        int pos[PGP_MAXK];
        for (int i = 0; i < c; ++i) pos[seq[i]] = i;
        bool ok = true;
        for (int a : seq)
            for (int b : seq)
                if (cl.less[a][b] && pos[a] > pos[b]) ok = false;
        if (!ok) continue;
        uint32_t bound = 1u << seq[c - 1];
        for (int step = 1; step < c; ++step) {
            int pick = -1;
            for (int i = c - 1; i >= 0 && pick < 0; --i) {
                const int u = seq[i];
                if (bound >> u & 1) continue;
                for (int x = 0; x < p.k; ++x)
                    if ((bound >> x & 1) && p.rel[u][x] == 1) { pick = u; break; }
            }
            bool cheap = false;
            for (int x = 0; x < p.k; ++x)
                if ((bound >> x & 1) && p.rel[pick][x] == 1 && pos[x] > pos[pick]) cheap = true;
            cost += cheap ? 0 : 1;
            bound |= 1u << pick;
        }
    } while (std::next_permutation(seq.begin(), seq.end()));
    return cost;
}

// Anti-vertex a: its regular neighbours, and those plus their pattern
// neighbours (every regular vertex its check reads).
struct AntiSpec {
    uint32_t nbrs, reads;
};

// computeMatchingOrders (Section 4.1) and the lowering of each order into a
// level program.  groups: the non-core groups; counted: index of the group
// counted from its set's cardinality (-1: every vertex enumerated); partner:
// index of a single-vertex group counted jointly with it (-1: none).
int lower_orders(const PgPattern &p, const Closure &cl, uint32_t best, const std::vector<std::vector<int>> &groups,
                 int counted, int partner, const std::vector<AntiSpec> &avs, std::vector<PgOrder> &orders,
                 std::string &err) {
    const int k = p.k;
    std::vector<int> core;
    for (int u = 0; u < k; ++u)
        if (best >> u & 1) core.push_back(u);
    const int c = (int)core.size();
    std::vector<int> seq = core;
    std::sort(seq.begin(), seq.end());
    do {
        int pos[PGP_MAXK];
        for (int i = 0; i < k; ++i) pos[i] = -1;
        for (int i = 0; i < c; ++i) pos[seq[i]] = i;
        bool ok = true;
        for (int a : core)
            for (int b : core)
                if (cl.less[a][b] && pos[a] > pos[b]) ok = false;
        if (!ok) continue;
        if (orders.size() >= PGP_MAX_ORDERS) { err = "too many matching orders"; return PG_EINVAL; }

        // Exploration order: start from the highest sequence position (the
        // task's start vertex, Section 5.2 high-to-low), then repeatedly the
        // highest-position core vertex adjacent to one already bound.
        int lvl_of[PGP_MAXK];
        for (int i = 0; i < k; ++i) lvl_of[i] = -1;
        std::vector<int> bound_order;
        bound_order.push_back(seq[c - 1]);
        lvl_of[seq[c - 1]] = 0;
        while ((int)bound_order.size() < c) {
            int pick = -1;
            for (int i = c - 1; i >= 0 && pick < 0; --i) {
                int u = seq[i];
                if (lvl_of[u] >= 0) continue;
                for (int x : bound_order)
                    if (p.rel[u][x] == 1) { pick = u; break; }
            }
            lvl_of[pick] = (int)bound_order.size();
            bound_order.push_back(pick);
        }
        // non-core: enumerated groups first (chain order), counted group last;
        // a single counted vertex is paired with another single non-core
        // vertex placed right before it (joint counting of the last two)
        std::vector<int> nc_order;
        for (int i = 0; i < (int)groups.size(); ++i)
            if (i != counted && i != partner)
                for (int u : groups[i]) nc_order.push_back(u);
        if (partner >= 0) nc_order.push_back(groups[partner][0]);
        for (int u : nc_order) {
            lvl_of[u] = (int)bound_order.size();
            bound_order.push_back(u);
        }
        int counted_first = -1;
        if (counted >= 0) {
            counted_first = groups[counted][0];
            lvl_of[counted_first] = (int)bound_order.size();
            bound_order.push_back(counted_first);
        }

        PgOrder ord;
        std::memset(&ord, 0, sizeof(ord));
        ord.n_levels = (int)bound_order.size();
        ord.n_core = c;
        for (int l = 0; l < ord.n_levels; ++l) {
            const int u = bound_order[l];
            PgLevel &L = ord.lv[l];
            L.pattern_vertex = (int8_t)u;
            L.is_core = (int8_t)((best >> u) & 1);
            L.label = p.label[u];
            L.group = (int8_t)((u == counted_first) ? (int)groups[counted].size() : 1);
            L.joint = (int8_t)(u == counted_first && partner >= 0);
            if (l == 0) continue;
            const bool core_level = L.is_core;
            int lo_core = -1, hi_core = -1; // tightest core bounds (by position)
            for (int j = 0; j < l; ++j) {
                const int x = bound_order[j];
                if (p.rel[u][x] == 1) L.int_src[L.n_int++] = (int8_t)j;
                if (p.rel[u][x] == 2) L.diff_src[L.n_diff++] = (int8_t)j;
                const bool x_core = (best >> x) & 1;
                bool below, above; // m(x) < m(u) / m(x) > m(u) required
                if (core_level && x_core) {
                    below = pos[x] < pos[u];
                    above = pos[x] > pos[u];
                } else {
                    below = cl.less[x][u];
                    above = cl.less[u][x];
                }
                if (x_core && (below || above)) {
                    if (below && (lo_core < 0 || pos[x] > pos[bound_order[lo_core]])) lo_core = j;
                    if (above && (hi_core < 0 || pos[x] < pos[bound_order[hi_core]])) hi_core = j;
                } else {
                    if (below) L.lo_src[L.n_lo++] = (int8_t)j;
                    if (above) L.hi_src[L.n_hi++] = (int8_t)j;
                }
            }
            if (lo_core >= 0) L.lo_src[L.n_lo++] = (int8_t)lo_core;
            if (hi_core >= 0) L.hi_src[L.n_hi++] = (int8_t)hi_core;
            // candidates adjacent to a bound vertex x and ranked below it lie
            // in N+(x): at most max out-degree of them
            {
                bool bounded = false;
                for (int i = 0; i < L.n_int && !bounded; ++i) {
                    const int x = bound_order[L.int_src[i]];
                    const bool x_core = (best >> x) & 1;
                    if (cl.less[u][x]) bounded = true;
                    if (x_core && hi_core >= 0 && pos[bound_order[hi_core]] <= pos[x]) bounded = true;
                    if (core_level && x_core && pos[x] > pos[u]) bounded = true;
                }
                L.out_bounded = (int8_t)bounded;
            }
            // injectivity: exclude every earlier image not already ruled out
            for (int j = 0; j < l; ++j) {
                const int x = bound_order[j];
                const bool x_core = (best >> x) & 1;
                bool out_of_set = false;
                for (int i = 0; i < L.n_int && !out_of_set; ++i) {
                    int y = bound_order[L.int_src[i]];
                    if (y == x || p.rel[x][y] == 2) out_of_set = true; // m(x) not in adj(m(y))
                }
                for (int i = 0; i < L.n_diff && !out_of_set; ++i)
                    if (p.rel[x][bound_order[L.diff_src[i]]] == 1) out_of_set = true;
                for (int i = 0; i < L.n_lo && !out_of_set; ++i) {
                    int y = bound_order[L.lo_src[i]];
                    if (y == x || (x_core && ((best >> y) & 1) && pos[x] <= pos[y])) out_of_set = true;
                }
                for (int i = 0; i < L.n_hi && !out_of_set; ++i) {
                    int y = bound_order[L.hi_src[i]];
                    if (y == x || (x_core && ((best >> y) & 1) && pos[x] >= pos[y])) out_of_set = true;
                }
                if (!out_of_set && L.label >= 0 && p.label[x] >= 0 && p.label[x] != L.label) out_of_set = true;
                if (!out_of_set) L.excl_src[L.n_excl++] = (int8_t)j;
            }
        }
        // anti-vertex checks, each at the level binding the last vertex it reads
        for (const AntiSpec &a : avs) {
            PgAntiCheck &C = ord.chk[ord.n_checks++];
            int at = 0;
            for (int u = 0; u < p.k; ++u)
                if (a.reads >> u & 1) at = std::max(at, lvl_of[u]);
            C.level = (int8_t)at;
            for (int u = 0; u < p.k; ++u) {
                if (a.nbrs >> u & 1) C.int_src[C.n_int++] = (int8_t)lvl_of[u];
                else if (a.reads >> u & 1) C.excl_src[C.n_excl++] = (int8_t)lvl_of[u];
            }
            ord.lv[at].n_anti++;
        }
        orders.push_back(ord);
    } while (std::next_permutation(seq.begin(), seq.end()));
    return PG_OK;
}

}  // namespace

int pg_plan_compile(const PgPattern &in, bool vertex_induced, PgPlanHost &out, std::string &err) {
    auto t0 = std::chrono::steady_clock::now();
    PgPattern p = in;
    const int k = p.k;
    if (k < 1 || k > PGP_MAXK) { err = "pattern size must be 1..8"; return PG_EINVAL; }
    uint32_t reg = 0;
    for (int u = 0; u < k; ++u) {
        if (p.rel[u][u]) { err = "self loop in pattern"; return PG_EINVAL; }
        if (p.label[u] < -1) { err = "pattern label must be >= -1"; return PG_EINVAL; }
        for (int w = 0; w < k; ++w) {
            if (p.rel[u][w] != p.rel[w][u] || p.rel[u][w] > 2) { err = "bad pattern relation"; return PG_EINVAL; }
            if ((p.anti_vertex[u] || p.anti_vertex[w]) && p.rel[u][w] == 1) {
                err = "an anti-vertex may only have anti-edges";
                return PG_EINVAL;
            }
        }
        if (!p.anti_vertex[u]) reg |= 1u << u;
    }
    for (int u = 0; u < k; ++u)
        if (p.anti_vertex[u]) {
            bool any = false;
            for (int w = 0; w < k; ++w) any |= (p.rel[u][w] == 2 && !p.anti_vertex[w]);
            if (!any) { err = "an anti-vertex needs at least one anti-edge to a regular vertex"; return PG_EINVAL; }
        }
    if (!reg) { err = "pattern has no regular vertex"; return PG_EINVAL; }
    if (!connected_by_edges(p, reg)) { err = "regular pattern vertices must be connected by edges"; return PG_EINVAL; }
    for (int u = 0; u < k; ++u)
        if (p.anti_vertex[u]) {
            if (p.label[u] >= 0) { err = "anti-vertices carry no label"; return PG_EINVAL; }
            for (int w = 0; w < k; ++w)
                if (p.anti_vertex[w] && p.rel[u][w]) { err = "anti-vertices may not be related to each other"; return PG_EINVAL; }
        }

    // Theorem of Section 3.1.3: vertex-induced == anti-edges on all non-adjacent pairs.
    if (vertex_induced)
        for (int u = 0; u < k; ++u)
            for (int w = 0; w < k; ++w)
                if (u != w && (reg >> u & 1) && (reg >> w & 1) && p.rel[u][w] == 0) p.rel[u][w] = 2;

    out = PgPlanHost{};
    out.pat = p;
    out.n_regular = popcount(reg);
    for (int u = 0; u < k; ++u) out.labeled |= p.label[u] >= 0;

    // ---- breakSymmetries (Section 4.1; Grochow-Kellis) -------------------
    std::vector<Perm> group = automorphisms(p);
    {
        std::vector<uint64_t> codes;
        for (auto &s : group) {
            uint64_t code = 0;
            for (int u = 0; u < k; ++u) code = code * 8 + (uint64_t)((reg >> u & 1) ? s[u] : 0);
            codes.push_back(code);
        }
        std::sort(codes.begin(), codes.end());
        out.aut = (uint64_t)(std::unique(codes.begin(), codes.end()) - codes.begin());
    }
    // Which symmetric vertex to order first is free (Grochow-Kellis; any
    // choice gives the same count).  Ordering a vertex that every minimum
    // connected vertex cover contains puts the order on core vertices, where
    // it halves the enumerated core matches, and leaves the non-core
    // vertices unordered, where their completion needs only membership tests
    // (e.g. the path 0-1-2-3 orders 1 < 2 instead of 0 < 3).
    uint32_t in_every_cover = reg;
    {
        int min_size = 0;
        for (int size = 1; size <= popcount(reg) && !min_size; ++size)
            for (uint32_t mask = 1; mask < (1u << k); ++mask) {
                if ((mask & ~reg) || popcount(mask) != size) continue;
                bool covers = true;
                for (int u = 0; u < k && covers; ++u)
                    for (int w = u + 1; w < k && covers; ++w)
                        if ((reg >> u & 1) && (reg >> w & 1) && p.rel[u][w] && !(mask >> u & 1) && !(mask >> w & 1))
                            covers = false;
                if (!covers || !connected_by_edges(p, mask)) continue;
                min_size = size;
                in_every_cover &= mask;
            }
        if (popcount(reg) == 1) in_every_cover = reg;
    }
    for (;;) {
        int v = -1;
        uint32_t orbit = 0;
        for (int pass = 0; pass < 2 && v < 0; ++pass)
            for (int u = 0; u < k && v < 0; ++u) {
                if (!(reg >> u & 1)) continue;
                if (pass == 0 && !(in_every_cover >> u & 1)) continue;
                uint32_t o = 0;
                for (auto &s : group) o |= 1u << s[u];
                if (popcount(o) > 1) { v = u; orbit = o; }
            }
        if (v < 0) break;
        for (int w = 0; w < k; ++w)
            if (w != v && (orbit >> w & 1)) out.po.push_back({v, w});
        std::vector<Perm> stab;
        for (auto &s : group)
            if (s[v] == v) stab.push_back(s);
        group.swap(stab);
    }
    const Closure cl = close_po(k, out.po);

    // ---- minConnectedVertexCover (Sections 4.1, 4.2) ------------------------
    // covers every edge and every anti-edge between regular vertices, connected
    // through true edges.  Among minimum covers: fewest core levels, over all
    // matching orders, whose candidates cannot be drawn from the
    // out-neighbourhood of an already bound neighbour (under the degree
    // ranking such a level scans a high-degree vertex's lower-degree
    // neighbours); then fewest non-core groups; then non-core vertices below
    // core vertices in the partial order (their sets are bounded above); then
    // the smallest vertex mask.
    uint32_t best = 0;
    if (out.n_regular == 1) {
        best = reg;
    } else {
        int best_cost = 1 << 30, best_groups = 1 << 30, best_below = -(1 << 30);
        for (int size = 1; size <= out.n_regular && !best; ++size) {
            for (uint32_t mask = 1; mask < (1u << k); ++mask) {
                if ((mask & ~reg) || popcount(mask) != size) continue;
                bool covers = true;
                for (int u = 0; u < k && covers; ++u)
                    for (int w = u + 1; w < k && covers; ++w)
                        if ((reg >> u & 1) && (reg >> w & 1) && p.rel[u][w] && !(mask >> u & 1) && !(mask >> w & 1))
                            covers = false;
                if (!covers || !connected_by_edges(p, mask)) continue;
                uint32_t nc = reg & ~mask;
                const int cost = core_scan_cost(p, cl, mask);
                int ng = (int)noncore_groups(p, cl, nc).size();
                int below = 0;
                for (int u = 0; u < k; ++u)
                    if (nc >> u & 1)
                        for (int x = 0; x < k; ++x)
                            if (mask >> x & 1) below += (int)cl.less[u][x] - (int)cl.less[x][u];
                if (!best || cost < best_cost || (cost == best_cost && ng < best_groups) ||
                    (cost == best_cost && ng == best_groups && below > best_below)) {
                    best = mask;
                    best_cost = cost;
                    best_groups = ng;
                    best_below = below;
                }
            }
        }
    }
    out.core_mask = best;
    const uint32_t noncore = reg & ~best;

    // anti-vertices: the regular vertices each check reads (Section 4.3,
    // "Checking Anti-Vertices"): its neighbours, and their pattern neighbours
    // whose images are excluded as witnesses
    std::vector<AntiSpec> avs;
    uint32_t involved = 0;
    for (int a = 0; a < k; ++a) {
        if (!p.anti_vertex[a]) continue;
        AntiSpec sp{0, 0};
        for (int u = 0; u < k; ++u)
            if (p.rel[a][u] == 2 && (reg >> u & 1)) sp.nbrs |= 1u << u;
        sp.reads = sp.nbrs;
        for (int u = 0; u < k; ++u)
            if (sp.nbrs >> u & 1)
                for (int w = 0; w < k; ++w)
                    if (p.rel[u][w] == 1 && (reg >> w & 1)) sp.reads |= 1u << w;
        involved |= sp.reads;
        avs.push_back(sp);
    }
    out.anti_vertices = !avs.empty();

    // non-core groups; the largest is counted (an uninvolved one on ties),
    // the rest enumerated.  Vertices an anti-vertex check reads are single.
    std::vector<std::vector<int>> groups = noncore_groups(p, cl, noncore, involved);
    int counted = -1;
    for (int i = 0; i < (int)groups.size(); ++i) {
        if (counted < 0 || groups[i].size() > groups[counted].size()) { counted = i; continue; }
        if (groups[i].size() == groups[counted].size() && (involved >> groups[counted][0] & 1) &&
            !(involved >> groups[i][0] & 1))
            counted = i;
    }
    out.counted_group = counted < 0 ? 1 : (int)groups[counted].size();
    // joint partner: another single-vertex group (fewest regular neighbours,
    // i.e. the set most expensive to enumerate); neither may be read by an
    // anti-vertex check
    int partner = -1;
    if (counted >= 0 && groups[counted].size() == 1 && !(involved >> groups[counted][0] & 1)) {
        auto nbrs = [&](int u) {
            int c = 0;
            for (int w = 0; w < k; ++w) c += p.rel[u][w] == 1;
            return c;
        };
        for (int i = 0; i < (int)groups.size(); ++i)
            if (i != counted && groups[i].size() == 1 && !(involved >> groups[i][0] & 1) &&
                (partner < 0 || nbrs(groups[i][0]) < nbrs(groups[partner][0])))
                partner = i;
    }
    int rc = lower_orders(p, cl, best, groups, counted, partner, avs, out.orders, err);
    if (rc) return rc;
    // listing program: every non-core vertex enumerated on its own level
    std::vector<std::vector<int>> singles;
    for (int u = 0; u < k; ++u)
        if (noncore >> u & 1) singles.push_back({u});
    rc = lower_orders(p, cl, best, singles, -1, -1, avs, out.list_orders, err);
    if (rc) return rc;

    // k-clique: complete on all vertices, unlabeled (vertex-induced or not)
    bool clique = !out.labeled;
    for (int u = 0; u < k; ++u)
        for (int w = 0; w < k; ++w)
            if (u != w && p.rel[u][w] != 1) clique = false;
    out.is_clique = clique && k >= 2;
    out.clique_k = out.is_clique ? k : 0;
    out.compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return PG_OK;
}
