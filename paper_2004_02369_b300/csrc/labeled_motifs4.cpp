// Labeled 4-motifs with label discovery (Section 6 labeled motif workloads;
// Section 3.2.1: a pattern's labels are discovered from the data rather than
// enumerated up front).
//
// Every vertex-induced 4-vertex match induces connected 3-vertex matches on
// the connected triples of its pattern (wedges and triangles).  So the labeled
// 3-motifs present in the graph (found by the labeled 3-motif kernels)
// discover the candidate labelings: a labeled 4-motif is counted only if
// each of its connected induced triples, with its labels, occurs.  The
// surviving labeled patterns are canonicalised under the shape's
// automorphisms and counted exactly as vertex-induced labeled plans, several
// per fused launch (the batch kernel, one task group per pattern, anti-edges
// expanded into edge-induced terms).  Only nonzero counts are reported.
#include <algorithm>
#include <array>
#include <cstring>
#include <set>
#include <vector>

#include "pg_internal.h"

namespace {

// The six connected 4-vertex shapes, in PG_MOTIF4_* order, vertex numbering
// as documented in pg.h.
const int kEdges[6][6][2] = {
    {{0, 1}, {1, 2}, {2, 3}},                          // path 0-1-2-3
    {{0, 1}, {0, 2}, {0, 3}},                          // star, centre 0
    {{0, 1}, {1, 2}, {2, 3}, {3, 0}},                  // cycle 0-1-2-3-0
    {{0, 1}, {0, 2}, {1, 2}, {0, 3}},                  // tailed triangle, tail 3 at 0
    {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {1, 3}},          // diamond, chord 1-3
    {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}},  // clique
};
const int kNumEdges[6] = {3, 3, 4, 4, 5, 6};
constexpr int kBatch = 8; // labeled plans per fused launch

struct ShapeInfo {
    bool adj[4][4];
    std::vector<std::array<int, 4>> aut; // vertex maps preserving edges
    // connected induced triples: (a, b, c) with b the centre of a wedge, or a triangle
    std::vector<std::array<int, 3>> wedges;    // (x, centre, y)
    std::vector<std::array<int, 3>> triangles;
};

ShapeInfo shape_info(int s) {
    ShapeInfo si;
    std::memset(si.adj, 0, sizeof(si.adj));
    for (int e = 0; e < kNumEdges[s]; ++e) {
        si.adj[kEdges[s][e][0]][kEdges[s][e][1]] = true;
        si.adj[kEdges[s][e][1]][kEdges[s][e][0]] = true;
    }
    std::array<int, 4> p = {0, 1, 2, 3};
    do {
        bool ok = true;
        for (int u = 0; u < 4 && ok; ++u)
            for (int w = 0; w < 4 && ok; ++w) ok = si.adj[u][w] == si.adj[p[u]][p[w]];
        if (ok) si.aut.push_back(p);
    } while (std::next_permutation(p.begin(), p.end()));
    for (int skip = 0; skip < 4; ++skip) {
        int t[3], n = 0;
        for (int u = 0; u < 4; ++u)
            if (u != skip) t[n++] = u;
        const int e = si.adj[t[0]][t[1]] + si.adj[t[0]][t[2]] + si.adj[t[1]][t[2]];
        if (e == 3) si.triangles.push_back({t[0], t[1], t[2]});
        if (e == 2) {
            // the centre is adjacent to both others
            for (int c = 0; c < 3; ++c) {
                const int x = t[(c + 1) % 3], y = t[(c + 2) % 3];
                if (si.adj[t[c]][x] && si.adj[t[c]][y]) si.wedges.push_back({x, t[c], y});
            }
        }
    }
    return si;
}

}  // namespace

int pg_labeled_motif4_run(pg_graph *g, pg_labeled_count4 *out, int64_t capacity, int64_t *n_out, cudaStream_t s) {
    *n_out = 0;
    if (!g->labeled) return pg_set_error(PG_EINVAL, "labeled motifs need a labeled graph");
    const int L = std::max(1, (int)g->n_labels);
    if (L > 32) return pg_set_error(PG_EUNSUPPORTED, "labeled motifs support labels 0..31");
    // 1. discovery: the labeled 3-motifs present (at most every labeled
    // wedge and triangle: L * L(L+1)/2 + L(L+1)(L+2)/6 of them)
    int64_t n3 = 0;
    std::vector<pg_labeled_count> m3((size_t)L * L * (L + 1) / 2 + (size_t)L * (L + 1) * (L + 2) / 6);
    int rc = pg_labeled_motif3_run(g, m3.data(), (int64_t)m3.size(), &n3, s);
    if (rc != PG_OK) return rc;
    std::set<std::array<int, 3>> tri, wedge; // sorted triples; (centre, x <= y)
    for (int64_t i = 0; i < n3; ++i) {
        const pg_labeled_count &r = m3[i];
        if (r.shape == PG_FSM_TRIANGLE) tri.insert({r.labels[0], r.labels[1], r.labels[2]});
        else wedge.insert({r.labels[0], r.labels[1], r.labels[2]});
    }
    // 2. candidates: labelings whose connected induced triples all occur,
    // one per automorphism class (smallest label tuple)
    struct Cand {
        int shape;
        std::array<int, 4> lab;
    };
    std::vector<Cand> cands;
    for (int sh = 0; sh < 6; ++sh) {
        const ShapeInfo si = shape_info(sh);
        std::set<std::array<int, 4>> seen;
        std::array<int, 4> lab;
        for (int code = 0; code < L * L * L * L; ++code) {
            lab = {code % L, code / L % L, code / (L * L) % L, code / (L * L * L)};
            bool ok = true;
            for (auto &t : si.triangles) {
                std::array<int, 3> k = {lab[t[0]], lab[t[1]], lab[t[2]]};
                std::sort(k.begin(), k.end());
                if (!tri.count(k)) { ok = false; break; }
            }
            for (size_t w = 0; w < si.wedges.size() && ok; ++w) {
                const auto &t = si.wedges[w];
                const int x = std::min(lab[t[0]], lab[t[2]]), y = std::max(lab[t[0]], lab[t[2]]);
                if (!wedge.count({lab[t[1]], x, y})) ok = false;
            }
            if (!ok) continue;
            std::array<int, 4> best = lab;
            for (auto &p : si.aut) {
                std::array<int, 4> q = {lab[p[0]], lab[p[1]], lab[p[2]], lab[p[3]]};
                best = std::min(best, q);
            }
            if (seen.insert(best).second) cands.push_back({sh, best});
        }
    }
    // 3. exact counts of the candidates, kBatch labeled plans per fused launch
    std::vector<pg_labeled_count4> found;
    unsigned long long *d_counts = nullptr;
    cudaError_t e = cudaMalloc(&d_counts, 2 * sizeof(uint64_t) * kBatch);
    if (e != cudaSuccess) return pg_cuda_error(e, "cudaMalloc (labeled 4-motifs)");
    for (size_t b0 = 0; b0 < cands.size() && rc == PG_OK; b0 += kBatch) {
        const size_t nb = std::min<size_t>(kBatch, cands.size() - b0);
        std::vector<pg_plan *> plans(nb, nullptr);
        for (size_t i = 0; i < nb && rc == PG_OK; ++i) {
            const Cand &c = cands[b0 + i];
            int32_t edges[12], labels[4];
            for (int k = 0; k < kNumEdges[c.shape]; ++k) {
                edges[2 * k] = kEdges[c.shape][k][0];
                edges[2 * k + 1] = kEdges[c.shape][k][1];
            }
            for (int u = 0; u < 4; ++u) labels[u] = c.lab[u];
            pg_pattern_desc d{4, kNumEdges[c.shape], edges, 0, nullptr, labels, nullptr, 1};
            rc = pg_compile_pattern(&d, &plans[i]);
        }
        pg_batch *batch = nullptr;
        if (rc == PG_OK) rc = pg_compile_batch(plans.data(), (int32_t)nb, PG_BATCH_EXPAND_ANTI, &batch);
        if (rc == PG_OK) rc = pg_count_batch(g, batch, (uint64_t *)d_counts, s);
        uint64_t h[2 * kBatch];
        if (rc == PG_OK) {
            e = cudaMemcpyAsync(h, d_counts, 2 * sizeof(uint64_t) * nb, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = pg_cuda_error(e, "labeled 4-motif counts");
        }
        if (rc == PG_OK)
            for (size_t i = 0; i < nb; ++i)
                if (h[2 * i] || h[2 * i + 1]) {
                    pg_labeled_count4 r;
                    std::memset(&r, 0, sizeof(r));
                    r.shape = PG_MOTIF4_PATH + cands[b0 + i].shape;
                    for (int u = 0; u < 4; ++u) r.labels[u] = cands[b0 + i].lab[u];
                    r.count_lo = h[2 * i];
                    r.count_hi = h[2 * i + 1];
                    found.push_back(r);
                }
        // the batch kernel may still read the batch image: free after the sync
        pg_free_batch(batch);
        for (auto *p : plans) pg_free_plan(p);
    }
    cudaFree(d_counts);
    if (rc) return rc;
    *n_out = (int64_t)found.size();
    for (size_t i = 0; i < found.size() && (int64_t)i < capacity; ++i) out[i] = found[i];
    if ((int64_t)found.size() > capacity) return pg_set_error(PG_ETRUNC, "more labeled motifs than capacity; *n_out is exact");
    return PG_OK;
}
