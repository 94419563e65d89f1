// Labeled frequent subgraph mining for any number of edges (Section 3.2,
// the FSM program: match the current patterns, keep those whose MNI support
// (Section 2.1) reaches the threshold, extend the survivors by one edge
// with extendByEdge, repeat; label discovery of Section 3.2.1 for the labels
// of new vertices).
//
// Domains (Section 5.5) are decided vertex by vertex: v lies in D(u) iff
// some edge-induced map sends pattern vertex u to v.  For each candidate
// labeled pattern and each orbit of its automorphism group (vertices of one
// orbit have equal domains) the host builds an anchored level program: u
// binds the task's vertex, the other pattern vertices follow in breadth-
// first order, each level intersecting the lists of its bound pattern
// neighbours and excluding earlier images (no partial order: domains are
// over all maps).  The domain kernel runs one warp per (program, vertex
// with u's label) and stops at the first complete match; |D(u)| is the
// number of hits.  A candidate's orbits are decided one round at a time and
// a candidate leaves as soon as one domain is below the threshold, so most
// infrequent candidates cost one domain.  Candidates of k + 1 edges come
// from the frequent k-edge patterns (one more edge between two vertices, or
// to a new vertex of any label), merged by isomorphism, and kept only if
// every connected k-edge sub-pattern is frequent (MNI is anti-monotone).
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "level_ops.cuh"

using namespace pgk;

namespace {

constexpr int kWarps = 8;
constexpr int kBlock = kWarps * 32;
constexpr int kMaxV = PGP_MAXK;

// ------------------------------------------------------------ device ----

struct DomArgs {
    DevGraph g;
    const PgOrder *orders;
    int n_orders;
    const long long *task_prefix;   // n_orders + 1: tasks of program i are [prefix[i], prefix[i+1])
    const int *bucket_start;        // program i's vertices: by_label[bucket_start[i] + j]
    const int *by_label;            // vertices grouped by label
    unsigned long long *hits;       // per program: vertices with a match
    int *scratch;
    long long warp_stride;
    long long lvl_off[PGP_MAXK];
    unsigned long long *queue;
    long long n_tasks;
    int chunk;
    PgRunCtl ctl;
};

// Does some match of program `ord` bind level 0 to v?  First hit ends it.
__device__ bool anchored_hit(const DomArgs &a, const PgOrder &ord, int v, int *wbuf, int lane) {
    const DevGraph &g = a.g;
    const int L = ord.n_levels;
    int m[PGP_MAXK], sz[PGP_MAXK], idx[PGP_MAXK];
    m[0] = v;
    if (L == 1) return true;
    int l = 1;
    for (;;) {
        const PgLevel &lv = ord.lv[l];
        if (l == L - 1) {
            if (count_last(g, lv, m, lane) > 0) return true;
        } else {
            sz[l] = fill_level(g, lv, m, wbuf + a.lvl_off[l], lane);
            idx[l] = 0;
        }
        while (l >= 1 && (l == L - 1 || idx[l] >= sz[l])) --l;
        if (l < 1) return false;
        m[l] = wbuf[a.lvl_off[l] + idx[l]];
        ++idx[l];
        ++l;
    }
}

__global__ void __launch_bounds__(kBlock) k_fsm_domains(DomArgs a) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    int *wbuf = a.scratch + gw * a.warp_stride;
    const bool polled = a.ctl.words != nullptr;
    if (polled && lane == 0) ctl_begin(a.ctl);
    int cur = -1;
    unsigned long long mine = 0; // hits of program `cur` not yet added
    for (;;) {
        if (polled && ctl_stop(a.ctl, lane)) break;
        long long t0 = 0;
        if (lane == 0) t0 = (long long)atomicAdd(a.queue, (unsigned long long)a.chunk);
        t0 = __shfl_sync(PG_FULL, t0, 0);
        if (t0 >= a.n_tasks) break;
        const long long t1 = min(t0 + a.chunk, a.n_tasks);
        for (long long t = t0; t < t1; ++t) {
            // program of task t: last i with task_prefix[i] <= t
            int lo = 0, hi = a.n_orders;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(a.task_prefix + mid) <= t) lo = mid; else hi = mid;
            }
            if (lo != cur) {
                if (lane == 0 && mine) atomicAdd(a.hits + cur, mine);
                mine = 0;
                cur = lo;
            }
            const int v = __ldg(a.by_label + __ldg(a.bucket_start + lo) + (t - __ldg(a.task_prefix + lo)));
            if (anchored_hit(a, a.orders[lo], v, wbuf, lane)) ++mine;
        }
    }
    if (lane == 0 && mine) atomicAdd(a.hits + cur, mine);
}

__global__ void k_label_count(DevGraph g, unsigned *hist) {
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v < g.n) atomicAdd(hist + __ldg(&g.vinfo[v].w), 1u);
}

__global__ void k_label_scatter(DevGraph g, unsigned *cursor, int *by_label) {
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v < g.n) by_label[atomicAdd(cursor + __ldg(&g.vinfo[v].w), 1u)] = (int)v;
}

// -------------------------------------------------------------- host ----

// A connected labeled pattern with edges only (edge-induced matching).
struct LPat {
    int k = 0;
    uint8_t adj[kMaxV] = {}; // bit w of adj[u]: edge (u, w)
    int lab[kMaxV] = {};
    int edges() const {
        int e = 0;
        for (int u = 0; u < k; ++u) e += __builtin_popcount(adj[u]);
        return e / 2;
    }
};

bool connected(const LPat &p) {
    if (p.k == 0) return false;
    unsigned seen = 1, frontier = 1;
    while (frontier) {
        unsigned next = 0;
        for (int u = 0; u < p.k; ++u)
            if (frontier >> u & 1) next |= p.adj[u];
        next &= ~seen;
        seen |= next;
        frontier = next;
    }
    return seen == (1u << p.k) - 1;
}

// Vertex permutations that respect the (label, degree) classes: the
// canonical form is the smallest code over them, and the automorphisms are
// among them.  perms[i][j] = original vertex placed at position j.
void class_perms(const LPat &p, std::vector<std::vector<int>> &perms) {
    std::vector<int> order(p.k);
    for (int i = 0; i < p.k; ++i) order[i] = i;
    auto key = [&](int u) { return std::make_pair(p.lab[u], __builtin_popcount(p.adj[u])); };
    std::sort(order.begin(), order.end(), [&](int x, int y) { return key(x) < key(y); });
    // class boundaries
    std::vector<std::pair<int, int>> cls;
    for (int i = 0; i < p.k;) {
        int j = i;
        while (j < p.k && key(order[j]) == key(order[i])) ++j;
        cls.push_back({i, j});
        i = j;
    }
    perms.clear();
    std::vector<int> cur = order;
    // odometer over per-class permutations
    std::vector<std::vector<int>> sub;
    for (auto &c : cls) {
        std::vector<int> v(order.begin() + c.first, order.begin() + c.second);
        std::sort(v.begin(), v.end());
        sub.push_back(v);
    }
    std::vector<std::vector<int>> state = sub;
    for (;;) {
        int pos = 0;
        for (auto &v : state)
            for (int x : v) cur[pos++] = x;
        perms.push_back(cur);
        int c = (int)state.size() - 1;
        while (c >= 0 && !std::next_permutation(state[c].begin(), state[c].end())) --c;
        if (c < 0) break;
    }
}

std::vector<int> code_of(const LPat &p, const std::vector<int> &perm) {
    std::vector<int> code;
    code.reserve(1 + p.k + p.k * (p.k - 1) / 2);
    code.push_back(p.k);
    for (int j = 0; j < p.k; ++j) code.push_back(p.lab[perm[j]]);
    for (int i = 0; i < p.k; ++i)
        for (int j = i + 1; j < p.k; ++j) code.push_back((p.adj[perm[i]] >> perm[j]) & 1);
    return code;
}

// Canonical form (relabelled pattern) and its code.
LPat canonical(const LPat &p, std::vector<int> *code_out) {
    std::vector<std::vector<int>> perms;
    class_perms(p, perms);
    std::vector<int> best;
    int bi = 0;
    for (size_t i = 0; i < perms.size(); ++i) {
        std::vector<int> c = code_of(p, perms[i]);
        if (best.empty() || c < best) {
            best = c;
            bi = (int)i;
        }
    }
    const std::vector<int> &pm = perms[bi];
    int inv[kMaxV];
    for (int j = 0; j < p.k; ++j) inv[pm[j]] = j;
    LPat q;
    q.k = p.k;
    for (int j = 0; j < p.k; ++j) {
        q.lab[j] = p.lab[pm[j]];
        uint8_t a = 0;
        for (int w = 0; w < p.k; ++w)
            if (p.adj[pm[j]] >> w & 1) a |= (uint8_t)(1u << inv[w]);
        q.adj[j] = a;
    }
    if (code_out) *code_out = best;
    return q;
}

// Orbits of the automorphism group (labels and edges preserved): one
// representative per orbit.
std::vector<int> orbit_reps(const LPat &p) {
    std::vector<std::vector<int>> perms;
    class_perms(p, perms);
    int rep[kMaxV];
    for (int u = 0; u < p.k; ++u) rep[u] = u;
    for (auto &pm : perms) {
        // pm maps position j -> vertex pm[j]; as a vertex map: sigma(order[j]) = pm[j]
        // with order = perms[0] (the class-sorted identity arrangement)
        const std::vector<int> &base = perms[0];
        int sigma[kMaxV];
        for (int j = 0; j < p.k; ++j) sigma[base[j]] = pm[j];
        bool aut = true;
        for (int u = 0; u < p.k && aut; ++u)
            for (int w = 0; w < p.k && aut; ++w)
                if (((p.adj[u] >> w) & 1) != ((p.adj[sigma[u]] >> sigma[w]) & 1)) aut = false;
        if (!aut) continue;
        for (int u = 0; u < p.k; ++u) {
            const int a = std::min(rep[u], rep[sigma[u]]);
            rep[u] = rep[sigma[u]] = a;
        }
    }
    // close the union (representatives are minima of their orbit)
    bool changed = true;
    while (changed) {
        changed = false;
        for (auto &pm : perms) {
            const std::vector<int> &base = perms[0];
            int sigma[kMaxV];
            for (int j = 0; j < p.k; ++j) sigma[base[j]] = pm[j];
            bool aut = true;
            for (int u = 0; u < p.k && aut; ++u)
                for (int w = 0; w < p.k && aut; ++w)
                    if (((p.adj[u] >> w) & 1) != ((p.adj[sigma[u]] >> sigma[w]) & 1)) aut = false;
            if (!aut) continue;
            for (int u = 0; u < p.k; ++u)
                if (rep[u] != rep[sigma[u]]) {
                    const int a = std::min(rep[u], rep[sigma[u]]);
                    rep[u] = rep[sigma[u]] = a;
                    changed = true;
                }
        }
    }
    std::vector<int> out;
    for (int u = 0; u < p.k; ++u)
        if (rep[u] == u) out.push_back(u);
    return out;
}

// Anchored level program of p rooted at u: breadth-first binding order,
// each level intersecting its bound neighbours' lists, excluding the
// earlier images that could lie in that set, labels checked.
PgOrder anchored_order(const LPat &p, int root) {
    PgOrder ord;
    std::memset(&ord, 0, sizeof(ord));
    int seq[kMaxV], lvl_of[kMaxV];
    for (int i = 0; i < kMaxV; ++i) lvl_of[i] = -1;
    int n = 0;
    seq[n] = root;
    lvl_of[root] = n++;
    for (int i = 0; i < n; ++i)
        for (int w = 0; w < p.k; ++w)
            if ((p.adj[seq[i]] >> w & 1) && lvl_of[w] < 0) {
                seq[n] = w;
                lvl_of[w] = n++;
            }
    ord.n_levels = n;
    ord.n_core = n;
    for (int l = 0; l < n; ++l) {
        const int u = seq[l];
        PgLevel &L = ord.lv[l];
        L.pattern_vertex = (int8_t)u;
        L.is_core = 1;
        L.label = p.lab[u];
        L.group = 1;
        for (int j = 0; j < l; ++j)
            if (p.adj[u] >> seq[j] & 1) L.int_src[L.n_int++] = (int8_t)j;
        for (int j = 0; j < l; ++j) {
            const int x = seq[j];
            bool out_of_set = p.adj[u] >> x & 1; // x is an intersected list's owner: not in its own list
            if (!out_of_set && p.lab[x] != p.lab[u]) out_of_set = true;
            if (!out_of_set) L.excl_src[L.n_excl++] = (int8_t)j;
        }
    }
    return ord;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    int alloc(size_t bytes) {
        if (p) cudaFree(p);
        p = nullptr;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
        return e == cudaSuccess ? PG_OK : pg_cuda_error(e, "cudaMalloc (FSM)");
    }
};

struct Cand {
    LPat p;
    std::vector<int> code;
    std::vector<int> reps;     // orbit representatives, smallest label bucket first
    unsigned long long support = ~0ull;
    bool alive = true;
};

}  // namespace

int pg_fsm_general_run(pg_graph *g, int max_edges, unsigned long long threshold, pg_fsm_general_pattern *out,
                       int64_t capacity, int64_t *n_frequent, cudaStream_t s) {
    if (!g->labeled) return pg_set_error(PG_EINVAL, "frequent subgraph mining needs a labeled graph");
    if (max_edges < 1 || max_edges > PG_FSM_MAX_EDGES)
        return pg_set_error(PG_EINVAL, "max_edges must be 1..7");
    if (threshold < 1) return pg_set_error(PG_EINVAL, "threshold must be >= 1");
    *n_frequent = 0;
    if (g->n == 0) return PG_OK;
    const int nl = std::max(1, g->n_labels);
    // vertices grouped by label
    DevBuf hist, by_label;
    int rc = hist.alloc(2 * (nl + 1) * sizeof(unsigned));
    if (!rc) rc = by_label.alloc(g->n * sizeof(int));
    if (rc) return rc;
    unsigned *h = (unsigned *)hist.p, *cursor = h + nl + 1;
    PG_CUDA(cudaMemsetAsync(h, 0, 2 * (nl + 1) * sizeof(unsigned), s));
    const unsigned nb = (unsigned)((g->n + 255) / 256);
    k_label_count<<<nb, 256, 0, s>>>(g->d, h);
    PG_CUDA(cudaGetLastError());
    std::vector<unsigned> cnt(nl), start(nl + 1, 0);
    PG_CUDA(cudaMemcpyAsync(cnt.data(), h, nl * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    for (int l = 0; l < nl; ++l) start[l + 1] = start[l] + cnt[l];
    PG_CUDA(cudaMemcpyAsync(cursor, start.data(), nl * sizeof(unsigned), cudaMemcpyHostToDevice, s));
    k_label_scatter<<<nb, 256, 0, s>>>(g->d, cursor, (int *)by_label.p);
    PG_CUDA(cudaGetLastError());

    // per-warp level buffers (no order bounds: any list length)
    const long long cap = (g->max_deg + 31) & ~31ll;
    long long lvl_off[PGP_MAXK];
    long long per_warp = 0;
    for (int l = 0; l < PGP_MAXK; ++l) {
        lvl_off[l] = per_warp;
        if (l >= 1 && l <= max_edges) per_warp += cap; // levels 1 .. k-2 are materialised (k <= max_edges + 1)
    }
    int per_sm = 0;
    PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fsm_domains, kBlock, 0));
    long long blocks = (long long)std::max(1, per_sm) * g->num_sms;
    // keep the buffers within 8 GiB
    const long long max_blocks = std::max<long long>(1, (8ll << 30) / (per_warp * 4 * kWarps + 1));
    blocks = std::max<long long>(1, std::min(blocks, max_blocks));
    rc = pg_ensure_scratch(g, (size_t)blocks * kWarps * per_warp * sizeof(int) + 16, s);
    if (rc) return rc;
    DevBuf d_queue;
    if ((rc = d_queue.alloc(sizeof(unsigned long long)))) return rc;

    // level 1: every label pair present in the graph
    std::vector<Cand> cands;
    std::map<std::vector<int>, int> seen;
    auto add_cand = [&](const LPat &p) {
        std::vector<int> code;
        LPat c = canonical(p, &code);
        if (seen.count(code)) return;
        seen[code] = (int)cands.size();
        Cand cd;
        cd.p = c;
        cd.code = code;
        cd.reps = orbit_reps(c);
        std::sort(cd.reps.begin(), cd.reps.end(),
                  [&](int x, int y) { return cnt[c.lab[x]] < cnt[c.lab[y]]; });
        cands.push_back(cd);
    };
    for (int x = 0; x < nl; ++x)
        for (int y = x; y < nl; ++y)
            if (cnt[x] && cnt[y]) {
                LPat p;
                p.k = 2;
                p.adj[0] = 2;
                p.adj[1] = 1;
                p.lab[0] = x;
                p.lab[1] = y;
                add_cand(p);
            }
    std::vector<Cand> frequent_all;
    for (int k = 1; k <= max_edges && !cands.empty(); ++k) {
        // domain rounds: round r decides the r-th orbit of every live candidate
        for (int r = 0;; ++r) {
            std::vector<int> which;
            for (int i = 0; i < (int)cands.size(); ++i)
                if (cands[i].alive && r < (int)cands[i].reps.size()) which.push_back(i);
            if (which.empty()) break;
            const int n_prog = (int)which.size();
            std::vector<PgOrder> orders(n_prog);
            std::vector<long long> prefix(n_prog + 1, 0);
            std::vector<int> bstart(n_prog);
            for (int j = 0; j < n_prog; ++j) {
                const Cand &c = cands[which[j]];
                const int u = c.reps[r];
                orders[j] = anchored_order(c.p, u);
                bstart[j] = (int)start[c.p.lab[u]];
                prefix[j + 1] = prefix[j] + cnt[c.p.lab[u]];
            }
            DevBuf d_orders, d_prefix, d_bstart, d_hits;
            if ((rc = d_orders.alloc(n_prog * sizeof(PgOrder))) || (rc = d_prefix.alloc((n_prog + 1) * sizeof(long long))) ||
                (rc = d_bstart.alloc(n_prog * sizeof(int))) || (rc = d_hits.alloc(n_prog * sizeof(unsigned long long))))
                return rc;
            PG_CUDA(cudaMemcpyAsync(d_orders.p, orders.data(), n_prog * sizeof(PgOrder), cudaMemcpyHostToDevice, s));
            PG_CUDA(cudaMemcpyAsync(d_prefix.p, prefix.data(), (n_prog + 1) * sizeof(long long), cudaMemcpyHostToDevice, s));
            PG_CUDA(cudaMemcpyAsync(d_bstart.p, bstart.data(), n_prog * sizeof(int), cudaMemcpyHostToDevice, s));
            PG_CUDA(cudaMemsetAsync(d_hits.p, 0, n_prog * sizeof(unsigned long long), s));
            PG_CUDA(cudaMemsetAsync(d_queue.p, 0, sizeof(unsigned long long), s));
            DomArgs a;
            a.g = g->d;
            a.orders = (const PgOrder *)d_orders.p;
            a.n_orders = n_prog;
            a.task_prefix = (const long long *)d_prefix.p;
            a.bucket_start = (const int *)d_bstart.p;
            a.by_label = (const int *)by_label.p;
            a.hits = (unsigned long long *)d_hits.p;
            a.scratch = (int *)g->ex->scratch;
            a.warp_stride = per_warp;
            for (int l = 0; l < PGP_MAXK; ++l) a.lvl_off[l] = lvl_off[l];
            a.queue = (unsigned long long *)d_queue.p;
            a.n_tasks = prefix[n_prog];
            a.chunk = 8;
            a.ctl = PgRunCtl{};
            if (a.n_tasks > 0) {
                k_fsm_domains<<<(unsigned)blocks, kBlock, 0, s>>>(a);
                PG_CUDA(cudaGetLastError());
            }
            std::vector<unsigned long long> hits(n_prog);
            PG_CUDA(cudaMemcpyAsync(hits.data(), d_hits.p, n_prog * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            PG_CUDA(cudaStreamSynchronize(s));
            for (int j = 0; j < n_prog; ++j) {
                Cand &c = cands[which[j]];
                c.support = std::min(c.support, hits[j]);
                if (hits[j] < threshold) c.alive = false;
            }
        }
        std::vector<Cand> freq;
        std::map<std::vector<int>, bool> freq_codes;
        for (auto &c : cands)
            if (c.alive) {
                freq.push_back(c);
                freq_codes[c.code] = true;
            }
        for (auto &c : freq) frequent_all.push_back(c);
        if (k == max_edges) break;
        // extendByEdge with label discovery, anti-monotone pruning
        cands.clear();
        seen.clear();
        auto all_subs_frequent = [&](const LPat &q) {
            for (int u = 0; u < q.k; ++u)
                for (int w = u + 1; w < q.k; ++w) {
                    if (!(q.adj[u] >> w & 1)) continue;
                    LPat r = q;
                    r.adj[u] &= (uint8_t)~(1u << w);
                    r.adj[w] &= (uint8_t)~(1u << u);
                    // drop a vertex left without edges
                    int drop = -1;
                    if (!r.adj[u]) drop = u;
                    else if (!r.adj[w]) drop = w;
                    if (drop >= 0) {
                        LPat t;
                        t.k = r.k - 1;
                        int map[kMaxV], j = 0;
                        for (int x = 0; x < r.k; ++x) map[x] = x == drop ? -1 : j++;
                        for (int x = 0; x < r.k; ++x) {
                            if (map[x] < 0) continue;
                            t.lab[map[x]] = r.lab[x];
                            for (int y = 0; y < r.k; ++y)
                                if ((r.adj[x] >> y & 1) && map[y] >= 0) t.adj[map[x]] |= (uint8_t)(1u << map[y]);
                        }
                        r = t;
                    }
                    if (!connected(r)) continue; // not a connected sub-pattern
                    std::vector<int> code;
                    canonical(r, &code);
                    if (!freq_codes.count(code)) return false;
                }
            return true;
        };
        for (auto &c : freq) {
            const LPat &p = c.p;
            for (int u = 0; u < p.k; ++u)
                for (int w = u + 1; w < p.k; ++w)
                    if (!(p.adj[u] >> w & 1)) {
                        LPat q = p;
                        q.adj[u] |= (uint8_t)(1u << w);
                        q.adj[w] |= (uint8_t)(1u << u);
                        if (all_subs_frequent(q)) add_cand(q);
                    }
            if (p.k < kMaxV)
                for (int u = 0; u < p.k; ++u)
                    for (int l = 0; l < nl; ++l) {
                        if (!cnt[l]) continue;
                        LPat q = p;
                        q.k = p.k + 1;
                        q.lab[p.k] = l;
                        q.adj[p.k] = (uint8_t)(1u << u);
                        q.adj[u] |= (uint8_t)(1u << p.k);
                        if (all_subs_frequent(q)) add_cand(q);
                    }
        }
    }
    std::sort(frequent_all.begin(), frequent_all.end(), [](const Cand &x, const Cand &y) {
        const int ex = x.p.edges(), ey = y.p.edges();
        if (ex != ey) return ex < ey;
        return x.code < y.code;
    });
    *n_frequent = (int64_t)frequent_all.size();
    for (size_t i = 0; i < frequent_all.size() && (int64_t)i < capacity; ++i) {
        const LPat &p = frequent_all[i].p;
        pg_fsm_general_pattern &o = out[i];
        std::memset(&o, 0, sizeof(o));
        o.k = p.k;
        for (int u = 0; u < PG_MAX_PATTERN; ++u) o.labels[u] = u < p.k ? p.lab[u] : -1;
        for (int u = 0; u < p.k; ++u)
            for (int w = u + 1; w < p.k; ++w)
                if (p.adj[u] >> w & 1) {
                    o.edges[2 * o.n_edges] = u;
                    o.edges[2 * o.n_edges + 1] = w;
                    ++o.n_edges;
                }
        o.support = frequent_all[i].support;
    }
    if ((int64_t)frequent_all.size() > capacity) return pg_set_error(PG_ETRUNC, "output capacity smaller than the frequent set");
    return PG_OK;
}
