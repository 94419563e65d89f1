// Batched counting: many plans in one persistent launch.
//
// Every plan contributes one level program per matching order (Section 4.1);
// every program starts at the task's start vertex (Section 5.1).  The
// programs of a counted pattern are merged into a prefix tree: two programs
// share a node at depth l when their level specifications 1..l are
// identical (same intersected / subtracted / bounding / excluded earlier
// levels and label), so the candidate set of a shared prefix is computed
// once per start vertex and its candidates are extended into every program
// below it.  A node where one or more programs end is counted once by
// cardinality and adds C(|S|, g) into each such plan's counter.  Two counted
// patterns leave the tree for kernels of their own: unlabeled k-cliques (the
// bitmap clique kernel) and the unlabeled edge-induced 4-cycle (co-degree
// accumulation).
//
// Task groups: by default each counted pattern is a group of its own and a
// task is a (group, start vertex) pair, handed out group by group, so the
// warps of an SM mostly run one pattern's set operations at a time (the
// fused walk of several patterns' trees per start vertex measured slower
// than the same trees one after another: more code in flight per SM, and
// the instruction fetch stall is this kernel's largest).  With
// PG_BATCH_SHARE_PREFIXES all patterns form one tree walked once per start
// vertex, sharing identical prefixes across patterns.
//
// GPU mapping: one warp per task (device atomic queue, highest degree first
// within a group, Section 5.2); depth-first walk of the tree with an
// explicit per-depth stack; per-depth candidate buffers in a per-warp scratch
// region; per-warp 128-bit counters per plan in shared memory, flushed once
// per warp.
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "level_ops.cuh"

using namespace pgk;

// Children of a node: n_children plain ones from first_child, then n_joint
// joint leaves (counted together with this node's vertex, see plan.h).
struct PgTrieNode {
    PgLevel spec;
    int32_t depth;
    int32_t first_child, n_children;
    int32_t first_term, n_terms;
    int32_t n_joint;
    int32_t group; // roots: the task group that walks this tree
};

struct PgTrieTerm {
    int32_t slot;
    int32_t group;
};

namespace {

constexpr int kMaxSlots = PG_MAX_QUEUES;

struct BatchArgs {
    DevGraph g;
    const PgTrieNode *nodes;
    const PgTrieTerm *terms;
    int n_roots; // roots are nodes[0 .. n_roots)
    int n_groups; // task t walks group t / n_tasks over start-vertex task t % n_tasks
    int n_slots;
    int *scratch;
    long long warp_stride;
    long long lvl_off[PGP_MAXK];
    unsigned long long *queue;
    int n;
    int chunk;                  // tasks per queue grab
    long long stride, offset;   // task selection: offset, offset + stride, ... (samples, partition)
    long long n_tasks;          // selected tasks of the n_split_tasks + n - n_split
    // Ranks 0..n_split-1 (the highest degrees) are split: rank r owns tasks
    // split_prefix[r] .. split_prefix[r+1]-1, task j of S walking the level-1
    // candidates with index = j (mod S).  Later ranks are one task each.
    const long long *split_prefix;
    int n_split;
    long long n_split_tasks;
    unsigned long long *counts; // 2 words per slot
    PgRunCtl ctl;               // work budget (polled between tasks and first-level candidates)
};

__device__ __forceinline__ void add_slot(unsigned long long *acc, int slot, unsigned __int128 x) {
    // acc: per-warp (low, high) pairs in shared memory, single writer (lane 0)
    unsigned long long lo = acc[2 * slot];
    const unsigned long long add = (unsigned long long)x;
    acc[2 * slot] = lo + add;
    acc[2 * slot + 1] += (unsigned long long)(x >> 64) + (lo + add < lo ? 1ull : 0ull);
}

__device__ void count_terms(const BatchArgs &a, const PgTrieNode &C, const int *m, int lane,
                            unsigned long long *acc) {
    const unsigned long long c = count_last(a.g, C.spec, m, lane);
    if (lane == 0 && c)
        for (int t = 0; t < C.n_terms; ++t) {
            const PgTrieTerm tm = a.terms[C.first_term + t];
            add_slot(acc, tm.slot, choose_u128(c, tm.group));
        }
}

// W warps per CTA.  CAP limits the registers per thread so that more warps
// are resident to hide the latency of the searches, at the price of some
// spilling: 1 = 32 / W CTAs per SM (64 registers), 2 = 20 / W CTAs per SM
// (about 100 registers); 0 = the compiler's choice.
template <int W, int CAP>
__global__ void __launch_bounds__(W * 32, CAP == 1 ? 32 / W : CAP == 2 ? 20 / W : 0) k_count_batched(BatchArgs a) {
    __shared__ unsigned long long s_acc[W][2 * kMaxSlots];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    int *wbuf = a.scratch + gw * a.warp_stride;
    unsigned long long *acc = s_acc[wib];
    for (int i = lane; i < 2 * kMaxSlots; i += 32) acc[i] = 0;
    __syncwarp();
    const DevGraph &g = a.g;
    int m[PGP_MAXK], node[PGP_MAXK], sz[PGP_MAXK], ci[PGP_MAXK], ch[PGP_MAXK];
    long long task = 0, task_end = 0;
    const bool polled = a.ctl.words != nullptr;
    if (polled && lane == 0) ctl_begin(a.ctl);
    for (;;) {
        if (polled && ctl_stop(a.ctl, lane)) break;
        if (task >= task_end) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(a.queue, (unsigned long long)a.chunk);
            task = (long long)__shfl_sync(PG_FULL, t, 0);
            if (task >= a.n_groups * a.n_tasks) break;
            task_end = min(task + a.chunk, a.n_groups * a.n_tasks); // may cross into the next group
        }
        const int grp = (int)(task / a.n_tasks);
        const long long tg = a.offset + (task - grp * a.n_tasks) * a.stride;
        ++task;
        int v, part = 0, parts = 1;
        if (tg < a.n_split_tasks) {
            int lo = 0, hi = a.n_split; // last r with split_prefix[r] <= tg
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(a.split_prefix + mid) <= tg) lo = mid; else hi = mid;
            }
            v = lo;
            part = (int)(tg - __ldg(a.split_prefix + lo));
            parts = (int)(__ldg(a.split_prefix + lo + 1) - __ldg(a.split_prefix + lo));
        } else {
            v = a.n_split + (int)(tg - a.n_split_tasks);
        }
        const int label = g.labeled ? __ldg(&g.vinfo[v].w) : 0;
        for (int r = 0; r < a.n_roots; ++r) {
            const PgTrieNode &R = a.nodes[r];
            if (R.group != grp || (R.spec.label >= 0 && R.spec.label != label)) continue;
            if (lane == 0 && part == 0)
                for (int t = 0; t < R.n_terms; ++t) add_slot(acc, a.terms[R.first_term + t].slot, 1);
            if (R.n_children == 0) continue;
            int l = 0;
            node[0] = r;
            sz[0] = 1;
            ci[0] = 0;
            ch[0] = 0;
            m[0] = v;
            for (;;) {
                const PgTrieNode &N = a.nodes[node[l]];
                if (ch[l] >= N.n_children) {
                    ch[l] = 0;
                    if ((ci[l] += (l == 1 ? parts : 1)) >= sz[l]) {
                        if (l == 0) break;
                        --l;
                        ++ch[l];
                        continue;
                    }
                }
                // poll at each new candidate of the first three levels, so a
                // stop or a spent budget ends even a hub's long task soon
                if (polled && ch[l] == 0 && l >= 1 && l <= 3 && ctl_stop(a.ctl, lane)) break;
                if (l > 0) m[l] = wbuf[a.lvl_off[l] + ci[l]];
                const int child = N.first_child + ch[l];
                const PgTrieNode &C = a.nodes[child];
                // what depends on the start vertex alone is counted by part 0
                if (C.n_terms && (l > 0 || part == 0)) count_terms(a, C, m, lane, acc);
                for (int j = 0; j < C.n_joint && (l > 0 || part == 0); ++j) {
                    const PgTrieNode &J = a.nodes[C.first_child + C.n_children + j];
                    const unsigned long long c =
                        count_joint(g, C.spec, J.spec, l + 1, m, wbuf + a.lvl_off[l + 1], wbuf + a.lvl_off[l + 2], lane);
                    if (lane == 0 && c)
                        for (int t = 0; t < J.n_terms; ++t) add_slot(acc, a.terms[J.first_term + t].slot, c);
                }
                if (C.n_children) {
                    const int s = fill_level(g, C.spec, m, wbuf + a.lvl_off[l + 1], lane);
                    const int first = l == 0 ? part : 0; // a part's first level-1 candidate
                    if (s > first) {
                        ++l;
                        node[l] = child;
                        sz[l] = s;
                        ci[l] = first;
                        ch[l] = 0;
                        continue;
                    }
                }
                ++ch[l];
            }
        }
    }
    __syncwarp();
    if (lane < a.n_slots) {
        const unsigned __int128 x =
            ((unsigned __int128)acc[2 * lane + 1] << 64) | (unsigned __int128)acc[2 * lane];
        if (x) atomic_add_u128(a.counts + 2 * lane, x);
    }
    if (a.n_slots > 32 && lane + 32 < a.n_slots) {
        const int s = lane + 32;
        const unsigned __int128 x = ((unsigned __int128)acc[2 * s + 1] << 64) | (unsigned __int128)acc[2 * s];
        if (x) atomic_add_u128(a.counts + 2 * s, x);
    }
}

// Output counts from slot counts: out[i] = (sum_t coef_t * slot[t]) / div[i]
// in wrapping 128-bit arithmetic (the true value is non-negative, < 2^128).
__global__ void k_combine(const unsigned long long *slot_counts, const int *term_slot, const long long *term_coef,
                          const int *out_first, const int *out_n, const unsigned long long *out_div, int n_out,
                          unsigned long long *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_out) return;
    unsigned __int128 acc = 0;
    for (int t = out_first[i]; t < out_first[i] + out_n[i]; ++t) {
        const int s = term_slot[t];
        const unsigned __int128 c = ((unsigned __int128)slot_counts[2 * s + 1] << 64) | slot_counts[2 * s];
        acc += (unsigned __int128)(__int128)term_coef[t] * c;
    }
    acc /= out_div[i];
    out[2 * i] = (unsigned long long)acc;
    out[2 * i + 1] = (unsigned long long)(acc >> 64);
}

int batched_warps(const pg_graph *g) {
    const int w = g->tune.batched_warps;
    return (w == 2 || w == 8) ? w : 4;
}

template <int CAP>
void batched_kernel(int w, void **fn) {
    *fn = w == 2 ? (void *)k_count_batched<2, CAP> : w == 4 ? (void *)k_count_batched<4, CAP>
                                                             : (void *)k_count_batched<8, CAP>;
}

void *batched_fn(const pg_graph *g) {
    void *fn = nullptr;
    if (g->tune.batched_regcap == 1) batched_kernel<1>(batched_warps(g), &fn);
    else if (g->tune.batched_regcap == 2) batched_kernel<2>(batched_warps(g), &fn);
    else batched_kernel<0>(batched_warps(g), &fn);
    return fn;
}

int batched_grid(const pg_graph *g) {
    const int w = batched_warps(g);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_fn(g), w * 32, 0);
    if (per_sm < 1) per_sm = 1;
    if (g->tune.batched_blocks_per_sm > 0) per_sm = std::min(per_sm, g->tune.batched_blocks_per_sm);
    return per_sm * g->num_sms;
}

// ---- trie construction (host) --------------------------------------------

PgLevel normalized(const PgLevel &L) {
    PgLevel n;
    std::memset(&n, 0, sizeof(n));
    n.n_int = L.n_int;
    n.n_diff = L.n_diff;
    n.n_lo = L.n_lo;
    n.n_hi = L.n_hi;
    n.n_excl = L.n_excl;
    n.group = 1;
    n.joint = L.joint;
    n.label = L.label;
    std::memcpy(n.int_src, L.int_src, L.n_int);
    std::memcpy(n.diff_src, L.diff_src, L.n_diff);
    std::memcpy(n.lo_src, L.lo_src, L.n_lo);
    std::memcpy(n.hi_src, L.hi_src, L.n_hi);
    std::memcpy(n.excl_src, L.excl_src, L.n_excl);
    std::sort(n.int_src, n.int_src + n.n_int);
    std::sort(n.diff_src, n.diff_src + n.n_diff);
    std::sort(n.lo_src, n.lo_src + n.n_lo);
    std::sort(n.hi_src, n.hi_src + n.n_hi);
    std::sort(n.excl_src, n.excl_src + n.n_excl);
    return n;
}

bool same_spec(const PgLevel &x, const PgLevel &y) { return std::memcmp(&x, &y, sizeof(PgLevel)) == 0; }

}  // namespace

struct pg_batch {
    // counted patterns ("slots"): the plans themselves, or the edge-induced
    // terms their anti-edges expand into; output i = sum over its terms of
    // coef * slot count, divided by div[i]
    std::vector<PgPlanHost> slot_plans;
    std::vector<int> clique_k;          // per slot: k when counted by the clique kernel, else 0
    int clique_kmin = 0, clique_kmax = 0;
    int c4_slot = -1;                   // slot of the unlabeled edge-induced 4-cycle (co-degree kernel)
    std::vector<int> out_first, out_n;  // per output plan: range in out_terms
    std::vector<int> term_slot;
    std::vector<long long> term_coef;   // signed, includes |Aut| of the term pattern
    std::vector<unsigned long long> out_div;
    int n_out = 0;
    int *d_term_slot = nullptr;
    long long *d_term_coef = nullptr;
    int *d_out_first = nullptr, *d_out_n = nullptr;
    unsigned long long *d_out_div = nullptr;
    unsigned long long *d_slot_counts = nullptr; // 2 words per slot
    std::vector<PgTrieNode> nodes;
    std::vector<PgTrieTerm> terms;
    int n_roots = 0;
    int n_groups = 1;           // task groups (one per counted pattern unless prefixes are shared)
    bool share_prefixes = false;
    int n_slots = 0;
    int n_programs = 0;
    int n_levels_total = 0;     // sum over programs of their levels
    bool labeled = false;
    bool out_bounded[PGP_MAXK] = {};
    bool any_level[PGP_MAXK] = {};
    PgTrieNode *d_nodes = nullptr;
    PgTrieTerm *d_terms = nullptr;
    void *d_image = nullptr; // all device arrays of the batch, contiguous
    bool image_owned = false;
};

namespace {

// Canonical form of a pattern under vertex permutations (labels and
// relations), for merging isomorphic expansion terms.
std::vector<int> canonical(const PgPattern &q) {
    std::vector<int> best;
    int a[PGP_MAXK];
    for (int i = 0; i < q.k; ++i) a[i] = i;
    do {
        std::vector<int> code;
        code.reserve(q.k + q.k * q.k);
        for (int i = 0; i < q.k; ++i) code.push_back(q.label[a[i]]);
        for (int i = 0; i < q.k; ++i)
            for (int j = i + 1; j < q.k; ++j) code.push_back(q.rel[a[i]][a[j]]);
        if (best.empty() || code < best) best = code;
    } while (std::next_permutation(a, a + q.k));
    return best;
}

}  // namespace

// Anti-edge expansion (flags & PG_BATCH_EXPAND_ANTI): a plan whose regular
// vertices carry anti-edges A is counted as
//   maps(E, A) = sum over T subset of A of (-1)^|T| maps(E + T, no anti-edges)
// (inclusion-exclusion over the events "an anti-edge pair is adjacent", the
// pattern-level form of the set differences of Section 4.2; with the Theorem
// of Section 3.1.3 this covers vertex-induced patterns), maps(q) = |Aut(q)|
// count(q), and count = maps / |Aut|.  Isomorphic terms of all plans are
// merged and counted once by their own (edge-induced) plans.
int pg_batch_build(pg_plan *const *plans, int n_plans, int flags, pg_batch **out) {
    if (n_plans < 1 || n_plans > kMaxSlots) return pg_set_error(PG_EINVAL, "a batch holds 1..64 plans");
    for (int i = 0; i < n_plans; ++i)
        if (plans[i]->h.big_clique)
            return pg_set_error(PG_EUNSUPPORTED, "cliques above 8 vertices run on the k-clique kernel only (pg_count)");
    for (int i = 0; i < n_plans; ++i)
        if (plans[i]->h.anti_vertices)
            return pg_set_error(PG_EUNSUPPORTED, "anti-vertex patterns run on the plan interpreter (PG_KERNEL_GENERIC)");
    pg_batch *bb = new (std::nothrow) pg_batch();
    if (!bb) return pg_set_error(PG_ENOMEM, "host allocation failed");
    std::map<std::vector<int>, int> slot_of;
    auto slot_for = [&](const PgPattern &q, bool is_plain_plan, const PgPlanHost *ready, int *slot) -> int {
        std::vector<int> key = canonical(q);
        key.push_back(is_plain_plan ? 0 : 1);
        auto it = slot_of.find(key);
        if (it != slot_of.end()) { *slot = it->second; return PG_OK; }
        if ((int)bb->slot_plans.size() >= kMaxSlots) return PG_EUNSUPPORTED;
        PgPlanHost h;
        if (ready) {
            h = *ready;
        } else {
            std::string err;
            int rc = pg_plan_compile(q, false, h, err);
            if (rc) return pg_set_error(rc, err);
        }
        bb->slot_plans.push_back(h);
        *slot = (int)bb->slot_plans.size() - 1;
        slot_of[key] = *slot;
        return PG_OK;
    };
    bb->n_out = n_plans;
    for (int p = 0; p < n_plans; ++p) {
        const PgPlanHost &h = plans[p]->h;
        std::vector<std::pair<int, int>> anti;
        bool has_anti_vertex = false;
        for (int u = 0; u < h.pat.k; ++u) {
            has_anti_vertex |= h.pat.anti_vertex[u] != 0;
            for (int w = u + 1; w < h.pat.k; ++w)
                if (h.pat.rel[u][w] == 2) anti.push_back({u, w});
        }
        bb->out_first.push_back((int)bb->term_slot.size());
        bool expanded = false;
        // room for this plan's terms while keeping one slot per later plan
        const int room = kMaxSlots - (int)bb->slot_plans.size() - (n_plans - p - 1);
        long long perms = 1;
        for (int i = 2; i <= h.pat.k; ++i) perms *= i;
        // host cost of classifying the 2^|A| terms: at most about 5M permutations
        if ((flags & PG_BATCH_EXPAND_ANTI) && !anti.empty() && !has_anti_vertex && anti.size() <= 10 &&
            (perms << anti.size()) <= 5000000) {
            // signed terms merged by isomorphism class first; only classes
            // whose coefficients do not cancel need a slot
            std::map<std::vector<int>, std::pair<long long, PgPattern>> terms;
            for (unsigned T = 0; T < (1u << anti.size()); ++T) {
                PgPattern q = h.pat;
                for (size_t i = 0; i < anti.size(); ++i)
                    q.rel[anti[i].first][anti[i].second] = q.rel[anti[i].second][anti[i].first] =
                        (T >> i & 1) ? 1 : 0;
                std::vector<int> key = canonical(q);
                key.push_back(1);
                auto it = terms.find(key);
                if (it == terms.end()) it = terms.emplace(key, std::make_pair(0ll, q)).first;
                it->second.first += (__builtin_popcount(T) & 1) ? -1 : 1;
            }
            int new_slots = 0;
            for (auto &kv : terms)
                if (kv.second.first && !slot_of.count(kv.first)) ++new_slots;
            if (new_slots <= room) {
                std::map<int, long long> coef;
                for (auto &kv : terms) {
                    if (!kv.second.first) continue;
                    int slot;
                    int rc = slot_for(kv.second.second, false, nullptr, &slot);
                    if (rc) { pg_batch_free(bb); return rc == PG_EUNSUPPORTED ? pg_set_error(rc, "batch slots exhausted") : rc; }
                    coef[slot] += kv.second.first;
                }
                for (auto &kv : coef)
                    if (kv.second) {
                        bb->term_slot.push_back(kv.first);
                        bb->term_coef.push_back(kv.second * (long long)bb->slot_plans[kv.first].aut);
                    }
                bb->out_div.push_back(h.aut);
                expanded = true;
            }
        }
        if (!expanded) {
            int slot;
            int rc = slot_for(h.pat, true, &h, &slot);
            if (rc) { pg_batch_free(bb); return rc == PG_EUNSUPPORTED ? pg_set_error(rc, "batch needs more than 64 counted patterns") : rc; }
            bb->term_slot.push_back(slot);
            bb->term_coef.push_back(1);
            bb->out_div.push_back(1);
        }
        bb->out_n.push_back((int)bb->term_slot.size() - bb->out_first.back());
    }
    bb->share_prefixes = (flags & PG_BATCH_SHARE_PREFIXES) != 0;
    int rc = pg_batch_build_trie(bb);
    if (!rc && !(flags & PG_BATCH_HOST_ONLY)) rc = pg_batch_upload(bb);
    if (rc) { pg_batch_free(bb); return rc; }
    *out = bb;
    return PG_OK;
}

namespace {
// Unlabeled edge-induced 4-cycle without anti-edges or anti-vertices.
bool is_plain_c4(const PgPlanHost &h) {
    if (h.big_clique || h.labeled || h.anti_vertices || h.pat.k != 4) return false;
    int edges = 0;
    for (int u = 0; u < 4; ++u) {
        int d = 0;
        for (int w = 0; w < 4; ++w) {
            if (h.pat.rel[u][w] == 2) return false;
            d += h.pat.rel[u][w] == 1;
        }
        if (d != 2) return false;
        edges += d;
    }
    return edges == 8; // 2-regular on 4 vertices, connected (plans are): the 4-cycle
}
}  // namespace

int pg_batch_build_trie(pg_batch *b) {
    const int n_plans = (int)b->slot_plans.size();
    // tree with child lists, then laid out so that siblings are contiguous
    struct TNode {
        PgLevel spec;
        int depth;
        std::vector<int> kids;
        std::vector<PgTrieTerm> terms;
    };
    std::vector<TNode> t;
    std::vector<int> roots, root_group;
    int n_groups = 0;
    for (int i = 0; i < PGP_MAXK; ++i) b->out_bounded[i] = true;
    b->n_slots = n_plans;
    b->clique_k.assign(n_plans, 0);
    for (int p = 0; p < n_plans; ++p) {
        b->labeled = b->labeled || b->slot_plans[p].labeled;
        const PgPlanHost &sp = b->slot_plans[p];
        if (sp.is_clique && sp.pat.k >= 3) {
            // unlabeled k-cliques go to the bitmap clique kernel (one launch
            // for all clique sizes of the batch)
            b->clique_k[p] = sp.pat.k;
            b->clique_kmin = b->clique_kmin ? std::min(b->clique_kmin, sp.pat.k) : sp.pat.k;
            b->clique_kmax = std::max(b->clique_kmax, sp.pat.k);
            continue;
        }
        if (b->c4_slot < 0 && is_plain_c4(sp)) {
            b->c4_slot = p;
            continue;
        }
        // programs of one pattern always share prefixes; of different
        // patterns only with share_prefixes (else each pattern is a task
        // group of its own, walked over all start vertices in turn)
        const int grp = b->share_prefixes ? 0 : n_groups;
        n_groups = b->share_prefixes ? 1 : n_groups + 1;
        for (const PgOrder &o : b->slot_plans[p].orders) {
            b->n_programs++;
            b->n_levels_total += o.n_levels;
            PgLevel root_spec;
            std::memset(&root_spec, 0, sizeof(root_spec));
            root_spec.group = 1;
            root_spec.label = o.lv[0].label;
            int cur = -1;
            for (size_t i = 0; i < roots.size(); ++i)
                if (root_group[i] == grp && same_spec(t[roots[i]].spec, root_spec)) cur = roots[i];
            if (cur < 0) {
                t.push_back({root_spec, 0, {}, {}});
                cur = (int)t.size() - 1;
                roots.push_back(cur);
                root_group.push_back(grp);
            }
            for (int l = 1; l < o.n_levels; ++l) {
                const PgLevel spec = normalized(o.lv[l]);
                const bool is_last = l == o.n_levels - 1;
                const bool joint_pair = o.lv[o.n_levels - 1].joint && l >= o.n_levels - 2;
                if (joint_pair) {
                    b->any_level[l] = true; // both sets may be materialised
                    b->out_bounded[l] = false;
                } else if (!is_last) {
                    b->any_level[l] = true;
                    b->out_bounded[l] = b->out_bounded[l] && o.lv[l].out_bounded;
                }
                int nxt = -1;
                for (int k : t[cur].kids)
                    if (same_spec(t[k].spec, spec)) nxt = k;
                if (nxt < 0) {
                    t.push_back({spec, l, {}, {}});
                    nxt = (int)t.size() - 1;
                    t[cur].kids.push_back(nxt);
                }
                cur = nxt;
            }
            t[cur].terms.push_back({p, o.n_levels == 1 ? 1 : o.lv[o.n_levels - 1].group});
        }
    }
    // layout: roots first, then breadth-first so each node's children are contiguous
    for (auto &n : t)
        std::stable_partition(n.kids.begin(), n.kids.end(), [&](int k) { return !t[k].spec.joint; });
    std::vector<int> order(roots.begin(), roots.end());
    for (size_t i = 0; i < order.size(); ++i)
        for (int k : t[order[i]].kids) order.push_back(k);
    std::vector<int> pos(t.size());
    for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int)i;
    b->nodes.resize(order.size());
    for (size_t i = 0; i < order.size(); ++i) {
        const TNode &n = t[order[i]];
        PgTrieNode &d = b->nodes[i];
        std::memset(&d, 0, sizeof(d));
        d.spec = n.spec;
        d.depth = n.depth;
        int nj = 0;
        for (int k : n.kids) nj += t[k].spec.joint ? 1 : 0;
        d.n_children = (int)n.kids.size() - nj;
        d.n_joint = nj;
        d.first_child = n.kids.empty() ? 0 : pos[n.kids[0]];
        for (size_t k = 1; k < n.kids.size(); ++k)
            if (pos[n.kids[k]] != d.first_child + (int)k) return pg_set_error(PG_EINVAL, "internal: trie layout");
        d.first_term = (int)b->terms.size();
        d.n_terms = (int)n.terms.size();
        d.group = i < roots.size() ? root_group[i] : 0;
        for (auto &tm : n.terms) b->terms.push_back(tm);
    }
    b->n_roots = (int)roots.size();
    b->n_groups = std::max(1, n_groups);
    return PG_OK;
}

namespace {
// Device arrays of a batch, in one contiguous layout: nodes, terms, term
// slots, term coefficients, output ranges / divisors, slot counts.
struct BatchImage {
    size_t off[8];
    size_t bytes;
};

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

BatchImage batch_image(const pg_batch *b) {
    const size_t sz[8] = {b->nodes.size() * sizeof(PgTrieNode), b->terms.size() * sizeof(PgTrieTerm),
                          b->term_slot.size() * sizeof(int), b->term_coef.size() * sizeof(long long),
                          b->out_first.size() * sizeof(int), b->out_n.size() * sizeof(int),
                          b->out_div.size() * sizeof(unsigned long long),
                          2 * sizeof(unsigned long long) * (size_t)b->n_slots};
    BatchImage im;
    size_t o = 0;
    for (int i = 0; i < 8; ++i) {
        im.off[i] = o;
        o += align16(std::max<size_t>(sz[i], 16));
    }
    im.bytes = o;
    return im;
}

void batch_fill_host(const pg_batch *b, const BatchImage &im, unsigned char *h) {
    auto put = [&](int i, const void *src, size_t bytes) {
        if (bytes) std::memcpy(h + im.off[i], src, bytes);
    };
    put(0, b->nodes.data(), b->nodes.size() * sizeof(PgTrieNode));
    put(1, b->terms.data(), b->terms.size() * sizeof(PgTrieTerm));
    put(2, b->term_slot.data(), b->term_slot.size() * sizeof(int));
    put(3, b->term_coef.data(), b->term_coef.size() * sizeof(long long));
    put(4, b->out_first.data(), b->out_first.size() * sizeof(int));
    put(5, b->out_n.data(), b->out_n.size() * sizeof(int));
    put(6, b->out_div.data(), b->out_div.size() * sizeof(unsigned long long));
}

void batch_point(pg_batch *b, const BatchImage &im, unsigned char *d) {
    b->d_nodes = (PgTrieNode *)(d + im.off[0]);
    b->d_terms = (PgTrieTerm *)(d + im.off[1]);
    b->d_term_slot = (int *)(d + im.off[2]);
    b->d_term_coef = (long long *)(d + im.off[3]);
    b->d_out_first = (int *)(d + im.off[4]);
    b->d_out_n = (int *)(d + im.off[5]);
    b->d_out_div = (unsigned long long *)(d + im.off[6]);
    b->d_slot_counts = (unsigned long long *)(d + im.off[7]);
}
}  // namespace

// Device copy owned by the batch (public batches, pg_count_ex's cache).
int pg_batch_upload(pg_batch *b) {
    const BatchImage im = batch_image(b);
    std::vector<unsigned char> h(im.bytes, 0);
    batch_fill_host(b, im, h.data());
    void *d = nullptr;
    PG_CUDA(cudaMalloc(&d, im.bytes));
    cudaError_t e = cudaMemcpy(d, h.data(), im.bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return pg_cuda_error(e, "batch upload");
    }
    b->d_image = d;
    b->image_owned = true;
    batch_point(b, im, (unsigned char *)d);
    return PG_OK;
}

// Device copy staged into caller areas with an asynchronous copy on stream
// s: `host` must be pinned and stay untouched until the copy is done; no
// allocation.  PG_ENOMEM if the image is larger than the areas.
int pg_batch_stage(pg_batch *b, void *dev_area, void *host_area, size_t area_bytes, cudaStream_t s) {
    const BatchImage im = batch_image(b);
    if (im.bytes > area_bytes) return pg_set_error(PG_ENOMEM, "batch image larger than the staging area");
    batch_fill_host(b, im, (unsigned char *)host_area);
    PG_CUDA(cudaMemcpyAsync(dev_area, host_area, im.bytes, cudaMemcpyHostToDevice, s));
    b->d_image = dev_area;
    b->image_owned = false;
    batch_point(b, im, (unsigned char *)dev_area);
    return PG_OK;
}

void pg_batch_free(pg_batch *b) {
    if (!b) return;
    if (b->image_owned && b->d_image) cudaFree(b->d_image);
    delete b;
}

int pg_batch_slots(const pg_batch *b) { return b->n_out; }
bool pg_batch_labeled(const pg_batch *b) { return b->labeled; }

void pg_batch_stats(const pg_batch *b, int *nodes, int *programs, int *levels_total) {
    *nodes = (int)b->nodes.size();
    *programs = b->n_programs;
    *levels_total = b->n_levels_total;
}

namespace {
long long batch_layout(const pg_graph *g, const pg_batch *b, long long *off) {
    const long long cap_out = (g->max_out + 31) & ~31ll, cap_all = (g->max_deg + 31) & ~31ll;
    long long total = 0;
    for (int l = 0; l < PGP_MAXK; ++l) {
        off[l] = total;
        if (b->any_level[l]) total += b->out_bounded[l] ? cap_out : cap_all;
    }
    return total;
}
}  // namespace

size_t pg_batch_scratch_bytes(const pg_graph *g, const pg_batch *b) {
    long long off[PGP_MAXK];
    size_t bytes = (size_t)batched_grid(g) * batched_warps(g) * (size_t)batch_layout(g, b, off) * sizeof(int);
    if (b->clique_kmax) bytes = std::max(bytes, pg_clique_scratch_bytes(g, b->clique_kmax));
    if (b->c4_slot >= 0) bytes = std::max(bytes, pg_c4_scratch_bytes(g));
    return bytes;
}

int pg_launch_batched(pg_graph *g, const pg_batch *b, unsigned long long *counts_dev, int queue_slot,
                      cudaStream_t s, const PgRunCtl *ctl) {
    if (g->n == 0) {
        PG_CUDA(cudaMemsetAsync(counts_dev, 0, 2 * sizeof(unsigned long long) * (size_t)b->n_out, s));
        return PG_OK;
    }
    BatchArgs a;
    a.g = g->d;
    a.nodes = b->d_nodes;
    a.terms = b->d_terms;
    a.n_roots = b->n_roots;
    a.n_groups = b->n_groups;
    a.n_slots = b->n_slots;
    a.scratch = (int *)g->ex->scratch;
    a.warp_stride = batch_layout(g, b, a.lvl_off);
    a.queue = g->ex->queues + queue_slot;
    a.n = (int)g->n;
    a.chunk = std::max(1, g->tune.batched_chunk);
    const PgTaskSel sel = pg_task_sel(g);
    a.stride = sel.stride;
    a.offset = sel.offset;
    a.split_prefix = g->split_prefix;
    a.n_split = g->n_split;
    a.n_split_tasks = g->n_split_tasks;
    a.n_tasks = sel.count(g->n_split_tasks + (g->n - g->n_split));
    a.counts = b->d_slot_counts;
    a.ctl = ctl ? *ctl : PgRunCtl{};
    PG_CUDA(cudaMemsetAsync(b->d_slot_counts, 0, 2 * sizeof(unsigned long long) * (size_t)b->n_slots, s));
    if (b->n_roots > 0 && a.n_tasks > 0) {
        PG_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s));
        void *args[] = {&a};
        PG_CUDA(cudaLaunchKernel(batched_fn(g), dim3(batched_grid(g)), dim3(batched_warps(g) * 32), args, 0, s));
        PG_CUDA(cudaGetLastError());
    }
    if (b->clique_kmax) {
        if (g->max_out >= 65536) return pg_set_error(PG_EUNSUPPORTED, "clique kernel needs out-degrees below 65536");
        const int span = b->clique_kmax - b->clique_kmin + 1;
        PG_CUDA(cudaMemsetAsync(g->ex->tmp_counts, 0, 2 * sizeof(unsigned long long) * span, s));
        int rc = pg_launch_clique(g, b->clique_kmin, b->clique_kmax, g->ex->tmp_counts, queue_slot + 2, s, ctl);
        if (rc) return rc;
        for (int p = 0; p < b->n_slots; ++p)
            if (b->clique_k[p])
                PG_CUDA(cudaMemcpyAsync(b->d_slot_counts + 2 * p, g->ex->tmp_counts + 2 * (b->clique_k[p] - b->clique_kmin),
                                        2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
    }
    if (b->c4_slot >= 0) {
        int rc = pg_launch_c4(g, b->d_slot_counts + 2 * b->c4_slot, queue_slot + 4, s, ctl);
        if (rc) return rc;
    }
    k_combine<<<(b->n_out + 63) / 64, 64, 0, s>>>(b->d_slot_counts, b->d_term_slot, b->d_term_coef, b->d_out_first,
                                                 b->d_out_n, b->d_out_div, b->n_out, counts_dev);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}
