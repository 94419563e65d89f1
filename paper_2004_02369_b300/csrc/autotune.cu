// Launch-parameter tuning of the persistent kernels (pg_get_tuning,
// pg_set_tuning, pg_autotune).
//
// The paper sets its runtime's task granularity by hand (Section 5.5: tasks
// are start vertices handed out in chunks).  On a GPU the same choices are
// the number of start vertices a warp takes per work-queue grab, the CTA
// shape and count, the out-degree above which a k-clique start vertex gets a
// whole CTA, and how many high-degree vertices get membership bitmaps.  The
// best values depend on the graph's degree distribution, so they are chosen
// by measurement: coordinate descent over the knobs of the kernel family that
// would run, each value timed with CUDA events, optionally on a strided
// sample of start vertices.  Counts never depend on the values.
#include <chrono>
#include <cmath>
#include <cstring>

#include "pg_internal.h"

namespace {

struct DevCounts {
    void *p = nullptr;
    ~DevCounts() { if (p) cudaFree(p); }
};

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

int check_tuning(const pg_tuning &t) {
    if (t.clique_chunk < 1 || t.clique_chunk > 64) return pg_set_error(PG_EINVAL, "clique_chunk must be 1..64");
    if (t.clique_blocks_per_sm < 0 || t.batched_blocks_per_sm < 0)
        return pg_set_error(PG_EINVAL, "blocks per SM must be >= 0");
    if (t.clique_heavy_min < 8 || t.clique_heavy_min > PG_CLIQUE_LIGHT_D)
        return pg_set_error(PG_EINVAL, "clique_heavy_min must be 8..64");
    if (t.batched_warps != 2 && t.batched_warps != 4 && t.batched_warps != 8)
        return pg_set_error(PG_EINVAL, "batched_warps must be 2, 4 or 8");
    if (t.batched_chunk < 1 || t.batched_chunk > 64) return pg_set_error(PG_EINVAL, "batched_chunk must be 1..64");
    if (t.hub_min_degree < 1 || t.hub_max < 0 || t.hub_max > 65536)
        return pg_set_error(PG_EINVAL, "hub_min_degree must be >= 1 and hub_max 0..65536");
    if (t.clique_min_blocks != 3 && t.clique_min_blocks != 4)
        return pg_set_error(PG_EINVAL, "clique_min_blocks must be 3 or 4");
    if (t.batched_regcap < 0 || t.batched_regcap > 2) return pg_set_error(PG_EINVAL, "batched_regcap must be 0, 1 or 2");
    if (t.batched_split_grain != 0 && t.batched_split_grain < 16)
        return pg_set_error(PG_EINVAL, "batched_split_grain must be 0 or >= 16");
    return PG_OK;
}

int apply(pg_graph *g, const pg_tuning &t, cudaStream_t s) {
    int rc = check_tuning(t);
    if (rc) return rc;
    if (t.hub_min_degree != g->tune.hub_min_degree || t.hub_max != g->tune.hub_max) {
        rc = pg_graph_build_hubs(g, t.hub_min_degree, t.hub_max, s);
        if (rc) return rc;
    }
    if (t.clique_heavy_min != g->heavy_min_built) {
        rc = pg_graph_build_heavy(g, t.clique_heavy_min, s);
        if (rc) return rc;
    }
    if (t.batched_split_grain != g->split_grain_built) {
        rc = pg_graph_build_split(g, t.batched_split_grain, s);
        if (rc) return rc;
    }
    g->tune = t;
    return PG_OK;
}

// One untimed count, then the best of two timed ones (milliseconds).
int time_count(pg_graph *g, pg_plan *const *plans, int n, int kernel, uint64_t *d_counts, cudaStream_t s,
               const Events &ev, double *ms) {
    int rc = pg_count_ex(g, plans, n, d_counts, kernel, s);
    if (rc) return rc;
    double best = INFINITY;
    for (int r = 0; r < 2; ++r) {
        PG_CUDA(cudaEventRecord(ev.a, s));
        rc = pg_count_ex(g, plans, n, d_counts, kernel, s);
        if (rc) return rc;
        PG_CUDA(cudaEventRecord(ev.b, s));
        PG_CUDA(cudaEventSynchronize(ev.b));
        float t = 0;
        PG_CUDA(cudaEventElapsedTime(&t, ev.a, ev.b));
        best = std::min(best, (double)t);
    }
    *ms = best;
    return PG_OK;
}

struct Knob {
    int32_t pg_tuning::*field;
    std::vector<int32_t> values;
};

}  // namespace

extern "C" int pg_get_tuning(const pg_graph *g, pg_tuning *out) {
    if (!g || !out) return pg_set_error(PG_EINVAL, "NULL argument");
    *out = g->tune;
    return PG_OK;
}

extern "C" int pg_set_tuning(pg_graph *g, const pg_tuning *t, void *stream) {
    if (!g || !t) return pg_set_error(PG_EINVAL, "NULL argument");
    if (g->servers > 0) return pg_set_error(PG_EINVAL, "a server is running on this graph");
    return apply(g, *t, (cudaStream_t)stream);
}

extern "C" int pg_autotune(pg_graph *g, pg_plan *const *plans, int32_t n_plans, int32_t sample_stride,
                           pg_tune_report *report, void *stream) {
    if (!g || !plans || n_plans < 1) return pg_set_error(PG_EINVAL, "NULL argument");
    if (n_plans > PG_MAX_QUEUES) return pg_set_error(PG_EINVAL, "at most 64 plans per call");
    if (sample_stride < 1) return pg_set_error(PG_EINVAL, "sample_stride must be >= 1");
    if (g->servers > 0) return pg_set_error(PG_EINVAL, "a server is running on this graph");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    bool all_clique = true, any_clique = false;
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i]) return pg_set_error(PG_EINVAL, "NULL plan");
        const PgPlanHost &h = plans[i]->h;
        if (h.anti_vertices) return pg_set_error(PG_EUNSUPPORTED, "anti-vertex plans run untuned on PG_KERNEL_GENERIC");
        const bool c = h.is_clique && pg_plan_size(h) >= 3;
        all_clique &= c;
        any_clique |= c;
    }
    const int kernel = (all_clique && g->max_out < 65536) ? PG_KERNEL_CLIQUE : PG_KERNEL_BATCHED;

    std::vector<Knob> knobs;
    const std::vector<Knob> clique_knobs = {
        {&pg_tuning::clique_heavy_min, {16, 32, 48, 64}},
        {&pg_tuning::clique_chunk, {1, 2, 4, 8, 16}},
        {&pg_tuning::clique_blocks_per_sm, {1, 2, 0}},
        {&pg_tuning::clique_min_blocks, {3, 4}},
    };
    if (kernel == PG_KERNEL_BATCHED) {
        knobs.push_back({&pg_tuning::batched_split_grain, {0, 128, 512, 2048}});
        knobs.push_back({&pg_tuning::batched_warps, {2, 4, 8}});
        knobs.push_back({&pg_tuning::batched_regcap, {0, 1, 2}});
        knobs.push_back({&pg_tuning::batched_chunk, {1, 2, 4, 8}});
        knobs.push_back({&pg_tuning::batched_blocks_per_sm, {1, 2, 4, 0}});
        knobs.push_back({&pg_tuning::hub_min_degree, {256, 1024, 4096}});
        knobs.push_back({&pg_tuning::hub_max, {0, 128, 512, 2048}});
    }
    if (kernel == PG_KERNEL_CLIQUE || (any_clique && g->max_out < 65536))
        knobs.insert(knobs.end(), clique_knobs.begin(), clique_knobs.end());

    DevCounts dc;
    PG_CUDA(cudaMalloc(&dc.p, 2 * sizeof(uint64_t) * n_plans));
    Events ev;
    PG_CUDA(cudaEventCreate(&ev.a));
    PG_CUDA(cudaEventCreate(&ev.b));

    const pg_tuning start = g->tune;
    g->sample_stride = sample_stride;
    int trials = 0, rc = PG_OK;
    double base_ms = 0, best_ms = 0;
    pg_tuning best = start;
    do {
        rc = time_count(g, plans, n_plans, kernel, (uint64_t *)dc.p, s, ev, &base_ms);
        if (rc) break;
        ++trials;
        best_ms = base_ms;
        for (const Knob &k : knobs) {
            const int32_t keep = best.*(k.field);
            for (int32_t v : k.values) {
                if (v == keep) continue;
                pg_tuning cand = best;
                cand.*(k.field) = v;
                if ((rc = apply(g, cand, s)) != PG_OK) break;
                double ms = 0;
                if ((rc = time_count(g, plans, n_plans, kernel, (uint64_t *)dc.p, s, ev, &ms)) != PG_OK) break;
                ++trials;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = cand;
                }
            }
            if (rc) break;
        }
    } while (0);
    g->sample_stride = 1;
    // a choice made on a sample is kept only if the full launch agrees
    double full_start = -1, full_best = -1;
    if (!rc && sample_stride > 1 && std::memcmp(&best, &start, sizeof(best)) != 0) {
        do {
            if ((rc = apply(g, start, s)) != PG_OK) break;
            if ((rc = time_count(g, plans, n_plans, kernel, (uint64_t *)dc.p, s, ev, &full_start)) != PG_OK) break;
            if ((rc = apply(g, best, s)) != PG_OK) break;
            if ((rc = time_count(g, plans, n_plans, kernel, (uint64_t *)dc.p, s, ev, &full_best)) != PG_OK) break;
            trials += 2;
            if (full_best >= full_start) best = start;
        } while (0);
    }
    const int rc2 = apply(g, rc ? start : best, s);
    if (rc) return rc;
    if (rc2) return rc2;
    if (report) {
        report->chosen = best;
        report->default_ms = base_ms;
        report->tuned_ms = best_ms;
        report->full_default_ms = full_start;
        report->full_tuned_ms = full_best;
        report->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        report->trials = trials;
        report->kernel = kernel;
        report->sample_stride = sample_stride;
        report->pad = 0;
    }
    return PG_OK;
}
