// Serving runtime: a request loop over a resident graph.
//
// Queries (patterns) arrive through pg_server_submit at any time; their
// plans are compiled once and cached.  A worker thread admits waiting
// queries into batches whenever one of the server's streams is free and the
// batch's scratch requirement fits that stream's preallocated arena (device
// memory admission), counts each batch in one launch of the batched kernel
// (one task group per pattern, cliques through the clique kernel), and
// publishes the results with their submit / start / completion times.
// Batches on different streams run concurrently on the device (continuous
// batching: queries that arrive while others are on the GPU are admitted as
// soon as a stream frees up).  With serial = 1 the same kernels run one
// query per launch, one launch at a time -- the one-query-at-a-time
// baseline.
//
// Admission by measured cost: the first query of a pattern runs alone and
// its service time is kept with the cached plan; patterns that took longer
// than the batch limit alone keep running alone.  A free stream takes the
// oldest waiting query if it must run alone, else a batch of the waiting
// short queries (which so overtake long ones), so a long query never holds
// a batch of short ones and short queries are still fused into one launch.
// With several streams the launches of queries that run alone (together
// with the waiting queries of the same pattern, which a batch counts once)
// hold at most all streams but one (one, under a query time limit),
// optionally on a share of the SMs (a smaller persistent grid), so that
// short batches always find a stream.
//
// A query time limit (query_timeout_s) becomes the device work budget of
// the launch that counts it (the smallest remaining time over the batch):
// the kernels stop when it runs out, so one slow pattern cannot hold a
// stream indefinitely.  A launch of one pattern (one query, or several
// queries of the same pattern) gets the least time left among its queries;
// when it runs out, the queries with more time left than the launch ran go
// to the back of the queue and the others get PG_ETIMEOUT.  A batch of
// several patterns gets half the least time left; if it runs out, its
// queries (it is not known which one was slow) go back to the front of the
// queue to be launched one by one, first with a quarter of the time they
// have left, which isolates the straggler.  The measuring run of a new
// pattern likewise gets at most a quarter of the limit, so queries behind it
// are not held for its whole limit.  Waiting queries fail with PG_ETIMEOUT as
// soon as their limit passes.  A stream whose launch fails with a device
// error is retired and its queries get PG_EDEVICE; when no stream is left,
// waiting queries fail the same way.
//
// Section 5.1 processing model (tasks = start vertices) applied to a stream
// of patterns; the paper itself runs one mining program at a time.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pg_internal.h"

namespace {

struct ServerQuery {
    uint64_t ticket;
    pg_plan *plan;
    double t_submit;
    bool alone = false; // isolated after its batch ran out of time: launched by itself
    double cap_s = 0;   // > 0: budget cap of a measuring run (re-queued if it runs out)
    bool requeued = false;
};

// Measured service time of a pattern (worker thread only).
struct PatternCost {
    double alone_s = -1; // last time of a launch of this pattern alone; < 0: not measured
    bool slow = false;   // longer than the batch limit alone, or ran out of time
};

struct Slot {
    pg_exec ex;
    pg_graph view;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void *d_area = nullptr, *h_area = nullptr;
    size_t area_bytes = 0;
    uint64_t *d_counts = nullptr, *h_counts = nullptr;
    std::vector<ServerQuery> qs;
    pg_batch *batch = nullptr;
    double t_start = 0;
    bool busy = false;
    bool dead = false;     // retired after a device error
    std::vector<uint64_t> cancelled; // cancelled queries of the launch in flight
    PgRunCtl ctl;          // run control of the launch in flight
    bool long_class = false; // the launch in flight runs a query alone (long or unmeasured)
    double deadline = 0;   // host time the launch in flight must end by (0: none)
    bool deadline_raised = false;
    cudaEvent_t raised = nullptr; // after the last stop-word copy on the control stream
    bool raise_pending = false;   // the next launch on this slot must wait for it
};

constexpr size_t kAreaBytes = 4u << 20;

}  // namespace

struct pg_server {
    pg_graph *g = nullptr;
    pg_server_config cfg{};
    std::vector<Slot> slots;
    std::mutex mu;
    std::deque<ServerQuery> pending;
    std::deque<pg_query_result> results;
    std::mutex plan_mu;
    std::unordered_map<std::string, pg_plan *> plans;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::atomic<int64_t> outstanding{0};
    std::chrono::steady_clock::time_point t0;
    int device = 0;
    uint64_t next_ticket = 1;
    std::atomic<int64_t> batches{0}, launched_queries{0};
    std::vector<uint64_t> cancelled;     // tickets to cancel (worker applies them)
    std::unordered_map<const pg_plan *, PatternCost> cost; // worker thread only
    double batch_limit_s = 0.02;         // < 0: batch everything
    double alone_share = 1.0;            // share of the SMs for queries that run alone
    cudaStream_t ctl_stream = nullptr;   // raises stop words of running launches
    unsigned long long *h_one = nullptr; // pinned host word holding 1: the source of those
                                         // copies (host-to-device, done by a copy engine
                                         // while the running kernel holds every SM)

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

std::string pattern_key(const pg_pattern_desc *d) {
    std::string k = std::to_string(d->k) + "|" + std::to_string(d->vertex_induced) + "|";
    auto pairs = [&](const int32_t *p, int n) {
        std::vector<std::pair<int, int>> v;
        for (int i = 0; i < n; ++i) v.push_back({std::min(p[2 * i], p[2 * i + 1]), std::max(p[2 * i], p[2 * i + 1])});
        std::sort(v.begin(), v.end());
        for (auto &e : v) k += std::to_string(e.first) + "-" + std::to_string(e.second) + ",";
        k += "|";
    };
    pairs(d->edges, d->n_edges);
    pairs(d->anti_edges, d->n_anti);
    for (int u = 0; u < d->k; ++u) k += std::to_string(d->labels ? d->labels[u] : -1) + ",";
    k += "|";
    for (int u = 0; u < d->k; ++u) k += std::to_string(d->anti_vertex ? (int)d->anti_vertex[u] : 0);
    return k;
}

void emit(pg_server *S, const ServerQuery &q, int status, const uint64_t *cnt, double t_start, double t_done, int bs) {
    pg_query_result r;
    std::memset(&r, 0, sizeof(r));
    r.ticket = q.ticket;
    r.status = status;
    r.count_lo = cnt ? cnt[0] : 0;
    r.count_hi = cnt ? cnt[1] : 0;
    r.t_submit = q.t_submit;
    r.t_start = t_start;
    r.t_done = t_done;
    r.batch_size = bs;
    std::lock_guard<std::mutex> lock(S->mu);
    S->results.push_back(r);
}

// Queries of qs with no time left fail with PG_ETIMEOUT and leave qs.
void drop_expired(pg_server *S, std::vector<ServerQuery> &qs) {
    if (S->cfg.query_timeout_s <= 0) return;
    const double now = S->now();
    size_t k = 0;
    for (auto &q : qs) {
        if (S->cfg.query_timeout_s - (now - q.t_submit) > 0) {
            qs[k++] = q;
        } else {
            emit(S, q, PG_ETIMEOUT, nullptr, now, now, 1);
            S->outstanding--;
        }
    }
    qs.resize(k);
}

// Work budget of a launch counting qs (ns), 0 without a limit: the smallest
// remaining query time when every query is of one pattern (at most the cap
// of a measuring run); half of it for a batch of several patterns, so that
// when a batch runs out every query still has at least half its time to run
// alone.  False if some query has no time left (reported).
bool set_budget(pg_server *S, Slot &s, std::vector<ServerQuery> &qs) {
    s.view.budget_ns = 0;
    s.deadline = 0;
    s.deadline_raised = false;
    if (s.raise_pending) {
        // a stop word raised for the previous launch lands before this
        // launch resets it
        cudaStreamWaitEvent(s.stream, s.raised, 0);
        s.raise_pending = false;
    }
    if (S->cfg.query_timeout_s <= 0) return true;
    const double now = S->now();
    double left = 1e300;
    bool one_pattern = true;
    for (auto &q : qs) {
        left = std::min(left, S->cfg.query_timeout_s - (now - q.t_submit));
        one_pattern &= q.plan == qs[0].plan;
    }
    if (!one_pattern) left *= 0.5;
    else if (qs[0].cap_s > 0 && left > 0) left = std::min(left, qs[0].cap_s);
    if (left <= 0) {
        for (auto &q : qs) emit(S, q, PG_ETIMEOUT, nullptr, now, now, (int)qs.size());
        S->outstanding -= (int64_t)qs.size();
        return false;
    }
    s.view.budget_ns = (unsigned long long)(left * 1e9) + 1;
    s.deadline = now + left;
    return true;
}

// After the counts: copy the timed-out flag of the launch behind the host
// counts, then record completion.
void finish_launch(Slot &s, size_t n) {
    unsigned long long *flag = (unsigned long long *)(s.h_counts + 2 * PG_MAX_QUEUES);
    *flag = 0;
    cudaMemcpyAsync(s.h_counts, s.d_counts, 2 * sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, s.stream);
    if (s.ctl.words)
        cudaMemcpyAsync(flag, s.ctl.words + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s.stream);
    cudaEventRecord(s.done, s.stream);
}

// An anti-vertex query runs alone on the plan interpreter (batches refuse
// anti-vertex plans); returns 1 if launched.
int launch_alone(pg_server *S, Slot &s, const ServerQuery &q) {
    std::vector<ServerQuery> one{q};
    if (!set_budget(S, s, one)) return 0;
    int rc = pg_plan_upload(q.plan);
    if (rc == PG_OK && pg_generic_scratch_bytes(&s.view, q.plan, true) > s.ex.scratch_bytes) rc = PG_ENOMEM;
    if (rc == PG_OK && cudaMemsetAsync(s.d_counts, 0, 2 * sizeof(uint64_t), s.stream) != cudaSuccess) rc = PG_EDEVICE;
    if (rc == PG_OK) rc = pg_run_ctl(&s.view, 0, s.stream, &s.ctl, true);
    if (rc == PG_OK) {
        s.t_start = S->now();
        rc = pg_launch_generic(&s.view, q.plan, (unsigned long long *)s.d_counts, 0, true, s.stream, &s.ctl);
    }
    if (rc != PG_OK) {
        emit(S, q, rc, nullptr, S->now(), S->now(), 1);
        S->outstanding--;
        return 0;
    }
    finish_launch(s, 1);
    s.batch = nullptr;
    s.qs = {q};
    s.busy = true;
    S->batches++;
    S->launched_queries += 1;
    return 1;
}

// Try to launch up to `take` queries on slot s; returns queries launched.
int launch_batch(pg_server *S, Slot &s, std::vector<ServerQuery> qs) {
    drop_expired(S, qs);
    for (size_t i = 0; i < qs.size(); ++i) {
        if (!qs[i].plan->h.anti_vertices) continue;
        // the first anti-vertex query goes alone; the rest return to the queue front
        {
            std::lock_guard<std::mutex> lock(S->mu);
            for (size_t j = qs.size(); j-- > 0;)
                if (j != i) S->pending.push_front(qs[j]);
        }
        return launch_alone(S, s, qs[i]);
    }
    while (!qs.empty()) {
        std::vector<pg_plan *> plans;
        for (auto &q : qs) plans.push_back(q.plan);
        pg_batch *b = nullptr;
        int rc = pg_batch_build(plans.data(), (int)plans.size(), PG_BATCH_EXPAND_ANTI | PG_BATCH_HOST_ONLY, &b);
        if (rc == PG_OK) {
            const size_t need = pg_batch_scratch_bytes(&s.view, b);
            if (need <= s.ex.scratch_bytes) {
                if (!set_budget(S, s, qs)) {
                    pg_batch_free(b);
                    return 0;
                }
                rc = pg_batch_stage(b, s.d_area, s.h_area, s.area_bytes, s.stream);
                if (rc == PG_OK) rc = pg_run_ctl(&s.view, 0, s.stream, &s.ctl, true);
                if (rc == PG_OK) {
                    s.t_start = S->now();
                    rc = pg_launch_batched(&s.view, b, (unsigned long long *)s.d_counts, 0, s.stream, &s.ctl);
                }
                if (rc == PG_OK) {
                    finish_launch(s, qs.size());
                    s.batch = b;
                    s.qs = qs;
                    s.busy = true;
                    S->batches++;
                    S->launched_queries += (int64_t)qs.size();
                    return (int)qs.size();
                }
            } else {
                rc = PG_ENOMEM;
            }
            pg_batch_free(b);
        }
        if (qs.size() == 1) {
            // the query alone does not fit (or fails): report it
            emit(S, qs[0], rc, nullptr, S->now(), S->now(), 1);
            S->outstanding--;
            return 0;
        }
        // admit fewer: return the second half to the front of the queue
        const size_t keep = qs.size() / 2;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            for (size_t i = qs.size(); i-- > keep;) S->pending.push_front(qs[i]);
        }
        qs.resize(keep);
    }
    return 0;
}

// Fail every waiting query with `status` (no stream left to run them).
void fail_pending(pg_server *S, int status) {
    std::deque<ServerQuery> qs;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        qs.swap(S->pending);
    }
    const double t = S->now();
    for (auto &q : qs) emit(S, q, status, nullptr, t, t, 0);
    S->outstanding -= (int64_t)qs.size();
}

// Raises the stop word of slot s's launch in flight (and its timed-out word
// first, for a deadline) by host-to-device copies on the control stream:
// a copy engine delivers them while the running kernel holds every SM.
void raise_stop(pg_server *S, Slot &s, bool timed_out) {
    if (timed_out)
        cudaMemcpyAsync(s.ctl.words + 1, S->h_one, sizeof(unsigned long long), cudaMemcpyHostToDevice, S->ctl_stream);
    cudaMemcpyAsync(s.ctl.words, S->h_one, sizeof(unsigned long long), cudaMemcpyHostToDevice, S->ctl_stream);
    cudaEventRecord(s.raised, S->ctl_stream);
    s.raise_pending = true;
}

// Launches past their deadline on the host clock get their stop and
// timed-out words raised: the device budget counts from the kernel's own
// start, which may come late when other launches hold the SMs.
void enforce_deadlines(pg_server *S) {
    if (S->cfg.query_timeout_s <= 0) return;
    const double now = S->now();
    for (Slot &s : S->slots)
        if (s.busy && s.ctl.words && s.deadline > 0 && !s.deadline_raised && now > s.deadline) {
            raise_stop(S, s, true);
            s.deadline_raised = true;
        }
}

// Cancellations: waiting queries leave the queue with PG_ECANCELED; a
// running launch that holds a cancelled query gets its stop word raised.
void apply_cancels(pg_server *S) {
    std::vector<uint64_t> todo;
    std::deque<ServerQuery> gone;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        todo.swap(S->cancelled);
        for (uint64_t t : todo)
            for (auto it = S->pending.begin(); it != S->pending.end(); ++it)
                if (it->ticket == t) {
                    gone.push_back(*it);
                    S->pending.erase(it);
                    break;
                }
    }
    const double now = S->now();
    for (auto &q : gone) emit(S, q, PG_ECANCELED, nullptr, now, now, 0);
    S->outstanding -= (int64_t)gone.size();
    for (uint64_t t : todo)
        for (Slot &s : S->slots) {
            if (!s.busy || !s.ctl.words) continue;
            bool mine = false;
            for (auto &q : s.qs) mine |= q.ticket == t;
            if (!mine) continue;
            if (s.cancelled.empty()) raise_stop(S, s, false);
            s.cancelled.push_back(t);
        }
    // a ticket found nowhere already has its result: nothing to do
}

// Waiting queries whose time limit has passed fail now with PG_ETIMEOUT
// (not when a stream would take them).
void expire_waiting(pg_server *S) {
    if (S->cfg.query_timeout_s <= 0) return;
    std::vector<ServerQuery> gone;
    const double now = S->now();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        for (auto it = S->pending.begin(); it != S->pending.end();) {
            if (S->cfg.query_timeout_s - (now - it->t_submit) <= 0) {
                gone.push_back(*it);
                it = S->pending.erase(it);
            } else {
                ++it;
            }
        }
    }
    for (auto &q : gone) emit(S, q, PG_ETIMEOUT, nullptr, now, now, 0);
    S->outstanding -= (int64_t)gone.size();
}

// Whether query q must be launched by itself: isolated after a batch ran
// out of time, an anti-vertex pattern, or a pattern not yet measured or
// measured longer than the batch limit.
bool goes_alone(pg_server *S, const ServerQuery &q) {
    if (q.alone || q.requeued || q.plan->h.anti_vertices) return true;
    if (S->batch_limit_s < 0) return false;
    auto it = S->cost.find(q.plan);
    return it == S->cost.end() || it->second.slow;
}

void worker_loop(pg_server *S) {
    cudaSetDevice(S->device);
    const int max_batch = S->cfg.serial ? 1 : std::max(1, std::min(S->cfg.max_batch, (int)PG_MAX_QUEUES));
    while (!S->stop.load()) {
        bool progress = false;
        apply_cancels(S);
        enforce_deadlines(S);
        for (Slot &s : S->slots) {
            if (!s.busy) continue;
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaErrorNotReady) continue;
            const double t = S->now();
            if (e != cudaSuccess) {
                // a failed launch or a device error: these queries fail, the
                // stream is retired
                cudaGetLastError();
                for (auto &q : s.qs) emit(S, q, PG_EDEVICE, nullptr, s.t_start, t, (int)s.qs.size());
                s.dead = true;
            } else if (!s.cancelled.empty()) {
                // the launch was stopped: its cancelled queries end here, the
                // others go back to the front of the queue
                std::vector<ServerQuery> again;
                int64_t ended = 0;
                for (auto &q : s.qs) {
                    bool c = false;
                    for (uint64_t x : s.cancelled) c |= x == q.ticket;
                    if (c) {
                        emit(S, q, PG_ECANCELED, nullptr, s.t_start, t, (int)s.qs.size());
                        ++ended;
                    } else {
                        again.push_back(q);
                    }
                }
                {
                    std::lock_guard<std::mutex> lock(S->mu);
                    for (size_t i = again.size(); i-- > 0;) S->pending.push_front(again[i]);
                }
                S->outstanding -= ended;
                pg_batch_free(s.batch);
                s.batch = nullptr;
                s.qs.clear();
                s.cancelled.clear();
                s.busy = false;
                progress = true;
                continue;
            } else {
                const bool timed_out = *(const unsigned long long *)(s.h_counts + 2 * PG_MAX_QUEUES) != 0;
                bool one_pattern = true;
                for (auto &q : s.qs) one_pattern &= q.plan == s.qs[0].plan;
                if (one_pattern) {
                    // a launch of one pattern measures it
                    const double ran = t - s.t_start;
                    PatternCost &c = S->cost[s.qs[0].plan];
                    c.alone_s = ran;
                    c.slow = timed_out || (S->batch_limit_s >= 0 && ran > S->batch_limit_s);
                    if (timed_out) {
                        // the pattern needs more than this launch had: its
                        // queries with more time left than that go to the
                        // back of the queue (uncapped), the others fail
                        std::vector<ServerQuery> again;
                        for (auto &q : s.qs) {
                            if (S->cfg.query_timeout_s - (t - q.t_submit) > ran) {
                                ServerQuery r = q;
                                r.cap_s = 0;
                                r.requeued = true;
                                r.alone = false;
                                again.push_back(r);
                            } else {
                                emit(S, q, PG_ETIMEOUT, nullptr, s.t_start, t, (int)s.qs.size());
                                S->outstanding--;
                            }
                        }
                        {
                            std::lock_guard<std::mutex> lock(S->mu);
                            for (auto &r : again) S->pending.push_back(r);
                        }
                        pg_batch_free(s.batch);
                        s.batch = nullptr;
                        s.qs.clear();
                        s.busy = false;
                        progress = true;
                        continue;
                    }
                }
                if (timed_out && s.qs.size() > 1) {
                    // isolate: every query of the batch runs again by itself,
                    // first with a quarter of the time it has left (the slow
                    // one then goes to the back of the queue)
                    std::lock_guard<std::mutex> lock(S->mu);
                    for (size_t i = s.qs.size(); i-- > 0;) {
                        ServerQuery q = s.qs[i];
                        q.alone = true;
                        q.cap_s = 0.25 * (S->cfg.query_timeout_s - (t - q.t_submit));
                        S->pending.push_front(q);
                    }
                    pg_batch_free(s.batch);
                    s.batch = nullptr;
                    s.qs.clear();
                    s.busy = false;
                    progress = true;
                    continue;
                }
                for (size_t i = 0; i < s.qs.size(); ++i)
                    emit(S, s.qs[i], timed_out ? PG_ETIMEOUT : PG_OK, timed_out ? nullptr : s.h_counts + 2 * i,
                         s.t_start, t, (int)s.qs.size());
            }
            S->outstanding -= (int64_t)s.qs.size();
            pg_batch_free(s.batch);
            s.batch = nullptr;
            s.qs.clear();
            s.busy = false;
            progress = true;
        }
        expire_waiting(S);
        // With several streams, queries that run alone (long, unmeasured or
        // isolated ones) hold at most all streams but one (optionally on a
        // share of the SMs), so that short batches always find a stream.
        const bool multi = S->slots.size() > 1;
        // launches that run alone may hold all streams but one; with a time
        // limit only one at a time: a persistent launch keeps the SMs it
        // starts on until it ends, so a second one would wait for them (and
        // could not see its stop word) past its queries' deadlines
        const int long_max = S->cfg.query_timeout_s > 0 ? 1 : std::max(1, (int)S->slots.size() - 1);
        int long_running = 0;
        for (Slot &s : S->slots) long_running += s.busy && s.long_class ? 1 : 0;
        bool any_alive = false;
        for (Slot &s : S->slots) {
            any_alive |= !s.dead;
            if (s.busy || s.dead) continue;
            std::vector<ServerQuery> take;
            bool is_long = false;
            {
                std::lock_guard<std::mutex> lock(S->mu);
                if (!S->pending.empty()) {
                    ServerQuery &f = S->pending.front();
                    if ((max_batch == 1 || goes_alone(S, f)) && !(multi && long_running >= long_max)) {
                        // the oldest query runs by itself: isolated, measuring
                        // its pattern, known long, or anti-vertex
                        if (!S->cfg.serial && S->cfg.query_timeout_s > 0 && !f.requeued && !f.alone &&
                            !S->cost.count(f.plan))
                            f.cap_s = 0.25 * S->cfg.query_timeout_s;
                        take.push_back(f);
                        S->pending.pop_front();
                        is_long = true;
                        // waiting queries of the same pattern ride along: a
                        // batch counts each distinct pattern once
                        if (max_batch > 1 && !take[0].plan->h.anti_vertices && !take[0].alone && take[0].cap_s <= 0)
                            for (auto it = S->pending.begin(); it != S->pending.end() && (int)take.size() < max_batch;) {
                                if (it->plan == take[0].plan && !it->alone) {
                                    take.push_back(*it);
                                    it = S->pending.erase(it);
                                } else {
                                    ++it;
                                }
                            }
                    } else if (max_batch > 1) {
                        // a batch of the waiting short queries, oldest first
                        for (auto it = S->pending.begin(); it != S->pending.end() && (int)take.size() < max_batch;) {
                            if (goes_alone(S, *it)) {
                                ++it;
                            } else {
                                take.push_back(*it);
                                it = S->pending.erase(it);
                            }
                        }
                    }
                }
            }
            if (take.empty()) break;
            s.view.num_sms = is_long && multi ? std::max(1, (int)(S->g->num_sms * S->alone_share)) : S->g->num_sms;
            launch_batch(S, s, take);
            s.long_class = is_long && s.busy;
            long_running += s.long_class ? 1 : 0;
            progress = true;
            if (S->cfg.serial) break;
        }
        if (!any_alive) {
            fail_pending(S, PG_EDEVICE);
            progress = false;
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" int pg_server_create(pg_graph *g, const pg_server_config *cfg, pg_server **out) {
    if (!g || !cfg || !out) return pg_set_error(PG_EINVAL, "NULL argument");
    if (!(cfg->query_timeout_s >= 0.0)) return pg_set_error(PG_EINVAL, "query_timeout_s must be >= 0");
    if (cfg->batch_limit_ms != cfg->batch_limit_ms) return pg_set_error(PG_EINVAL, "batch_limit_ms is NaN");
    if (!(cfg->alone_sm_fraction >= 0.0) || cfg->alone_sm_fraction > 1.0)
        return pg_set_error(PG_EINVAL, "alone_sm_fraction must lie in [0, 1]");
    *out = nullptr;
    pg_server *S = new (std::nothrow) pg_server();
    if (!S) return pg_set_error(PG_ENOMEM, "host allocation failed");
    S->g = g;
    g->servers++; // views copy the graph's hub and heavy pointers: no retuning meanwhile
    S->cfg = *cfg;
    if (cfg->batch_limit_ms > 0) S->batch_limit_s = cfg->batch_limit_ms * 1e-3;
    if (cfg->batch_limit_ms < 0) S->batch_limit_s = -1;
    if (cfg->alone_sm_fraction > 0) S->alone_share = std::min(1.0, cfg->alone_sm_fraction);
    S->t0 = std::chrono::steady_clock::now();
    const int n_streams = cfg->serial ? 1 : std::max(1, std::min(cfg->n_streams, 16));
    int rc = PG_OK;
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) {
        delete S;
        return pg_cuda_error(e, "cudaGetDevice");
    }
    if ((e = cudaStreamCreateWithFlags(&S->ctl_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMallocHost(&S->h_one, sizeof(unsigned long long))) != cudaSuccess) {
        rc = pg_cuda_error(e, "server control stream");
        pg_server_free(S);
        return rc;
    }
    *S->h_one = 1;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    size_t budget = cfg->memory_budget > 0 ? (size_t)cfg->memory_budget : std::min<size_t>(free_b / 5 * 2, 64ull << 30);
    const size_t per_stream = budget / n_streams;
    S->slots.resize(n_streams);
    for (Slot &s : S->slots) {
        if ((rc = pg_exec_init(&s.ex)) != PG_OK) break;
        if ((rc = pg_dalloc(&s.ex.scratch, per_stream, nullptr)) != PG_OK) break;
        if ((e = cudaStreamSynchronize(nullptr)) != cudaSuccess) { rc = pg_cuda_error(e, "server scratch"); break; }
        s.ex.scratch_bytes = per_stream;
        s.view = *g;
        s.view.ex = &s.ex;
        s.view.is_view = true;
        s.view.batch_cache = nullptr;
        s.view.batch_key.clear();
        s.view.budget_ns = 0;
        if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s.raised, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaMalloc(&s.d_area, kAreaBytes)) != cudaSuccess ||
            (e = cudaMallocHost(&s.h_area, kAreaBytes)) != cudaSuccess ||
            (e = cudaMalloc(&s.d_counts, 2 * sizeof(uint64_t) * PG_MAX_QUEUES)) != cudaSuccess ||
            (e = cudaMallocHost(&s.h_counts, 2 * sizeof(uint64_t) * PG_MAX_QUEUES + sizeof(uint64_t))) != cudaSuccess) {
            rc = pg_cuda_error(e, "server stream setup");
            break;
        }
        s.area_bytes = kAreaBytes;
    }
    if (rc) {
        pg_server_free(S);
        return rc;
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return PG_OK;
}

extern "C" int pg_server_submit(pg_server *S, const pg_pattern_desc *q, uint64_t *ticket) {
    if (!S || !q || !ticket) return pg_set_error(PG_EINVAL, "NULL argument");
    const double t = S->now();
    pg_plan *plan = nullptr;
    {
        std::lock_guard<std::mutex> lock(S->plan_mu);
        const std::string key = pattern_key(q);
        auto it = S->plans.find(key);
        if (it != S->plans.end()) {
            plan = it->second;
        } else {
            int rc = pg_compile_pattern(q, &plan);
            if (rc) return rc;
            if (plan->h.labeled && !S->g->labeled) {
                pg_free_plan(plan);
                return pg_set_error(PG_EINVAL, "labeled pattern on an unlabeled graph");
            }
            S->plans[key] = plan;
        }
    }
    std::lock_guard<std::mutex> lock(S->mu);
    *ticket = S->next_ticket++;
    S->pending.push_back({*ticket, plan, t});
    S->outstanding++;
    return PG_OK;
}

extern "C" int pg_server_poll(pg_server *S, pg_query_result *out, int32_t max_results, int32_t *n_out) {
    if (!S || !n_out || (max_results > 0 && !out)) return pg_set_error(PG_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    int n = 0;
    while (n < max_results && !S->results.empty()) {
        out[n++] = S->results.front();
        S->results.pop_front();
    }
    *n_out = n;
    return PG_OK;
}

extern "C" int pg_server_drain(pg_server *S, double timeout_s) {
    if (!S) return pg_set_error(PG_EINVAL, "NULL argument");
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (S->outstanding.load() > 0) {
        if (std::chrono::steady_clock::now() > until) return pg_set_error(PG_ETIMEOUT, "queries still outstanding");
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    return PG_OK;
}

extern "C" int pg_server_get_stats(pg_server *S, pg_server_stats *out) {
    if (!S || !out) return pg_set_error(PG_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->n_streams = (int32_t)S->slots.size();
    out->batches = S->batches.load();
    out->launched_queries = S->launched_queries.load();
    out->outstanding = S->outstanding.load();
    out->cached_plans = (int64_t)S->plans.size();
    out->scratch_bytes_per_stream = S->slots.empty() ? 0 : (int64_t)S->slots[0].ex.scratch_bytes;
    out->now = S->now();
    return PG_OK;
}

extern "C" void pg_server_free(pg_server *S) {
    if (!S) return;
    S->stop = true;
    if (S->worker.joinable()) S->worker.join();
    for (Slot &s : S->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.batch) pg_batch_free(s.batch);
        if (s.done) cudaEventDestroy(s.done);
        if (s.raised) cudaEventDestroy(s.raised);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.d_area) cudaFree(s.d_area);
        if (s.h_area) cudaFreeHost(s.h_area);
        if (s.d_counts) cudaFree(s.d_counts);
        if (s.h_counts) cudaFreeHost(s.h_counts);
        pg_exec_release(&s.ex);
    }
    for (auto &kv : S->plans) pg_free_plan(kv.second);
    if (S->ctl_stream) {
        cudaStreamSynchronize(S->ctl_stream);
        cudaStreamDestroy(S->ctl_stream);
    }
    if (S->h_one) cudaFreeHost(S->h_one);
    if (S->g) S->g->servers--;
    delete S;
}

extern "C" int pg_server_cancel(pg_server *S, uint64_t ticket) {
    if (!S) return pg_set_error(PG_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    if (ticket == 0 || ticket >= S->next_ticket) return pg_set_error(PG_EINVAL, "no such ticket");
    S->cancelled.push_back(ticket);
    return PG_OK;
}
