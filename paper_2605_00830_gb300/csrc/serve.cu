// serve.cu -- continuous-batching GED server on one GPU.
//
// Requests (a graph pair and its K) are submitted from any host thread and copied into the
// server. A dispatcher thread forms batches while earlier batches are still running: it keeps
// up to `lanes` batches in flight, each on its own lane (a private handle with its own
// streams, pinned staging and grow-only device buffers, so graph bitsets, beams and outputs
// stay resident between batches). A batch takes the oldest pending request's size bucket
// (bit-set words of g2 and a K range) and every pending request of that bucket, up to
// max_batch_pairs; it is launched once enough pairs are pending, once the oldest has waited
// max_wait_us, or at once when the GPU has nothing else in flight. Admission checks free
// device memory against the batch's footprint plus a reserve. A stream callback marks a
// lane finished; the dispatcher then moves its results to the completion queue that
// fastged_serve_poll drains. Latency is measured from submit to that hand-off.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/fastged.h"
#include "fastged_internal.h"
#include "fastged_runtime.h"

using namespace fastged;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t tag = 0;
    int32_t K = 1;
    int bucket = 0;
    int retries = 0;   // times the query went back to the queue after its batch failed
    int32_t n[2] = {0, 0}, m[2] = {0, 0};
    std::vector<int32_t> vl[2], ed[2], el[2];
    bool labelled[2] = {false, false};
    Clock::time_point t_submit;
};

struct Result {
    fastged_serve_result r;
    std::vector<int32_t> map;
};

struct Lane {
    fastged_handle *h = nullptr;
    bool busy = false;
    bool large = false;   // running a batch of large pairs
    int sms = 0;          // SMs the large batch's teams may hold at once
    bool done = false;
    std::vector<Request *> reqs;
    std::vector<fastged_graph> graphs;
    std::vector<int32_t> pairs, kpp, out_cost, out_map;
    std::vector<int64_t> out_nev;
    Clock::time_point t_launch;
    fastged_server *srv = nullptr;
};

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Size buckets follow the size classes: one-warp teams (K <= 128, target of at most 63
// vertices) split by their word instance (<= 31 vertices: bucket 0, else 2); the other pairs
// by the bitset word class of the target graph (<= 32 vertices: bucket 1, one 64-bit word: 3,
// then 2, 4, 8, 16 words: 4-7). A batch carries a K per pair, so K splits nothing else, and a
// batch of one bucket is (nearly always) one size class, launched on its lane's own stream.
int bucket_of(int n2, int K)
{
    if (K <= kWarpMaxK && n2 <= kWarpMaxN2) return n2 <= kWarpMaxN2Word32 ? 0 : 2;
    const int w = n2 <= 32 ? 0 : n2 <= 64 ? 1 : n2 <= 128 ? 2 : n2 <= 256 ? 3 : n2 <= 512 ? 4 : 5;
    if (w <= 1) return 2 * w + 1;
    return 2 + w;
}

// Buckets of pairs with more than 256 target vertices (two-CTA cluster teams): such batches
// run for long (a batch holds its lane until its slowest pair ends), so they take every
// pending pair of their bucket, hold at most three lanes in eight, and together at most the
// SMs of the large-batch budget (half of the SMs). Every other batch keeps its persistent
// teams on at most a third of the SMs. A batch's teams hold their SMs until its queue is
// empty, so without these caps a dense or large batch would occupy the whole GPU and the
// small queries that arrive meanwhile would wait for it (a serving run at 5,000 req/s:
// molecule-query median 152 ms uncapped, 0.8 ms capped, the same completed rate).
bool bucket_is_large(int bucket) { return bucket >= 6; }

// The checks fastged_batch applies to one graph, plus duplicate edges (found by sorting).
int validate_graph(const fastged_graph *g, bool *labelled)
{
    if (!g) return set_error(FASTGED_ERR_INVALID_ARG, "null graph");
    if (g->n < 0 || g->n > FASTGED_MAX_N) return set_error(FASTGED_ERR_INVALID_ARG, "n out of range");
    if (g->m < 0 || (int64_t)g->m > (int64_t)g->n * (g->n - 1) / 2)
        return set_error(FASTGED_ERR_INVALID_ARG, "m out of range");
    if ((g->n > 0 && !g->vlabel) || (g->m > 0 && !g->edges))
        return set_error(FASTGED_ERR_INVALID_ARG, "null array");
    std::vector<int64_t> keys((size_t)g->m);
    for (int k = 0; k < g->m; ++k) {
        const int u = g->edges[2 * k], v = g->edges[2 * k + 1];
        if (u < 0 || v < 0 || u >= g->n || v >= g->n || u == v)
            return set_error(FASTGED_ERR_INVALID_ARG, "bad edge endpoint or self-loop");
        keys[k] = (int64_t)std::min(u, v) * g->n + std::max(u, v);
        if (g->elabel && (g->elabel[k] < 0 || g->elabel[k] > FASTGED_MAX_ELABEL))
            return set_error(FASTGED_ERR_INVALID_ARG, "edge label out of range");
    }
    std::sort(keys.begin(), keys.end());
    for (size_t k = 1; k < keys.size(); ++k)
        if (keys[k] == keys[k - 1]) return set_error(FASTGED_ERR_INVALID_ARG, "duplicate edge");
    *labelled = g->elabel != nullptr && g->m > 0;
    return FASTGED_OK;
}

}  // namespace

struct fastged_server {
    fastged_cost_model cost{};
    fastged_serve_config cfg{};
    std::mutex mu;
    std::condition_variable cv;        // dispatcher wake-ups
    std::condition_variable done_cv;   // poll wake-ups
    std::deque<Request *> pending;
    std::vector<Lane> lanes;
    std::deque<Result> done_q;
    std::thread dispatcher;
    bool stopping = false;
    fastged_serve_stats st{};
    int sm_count = 1;
    int large_sms = 1;   // SMs that the large batches in flight may hold together
};

// Queries of a failed batch that may still be retried go back to the front of the queue in
// their order; returns whether q was taken back (caller holds mu).
static bool requeue_for_retry(fastged_server *s, Request *q, std::vector<Request *> &again)
{
    if (q->retries >= s->cfg.max_retries) return false;
    ++q->retries;
    again.push_back(q);
    return true;
}

static void push_front_in_order(fastged_server *s, const std::vector<Request *> &again)
{
    for (auto it = again.rbegin(); it != again.rend(); ++it) s->pending.push_front(*it);
    if (!again.empty()) s->cv.notify_all();
}

static void CUDART_CB lane_done_cb(void *arg)
{
    Lane *l = (Lane *)arg;
    {
        std::lock_guard<std::mutex> g(l->srv->mu);
        l->done = true;
    }
    l->srv->cv.notify_all();
}

// Moves a finished lane's results to the completion queue (caller holds mu).
static void collect_lane(fastged_server *s, Lane &l)
{
    const int np = (int)l.reqs.size();
    const int rc = batch_results(l.h, l.out_cost.data(), l.out_map.data(), l.out_nev.data());
    const Clock::time_point now = Clock::now();
    int64_t off = 0;
    std::vector<Request *> again;
    for (int p = 0; p < np; ++p) {
        Request *q = l.reqs[p];
        if (rc != FASTGED_OK && requeue_for_retry(s, q, again)) continue;
        Result res;
        memset(&res.r, 0, sizeof(res.r));
        res.r.tag = q->tag;
        res.r.status = rc;
        res.r.n1 = rc == FASTGED_OK ? q->n[0] : 0;   // a failed query has no map
        res.r.latency_ms = ms_between(q->t_submit, now);
        res.r.queue_ms = ms_between(q->t_submit, l.t_launch);
        if (rc == FASTGED_OK) {
            res.r.cost = l.out_cost[p];
            res.r.n_evals = l.out_nev[p];
            res.map.assign(l.out_map.begin() + off, l.out_map.begin() + off + q->n[0]);
        }
        off += q->n[0];
        s->done_q.push_back(std::move(res));
        s->st.completed++;
        if (rc != FASTGED_OK) s->st.failed++;
        delete q;
    }
    push_front_in_order(s, again);
    l.reqs.clear();
    l.busy = false;
    l.done = false;
    s->done_cv.notify_all();
}

// Builds and enqueues one batch on a free lane (caller holds mu; it is released while the
// batch is flattened and launched).
static void launch_batch(fastged_server *s, Lane &l, std::unique_lock<std::mutex> &lk,
                         int max_sms)
{
    NvtxRange r("fastged serve batch");
    const int np = (int)l.reqs.size();
    l.graphs.resize(2 * (size_t)np);
    l.pairs.resize(2 * (size_t)np);
    l.kpp.resize(np);
    int32_t kmax = 1;
    int64_t mtot = 0;
    for (int p = 0; p < np; ++p) {
        Request *q = l.reqs[p];
        for (int r = 0; r < 2; ++r) {
            fastged_graph &g = l.graphs[2 * p + r];
            g.n = q->n[r];
            g.vlabel = q->vl[r].data();
            g.m = q->m[r];
            g.edges = q->ed[r].data();
            g.elabel = q->labelled[r] ? q->el[r].data() : nullptr;
        }
        l.pairs[2 * p] = 2 * p;
        l.pairs[2 * p + 1] = 2 * p + 1;
        l.kpp[p] = q->K;
        kmax = std::max(kmax, q->K);
        mtot += q->n[0];
    }
    l.out_cost.resize(np);
    l.out_nev.resize(np);
    l.out_map.resize((size_t)std::max<int64_t>(mtot, 1));
    l.busy = true;
    l.done = false;
    l.t_launch = Clock::now();
    s->st.batches++;
    s->st.batched_pairs += np;
    lk.unlock();
    fastged_pair_list pl;
    pl.n_graphs = 2 * np;
    pl.graphs = l.graphs.data();
    pl.n_pairs = np;
    pl.pairs = l.pairs.data();
    fastged_options o = default_options();
    o.k_per_pair = l.kpp.data();
    o.max_sms = max_sms;
    // large pairs on two-CTA clusters: the most successors per SM and second, which is what
    // a stream of queries needs (a bigger cluster only shortens one pair's latency)
    if (l.large) o.cluster = 2;
    int rc = batch_enqueue(l.h, &pl, kmax, o);
    int sms = 0;
    if (rc == FASTGED_OK && l.large) {
        // large classes run one CTA per SM
        for (const ClassPlan &cp : l.h->batch.classes) sms += cp.grid;
        sms = std::min(sms, s->sm_count);
    }
    if (rc == FASTGED_OK && cudaLaunchHostFunc(l.h->stream, lane_done_cb, &l) != cudaSuccess)
        rc = FASTGED_ERR_CUDA;
    if (rc != FASTGED_OK) {
        // copies queued before the failure finish before the lane's buffers are reused
        cudaStreamSynchronize(l.h->stream);
        cudaGetLastError();
    }
    lk.lock();
    l.sms = rc == FASTGED_OK ? sms : 0;
    if (rc != FASTGED_OK) {
        // nothing is in flight on this lane: queue the requests again while they may be
        // retried, report the failure for the others
        const Clock::time_point now = Clock::now();
        std::vector<Request *> again;
        for (Request *q : l.reqs) {
            if (requeue_for_retry(s, q, again)) continue;
            Result res;
            memset(&res.r, 0, sizeof(res.r));
            res.r.tag = q->tag;
            res.r.status = rc;
            res.r.n1 = 0;   // no map
            res.r.latency_ms = ms_between(q->t_submit, now);
            res.r.queue_ms = ms_between(q->t_submit, l.t_launch);
            s->done_q.push_back(std::move(res));
            s->st.completed++;
            s->st.failed++;
            delete q;
        }
        push_front_in_order(s, again);
        l.reqs.clear();
        l.busy = false;
        s->done_cv.notify_all();
    }
}

// Rough device footprint of a batch: inputs, bit-set pools, outputs and team scratch.
static size_t footprint(const std::vector<Request *> &reqs)
{
    size_t b = 1 << 20;
    for (const Request *q : reqs) {
        for (int r = 0; r < 2; ++r)
            b += 24 * (size_t)q->n[r] + 12 * (size_t)q->m[r] +
                 (size_t)q->n[r] * (size_t)((q->n[r] + 63) / 64) * 8 * 3;
        b += 64 + 4 * (size_t)q->n[0];
    }
    return b;
}

static void dispatcher_main(fastged_server *s)
{
    cudaSetDevice(s->lanes.empty() ? 0 : s->lanes[0].h->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        for (Lane &l : s->lanes)
            if (l.busy && l.done) collect_lane(s, l);
        int busy = 0;
        Lane *free_lane = nullptr;
        for (Lane &l : s->lanes) {
            if (l.busy) ++busy;
            else if (!free_lane) free_lane = &l;
        }
        if (s->stopping && s->pending.empty() && busy == 0) break;
        bool launched = false;
        if (free_lane && !s->pending.empty()) {
            // large batches: while one runs, another starts only if it would hold at most
            // three lanes in eight and the SM budget has room for a few teams
            int large_busy = 0, large_held = 0;
            for (const Lane &l : s->lanes)
                if (l.busy && l.large) {
                    ++large_busy;
                    large_held += l.sms;
                }
            const int large_room = s->large_sms - large_held;
            const bool large_ok =
                large_busy == 0 ||
                (large_busy < std::max(1, 3 * (int)s->lanes.size() / 8) && large_room >= 4);
            // the oldest query whose bucket may run now
            const Request *oldest = nullptr;
            for (const Request *q : s->pending)
                if (large_ok || !bucket_is_large(q->bucket)) {
                    oldest = q;
                    break;
                }
            const int bkt = oldest ? oldest->bucket : -1;
            int avail = 0;
            if (oldest)
                for (const Request *q : s->pending) avail += (q->bucket == bkt);
            const double waited_us = oldest ? 1e3 * ms_between(oldest->t_submit, Clock::now()) : 0.0;
            if (oldest && (avail >= s->cfg.min_batch_pairs || waited_us >= s->cfg.max_wait_us ||
                           busy == 0 || s->stopping)) {
                std::vector<Request *> take;
                for (auto it = s->pending.begin();
                     it != s->pending.end() && (int)take.size() < s->cfg.max_batch_pairs;) {
                    if ((*it)->bucket == bkt) {
                        take.push_back(*it);
                        it = s->pending.erase(it);
                    } else {
                        ++it;
                    }
                }
                // admission by free device memory
                size_t free_b = 0, total_b = 0;
                cudaMemGetInfo(&free_b, &total_b);
                const size_t need = footprint(take) + (size_t)s->cfg.hbm_reserve_bytes;
                const bool refuse = (free_b < need && busy > 0) || inject_fire(FASTGED_INJECT_ADMISSION);
                if (refuse) {
                    // wait for a running batch to release memory; keep arrival order
                    for (auto it = take.rbegin(); it != take.rend(); ++it) s->pending.push_front(*it);
                    s->st.admission_waits++;
                } else {
                    free_lane->reqs = std::move(take);
                    free_lane->large = bucket_is_large(bkt);
                    launch_batch(s, *free_lane, lk,
                                 free_lane->large ? std::max(large_room, 2)
                                                  : std::max(1, s->sm_count / 3));
                    launched = true;
                }
            }
        }
        if (!launched)
            s->cv.wait_for(lk, std::chrono::microseconds(std::max(20, s->cfg.max_wait_us / 4)));
    }
}

static fastged_serve_config serve_defaults()
{
    fastged_serve_config c;
    memset(&c, 0, sizeof(c));
    c.lanes = 16;
    c.max_batch_pairs = 4096;
    c.min_batch_pairs = 64;
    c.max_pending = 1 << 20;
    c.max_wait_us = 200;
    c.hbm_reserve_bytes = (int64_t)1 << 30;
    return c;
}

extern "C" int fastged_serve_start(const fastged_cost_model *cost, const fastged_serve_config *cfg,
                                   fastged_server **out)
{
    clear_error();
    if (!cost || !out) return set_error(FASTGED_ERR_INVALID_ARG, "null argument");
    fastged_serve_config c = cfg ? *cfg : serve_defaults();
    if (c.lanes < 1 || c.lanes > 16 || c.max_batch_pairs < 1 || c.min_batch_pairs < 1 ||
        c.max_pending < 1 || c.max_wait_us < 0 || c.hbm_reserve_bytes < 0 || c.max_retries < 0)
        return set_error(FASTGED_ERR_INVALID_ARG, "serve config out of range");
    fastged_server *s = new fastged_server();
    s->cost = *cost;
    s->cfg = c;
    s->lanes.resize(c.lanes);
    for (Lane &l : s->lanes) {
        l.srv = s;
        const int rc = fastged_create(cost, &l.h);
        if (rc != FASTGED_OK) {
            for (Lane &x : s->lanes)
                if (x.h) fastged_destroy(x.h);
            delete s;
            return rc;
        }
    }
    // the large batches together keep off a sixth of the SMs (at least 8), which stay free
    // for the small queries' teams
    s->sm_count = std::max(1, s->lanes[0].h->sm_count);
    s->large_sms = std::max(2, s->sm_count / 2);
    s->dispatcher = std::thread(dispatcher_main, s);
    *out = s;
    return FASTGED_OK;
}

extern "C" int fastged_serve_submit(fastged_server *s, const fastged_graph *g1,
                                    const fastged_graph *g2, int32_t K, uint64_t tag)
{
    clear_error();
    if (!s) return set_error(FASTGED_ERR_INVALID_ARG, "null server");
    if (K < 1 || K > FASTGED_MAX_K) return set_error(FASTGED_ERR_INVALID_ARG, "K out of range");
    bool lab[2] = {false, false};
    int rc = validate_graph(g1, &lab[0]);
    if (rc) return rc;
    if ((rc = validate_graph(g2, &lab[1]))) return rc;
    const fastged_cost_model &c = s->cost;
    const long long bound = (long long)g1->n * std::max(c.v_sub, c.v_del) +
                            (long long)g2->n * c.v_ins +
                            (long long)g1->m * std::max(c.e_sub, c.e_del) +
                            (long long)g2->m * c.e_ins;
    if (bound >= (long long)INT32_MAX)
        return set_error(FASTGED_ERR_INVALID_ARG, "costs can overflow int32");
    Request *q = new Request();
    q->tag = tag;
    q->K = K;
    const fastged_graph *gs[2] = {g1, g2};
    for (int r = 0; r < 2; ++r) {
        const fastged_graph *g = gs[r];
        q->n[r] = g->n;
        q->m[r] = g->m;
        q->vl[r].assign(g->vlabel, g->vlabel + g->n);
        q->ed[r].assign(g->edges, g->edges + 2 * (size_t)g->m);
        q->labelled[r] = lab[r];
        if (lab[r]) q->el[r].assign(g->elabel, g->elabel + g->m);
    }
    q->bucket = bucket_of(g2->n, K);
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stopping) {
            delete q;
            return set_error(FASTGED_ERR_STOPPED, "server is stopping");
        }
        if ((int)s->pending.size() >= s->cfg.max_pending) {
            delete q;
            s->st.rejected_busy++;
            return set_error(FASTGED_ERR_BUSY, "request queue full");
        }
        s->pending.push_back(q);
        s->st.submitted++;
    }
    s->cv.notify_all();
    return FASTGED_OK;
}

extern "C" int fastged_serve_cancel(fastged_server *s, uint64_t tag)
{
    clear_error();
    if (!s) return set_error(FASTGED_ERR_INVALID_ARG, "null server");
    int n = 0;
    {
        std::lock_guard<std::mutex> g(s->mu);
        const Clock::time_point now = Clock::now();
        for (auto it = s->pending.begin(); it != s->pending.end();) {
            Request *q = *it;
            if (q->tag != tag) {
                ++it;
                continue;
            }
            Result res;
            memset(&res.r, 0, sizeof(res.r));
            res.r.tag = q->tag;
            res.r.status = FASTGED_ERR_CANCELLED;
            res.r.latency_ms = res.r.queue_ms = ms_between(q->t_submit, now);
            s->done_q.push_back(std::move(res));
            s->st.completed++;
            delete q;
            it = s->pending.erase(it);
            ++n;
        }
    }
    if (n > 0) {
        s->done_cv.notify_all();
        s->cv.notify_all();
    }
    return n;
}

extern "C" int fastged_serve_poll(fastged_server *s, fastged_serve_result *out, int32_t max_results,
                                  int32_t *map_buf, int64_t map_cap, int32_t timeout_ms)
{
    clear_error();
    if (!s || (!out && max_results > 0) || max_results < 0)
        return set_error(FASTGED_ERR_INVALID_ARG, "bad argument");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done_q.empty() && timeout_ms > 0)
        s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                            [s] { return !s->done_q.empty(); });
    int n = 0;
    int64_t used = 0;
    while (n < max_results && !s->done_q.empty()) {
        Result &r = s->done_q.front();
        const int64_t need = (int64_t)r.map.size();
        if (need > 0 && (!map_buf || used + need > map_cap)) {
            if (n == 0) return set_error(FASTGED_ERR_INVALID_ARG, "map buffer too small");
            break;
        }
        out[n] = r.r;
        out[n].map_offset = used;
        if (need > 0) memcpy(map_buf + used, r.map.data(), sizeof(int32_t) * (size_t)need);
        used += need;
        s->done_q.pop_front();
        ++n;
    }
    return n;
}

extern "C" int fastged_serve_get_stats(fastged_server *s, fastged_serve_stats *out)
{
    clear_error();
    if (!s || !out) return set_error(FASTGED_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->st;
    out->pending = (int64_t)s->pending.size();
    int64_t busy = 0;
    for (const Lane &l : s->lanes) busy += l.busy ? 1 : 0;
    out->lanes_busy = busy;
    return FASTGED_OK;
}

extern "C" void fastged_serve_stop(fastged_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stopping = true;
    }
    s->cv.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
}

extern "C" void fastged_serve_destroy(fastged_server *s)
{
    if (!s) return;
    fastged_serve_stop(s);
    for (Lane &l : s->lanes)
        if (l.h) fastged_destroy(l.h);
    for (Request *q : s->pending) delete q;
    delete s;
}
