// Test driver for the host runtime under sanitizers (tests/test_host_sanitizers.py builds it
// with ThreadSanitizer, and with AddressSanitizer + UndefinedBehaviorSanitizer, against the
// fakes of fake_cuda.cpp). Through the public C API it runs, on seeded random graphs of every
// size class: batches from two handles on two threads at once (one of them contends for the
// shared host thread pool), invalid batches, the degree order, an autotuned plan replayed as
// a graph, and the server fed by three submitting threads while the main thread cancels a few
// queries and polls. It
// prints one summary line and exits 0 only if every call returned what it should.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "fastged.h"

extern "C" void fake_set_host_fn_delay_us(int us);

namespace {

std::atomic<int> g_failures{0};

void expect(bool ok, const char *what)
{
    if (!ok) {
        ++g_failures;
        std::fprintf(stderr, "FAILED: %s (%s)\n", what, fastged_last_error(nullptr));
    }
}

// splitmix64
struct Rng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    int below(int n) { return (int)(next() % (uint64_t)n); }
};

struct Graph {
    int n = 0;
    std::vector<int32_t> vl, ed, el;
};

Graph random_graph(Rng &r, int n, int per_mille, bool labelled)
{
    Graph g;
    g.n = n;
    for (int v = 0; v < n; ++v) g.vl.push_back(r.below(8));
    for (int u = 0; u < n; ++u)
        for (int v = u + 1; v < n; ++v)
            if (r.below(1000) < per_mille) {
                g.ed.push_back(u);
                g.ed.push_back(v);
                if (labelled) g.el.push_back(r.below(3));
            }
    return g;
}

struct Batch {
    std::vector<Graph> graphs;
    std::vector<fastged_graph> view;
    std::vector<int32_t> pairs;
    fastged_pair_list pl{};
    int64_t map_total = 0;

    void finish()
    {
        view.clear();
        for (const Graph &g : graphs) {
            fastged_graph v;
            v.n = g.n;
            v.vlabel = g.vl.data();
            v.m = (int32_t)(g.ed.size() / 2);
            v.edges = g.ed.data();
            v.elabel = g.el.empty() ? nullptr : g.el.data();
            view.push_back(v);
        }
        pl.n_graphs = (int32_t)view.size();
        pl.graphs = view.data();
        pl.n_pairs = (int32_t)(pairs.size() / 2);
        pl.pairs = pairs.data();
        map_total = 0;
        for (size_t p = 0; p < pairs.size(); p += 2) map_total += graphs[pairs[p]].n;
    }
};

// pairs of every size class: mostly small, some of 33-64, 65-300 and a few of 300-600 vertices
Batch random_batch(uint64_t seed, int n_pairs)
{
    Rng r{seed};
    Batch b;
    for (int p = 0; p < n_pairs; ++p) {
        const int c = r.below(100);
        const int lo = c < 70 ? 5 : c < 85 ? 33 : c < 97 ? 65 : 300;
        const int hi = c < 70 ? 32 : c < 85 ? 64 : c < 97 ? 300 : 600;
        const int pm = hi > 100 ? 20 : 120;
        const bool lab = r.below(2) == 0;
        for (int k = 0; k < 2; ++k) b.graphs.push_back(random_graph(r, lo + r.below(hi - lo + 1), pm, lab));
        b.pairs.push_back(2 * p);
        b.pairs.push_back(2 * p + 1);
    }
    b.finish();
    return b;
}

int run_batch(fastged_handle *h, const Batch &b, int K, const fastged_options *o)
{
    std::vector<int32_t> cost(b.pl.n_pairs), map((size_t)std::max<int64_t>(b.map_total, 1));
    std::vector<int64_t> nev(b.pl.n_pairs);
    return fastged_batch_ex(h, &b.pl, K, o, cost.data(), map.data(), nev.data());
}

}  // namespace

int main()
{
    const fastged_cost_model cost = {2, 4, 4, 1, 2, 2};
    fastged_options opt;
    std::memset(&opt, 0, sizeof(opt));
    opt.use_cuda_graph = 1;

    // batches from two handles on two threads at once
    Batch big = random_batch(1, 3000), other = random_batch(2, 2000);
    std::thread t1([&] {
        fastged_handle *h = nullptr;
        expect(fastged_create(&cost, &h) == FASTGED_OK, "create 1");
        for (int k = 0; k < 4; ++k) expect(run_batch(h, big, 64, &opt) == FASTGED_OK, "batch 1");
        fastged_destroy(h);
    });
    std::thread t2([&] {
        fastged_handle *h = nullptr;
        expect(fastged_create(&cost, &h) == FASTGED_OK, "create 2");
        fastged_options o2 = opt;
        o2.vertex_order = FASTGED_ORDER_DEGREE;
        for (int k = 0; k < 4; ++k) expect(run_batch(h, other, 100, &o2) == FASTGED_OK, "batch 2");
        fastged_destroy(h);
    });
    t1.join();
    t2.join();

    // invalid batches: a bad pair index and a bad endpoint far into the batch
    {
        fastged_handle *h = nullptr;
        expect(fastged_create(&cost, &h) == FASTGED_OK, "create 3");
        Batch bad = random_batch(3, 2500);
        bad.pairs[2 * 2100 + 1] = 1 << 30;
        bad.finish();
        expect(run_batch(h, bad, 32, &opt) == FASTGED_ERR_INVALID_ARG, "bad pair rejected");
        Batch bad2 = random_batch(4, 2500);
        for (Graph &g : bad2.graphs)
            if (&g - bad2.graphs.data() == 3001 && !g.ed.empty()) g.ed[0] = g.n + 5;
        bad2.finish();
        const int rc = run_batch(h, bad2, 32, &opt);
        expect(rc == FASTGED_ERR_INVALID_ARG || bad2.graphs[3001].ed.empty(), "bad endpoint rejected");
        expect(run_batch(h, big, 16, &opt) == FASTGED_OK, "handle usable after errors");

        // an autotuned plan, run three times and read back
        fastged_plan *p = nullptr;
        fastged_options po = opt;
        po.autotune = 1;
        expect(fastged_plan_create(h, &big.pl, 64, &po, &p) == FASTGED_OK, "plan create");
        for (int k = 0; k < 3; ++k) expect(fastged_plan_run(p, nullptr) == FASTGED_OK, "plan run");
        std::vector<int32_t> c(big.pl.n_pairs), m((size_t)big.map_total);
        std::vector<int64_t> n(big.pl.n_pairs);
        expect(fastged_plan_read(p, c.data(), m.data(), n.data()) == FASTGED_OK, "plan read");
        fastged_plan_destroy(p);
        fastged_destroy(h);
    }

    // the server: three submitting threads, the main thread polls
    int served = 0;
    {
        fake_set_host_fn_delay_us(200);
        fastged_serve_config cfg;
        std::memset(&cfg, 0, sizeof(cfg));
        cfg.lanes = 3;
        cfg.max_batch_pairs = 32;
        cfg.min_batch_pairs = 4;
        cfg.max_pending = 64;
        cfg.max_wait_us = 200;
        cfg.hbm_reserve_bytes = 0;
        fastged_server *s = nullptr;
        expect(fastged_serve_start(&cost, &cfg, &s) == FASTGED_OK, "serve start");
        Batch q = random_batch(5, 300);
        const int per = 100;
        std::vector<std::thread> subs;
        for (int t = 0; t < 3; ++t)
            subs.emplace_back([&, t] {
                for (int k = t * per; k < (t + 1) * per; ++k) {
                    for (;;) {
                        const int rc = fastged_serve_submit(s, &q.view[q.pairs[2 * k]],
                                                            &q.view[q.pairs[2 * k + 1]], 32 << (k % 3),
                                                            (uint64_t)k);
                        if (rc == FASTGED_ERR_BUSY) {
                            std::this_thread::sleep_for(std::chrono::microseconds(200));
                            continue;
                        }
                        expect(rc == FASTGED_OK, "submit");
                        break;
                    }
                }
            });
        // cancel a few queries while the others are submitted and served (each is either still
        // queued, and comes back cancelled, or already in a batch, and runs)
        for (int k : {10, 150, 250}) expect(fastged_serve_cancel(s, (uint64_t)k) >= 0, "cancel");
        std::vector<fastged_serve_result> out(64);
        std::vector<int32_t> maps(1 << 16);
        std::vector<int> seen(3 * per, 0);
        const auto t0 = std::chrono::steady_clock::now();
        while (served < 3 * per &&
               std::chrono::steady_clock::now() - t0 < std::chrono::seconds(120)) {
            const int n = fastged_serve_poll(s, out.data(), (int32_t)out.size(), maps.data(),
                                             (int64_t)maps.size(), 20);
            expect(n >= 0, "poll");
            for (int i = 0; i < n; ++i) {
                const uint64_t t = out[i].tag;
                const bool may_cancel = t == 10 || t == 150 || t == 250;
                expect(out[i].status == FASTGED_OK ||
                           (may_cancel && out[i].status == FASTGED_ERR_CANCELLED && out[i].n1 == 0),
                       "served status");
                expect(out[i].tag < (uint64_t)(3 * per) && seen[out[i].tag]++ == 0, "served once");
                ++served;
            }
        }
        for (auto &t : subs) t.join();
        fastged_serve_stop(s);
        fastged_serve_stats st;
        expect(fastged_serve_get_stats(s, &st) == FASTGED_OK, "stats");
        expect(st.completed == 3 * per && st.failed == 0, "all served");
        fastged_serve_destroy(s);
        fake_set_host_fn_delay_us(0);
    }
    std::printf("host runtime driver: %d served, %d failures\n", served, g_failures.load());
    return g_failures.load() == 0 ? 0 : 1;
}
