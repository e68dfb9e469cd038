// Test infrastructure: runs the host runtime's batch flattening (fastged::flatten) on a
// handle set up for a 152-SM GPU, without a device (see fake_cuda.cpp), and exposes what it
// produced: the batch's sizes and offsets, the size classes with their pair orders, the graph
// table, the map offsets, the branching-order permutation and the pinned staging bytes.
#include <cstring>

#include "fastged_internal.h"
#include "fastged_runtime.h"

using namespace fastged;

static fastged_handle *probe_handle()
{
    static fastged_handle h;
    return &h;
}
static Batch g_b;

extern "C" int probe_flatten(const fastged_pair_list *pl, int32_t K, const fastged_options *opt,
                             const int32_t *cost)
{
    fastged_handle *h = probe_handle();
    h->cost = fastged_cost_model{cost[0], cost[1], cost[2], cost[3], cost[4], cost[5]};
    h->sm_count = 152;
    h->smem_optin = 232448;
    h->smem_per_sm = 233472;
    return flatten(h, pl, K, opt ? *opt : default_options(), g_b);
}

extern "C" const char *probe_error() { return fastged_last_error(nullptr); }

// n_graphs n_pairs K B labelled has_kpp n_vlab n_edges adj_words plane_words map_total
// off_meta off_vlab off_edges off_elab off_pairs off_order off_mapoff off_kpp in_bytes
// woff_err woff_cost woff_nev woff_map out_bytes woff_queue woff_pool woff_scratch work_bytes
// n_classes perm_size
extern "C" void probe_batch(int64_t *v)
{
    const Batch &b = g_b;
    const int64_t x[] = {b.n_graphs, b.n_pairs, b.K, b.B, b.labelled, b.has_kpp, b.n_vlab,
                         b.n_edges, b.adj_words, b.plane_words, b.map_total,
                         (int64_t)b.off_meta, (int64_t)b.off_vlab, (int64_t)b.off_edges,
                         (int64_t)b.off_elab, (int64_t)b.off_pairs, (int64_t)b.off_order,
                         (int64_t)b.off_mapoff, (int64_t)b.off_kpp, (int64_t)b.in_bytes,
                         (int64_t)b.woff_err, (int64_t)b.woff_cost, (int64_t)b.woff_nev,
                         (int64_t)b.woff_map, (int64_t)b.out_bytes, (int64_t)b.woff_queue,
                         (int64_t)b.woff_pool, (int64_t)b.woff_scratch, (int64_t)b.work_bytes,
                         (int64_t)b.classes.size(), (int64_t)b.perm.size()};
    memcpy(v, x, sizeof(x));
}

// W wide w32 pk cluster n1max n2max m1max kmax n_order order_off block grid slice_bytes
// scratch_off smem_bytes warp
extern "C" void probe_class(int k, int64_t *v)
{
    const ClassPlan &c = g_b.classes[k];
    const int64_t x[] = {c.W, c.wide, c.w32, c.pk, c.cluster, c.n1max, c.n2max, c.m1max,
                         c.kmax, (int64_t)c.order.size(), c.order_off, c.block, c.grid,
                         c.lay.slice_bytes, (int64_t)c.scratch_off, c.lay.smem_bytes, c.warp};
    memcpy(v, x, sizeof(x));
}

extern "C" void probe_class_order(int k, int32_t *out)
{
    const auto &o = g_b.classes[k].order;
    if (!o.empty()) memcpy(out, o.data(), 4 * o.size());
}

extern "C" void probe_meta(void *out)
{
    if (!g_b.meta.empty()) memcpy(out, g_b.meta.data(), sizeof(GraphMeta) * g_b.meta.size());
}

extern "C" void probe_map_off(int64_t *out)
{
    if (!g_b.map_off.empty()) memcpy(out, g_b.map_off.data(), 8 * g_b.map_off.size());
}

extern "C" void probe_perm(int32_t *out)
{
    if (!g_b.perm.empty()) memcpy(out, g_b.perm.data(), 4 * g_b.perm.size());
}

extern "C" const void *probe_staging() { return probe_handle()->pin.p; }

// drops the staging buffer, so that the next flatten allocates it again
extern "C" void probe_reset() { probe_handle()->pin.release(); }
