// paths.cu -- edit paths from vertex maps, partial application of an edit path, and GED
// matrices (host code around the K-Best batch).
//
// The edit path of a complete vertex map follows the operation and cost definitions of
// Sec. 2.2-2.4 (vertex and edge substitution, deletion, insertion); its total is the cost of
// the map. Sec. 6 uses an edit path for the crossover of two architectures (applying half of
// its operations) and a GED matrix for nearest-neighbour graph classification.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fastged.h"
#include "fastged_runtime.h"

using namespace fastged;

namespace {

// Sorted edge table of one graph: key (min << 32 | max) -> (label, input index).
struct EdgeTable {
    std::vector<uint64_t> key;
    std::vector<int32_t> lab, idx;
    int find(int u, int v) const
    {
        const uint64_t k = ((uint64_t)(uint32_t)std::min(u, v) << 32) | (uint32_t)std::max(u, v);
        auto it = std::lower_bound(key.begin(), key.end(), k);
        if (it == key.end() || *it != k) return -1;
        return (int)(it - key.begin());
    }
};

// Validates a graph (sizes, pointers, endpoints, self-loops, duplicate edges) and builds its
// edge table; false with the error set otherwise.
bool load_graph(const fastged_graph *g, const char *name, EdgeTable &t)
{
    if (!g) { set_error(FASTGED_ERR_INVALID_ARG, std::string("null ") + name); return false; }
    if (g->n < 0 || g->n > FASTGED_MAX_N || g->m < 0 ||
        (int64_t)g->m > (int64_t)g->n * (g->n - 1) / 2 || (g->n > 0 && !g->vlabel) ||
        (g->m > 0 && !g->edges)) {
        set_error(FASTGED_ERR_INVALID_ARG, std::string(name) + ": invalid sizes or arrays");
        return false;
    }
    std::vector<std::pair<uint64_t, int>> e((size_t)g->m);
    for (int k = 0; k < g->m; ++k) {
        const int u = g->edges[2 * k], v = g->edges[2 * k + 1];
        if (u < 0 || v < 0 || u >= g->n || v >= g->n || u == v) {
            set_error(FASTGED_ERR_INVALID_ARG, std::string(name) + ": bad edge endpoint or self-loop");
            return false;
        }
        e[k] = {((uint64_t)(uint32_t)std::min(u, v) << 32) | (uint32_t)std::max(u, v), k};
    }
    std::sort(e.begin(), e.end());
    t.key.resize(e.size());
    t.lab.resize(e.size());
    t.idx.resize(e.size());
    for (size_t k = 0; k < e.size(); ++k) {
        if (k > 0 && e[k].first == e[k - 1].first) {
            set_error(FASTGED_ERR_INVALID_ARG, std::string(name) + ": duplicate edge");
            return false;
        }
        t.key[k] = e[k].first;
        t.idx[k] = e[k].second;
        t.lab[k] = g->elabel ? g->elabel[e[k].second] : 0;
    }
    return true;
}

// The map's inverse on g2 (-1 = not an image); false with the error set if the map is not an
// injective partial map into g2.
bool invert_map(const fastged_graph *g1, const fastged_graph *g2, const int32_t *mapping,
                std::vector<int> &inv)
{
    inv.assign((size_t)g2->n, -1);
    if (g1->n > 0 && !mapping) { set_error(FASTGED_ERR_INVALID_ARG, "null mapping"); return false; }
    for (int v = 0; v < g1->n; ++v) {
        const int x = mapping[v];
        if (x < -1 || x >= g2->n || (x >= 0 && inv[x] >= 0)) {
            set_error(FASTGED_ERR_INVALID_ARG, "mapping is not an injective partial map into g2");
            return false;
        }
        if (x >= 0) inv[x] = v;
    }
    return true;
}

fastged_edit_op make_op(int kind, int cost, int a, int b, int x, int y)
{
    fastged_edit_op o;
    o.kind = kind;
    o.cost = cost;
    o.g1_u = a;
    o.g1_v = b;
    o.g2_u = x;
    o.g2_v = y;
    return o;
}

}  // namespace

extern "C" int fastged_edit_path(const fastged_cost_model *cost, const fastged_graph *g1,
                                 const fastged_graph *g2, const int32_t *mapping,
                                 fastged_edit_op *ops, int32_t cap, int32_t *n_ops,
                                 int64_t *total_cost)
{
    clear_error();
    if (!cost || !n_ops) return set_error(FASTGED_ERR_INVALID_ARG, "null argument");
    EdgeTable e1, e2;
    if (!load_graph(g1, "g1", e1) || !load_graph(g2, "g2", e2)) return FASTGED_ERR_INVALID_ARG;
    std::vector<int> inv;
    if (!invert_map(g1, g2, mapping, inv)) return FASTGED_ERR_INVALID_ARG;
    const fastged_cost_model &c = *cost;
    std::vector<fastged_edit_op> out;
    for (int x = 0; x < g2->n; ++x)
        if (inv[x] < 0) out.push_back(make_op(FASTGED_OP_VINS, c.v_ins, -1, -1, x, -1));
    for (int v = 0; v < g1->n; ++v) {
        const int x = mapping[v];
        if (x >= 0 && g1->vlabel[v] != g2->vlabel[x])
            out.push_back(make_op(FASTGED_OP_VSUB, c.v_sub, v, -1, x, -1));
    }
    // g1 edges in input order: deleted unless both ends map onto the ends of a g2 edge
    std::vector<int> img((size_t)g1->m, -1);   // g2 edge-table row of each g1 edge's image
    for (int k = 0; k < g1->m; ++k) {
        const int u = g1->edges[2 * k], v = g1->edges[2 * k + 1];
        if (mapping[u] >= 0 && mapping[v] >= 0) img[k] = e2.find(mapping[u], mapping[v]);
        if (img[k] < 0) out.push_back(make_op(FASTGED_OP_EDEL, c.e_del, u, v, -1, -1));
    }
    for (int k = 0; k < g1->m; ++k) {
        if (img[k] < 0) continue;
        const int l1 = g1->elabel ? g1->elabel[k] : 0;
        if (l1 != e2.lab[img[k]]) {
            const int u = g1->edges[2 * k], v = g1->edges[2 * k + 1];
            out.push_back(make_op(FASTGED_OP_ESUB, c.e_sub, u, v, mapping[u], mapping[v]));
        }
    }
    // g2 edges in input order: inserted unless they are the image of a g1 edge
    for (int k = 0; k < g2->m; ++k) {
        const int x = g2->edges[2 * k], y = g2->edges[2 * k + 1];
        if (inv[x] < 0 || inv[y] < 0 || e1.find(inv[x], inv[y]) < 0)
            out.push_back(make_op(FASTGED_OP_EINS, c.e_ins, -1, -1, x, y));
    }
    for (int v = 0; v < g1->n; ++v)
        if (mapping[v] < 0) out.push_back(make_op(FASTGED_OP_VDEL, c.v_del, v, -1, -1, -1));
    *n_ops = (int32_t)out.size();
    int64_t tot = 0;
    for (const auto &o : out) tot += o.cost;
    if (total_cost) *total_cost = tot;
    if (ops) {
        if (cap < (int32_t)out.size())
            return set_error(FASTGED_ERR_INVALID_ARG, "operation array too small");
        if (!out.empty()) memcpy(ops, out.data(), sizeof(fastged_edit_op) * out.size());
    }
    return FASTGED_OK;
}

extern "C" int fastged_apply_edit_ops(const fastged_graph *g1, const fastged_graph *g2,
                                      const int32_t *mapping, const fastged_edit_op *ops,
                                      int32_t n_apply, int32_t *out_n, int32_t *out_vlabel,
                                      int32_t *out_m, int32_t *out_edges, int32_t *out_elabel)
{
    clear_error();
    if (!out_n || !out_m || n_apply < 0 || (n_apply > 0 && !ops))
        return set_error(FASTGED_ERR_INVALID_ARG, "null argument or negative count");
    EdgeTable e1, e2;
    if (!load_graph(g1, "g1", e1) || !load_graph(g2, "g2", e2)) return FASTGED_ERR_INVALID_ARG;
    std::vector<int> inv;
    if (!invert_map(g1, g2, mapping, inv)) return FASTGED_ERR_INVALID_ARG;
    const int n1 = g1->n, n2 = g2->n;
    // node ids while editing: g1 vertex v -> v, inserted g2 vertex x -> n1 + x
    std::vector<char> alive((size_t)(n1 + n2), 0);
    std::vector<int32_t> lab((size_t)(n1 + n2), 0);
    for (int v = 0; v < n1; ++v) { alive[v] = 1; lab[v] = g1->vlabel[v]; }
    std::vector<int> ins_order;
    struct E { int u, v, lab; bool live; };
    std::vector<E> edges;
    for (int k = 0; k < g1->m; ++k)
        edges.push_back({g1->edges[2 * k], g1->edges[2 * k + 1], g1->elabel ? g1->elabel[k] : 0, true});
    auto find_live = [&](int a, int b) -> int {
        for (size_t k = 0; k < edges.size(); ++k)
            if (edges[k].live && ((edges[k].u == a && edges[k].v == b) || (edges[k].u == b && edges[k].v == a)))
                return (int)k;
        return -1;
    };
    auto node_of = [&](int x) -> int { return inv[x] >= 0 ? inv[x] : n1 + x; };
    auto bad = [&](const char *what) { return set_error(FASTGED_ERR_INVALID_ARG, what); };
    for (int q = 0; q < n_apply; ++q) {
        const fastged_edit_op &o = ops[q];
        switch (o.kind) {
        case FASTGED_OP_VINS:
            if (o.g2_u < 0 || o.g2_u >= n2 || inv[o.g2_u] >= 0 || alive[n1 + o.g2_u])
                return bad("vertex insertion of a mapped or present g2 vertex");
            alive[n1 + o.g2_u] = 1;
            lab[n1 + o.g2_u] = g2->vlabel[o.g2_u];
            ins_order.push_back(o.g2_u);
            break;
        case FASTGED_OP_VSUB:
            if (o.g1_u < 0 || o.g1_u >= n1 || o.g2_u < 0 || o.g2_u >= n2 || !alive[o.g1_u])
                return bad("vertex substitution of an absent vertex");
            lab[o.g1_u] = g2->vlabel[o.g2_u];
            break;
        case FASTGED_OP_EDEL: {
            const int k = find_live(o.g1_u, o.g1_v);
            if (o.g1_u < 0 || o.g1_u >= n1 || o.g1_v < 0 || o.g1_v >= n1 || k < 0)
                return bad("edge deletion of an absent edge");
            edges[k].live = false;
            break;
        }
        case FASTGED_OP_ESUB: {
            const int k = find_live(o.g1_u, o.g1_v);
            const int r = (o.g2_u >= 0 && o.g2_u < n2 && o.g2_v >= 0 && o.g2_v < n2)
                              ? e2.find(o.g2_u, o.g2_v) : -1;
            if (o.g1_u < 0 || o.g1_u >= n1 || o.g1_v < 0 || o.g1_v >= n1 || k < 0 || r < 0)
                return bad("edge substitution of an absent edge");
            edges[k].lab = e2.lab[r];
            break;
        }
        case FASTGED_OP_EINS: {
            if (o.g2_u < 0 || o.g2_u >= n2 || o.g2_v < 0 || o.g2_v >= n2)
                return bad("edge insertion with an endpoint outside g2");
            const int a = node_of(o.g2_u), b = node_of(o.g2_v);
            const int r = e2.find(o.g2_u, o.g2_v);
            if (!alive[a] || !alive[b] || r < 0 || find_live(a, b) >= 0)
                return bad("edge insertion between absent vertices, or of a present edge");
            edges.push_back({a, b, e2.lab[r], true});
            break;
        }
        case FASTGED_OP_VDEL:
            if (o.g1_u < 0 || o.g1_u >= n1 || !alive[o.g1_u])
                return bad("vertex deletion of an absent vertex");
            alive[o.g1_u] = 0;
            for (auto &e : edges)
                if (e.u == o.g1_u || e.v == o.g1_u) e.live = false;
            break;
        default:
            return bad("unknown operation kind");
        }
    }
    // renumber: surviving g1 vertices in order, then inserted vertices in insertion order
    std::vector<int> id((size_t)(n1 + n2), -1);
    int nn = 0;
    for (int v = 0; v < n1; ++v)
        if (alive[v]) id[v] = nn++;
    for (int x : ins_order) id[n1 + x] = nn++;
    int mm = 0;
    for (const auto &e : edges) mm += e.live ? 1 : 0;
    if ((nn > 0 && !out_vlabel) || (mm > 0 && !out_edges))
        return bad("null output array");
    for (int v = 0; v < n1 + n2; ++v)
        if (id[v] >= 0) out_vlabel[id[v]] = lab[v];
    int k2 = 0;
    for (const auto &e : edges) {
        if (!e.live) continue;
        out_edges[2 * k2] = id[e.u];
        out_edges[2 * k2 + 1] = id[e.v];
        if (out_elabel) out_elabel[k2] = e.lab;
        ++k2;
    }
    *out_n = nn;
    *out_m = mm;
    return FASTGED_OK;
}

extern "C" int fastged_cross(fastged_handle *h, const fastged_graph *graphs, int32_t n_graphs,
                             const int32_t *rows, int32_t n_rows, const int32_t *cols,
                             int32_t n_cols, int32_t K, const fastged_options *opt,
                             int32_t *out)
{
    clear_error();
    if (!h || n_rows < 0 || n_cols < 0) return set_error(FASTGED_ERR_INVALID_ARG, "null handle or negative count");
    if ((int64_t)n_rows * n_cols > (int64_t)INT32_MAX)
        return set_error(FASTGED_ERR_INVALID_ARG, "matrix too large");
    if (opt && opt->k_per_pair) return set_error(FASTGED_ERR_INVALID_ARG, "k_per_pair is not used here");
    if ((int64_t)n_rows * n_cols == 0) return FASTGED_OK;
    if (!rows || !cols || !out) return set_error(FASTGED_ERR_INVALID_ARG, "null rows, cols or out");
    std::vector<int32_t> pairs(2 * (size_t)n_rows * (size_t)n_cols);
    size_t q = 0;
    for (int r = 0; r < n_rows; ++r)
        for (int c = 0; c < n_cols; ++c) {
            pairs[q++] = rows[r];
            pairs[q++] = cols[c];
        }
    fastged_pair_list pl;
    pl.n_graphs = n_graphs;
    pl.graphs = graphs;
    pl.n_pairs = n_rows * n_cols;
    pl.pairs = pairs.data();
    return fastged_batch_ex(h, &pl, K, opt, out, nullptr, nullptr);
}
