/*
 * fastged_oracle.c -- plain serial CPU oracle for K-Best graph edit distance
 * (Dabah & Herten, "Efficient Accelerated Graph Edit Distance Computation on GPU").
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU
 * baseline load this file. It is deliberately slow and literal so that it can be checked
 * against the paper by eye, and it shares no code, header, table or helper with the CUDA
 * path.
 *
 * Graph representation (Sec. 2.1: simple, undirected, labelled, no loops): n vertices,
 * vertex labels alpha[n], and a dense byte adjacency matrix adj[n*n] with
 *     adj[a*n + b] == 0            when a and b are not adjacent,
 *     adj[a*n + b] == 1 + beta     when they are joined by an edge with label beta.
 * The matrix is symmetric with a zero diagonal.
 *
 * Cost model (Sec. 2.4 with the six explicit costs of Sec. 5):
 *     c[0] vertex substitution  (charged only when the two vertex labels differ)
 *     c[1] vertex deletion      c[2] vertex insertion
 *     c[3] edge substitution    (charged only when the two edge labels differ)
 *     c[4] edge deletion        c[5] edge insertion
 *
 * Functions
 *   ogo_full_cost    cost of the complete edit path a vertex map induces (Sec. 2.2-2.4)
 *   ogo_brute_ged    exact GED: minimum over every injective partial vertex map (Sec. 2.2)
 *   ogo_brute_square exact GED by a second, independent enumeration: every bijection of the
 *                    (n1+n2)-square extended vertex sets, edges scored pair by pair
 *   ogo_kbest        the K-Best search of Algorithm 1 (branching Sec. 4.1.1, evaluation
 *                    Sec. 4.1.2 and Algorithm 2, selection Sec. 4.2, insertions at the leaf)
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *   - g1 vertices are branched in index order v_0 .. v_{n1-1} ("ForEach v in V1").
 *   - successors of a node are enumerated as the substitutions v -> u_j for every u_j in
 *     R_V2 in increasing j, then the deletion v -> eps (written j = n2).
 *   - "best K" means the K smallest PED; ties are broken by (parent slot, j), which makes
 *     the kept list the first K entries of a sort on the key (PED, parent slot, j).
 *     The kept list is stored in that order, so a node's slot is its rank.
 *   - when fewer than K successors exist, all are kept.
 *   - insertions happen only once all g1 vertices are processed: every g2 vertex left in
 *     R_V2 costs c[2] and every g2 edge with an endpoint in R_V2 costs c[5].
 *   - the result is the kept leaf with the smallest completed cost; ties go to the lowest
 *     slot (variant 0). Variant 1 completes every last-level successor instead of only
 *     the best K, ties going to the lowest rank in the same key order.
 *   - n_evals counts every successor scored at every level plus every leaf completed.
 */
#include <limits.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n;
    const int *alpha;          /* vertex labels, length n                          */
    const unsigned char *adj;  /* n*n; 0 = no edge, 1 + edge label otherwise        */
} ogo_graph;

enum { C_VSUB = 0, C_VDEL = 1, C_VINS = 2, C_ESUB = 3, C_EDEL = 4, C_EINS = 5 };

static int ogo_edge(const ogo_graph *g, int a, int b)
{
    return g->adj[(size_t)a * (size_t)g->n + (size_t)b];
}

/* ------------------------------------------------------------------------------------ */
/* Cost of the complete edit path induced by a vertex map (Sec. 2.2-2.4).               */
/* map[i] is the g2 vertex that v_i is substituted by, or -1 when v_i is deleted. Every  */
/* g2 vertex outside the image is inserted. Edges are implied (Sec. 2.3.1): a g1 edge is  */
/* substituted when both endpoints are substituted and their images are adjacent in g2, */
/* otherwise it is deleted; a g2 edge that no g1 edge was substituted by is inserted.    */
/* Returns -1 if map is not an injective partial map into g2.                            */
/* ------------------------------------------------------------------------------------ */
long long ogo_full_cost(const ogo_graph *g1, const ogo_graph *g2, const int *c,
                        const int *map)
{
    int n1 = g1->n, n2 = g2->n;
    int *pre = (int *)malloc(sizeof(int) * (size_t)(n2 > 0 ? n2 : 1));
    long long cost = 0;
    int a, b, u;
    for (u = 0; u < n2; ++u) pre[u] = -1;
    for (a = 0; a < n1; ++a) {
        if (map[a] < -1 || map[a] >= n2) { free(pre); return -1; }
        if (map[a] >= 0) {
            if (pre[map[a]] >= 0) { free(pre); return -1; }
            pre[map[a]] = a;
        }
    }
    /* vertex operations (Sec. 2.3) */
    for (a = 0; a < n1; ++a) {
        if (map[a] < 0) cost += c[C_VDEL];
        else if (g1->alpha[a] != g2->alpha[map[a]]) cost += c[C_VSUB];
    }
    for (u = 0; u < n2; ++u)
        if (pre[u] < 0) cost += c[C_VINS];
    /* edges of g1 */
    for (a = 0; a < n1; ++a)
        for (b = a + 1; b < n1; ++b) {
            int e1 = ogo_edge(g1, a, b);
            if (!e1) continue;
            if (map[a] >= 0 && map[b] >= 0 && ogo_edge(g2, map[a], map[b])) {
                if (ogo_edge(g2, map[a], map[b]) != e1) cost += c[C_ESUB];
            } else {
                cost += c[C_EDEL];
            }
        }
    /* edges of g2 */
    for (a = 0; a < n2; ++a)
        for (b = a + 1; b < n2; ++b) {
            if (!ogo_edge(g2, a, b)) continue;
            if (!(pre[a] >= 0 && pre[b] >= 0 && ogo_edge(g1, pre[a], pre[b])))
                cost += c[C_EINS];
        }
    free(pre);
    return cost;
}

/* ------------------------------------------------------------------------------------ */
/* Exact GED, first enumeration: every injective partial map V1 -> V2 u {eps}.          */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    const ogo_graph *g1, *g2;
    const int *c;
    int *map, *used, *best_map;
    long long best;
    long long count;
} ogo_brute_state;

static void ogo_brute_rec(ogo_brute_state *st, int i)
{
    int u;
    if (i == st->g1->n) {
        long long v = ogo_full_cost(st->g1, st->g2, st->c, st->map);
        st->count++;
        if (v < st->best) {
            st->best = v;
            memcpy(st->best_map, st->map, sizeof(int) * (size_t)st->g1->n);
        }
        return;
    }
    for (u = 0; u < st->g2->n; ++u) {
        if (st->used[u]) continue;
        st->used[u] = 1;
        st->map[i] = u;
        ogo_brute_rec(st, i + 1);
        st->used[u] = 0;
    }
    st->map[i] = -1;
    ogo_brute_rec(st, i + 1);
}

/* Returns the exact GED (or -1 when n1 or n2 exceeds 10); fills out_map (n1 ints) with
   one optimal map and *out_count with the number of maps enumerated. */
long long ogo_brute_ged(const ogo_graph *g1, const ogo_graph *g2, const int *c,
                        int *out_map, long long *out_count)
{
    ogo_brute_state st;
    int n1 = g1->n, n2 = g2->n;
    if (n1 > 10 || n2 > 10) return -1;
    st.g1 = g1; st.g2 = g2; st.c = c;
    st.map = (int *)calloc((size_t)n1 + 1, sizeof(int));
    st.best_map = (int *)calloc((size_t)n1 + 1, sizeof(int));
    st.used = (int *)calloc((size_t)n2 + 1, sizeof(int));
    st.best = LLONG_MAX;
    st.count = 0;
    ogo_brute_rec(&st, 0);
    if (out_map) memcpy(out_map, st.best_map, sizeof(int) * (size_t)n1);
    if (out_count) *out_count = st.count;
    free(st.map); free(st.best_map); free(st.used);
    return st.best;
}

/* ------------------------------------------------------------------------------------ */
/* Exact GED, second enumeration (independent of ogo_full_cost): both vertex sets are    */
/* padded with eps vertices to N = n1 + n2 (rows: g1 then n2 eps; columns: g2 then n1    */
/* eps) and every bijection pi is scored directly: one vertex term per row and one edge  */
/* term per unordered row pair, eps vertices having no edges.                            */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    const ogo_graph *g1, *g2;
    const int *c;
    int N, n1, n2;
    int *pi, *taken;
    long long best;
} ogo_square_state;

static long long ogo_square_score(const ogo_square_state *st)
{
    long long cost = 0;
    int r, s, n1 = st->n1, n2 = st->n2;
    const int *c = st->c;
    for (r = 0; r < st->N; ++r) {
        int col = st->pi[r];
        int real_r = r < n1, real_c = col < n2;
        if (real_r && real_c) cost += (st->g1->alpha[r] != st->g2->alpha[col]) ? c[C_VSUB] : 0;
        else if (real_r) cost += c[C_VDEL];
        else if (real_c) cost += c[C_VINS];
    }
    for (r = 0; r < st->N; ++r)
        for (s = r + 1; s < st->N; ++s) {
            int e1 = (r < n1 && s < n1) ? ogo_edge(st->g1, r, s) : 0;
            int pr = st->pi[r], ps = st->pi[s];
            int e2 = (pr < n2 && ps < n2) ? ogo_edge(st->g2, pr, ps) : 0;
            if (e1 && e2) cost += (e1 != e2) ? c[C_ESUB] : 0;
            else if (e1) cost += c[C_EDEL];
            else if (e2) cost += c[C_EINS];
        }
    return cost;
}

static void ogo_square_rec(ogo_square_state *st, int r)
{
    int col;
    if (r == st->N) {
        long long v = ogo_square_score(st);
        if (v < st->best) st->best = v;
        return;
    }
    for (col = 0; col < st->N; ++col) {
        if (st->taken[col]) continue;
        st->taken[col] = 1;
        st->pi[r] = col;
        ogo_square_rec(st, r + 1);
        st->taken[col] = 0;
    }
}

/* Returns the exact GED, or -1 when n1 + n2 exceeds 10. */
long long ogo_brute_square(const ogo_graph *g1, const ogo_graph *g2, const int *c)
{
    ogo_square_state st;
    st.g1 = g1; st.g2 = g2; st.c = c;
    st.n1 = g1->n; st.n2 = g2->n; st.N = g1->n + g2->n;
    if (st.N > 10) return -1;
    if (st.N == 0) return 0;
    st.pi = (int *)calloc((size_t)st.N, sizeof(int));
    st.taken = (int *)calloc((size_t)st.N, sizeof(int));
    st.best = LLONG_MAX;
    ogo_square_rec(&st, 0);
    free(st.pi); free(st.taken);
    return st.best;
}

/* ------------------------------------------------------------------------------------ */
/* K-Best search, Algorithm 1.                                                          */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    long long ped;   /* PED(nd_j): cost of all operations in lambda(nd_j)        */
    int parent;      /* slot of the node it was branched from                      */
    int j;           /* 0..n2-1: substitution v -> u_j;  n2: deletion v -> eps     */
} ogo_cand;

static int ogo_cand_cmp(const void *x, const void *y)
{
    const ogo_cand *a = (const ogo_cand *)x, *b = (const ogo_cand *)y;
    if (a->ped != b->ped) return a->ped < b->ped ? -1 : 1;
    if (a->parent != b->parent) return a->parent < b->parent ? -1 : 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    return 0;
}

/* Evaluation of successor nd_j of a node whose lambda maps v_0..v_{i-1} as map[0..i-1]
   (Sec. 4.1.2, Algorithm 2): the cost of the new vertex operation on v_i plus the implied
   edge operations between v_i and every vertex already in lambda (Sec. 2.3.1). */
static long long ogo_step_cost(const ogo_graph *g1, const ogo_graph *g2, const int *c,
                               const int *map, int i, int j)
{
    long long cost = 0;
    int k, n2 = g2->n;
    if (j == n2) {                                   /* v_i -> eps */
        cost += c[C_VDEL];
        for (k = 0; k < i; ++k)
            if (ogo_edge(g1, i, k)) cost += c[C_EDEL];   /* its edges go with it */
        return cost;
    }
    if (g1->alpha[i] != g2->alpha[j]) cost += c[C_VSUB];   /* v_i -> u_j */
    for (k = 0; k < i; ++k) {
        int e1 = ogo_edge(g1, i, k);
        if (map[k] < 0) {                            /* v_k was deleted earlier */
            if (e1) cost += c[C_EDEL];
            continue;
        }
        {
            int e2 = ogo_edge(g2, j, map[k]);
            if (e1 && e2) { if (e1 != e2) cost += c[C_ESUB]; }   /* e1 -> e2 */
            else if (e1) cost += c[C_EDEL];                      /* e1 -> eps */
            else if (e2) cost += c[C_EINS];                      /* eps -> e2 */
        }
    }
    return cost;
}

/* The search itself. On return the final List (before the leaf insertions) is held in
   *p_map / *p_used / *p_ped (L entries, in slot order) and the caller frees them. */
static int ogo_search(const ogo_graph *g1, const ogo_graph *g2, const int *c, int K,
                      int variant, size_t *p_L, int **p_map, unsigned char **p_used,
                      long long **p_ped, long long *p_nevals)
{
    int n1 = g1->n, n2 = g2->n;
    size_t cap, maxcand;
    int *map_cur = NULL, *map_nxt = NULL;
    unsigned char *used_cur = NULL, *used_nxt = NULL;
    long long *ped_cur = NULL, *ped_nxt = NULL;
    ogo_cand *cand = NULL;
    size_t L = 1;
    long long nevals = 0;
    int i;
    size_t mrow = (size_t)(n1 > 0 ? n1 : 1), urow = (size_t)(n2 > 0 ? n2 : 1);

    if (K < 1 || n1 < 0 || n2 < 0) return -1;
    cap = (size_t)K;
    maxcand = cap * (size_t)(n2 + 1);
    if (variant == 1) cap = maxcand > cap ? maxcand : cap;

    map_cur = (int *)calloc(cap * mrow, sizeof(int));
    map_nxt = (int *)calloc(cap * mrow, sizeof(int));
    used_cur = (unsigned char *)calloc(cap * urow, 1);
    used_nxt = (unsigned char *)calloc(cap * urow, 1);
    ped_cur = (long long *)calloc(cap, sizeof(long long));
    ped_nxt = (long long *)calloc(cap, sizeof(long long));
    cand = (ogo_cand *)calloc(maxcand > 0 ? maxcand : 1, sizeof(ogo_cand));
    if (!map_cur || !map_nxt || !used_cur || !used_nxt || !ped_cur || !ped_nxt || !cand) {
        free(map_cur); free(map_nxt); free(used_cur); free(used_nxt);
        free(ped_cur); free(ped_nxt); free(cand);
        return -1;
    }

    /* List <- {initial problem}: lambda empty, R_V1 = V1, R_V2 = V2, PED 0 */
    L = 1;
    ped_cur[0] = 0;

    for (i = 0; i < n1; ++i) {                         /* ForEach v in V1 */
        size_t nc = 0, s, newL, r;
        int j;
        for (s = 0; s < L; ++s) {                      /* ForEach node in List */
            const int *map = map_cur + s * mrow;
            const unsigned char *used = used_cur + s * urow;
            for (j = 0; j <= n2; ++j) {                /* successors nd_j */
                if (j < n2 && used[j]) continue;       /* u_j not in R_V2 */
                cand[nc].ped = ped_cur[s] + ogo_step_cost(g1, g2, c, map, i, j);
                cand[nc].parent = (int)s;
                cand[nc].j = j;
                ++nc;
            }
        }
        nevals += (long long)nc;
        /* List <- best K nodes of list_tmp */
        qsort(cand, nc, sizeof(ogo_cand), ogo_cand_cmp);
        newL = nc;
        if (!(variant == 1 && i == n1 - 1) && newL > (size_t)K) newL = (size_t)K;
        for (r = 0; r < newL; ++r) {
            size_t p = (size_t)cand[r].parent;
            int *m = map_nxt + r * mrow;
            unsigned char *u = used_nxt + r * urow;
            memcpy(m, map_cur + p * mrow, sizeof(int) * mrow);
            memcpy(u, used_cur + p * urow, urow);
            if (cand[r].j < n2) { m[i] = cand[r].j; u[cand[r].j] = 1; }
            else m[i] = -1;
            ped_nxt[r] = cand[r].ped;
        }
        { int *t = map_cur; map_cur = map_nxt; map_nxt = t; }
        { unsigned char *t = used_cur; used_cur = used_nxt; used_nxt = t; }
        { long long *t = ped_cur; ped_cur = ped_nxt; ped_nxt = t; }
        L = newL;
    }
    free(map_nxt); free(used_nxt); free(ped_nxt); free(cand);
    *p_L = L; *p_map = map_cur; *p_used = used_cur; *p_ped = ped_cur;
    *p_nevals = nevals;
    return 0;
}

/* Runs the search. variant 0: keep the best K at every level, complete the kept leaves.
   variant 1: keep the best K at every level but the last, complete every last-level
   successor. On success returns 0 and writes *out_cost, out_map[0..n1-1] (-1 = deleted)
   and *out_nevals; returns -1 on bad arguments or allocation failure. */
int ogo_kbest(const ogo_graph *g1, const ogo_graph *g2, const int *c, int K, int variant,
              long long *out_cost, int *out_map, long long *out_nevals)
{
    int n1 = g1->n, n2 = g2->n;
    size_t L = 0, s, best_s = 0;
    int *map_cur = NULL;
    unsigned char *used_cur = NULL;
    long long *ped_cur = NULL, nevals = 0, best = LLONG_MAX;
    size_t mrow = (size_t)(n1 > 0 ? n1 : 1), urow = (size_t)(n2 > 0 ? n2 : 1);

    if (ogo_search(g1, g2, c, K, variant, &L, &map_cur, &used_cur, &ped_cur, &nevals) != 0)
        return -1;
    /* Insertions at the leaf: every remaining g2 vertex and every g2 edge with an
       endpoint in R_V2 is inserted; the best completed leaf is the result. */
    for (s = 0; s < L; ++s) {
        const unsigned char *used = used_cur + s * urow;
        long long total = ped_cur[s];
        int a, b;
        for (a = 0; a < n2; ++a) if (!used[a]) total += c[C_VINS];
        for (a = 0; a < n2; ++a)
            for (b = a + 1; b < n2; ++b)
                if (ogo_edge(g2, a, b) && (!used[a] || !used[b])) total += c[C_EINS];
        if (total < best) { best = total; best_s = s; }
    }
    nevals += (long long)L;
    if (out_cost) *out_cost = best;
    if (out_map && n1 > 0) memcpy(out_map, map_cur + best_s * mrow, sizeof(int) * (size_t)n1);
    if (out_nevals) *out_nevals = nevals;
    free(map_cur); free(used_cur); free(ped_cur);
    return 0;
}

/* The final List of the search (before the leaf insertions), in slot order: writes
   *out_L and, for the first min(L, cap) slots, leaf_ped[s] and leaf_map[s*n1 .. +n1).
   Returns 0, or -1 on bad arguments. */
int ogo_kbest_leaves(const ogo_graph *g1, const ogo_graph *g2, const int *c, int K,
                     int variant, int cap, int *out_L, long long *leaf_ped, int *leaf_map)
{
    int n1 = g1->n;
    size_t L = 0, s;
    int *map_cur = NULL;
    unsigned char *used_cur = NULL;
    long long *ped_cur = NULL, nevals = 0;
    size_t mrow = (size_t)(n1 > 0 ? n1 : 1);
    if (ogo_search(g1, g2, c, K, variant, &L, &map_cur, &used_cur, &ped_cur, &nevals) != 0)
        return -1;
    *out_L = (int)L;
    for (s = 0; s < L && s < (size_t)cap; ++s) {
        leaf_ped[s] = ped_cur[s];
        if (n1 > 0) memcpy(leaf_map + s * (size_t)n1, map_cur + s * mrow, sizeof(int) * (size_t)n1);
    }
    free(map_cur); free(used_cur); free(ped_cur);
    return 0;
}
