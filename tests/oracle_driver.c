/* Test driver for the oracle (tests/test_oracle_sanitizers.py): runs every oracle entry point
 * on seeded small graphs and prints the results, so that a build with AddressSanitizer and
 * UndefinedBehaviorSanitizer can be checked against a plain build. Test code only. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n;
    const int *alpha;
    const unsigned char *adj;
} ogo_graph;

long long ogo_full_cost(const ogo_graph *g1, const ogo_graph *g2, const int *c, const int *map);
long long ogo_brute_ged(const ogo_graph *g1, const ogo_graph *g2, const int *c, int *out_map,
                        long long *out_count);
long long ogo_brute_square(const ogo_graph *g1, const ogo_graph *g2, const int *c);
int ogo_kbest(const ogo_graph *g1, const ogo_graph *g2, const int *c, int K, int variant,
              long long *out_cost, int *out_map, long long *out_nevals);
int ogo_kbest_leaves(const ogo_graph *g1, const ogo_graph *g2, const int *c, int K, int variant,
                     int cap, int *out_L, long long *leaf_ped, int *leaf_map);

static unsigned long long rs = 0x9E3779B97F4A7C15ull;

static unsigned rnd(void)   /* xorshift64 */
{
    rs ^= rs << 13;
    rs ^= rs >> 7;
    rs ^= rs << 17;
    return (unsigned)(rs >> 11);
}

/* a random graph with n vertices, labels < 3, edge probability ~0.4, edge labels 0..2 */
static void make_graph(int n, int *alpha, unsigned char *adj)
{
    memset(adj, 0, (size_t)n * (size_t)n + 1);
    for (int v = 0; v < n; ++v) alpha[v] = (int)(rnd() % 3);
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b)
            if (rnd() % 10 < 4) adj[a * n + b] = adj[b * n + a] = (unsigned char)(1 + rnd() % 3);
}

int main(void)
{
    for (int t = 0; t < 80; ++t) {
        const int n1 = (int)(rnd() % 7), n2 = (int)(rnd() % 7);
        int a1[8], a2[8], c[6], map[8];
        unsigned char adj1[64], adj2[64];
        make_graph(n1, a1, adj1);
        make_graph(n2, a2, adj2);
        for (int k = 0; k < 6; ++k) c[k] = 1 + (int)(rnd() % 5);
        const ogo_graph g1 = {n1, a1, adj1}, g2 = {n2, a2, adj2};
        long long cnt = 0;
        const long long ged = ogo_brute_ged(&g1, &g2, c, map, &cnt);
        const long long sq = (n1 + n2 <= 10) ? ogo_brute_square(&g1, &g2, c) : -1;
        printf("case %d n1 %d n2 %d ged %lld maps %lld square %lld full %lld\n", t, n1, n2, ged,
               cnt, sq, ogo_full_cost(&g1, &g2, c, map));
        const int Ks[3] = {1, 3, 50};
        for (int ki = 0; ki < 3; ++ki)
            for (int variant = 0; variant < 2; ++variant) {
                long long cost = 0, nev = 0;
                int m[8];
                const int rc = ogo_kbest(&g1, &g2, c, Ks[ki], variant, &cost, m, &nev);
                printf("  K %d v %d rc %d cost %lld nev %lld full %lld map", Ks[ki], variant, rc,
                       cost, nev, ogo_full_cost(&g1, &g2, c, m));
                for (int v = 0; v < n1; ++v) printf(" %d", m[v]);
                printf("\n");
            }
        int L = 0;
        long long ped[3 * 7];
        int lm[3 * 7 * 7 + 1];
        const int rc = ogo_kbest_leaves(&g1, &g2, c, 3, 0, 3, &L, ped, lm);
        printf("  leaves rc %d L %d", rc, L);
        for (int k = 0; k < L && k < 3; ++k) printf(" %lld", ped[k]);
        printf("\n");
    }
    return 0;
}
