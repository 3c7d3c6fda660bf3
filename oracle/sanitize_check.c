/* Test infrastructure: drives every entry point of oracle.c on seeded random
 * graphs so that the oracle can be built with AddressSanitizer and
 * UndefinedBehaviorSanitizer (tests/test_oracle_sanitized.py compiles the two
 * files together with -fsanitize=address,undefined and runs this program).
 * Besides running clean, the entry points must agree with each other: the
 * Tomita search, the ordered search under all four pivot rules, the outer
 * loop of Alg. 3 and the root-children parts added up give the same maximal
 * cliques (count, hash, histogram), and the listed cliques hash to the same
 * value.  Exit status 0 when everything agreed. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

uint64_t oracle_clique_hash(const uint32_t *labels, uint32_t k);
int oracle_tomita(uint32_t n, const uint32_t *off, const uint32_t *adj, uint64_t *stats, uint64_t *hist,
                  uint32_t *list, uint64_t list_cap, uint64_t *list_used, uint64_t max_nodes);
int oracle_ordered(uint32_t n, const uint32_t *off, const uint32_t *adj, int mode, const uint32_t *order,
                   uint32_t *order_out, uint64_t *stats, uint64_t *hist, uint32_t *list, uint64_t list_cap,
                   uint64_t *list_used, int32_t *trace, uint64_t trace_cap, uint64_t *trace_used);
int oracle_root_children(uint32_t n, const uint32_t *off, const uint32_t *adj, int mode, const uint32_t *order,
                         uint32_t *sizes, uint32_t cap, uint32_t *count);
int oracle_ordered_part(uint32_t n, const uint32_t *off, const uint32_t *adj, int mode, const uint32_t *order,
                        const unsigned char *sel, uint32_t nsel, int count_root, uint64_t *stats, uint64_t *hist);
int oracle_outer(uint32_t n, const uint32_t *off, const uint32_t *adj, int mode, uint32_t *deg_order,
                 uint64_t *stats, uint64_t *hist, uint32_t *list, uint64_t list_cap, uint64_t *list_used);

static uint64_t lcg(uint64_t *s)
{
    *s = *s * 6364136223846793005ull + 1442695040888963407ull;
    return *s >> 11;
}

/* G(n, p) as sorted adjacency lists (CSR) */
static void gnp_csr(uint32_t n, double p, uint64_t seed, uint32_t **off_out, uint32_t **adj_out)
{
    unsigned char *a = (unsigned char *)calloc((size_t)n * n + 1, 1);
    uint64_t s = seed;
    for (uint32_t u = 0; u < n; ++u)
        for (uint32_t v = u + 1; v < n; ++v)
            if ((double)lcg(&s) / 9007199254740992.0 < p) a[(size_t)u * n + v] = a[(size_t)v * n + u] = 1;
    uint32_t *off = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    off[0] = 0;
    for (uint32_t u = 0; u < n; ++u) {
        uint32_t d = 0;
        for (uint32_t v = 0; v < n; ++v) d += a[(size_t)u * n + v];
        off[u + 1] = off[u] + d;
    }
    uint32_t *adj = (uint32_t *)malloc(((size_t)off[n] + 1) * sizeof(uint32_t));
    for (uint32_t u = 0, k = 0; u < n; ++u)
        for (uint32_t v = 0; v < n; ++v)
            if (a[(size_t)u * n + v]) adj[k++] = v;
    free(a);
    *off_out = off;
    *adj_out = adj;
}

static int check(uint32_t n, double p, uint64_t seed)
{
    uint32_t *off, *adj;
    gnp_csr(n, p, seed, &off, &adj);
    uint64_t ref[5], st[5], h0[64] = {0}, h1[64] = {0};
    int bad = 0;
    const uint64_t cap = 1u << 20;
    uint32_t *list = (uint32_t *)malloc(cap * sizeof(uint32_t));
    uint64_t used = 0;
    if (oracle_tomita(n, off, adj, ref, h0, list, cap, &used, 0) != 0) bad = 1;
    /* the listed cliques (size-prefixed records) hash to the reported hash */
    uint64_t hsum = 0, pos = 0, cnt = 0;
    while (!bad && pos < used) {
        const uint32_t k = list[pos];
        hsum += oracle_clique_hash(list + pos + 1, k);
        pos += 1 + k;
        ++cnt;
    }
    if (cnt != ref[0] || hsum != ref[4]) bad |= 2;
    for (int mode = 0; mode < 4 && !bad; ++mode) {
        memset(h1, 0, sizeof(h1));
        if (oracle_ordered(n, off, adj, mode, NULL, NULL, st, h1, NULL, 0, NULL, NULL, 0, NULL) != 0) bad |= 4;
        if (st[0] != ref[0] || st[4] != ref[4] || memcmp(h0, h1, sizeof(h0))) bad |= 8;
        /* root-children parts: even and odd children add up to the whole */
        uint32_t sizes[512], k = 0;
        if (oracle_root_children(n, off, adj, mode, NULL, sizes, 512, &k) != 0 || k > 512) bad |= 16;
        unsigned char sel[512];
        uint64_t tot[5] = {0}, ht[64] = {0};
        for (int part = 0; part < 2 && !bad; ++part) {
            for (uint32_t t = 0; t < k; ++t) sel[t] = (unsigned char)((t & 1u) == (uint32_t)part);
            uint64_t sp[5], hp[64] = {0};
            if (oracle_ordered_part(n, off, adj, mode, NULL, sel, k, part == 0, sp, hp) != 0) bad |= 32;
            for (int j = 0; j < 5; ++j) tot[j] += sp[j];
            for (int j = 0; j < 64; ++j) ht[j] += hp[j];
        }
        if (tot[0] != st[0] || tot[1] != st[1] || tot[4] != st[4] || memcmp(ht, h1, sizeof(ht))) bad |= 64;
        memset(h1, 0, sizeof(h1));
        if (oracle_outer(n, off, adj, mode, NULL, st, h1, NULL, 0, NULL) != 0) bad |= 128;
        /* Alg. 3 has one subproblem per vertex, so on a graph without vertices
         * it reports nothing, where Alg. 2 and 4 report the empty set as the
         * one maximal clique (the library runs Alg. 4 there) */
        if (n == 0) {
            if (st[0] != 0) bad |= 256;
        } else if (st[0] != ref[0] || st[4] != ref[4] || memcmp(h0, h1, sizeof(h0))) {
            bad |= 256;
        }
    }
    printf("n %u p %.2f seed %llu cliques %llu %s (%d)\n", n, p, (unsigned long long)seed,
           (unsigned long long)ref[0], bad ? "DIFFER" : "agree", bad);
    free(list);
    free(off);
    free(adj);
    return bad;
}

int main(void)
{
    int bad = 0;
    const uint32_t ns[] = {0, 1, 2, 5, 17, 40, 63};
    const double ps[] = {0.0, 0.3, 0.6, 1.0};
    uint64_t seed = 1;
    for (size_t i = 0; i < sizeof(ns) / sizeof(ns[0]); ++i)
        for (size_t j = 0; j < sizeof(ps) / sizeof(ps[0]); ++j) bad |= check(ns[i], ps[j], seed++);
    return bad ? 1 : 0;
}
