/* A C program that uses the library through include/mce.h alone: no Python,
 * no PyTorch.  It builds seeded G(n, p) edge lists with its own generator
 * (SplitMix64 as a plain counter-based stream), loads them, enumerates each
 * one alone (mce_enumerate), submits all of them to the served form
 * (mce_submit / mce_wait), runs them as one batch (mce_enumerate_batch), and
 * checks that the three forms give the same count, hash and search-tree
 * counters.  It prints one line per graph and a summary line
 *   served <requests> <seconds> <requests/s> <CUDA_DEVICE_MAX_CONNECTIONS>
 * and exits 0 when every graph agreed. */
#define _POSIX_C_SOURCE 199309L  /* clock_gettime */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "mce.h"

static uint64_t next64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* every pair (u < v) independently with probability p; returns m */
static uint64_t gnp(uint32_t n, double p, uint64_t seed, uint32_t **uv)
{
    uint64_t s = seed, m = 0, cap = 1024;
    uint32_t *e = (uint32_t *)malloc(cap * 2 * sizeof(uint32_t));
    for (uint32_t u = 0; u < n; ++u)
        for (uint32_t v = u + 1; v < n; ++v) {
            const double x = (double)(next64(&s) >> 11) * (1.0 / 9007199254740992.0);
            if (x < p) {
                if (m == cap) {
                    cap *= 2;
                    e = (uint32_t *)realloc(e, cap * 2 * sizeof(uint32_t));
                }
                e[2 * m] = u;
                e[2 * m + 1] = v;
                ++m;
            }
        }
    *uv = e;
    return m;
}

static double now_s(void)
{
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (double)t.tv_sec + 1e-9 * (double)t.tv_nsec;
}

static int same(const mce_result *a, const mce_result *b)
{
    return a->count == b->count && a->hash == b->hash && a->nodes == b->nodes &&
           a->internal_nodes == b->internal_nodes && a->dead_ends == b->dead_ends && a->max_size == b->max_size;
}

int main(int argc, char **argv)
{
    const uint32_t graphs = argc > 1 ? (uint32_t)atoi(argv[1]) : 64;
    const char *conn = getenv("CUDA_DEVICE_MAX_CONNECTIONS");
    mce_ctx *ctx = NULL;
    int rc = mce_ctx_create(0, 0, NULL, &ctx);
    if (rc) {
        fprintf(stderr, "mce_ctx_create: %s\n", mce_strerror(rc));
        return 2;
    }
    mce_graph **g = (mce_graph **)calloc(graphs, sizeof(mce_graph *));
    mce_result *alone = (mce_result *)calloc(graphs, sizeof(mce_result));
    mce_result *served = (mce_result *)calloc(graphs, sizeof(mce_result));
    mce_result *batched = (mce_result *)calloc(graphs, sizeof(mce_result));
    mce_ticket *t = (mce_ticket *)calloc(graphs, sizeof(mce_ticket));
    uint32_t *ns = (uint32_t *)calloc(graphs, sizeof(uint32_t));
    int bad = 0;
    for (uint32_t i = 0; i < graphs && !bad; ++i) {
        uint64_t s = 1000 + i;
        const uint32_t n = 40 + (uint32_t)(next64(&s) % 300);
        const double p = 0.15 + 0.3 * (double)(next64(&s) >> 11) * (1.0 / 9007199254740992.0);
        uint32_t *uv = NULL;
        const uint64_t m = gnp(n, p, next64(&s), &uv);
        ns[i] = n;
        rc = mce_load_edges(ctx, n, uv, m, &g[i]);
        free(uv);
        if (rc) {
            fprintf(stderr, "mce_load_edges %u: %s\n", i, mce_strerror(rc));
            bad = 1;
            break;
        }
        rc = mce_enumerate(g[i], NULL, &alone[i]);
        if (rc) {
            fprintf(stderr, "mce_enumerate %u: %s\n", i, mce_strerror(rc));
            bad = 1;
        }
    }
    double t0 = now_s();
    for (uint32_t i = 0; i < graphs && !bad; ++i)
        if ((rc = mce_submit(ctx, g[i], NULL, &t[i])) != MCE_OK) {
            fprintf(stderr, "mce_submit %u: %s\n", i, mce_strerror(rc));
            bad = 1;
        }
    for (uint32_t i = 0; i < graphs && !bad; ++i)
        if ((rc = mce_wait(ctx, t[i], 0, &served[i])) != MCE_OK) {
            fprintf(stderr, "mce_wait %u: %s\n", i, mce_strerror(rc));
            bad = 1;
        }
    const double secs = now_s() - t0;
    if (!bad && (rc = mce_enumerate_batch(ctx, g, graphs, NULL, batched)) != MCE_OK) {
        fprintf(stderr, "mce_enumerate_batch: %s\n", mce_strerror(rc));
        bad = 1;
    }
    for (uint32_t i = 0; i < graphs && !bad; ++i) {
        const int ok = same(&alone[i], &served[i]) && same(&alone[i], &batched[i]);
        printf("graph %u n %u count %llu hash %llu nodes %llu %s\n", i, ns[i], (unsigned long long)alone[i].count,
               (unsigned long long)alone[i].hash, (unsigned long long)alone[i].nodes, ok ? "agree" : "DIFFER");
        if (!ok) bad = 1;
    }
    if (!bad) printf("served %u %.6f %.1f %s\n", graphs, secs, graphs / secs, conn ? conn : "unset");
    for (uint32_t i = 0; i < graphs; ++i)
        if (g[i]) mce_graph_free(g[i]);
    mce_ctx_destroy(ctx);
    free(g);
    free(alone);
    free(served);
    free(batched);
    free(t);
    free(ns);
    return bad;
}
