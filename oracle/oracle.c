/*
 * oracle.c -- plain, slow CPU reference for maximal clique enumeration.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or helper with the CUDA library; the two meet only in the seeded
 * input generators.
 *
 * Graphs arrive in CSR form: vertex v's neighbours are
 * adj[off[v] .. off[v+1]), sorted ascending, symmetric, no self-loops,
 * vertices 0..n-1 (the paper's Section 2 numbers them 1..n).
 *
 * Two enumerators live here.
 *
 *  1. oracle_tomita: the Bron-Kerbosch recursion with pivoting (Alg. 2,
 *     Section 3.2) over sorted vertex arrays, with the Tomita pivot
 *     u = argmax_{u in P u X} |P n N(u)| (Section 3.2), ties to the smallest
 *     label.  It defines the *result*: the set of maximal cliques, which does
 *     not depend on ordering or pivot rule.
 *
 *  2. oracle_ordered: the paper's own search tree, so that search-node
 *     counts can be compared exactly.  It computes the maximum-degree-first
 *     ordering (Section 4.2), renumbers the graph by position (Section 4.2,
 *     "How we use the vertex ordering") and runs BKPivotOrdered with
 *     ChoosePivotOrdered (Alg. 4).  Pivot modes (Section 4.3):
 *       0 GreedyBB    p = first vertex of X in the order, else first of P;
 *       1 GreedyBBTX  p = argmax_{u in X} |P n N(u)|, else first of P;
 *       2 TomitaBB    p = argmax_{u in P u X} |P n N(u)|;
 *       3 GreedyBBNX  p = argmin_{u in X} |P n K(u)|, K(u) = V \ N(u) (u
 *                     included), else first of P; a candidate's count stops
 *                     as soon as it cannot beat the best so far (Naude's
 *                     early exit, as described in Section 4.3);
 *     argmax ties go to the vertex earliest in the order (Section 4.3).
 *     Its sets are sorted arrays of positions, so "first in the order" is
 *     element 0 -- no bitsets.
 *
 * Outputs shared by both (all counters modulo 2^64):
 *   count      number of maximal cliques
 *   hist[k]    number of maximal cliques with k vertices, k = 0..n
 *   hash       sum over cliques K of h(K), where
 *                S(K) = sum_{c in K} mix64(c + 1),  h(K) = mix64(S(K) ^ mix64(|K|))
 *              with c the original 0-based label and mix64 the SplitMix64
 *              finaliser (Steele, Lea, Flood, OOPSLA 2014).  h depends only on
 *              the set K, so the total equals a hash of the sorted cliques.
 *   nodes      invocations of the recursive procedure, root and leaves included
 *   internal   invocations with P non-empty
 *   dead_ends  invocations with P empty and X non-empty
 *   listing    optional: each clique as [k, c_1, ..., c_k] (original labels,
 *              ascending) appended to a flat array.
 *
 * n = 0 follows the BK definition: P = X = {} at the root, so R = {} is
 * reported once (hist[0] = 1).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* SplitMix64 output function. */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t oracle_mix64(uint64_t z) { return mix64(z); }

/* h(K) from the 0-based labels of K, in any order. */
uint64_t oracle_clique_hash(const uint32_t *labels, uint32_t k)
{
    uint64_t s = 0;
    for (uint32_t i = 0; i < k; ++i)
        s += mix64((uint64_t)labels[i] + 1);
    return mix64(s ^ mix64((uint64_t)k));
}

/* ------------------------------------------------------------------------ */
/* Sorted-array set operations.                                              */

/* out = a n b; returns |out|.  out may not alias a or b. */
static uint32_t set_and(const uint32_t *a, uint32_t na, const uint32_t *b, uint32_t nb, uint32_t *out)
{
    uint32_t i = 0, j = 0, k = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { out[k++] = a[i]; ++i; ++j; }
    }
    return k;
}

/* |a n b| */
static uint32_t set_and_count(const uint32_t *a, uint32_t na, const uint32_t *b, uint32_t nb)
{
    uint32_t i = 0, j = 0, k = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { ++k; ++i; ++j; }
    }
    return k;
}

/* out = a \ b; returns |out|. */
static uint32_t set_minus(const uint32_t *a, uint32_t na, const uint32_t *b, uint32_t nb, uint32_t *out)
{
    uint32_t i = 0, j = 0, k = 0;
    while (i < na) {
        if (j < nb && b[j] < a[i]) { ++j; continue; }
        if (j < nb && b[j] == a[i]) { ++i; ++j; continue; }
        out[k++] = a[i++];
    }
    return k;
}

/* Remove x from sorted a (present); returns new size. */
static uint32_t set_erase(uint32_t *a, uint32_t na, uint32_t x)
{
    uint32_t i = 0;
    while (i < na && a[i] != x) ++i;
    if (i < na) {
        memmove(a + i, a + i + 1, (size_t)(na - i - 1) * sizeof(uint32_t));
        return na - 1;
    }
    return na;
}

/* Insert x into sorted a (absent); returns new size. */
static uint32_t set_insert(uint32_t *a, uint32_t na, uint32_t x)
{
    uint32_t i = 0;
    while (i < na && a[i] < x) ++i;
    memmove(a + i + 1, a + i, (size_t)(na - i) * sizeof(uint32_t));
    a[i] = x;
    return na + 1;
}

/* ------------------------------------------------------------------------ */
/* Shared bookkeeping for one enumeration.                                   */

typedef struct {
    uint32_t n;
    const uint32_t *off, *adj;      /* neighbourhoods used by the recursion  */
    const uint32_t *label;          /* recursion vertex -> original label    */
    uint64_t count, nodes, internal, dead_ends, hash;
    uint64_t *hist;                 /* n + 1 entries                         */
    uint32_t *list;                 /* optional listing, may be NULL         */
    uint64_t list_cap, list_used;
    uint32_t *R;                    /* current clique (recursion vertices)   */
    uint32_t *tmp;                  /* n scratch words                       */
    uint32_t **lvl;                 /* per-depth buffers: P', X', L (3n)     */
    uint32_t depth_alloc;
    int mode;                       /* pivot rule of oracle_ordered          */
    int32_t *trace;                 /* optional: first internal nodes        */
    uint64_t trace_cap, trace_used;
    uint64_t max_nodes;             /* 0 = unlimited; else stop after this   */
    const unsigned char *root_sel;  /* optional: root children to expand    */
    uint32_t root_sel_n;            /* entries of root_sel                   */
    int count_root;                 /* with root_sel: count the root node    */
    int oom, stopped;
} run_t;

static uint32_t *level_buf(run_t *r, uint32_t d)
{
    if (d >= r->depth_alloc) {
        uint32_t na = r->depth_alloc ? r->depth_alloc * 2 : 16;
        while (na <= d) na *= 2;
        uint32_t **nl = (uint32_t **)realloc(r->lvl, (size_t)na * sizeof(uint32_t *));
        if (!nl) { r->oom = 1; return NULL; }
        for (uint32_t i = r->depth_alloc; i < na; ++i) nl[i] = NULL;
        r->lvl = nl;
        r->depth_alloc = na;
    }
    if (!r->lvl[d]) {
        r->lvl[d] = (uint32_t *)malloc((size_t)3 * (r->n + 1) * sizeof(uint32_t));
        if (!r->lvl[d]) { r->oom = 1; return NULL; }
    }
    return r->lvl[d];
}

static void report(run_t *r, uint32_t rn)
{
    r->count++;
    r->hist[rn]++;
    uint64_t s = 0;
    for (uint32_t i = 0; i < rn; ++i) {
        r->tmp[i] = r->label[r->R[i]];
        s += mix64((uint64_t)r->tmp[i] + 1);
    }
    r->hash += mix64(s ^ mix64((uint64_t)rn));
    if (r->list) {
        /* insertion sort: cliques are small */
        for (uint32_t i = 1; i < rn; ++i) {
            uint32_t x = r->tmp[i], j = i;
            while (j > 0 && r->tmp[j - 1] > x) { r->tmp[j] = r->tmp[j - 1]; --j; }
            r->tmp[j] = x;
        }
        if (r->list_used + rn + 1 <= r->list_cap) {
            r->list[r->list_used] = rn;
            memcpy(r->list + r->list_used + 1, r->tmp, (size_t)rn * sizeof(uint32_t));
        }
        r->list_used += rn + 1;
    }
}

static void record_trace(run_t *r, uint32_t rn, uint32_t p, const uint32_t *L, uint32_t nl)
{
    /* record: [depth, pivot label, |L|, L labels...] */
    if (!r->trace) return;
    if (r->trace_used + 3 + nl > r->trace_cap) return;
    int32_t *t = r->trace + r->trace_used;
    t[0] = (int32_t)rn;
    t[1] = (int32_t)r->label[p];
    t[2] = (int32_t)nl;
    for (uint32_t i = 0; i < nl; ++i) t[3 + i] = (int32_t)r->label[L[i]];
    r->trace_used += 3 + nl;
}

static const uint32_t *nbr(const run_t *r, uint32_t v, uint32_t *deg)
{
    *deg = r->off[v + 1] - r->off[v];
    return r->adj + r->off[v];
}

/* ------------------------------------------------------------------------ */
/* 1. BKPivot with the Tomita pivot (Alg. 2).                                */

static void bk_tomita(run_t *r, uint32_t *P, uint32_t np, uint32_t *X, uint32_t nx, uint32_t rn)
{
    if (r->oom || r->stopped) return;
    if (r->max_nodes && r->nodes >= r->max_nodes) { r->stopped = 1; return; }
    r->nodes++;
    if (np == 0 && nx == 0) { report(r, rn); return; }
    if (np == 0) { r->dead_ends++; return; }
    r->internal++;

    /* pivot: scan P u X in ascending label order; strict '>' keeps the
     * smallest label among ties */
    uint32_t best_u = 0, best_c = 0;
    int have = 0;
    uint32_t i = 0, j = 0;
    while (i < np || j < nx) {
        uint32_t u;
        if (j >= nx || (i < np && P[i] < X[j])) u = P[i++];
        else u = X[j++];
        uint32_t du;
        const uint32_t *nu = nbr(r, u, &du);
        uint32_t c = set_and_count(P, np, nu, du);
        if (!have || c > best_c) { best_c = c; best_u = u; have = 1; }
    }

    uint32_t *buf = level_buf(r, rn);
    if (!buf) return;
    uint32_t *L = buf + 2 * (r->n + 1);
    uint32_t dp;
    const uint32_t *np_ = nbr(r, best_u, &dp);
    uint32_t nl = set_minus(P, np, np_, dp, L);

    for (uint32_t t = 0; t < nl; ++t) {
        uint32_t v = L[t];
        uint32_t dv;
        const uint32_t *nv = nbr(r, v, &dv);
        /* child buffers live one level down */
        uint32_t *cb = level_buf(r, rn + 1);
        if (!cb) return;
        /* buf (level rn) holds this node's P' and X' scratch: reuse lvl[rn+1]
         * for the child's own sets so the child can mutate them. */
        uint32_t *cP = cb, *cX = cb + (r->n + 1);
        uint32_t ncp = set_and(P, np, nv, dv, cP);
        uint32_t ncx = set_and(X, nx, nv, dv, cX);
        r->R[rn] = v;
        bk_tomita(r, cP, ncp, cX, ncx, rn + 1);
        np = set_erase(P, np, v);
        nx = set_insert(X, nx, v);
    }
}

/* ------------------------------------------------------------------------ */
/* 2. BKPivotOrdered (Alg. 4) on the renumbered graph.                        */

static void bk_ordered(run_t *r, uint32_t *P, uint32_t np, uint32_t *X, uint32_t nx, uint32_t rn)
{
    if (r->oom) return;
    /* a part of the root's branching (root_sel): the root node itself is
     * counted by one part only */
    const int part_root = rn == 0 && r->root_sel != NULL;
    const int counted = !part_root || r->count_root;
    if (counted) r->nodes++;
    if (np == 0 && nx == 0) { if (counted) report(r, rn); return; }
    if (np == 0) { if (counted) r->dead_ends++; return; }
    if (counted) r->internal++;

    /* ChoosePivotOrdered.  Sets hold positions, so element 0 is the vertex
     * earliest in the order; scanning ascending with strict '>' gives the
     * earliest vertex among argmax ties. */
    uint32_t p;
    if (r->mode == 0) {
        p = nx ? X[0] : P[0];
    } else if (r->mode == 1) {
        if (nx) {
            uint32_t best_c = 0; p = X[0];
            for (uint32_t i = 0; i < nx; ++i) {
                uint32_t du; const uint32_t *nu = nbr(r, X[i], &du);
                uint32_t c = set_and_count(P, np, nu, du);
                if (i == 0 || c > best_c) { best_c = c; p = X[i]; }
            }
        } else {
            p = P[0];
        }
    } else if (r->mode == 3) {
        if (nx) {
            /* count P n K(u) by walking P against the sorted N(u); a
             * candidate is dropped once its count reaches the best one's */
            uint32_t best_k = UINT32_MAX; p = X[0];
            for (uint32_t i = 0; i < nx; ++i) {
                uint32_t du; const uint32_t *nu = nbr(r, X[i], &du);
                uint32_t k = 0, a = 0, b = 0;
                while (a < np && k < best_k) {
                    while (b < du && nu[b] < P[a]) ++b;
                    if (b >= du || nu[b] != P[a]) ++k;  /* P[a] not a neighbour of X[i] */
                    ++a;
                }
                if (a == np && k < best_k) { best_k = k; p = X[i]; }
            }
        } else {
            p = P[0];
        }
    } else {
        uint32_t best_c = 0; int have = 0; p = 0;
        uint32_t i = 0, j = 0;
        while (i < np || j < nx) {
            uint32_t u;
            if (j >= nx || (i < np && P[i] < X[j])) u = P[i++];
            else u = X[j++];
            uint32_t du; const uint32_t *nu = nbr(r, u, &du);
            uint32_t c = set_and_count(P, np, nu, du);
            if (!have || c > best_c) { best_c = c; p = u; have = 1; }
        }
    }

    uint32_t *buf = level_buf(r, rn);
    if (!buf) return;
    uint32_t *L = buf + 2 * (r->n + 1);
    uint32_t dp; const uint32_t *npv = nbr(r, p, &dp);
    /* L = P \ N(p); p itself stays in L when p is in P (p is not in N(p)) */
    uint32_t nl = set_minus(P, np, npv, dp, L);
    record_trace(r, rn, p, L, nl);

    /* branch on L in increasing position: v = argmin_{w in L} phi(w) */
    for (uint32_t t = 0; t < nl; ++t) {
        uint32_t v = L[t];
        uint32_t dv; const uint32_t *nv = nbr(r, v, &dv);
        uint32_t *cb = level_buf(r, rn + 1);
        if (!cb) return;
        uint32_t *cP = cb, *cX = cb + (r->n + 1);
        uint32_t ncp = set_and(P, np, nv, dv, cP);
        uint32_t ncx = set_and(X, nx, nv, dv, cX);
        r->R[rn] = v;
        /* a root child outside the part is skipped, but its move from P to
         * X below still happens: later siblings see exactly the sets of the
         * sequential loop */
        if (!part_root || (t < r->root_sel_n && r->root_sel[t]))
            bk_ordered(r, cP, ncp, cX, ncx, rn + 1);
        np = set_erase(P, np, v);
        nx = set_insert(X, nx, v);
    }
}

/* ------------------------------------------------------------------------ */
/* Maximum-degree-first ordering (Section 4.2): v_1 has maximum degree in G,
 * v_{i+1} has maximum degree in the subgraph induced by the vertices not yet
 * placed.  Ties go to the smallest original label (the paper does not say). */

void oracle_mdf_order(uint32_t n, const uint32_t *off, const uint32_t *adj, uint32_t *order)
{
    uint32_t *deg = (uint32_t *)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    unsigned char *placed = (unsigned char *)calloc(n ? n : 1, 1);
    for (uint32_t v = 0; v < n; ++v) deg[v] = off[v + 1] - off[v];
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t best = 0; int have = 0;
        for (uint32_t v = 0; v < n; ++v) {
            if (placed[v]) continue;
            if (!have || deg[v] > deg[best]) { best = v; have = 1; }
        }
        order[i] = best;
        placed[best] = 1;
        for (uint32_t e = off[best]; e < off[best + 1]; ++e)
            if (!placed[adj[e]]) deg[adj[e]]--;
    }
    free(deg);
    free(placed);
}

/* ------------------------------------------------------------------------ */
/* Entry points.  stats[] receives {count, nodes, internal, dead_ends, hash}.
 * Returns 0, or -2 when memory ran out. */

static int run_init(run_t *r, uint32_t n, uint64_t *hist, uint32_t *list, uint64_t list_cap)
{
    memset(r, 0, sizeof(*r));
    r->n = n;
    r->hist = hist;
    memset(hist, 0, (size_t)(n + 1) * sizeof(uint64_t));
    r->list = list;
    r->list_cap = list ? list_cap : 0;
    r->R = (uint32_t *)malloc((size_t)(n + 1) * sizeof(uint32_t));
    r->tmp = (uint32_t *)malloc((size_t)(n + 1) * sizeof(uint32_t));
    return (r->R && r->tmp) ? 0 : -2;
}

static void run_free(run_t *r)
{
    for (uint32_t i = 0; i < r->depth_alloc; ++i) free(r->lvl[i]);
    free(r->lvl);
    free(r->R);
    free(r->tmp);
}

static void run_stats(const run_t *r, uint64_t *stats, uint64_t *list_used)
{
    stats[0] = r->count;
    stats[1] = r->nodes;
    stats[2] = r->internal;
    stats[3] = r->dead_ends;
    stats[4] = r->hash;
    if (list_used) *list_used = r->list_used;
}

/* max_nodes > 0 stops the enumeration after that many search nodes (a
 * bounded sample for timing; the counters then cover the part explored) and
 * the return value is 1. */
int oracle_tomita(uint32_t n, const uint32_t *off, const uint32_t *adj,
                  uint64_t *stats, uint64_t *hist,
                  uint32_t *list, uint64_t list_cap, uint64_t *list_used, uint64_t max_nodes)
{
    run_t r;
    int rc = run_init(&r, n, hist, list, list_cap);
    r.max_nodes = max_nodes;
    uint32_t *ident = (uint32_t *)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    uint32_t *P = (uint32_t *)malloc((size_t)(n + 1) * sizeof(uint32_t));
    uint32_t *X = (uint32_t *)malloc((size_t)(n + 1) * sizeof(uint32_t));
    if (rc || !ident || !P || !X) { rc = -2; goto done; }
    for (uint32_t v = 0; v < n; ++v) { ident[v] = v; P[v] = v; }
    r.off = off; r.adj = adj; r.label = ident;
    bk_tomita(&r, P, n, X, 0, 0);
    rc = r.oom ? -2 : (r.stopped ? 1 : 0);
    run_stats(&r, stats, list_used);
done:
    free(ident); free(P); free(X);
    run_free(&r);
    return rc;
}

/* The graph renumbered by position (Section 4.2, "How we use the vertex
 * ordering"): position i is vertex ord[i]; its neighbours become positions,
 * sorted, so the order is kept inside every set. */
typedef struct {
    uint32_t *ord, *pos, *roff, *radj;
} renum_t;

static void renum_free(renum_t *g)
{
    free(g->ord); free(g->pos); free(g->roff); free(g->radj);
}

/* order: NULL -> maximum-degree-first; else order[i] = vertex at position i. */
static int renum_init(renum_t *g, uint32_t n, const uint32_t *off, const uint32_t *adj, const uint32_t *order)
{
    size_t nn = (size_t)(n ? n : 1);
    uint32_t m2 = n ? off[n] : 0;
    g->ord = (uint32_t *)malloc(nn * sizeof(uint32_t));
    g->pos = (uint32_t *)malloc(nn * sizeof(uint32_t));
    g->roff = (uint32_t *)malloc((nn + 1) * sizeof(uint32_t));
    g->radj = (uint32_t *)malloc((size_t)(m2 ? m2 : 1) * sizeof(uint32_t));
    if (!g->ord || !g->pos || !g->roff || !g->radj) return -2;
    if (order) memcpy(g->ord, order, (size_t)n * sizeof(uint32_t));
    else oracle_mdf_order(n, off, adj, g->ord);
    for (uint32_t i = 0; i < n; ++i) g->pos[g->ord[i]] = i;
    g->roff[0] = 0;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t v = g->ord[i], k = g->roff[i];
        for (uint32_t e = off[v]; e < off[v + 1]; ++e) g->radj[k++] = g->pos[adj[e]];
        g->roff[i + 1] = k;
        /* insertion sort of the new row (plain and obviously correct) */
        for (uint32_t a = g->roff[i] + 1; a < k; ++a) {
            uint32_t x = g->radj[a], b = a;
            while (b > g->roff[i] && g->radj[b - 1] > x) { g->radj[b] = g->radj[b - 1]; --b; }
            g->radj[b] = x;
        }
    }
    return 0;
}

/* order: NULL -> maximum-degree-first; else order[i] = vertex at position i.
 * order_out (optional) receives the order used. */
int oracle_ordered(uint32_t n, const uint32_t *off, const uint32_t *adj,
                   int mode, const uint32_t *order, uint32_t *order_out,
                   uint64_t *stats, uint64_t *hist,
                   uint32_t *list, uint64_t list_cap, uint64_t *list_used,
                   int32_t *trace, uint64_t trace_cap, uint64_t *trace_used)
{
    run_t r;
    renum_t g = {0};
    int rc = run_init(&r, n, hist, list, list_cap);
    uint32_t *P = (uint32_t *)malloc((size_t)(n + 1) * sizeof(uint32_t));
    uint32_t *X = (uint32_t *)malloc((size_t)(n + 1) * sizeof(uint32_t));
    if (rc || !P || !X || renum_init(&g, n, off, adj, order)) { rc = -2; goto done; }
    if (order_out) memcpy(order_out, g.ord, (size_t)n * sizeof(uint32_t));

    r.off = g.roff; r.adj = g.radj; r.label = g.ord; r.mode = mode;
    r.trace = trace; r.trace_cap = trace ? trace_cap : 0;
    for (uint32_t i = 0; i < n; ++i) P[i] = i;
    bk_ordered(&r, P, n, X, 0, 0);
    rc = r.oom ? -2 : 0;
    run_stats(&r, stats, list_used);
    if (trace_used) *trace_used = r.trace_used;
done:
    renum_free(&g); free(P); free(X);
    run_free(&r);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* The root's children as independent subtrees.  Alg. 3 (Section 3.3) splits
 * the enumeration into independent subproblems, one per vertex, because the
 * sequential loop of Alg. 2 hands each branch the sets P n N(v), X n N(v)
 * fixed by the branches before it.  The same holds for the root of Alg. 4:
 * child t (the t-th vertex v_t of the root's branching set L, in order) is
 * the search from R = {v_t}, P = (V minus v_1..v_{t-1}) n N(v_t),
 * X = {v_1..v_{t-1}} n N(v_t), whatever happens inside the other children.
 * So a set of children can be searched on its own and the counters of a
 * partition of the children add up (modulo 2^64) to the whole search, the
 * root node being counted by one part. */

/* The root's branching set: its size to *count and, for t < cap,
 * sizes[t] = |P_t| = |(V minus v_1..v_{t-1}) n N(v_t)|, the candidate set of
 * child t (an estimate of its subtree's size). */
int oracle_root_children(uint32_t n, const uint32_t *off, const uint32_t *adj, int mode, const uint32_t *order,
                         uint32_t *sizes, uint32_t cap, uint32_t *count)
{
    renum_t g = {0};
    uint32_t *P = (uint32_t *)malloc((size_t)(n + 1) * sizeof(uint32_t));
    uint32_t *L = (uint32_t *)malloc((size_t)(n + 1) * sizeof(uint32_t));
    int rc = 0;
    *count = 0;
    if (!P || !L || renum_init(&g, n, off, adj, order)) { rc = -2; goto done; }
    if (n == 0) goto done;
    for (uint32_t i = 0; i < n; ++i) P[i] = i;
    uint32_t np = n, p = 0;
    if (mode == 2) {
        /* TomitaBB with X empty: argmax over P of |P n N(u)| = the degree,
         * earliest position on ties */
        uint32_t best = 0;
        for (uint32_t u = 0; u < n; ++u) {
            uint32_t d = g.roff[u + 1] - g.roff[u];
            if (u == 0 || d > best) { best = d; p = u; }
        }
    }
    /* every other rule takes the first vertex of P when X is empty */
    uint32_t nl = set_minus(P, np, g.radj + g.roff[p], g.roff[p + 1] - g.roff[p], L);
    for (uint32_t t = 0; t < nl; ++t) {
        uint32_t v = L[t];
        uint32_t c = set_and_count(P, np, g.radj + g.roff[v], g.roff[v + 1] - g.roff[v]);
        if (t < cap) sizes[t] = c;
        np = set_erase(P, np, v);
    }
    *count = nl;
done:
    renum_free(&g); free(P); free(L);
    return rc;
}

/* Alg. 4 restricted to the root children t with sel[t] != 0 (t < nsel);
 * the root node is counted only when count_root. */
int oracle_ordered_part(uint32_t n, const uint32_t *off, const uint32_t *adj, int mode, const uint32_t *order,
                        const unsigned char *sel, uint32_t nsel, int count_root, uint64_t *stats, uint64_t *hist)
{
    run_t r;
    renum_t g = {0};
    int rc = run_init(&r, n, hist, NULL, 0);
    uint32_t *P = (uint32_t *)malloc((size_t)(n + 1) * sizeof(uint32_t));
    uint32_t *X = (uint32_t *)malloc((size_t)(n + 1) * sizeof(uint32_t));
    static const unsigned char none = 0;
    if (rc || !P || !X || renum_init(&g, n, off, adj, order)) { rc = -2; goto done; }
    r.off = g.roff; r.adj = g.radj; r.label = g.ord; r.mode = mode;
    r.root_sel = sel ? sel : &none;
    r.root_sel_n = sel ? nsel : 0;
    r.count_root = count_root;
    for (uint32_t i = 0; i < n; ++i) P[i] = i;
    bk_ordered(&r, P, n, X, 0, 0);
    rc = r.oom ? -2 : 0;
    run_stats(&r, stats, NULL);
done:
    renum_free(&g); free(P); free(X);
    run_free(&r);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* 3. The outer loop of Alg. 3 for large sparse graphs.                      */

/* Degeneracy ordering (Section 3.3): repeatedly remove a vertex of minimum
 * degree in the remaining graph; ties go to the smallest label. */
void oracle_degeneracy_order(uint32_t n, const uint32_t *off, const uint32_t *adj, uint32_t *order)
{
    uint32_t *deg = (uint32_t *)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    unsigned char *gone = (unsigned char *)calloc(n ? n : 1, 1);
    for (uint32_t v = 0; v < n; ++v) deg[v] = off[v + 1] - off[v];
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t best = 0; int have = 0;
        for (uint32_t v = 0; v < n; ++v) {
            if (gone[v]) continue;
            if (!have || deg[v] < deg[best]) { best = v; have = 1; }
        }
        order[i] = best;
        gone[best] = 1;
        for (uint32_t e = off[best]; e < off[best + 1]; ++e)
            if (!gone[adj[e]]) deg[adj[e]]--;
    }
    free(deg);
    free(gone);
}

/* Alg. 3 with the paper's ordered search inside.  For every vertex v, in
 * degeneracy order: the subproblem graph H = G[{v} u N(v)], its vertices
 * taken in increasing label, is ordered maximum-degree-first and renumbered
 * (Section 4.2), and BKPivotOrdered (Alg. 4, pivot rule `mode`) runs from
 * R = {v}, P = the neighbours of v after it in the degeneracy order, X = the
 * neighbours before it.  Every maximal clique is reported once, in the
 * subproblem of its vertex earliest in the degeneracy order.  `deg_order`
 * (optional, n entries) receives the outer order.  Adjacency lists must be
 * sorted.  stats/hist/list as for oracle_ordered. */
int oracle_outer(uint32_t n, const uint32_t *off, const uint32_t *adj, int mode, uint32_t *deg_order,
                 uint64_t *stats, uint64_t *hist, uint32_t *list, uint64_t list_cap, uint64_t *list_used)
{
    run_t r;
    int rc = run_init(&r, n, hist, list, list_cap);
    size_t nn = (size_t)(n ? n : 1);
    uint32_t maxd = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (off[v + 1] - off[v] > maxd) maxd = off[v + 1] - off[v];
    size_t hn = (size_t)maxd + 1;                       /* vertices of a subproblem */
    uint32_t *dord = (uint32_t *)malloc(nn * sizeof(uint32_t));
    uint32_t *dpos = (uint32_t *)malloc(nn * sizeof(uint32_t));
    uint32_t *U = (uint32_t *)malloc(hn * sizeof(uint32_t));
    uint32_t *hoff = (uint32_t *)malloc((hn + 1) * sizeof(uint32_t));
    uint32_t *hadj = (uint32_t *)malloc(hn * hn * sizeof(uint32_t));
    uint32_t *hord = (uint32_t *)malloc(hn * sizeof(uint32_t));
    uint32_t *hpos = (uint32_t *)malloc(hn * sizeof(uint32_t));
    uint32_t *roff = (uint32_t *)malloc((hn + 1) * sizeof(uint32_t));
    uint32_t *radj = (uint32_t *)malloc(hn * hn * sizeof(uint32_t));
    uint32_t *lab = (uint32_t *)malloc(hn * sizeof(uint32_t));
    uint32_t *P = (uint32_t *)malloc((nn + 1) * sizeof(uint32_t));
    uint32_t *X = (uint32_t *)malloc((nn + 1) * sizeof(uint32_t));
    if (rc || !dord || !dpos || !U || !hoff || !hadj || !hord || !hpos || !roff || !radj || !lab || !P || !X) {
        rc = -2;
        goto done;
    }
    oracle_degeneracy_order(n, off, adj, dord);
    if (deg_order) memcpy(deg_order, dord, (size_t)n * sizeof(uint32_t));
    for (uint32_t i = 0; i < n; ++i) dpos[dord[i]] = i;
    r.mode = mode;

    for (uint32_t i = 0; i < n && !r.oom; ++i) {
        const uint32_t v = dord[i];
        /* U = {v} u N(v) in increasing label */
        uint32_t h = 0, e = off[v];
        while (e < off[v + 1] && adj[e] < v) U[h++] = adj[e++];
        U[h++] = v;
        while (e < off[v + 1]) U[h++] = adj[e++];
        /* H's adjacency in local indices: N(a) n U for every a in U */
        hoff[0] = 0;
        for (uint32_t a = 0; a < h; ++a) {
            uint32_t k = hoff[a], x = off[U[a]], y = 0;
            while (x < off[U[a] + 1] && y < h) {
                if (adj[x] < U[y]) ++x;
                else if (adj[x] > U[y]) ++y;
                else { hadj[k++] = y; ++x; ++y; }
            }
            hoff[a + 1] = k;
        }
        /* maximum-degree-first order of H and renumbering by position */
        oracle_mdf_order(h, hoff, hadj, hord);
        for (uint32_t j = 0; j < h; ++j) hpos[hord[j]] = j;
        roff[0] = 0;
        for (uint32_t j = 0; j < h; ++j) {
            uint32_t a = hord[j], k = roff[j];
            for (uint32_t t = hoff[a]; t < hoff[a + 1]; ++t) radj[k++] = hpos[hadj[t]];
            roff[j + 1] = k;
            for (uint32_t s = roff[j] + 1; s < k; ++s) {
                uint32_t x = radj[s], b = s;
                while (b > roff[j] && radj[b - 1] > x) { radj[b] = radj[b - 1]; --b; }
                radj[b] = x;
            }
            lab[j] = U[a];
        }
        /* the root: R = {v}, P = later neighbours, X = earlier ones, as
         * sorted position lists */
        uint32_t np = 0, nx = 0, pv = 0;
        for (uint32_t j = 0; j < h; ++j) {
            const uint32_t u = lab[j];
            if (u == v) pv = j;
            else if (dpos[u] > i) P[np++] = j;
            else X[nx++] = j;
        }
        r.off = roff; r.adj = radj; r.label = lab;
        r.R[0] = pv;
        bk_ordered(&r, P, np, X, nx, 1);
    }
    rc = r.oom ? -2 : 0;
    run_stats(&r, stats, list_used);
done:
    free(dord); free(dpos); free(U); free(hoff); free(hadj); free(hord); free(hpos);
    free(roff); free(radj); free(lab); free(P); free(X);
    run_free(&r);
    return rc;
}

