/*
 * mce.h -- C ABI of libmce, a GB300 (sm_103a) implementation of maximal
 * clique enumeration by bit-parallel Bron-Kerbosch search with a static
 * maximum-degree-first vertex order and greedy pivot selection
 * (San Segundo, Artieda and Strash, "Efficiently Enumerating all Maximal
 * Cliques with Bit-Parallelism": Alg. 4, Sections 4.1-4.3).
 *
 * Problem (Section 1, Section 2): given a simple undirected graph
 * G = (V, E), V = {0, ..., n-1} (the paper numbers vertices from 1), report
 * every maximal clique: a set K of pairwise adjacent vertices such that no
 * vertex outside K is adjacent to all of K.  The library reports
 *
 *   count      |{maximal cliques}|
 *   hist[k]    number of maximal cliques with k vertices, k = 0..n
 *   hash       sum over cliques K of h(K) modulo 2^64, where
 *                S(K) = sum_{c in K} mix64(c + 1) (c = original 0-based label),
 *                h(K) = mix64(S(K) xor mix64(|K|)),
 *              mix64 = the SplitMix64 finaliser (Steele, Lea and Flood,
 *              OOPSLA 2014).  h depends only on the vertex set, so the total
 *              is an order-independent hash of the sorted cliques.
 *   nodes      search-tree nodes: invocations of BKPivotOrdered (Alg. 4),
 *              the root and the leaves included;
 *   internal   nodes with P non-empty;  dead_ends: P empty, X non-empty.
 *
 * n = 0 follows the Bron-Kerbosch definition (Alg. 1): the empty set is the
 * one maximal clique (hist[0] = 1).  Isolated vertices are maximal cliques of
 * size 1.
 *
 * Adjacency bitset layout (used by every call that takes "rows"): row v is
 * words_per_row consecutive uint32 words; vertex u is bit (u % 32) of word
 * (u / 32).  words_per_row >= ceil(n / 32).  A valid bitset is symmetric,
 * has a zero diagonal and zero bits at positions >= n.
 *
 * Return codes: every function returns one of the MCE_* codes below.
 * Device-level calls ("_device" suffix or taking d_* pointers) are
 * stream-ordered: they enqueue work on `stream` (a cudaStream_t; NULL =
 * legacy default stream) and return MCE_OK once it is enqueued; errors found
 * while the kernels run are written to d_out[MCE_OUT_STATUS].  Host-level
 * calls copy their inputs during the call (the caller keeps ownership) and
 * return after the result is on the host.
 *
 * Thread safety: handles (mce_ctx, mce_graph) must not be used from two host
 * threads at once.  Distinct contexts are independent.
 */
#ifndef MCE_H
#define MCE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------------- */
/* Return codes                                                              */

#define MCE_OK         0
#define MCE_PENDING    1   /* request not finished yet (mce_poll)            */
#define MCE_EINVAL    -1   /* bad argument: self-loop, id >= n, asymmetric or
                              padded-bit-set bitset, n > MCE_NMAX, NULL ptr  */
#define MCE_ENOMEM    -2   /* device or host allocation failed / too small   */
#define MCE_ECUDA     -3   /* a CUDA call failed                             */
#define MCE_ETRUNC    -4   /* listing or histogram buffer too small; the
                              *_needed fields are filled, counters are valid */
#define MCE_ETIMEOUT  -5   /* a bounded wait (device or host) gave up        */
#define MCE_EOVERFLOW -6   /* the device work queue overflowed               */
#define MCE_ENOTIMPL  -7   /* option combination not implemented             */
#define MCE_ECANCELED -8   /* the request was cancelled before it ran        */
#define MCE_EBUSY     -9   /* the request already runs (or ran): not cancelled */

#define MCE_NMAX 4096u     /* largest number of vertices on the bitset path  */
#define MCE_NMAX_SPARSE 65535u  /* largest graph mce_load_edges accepts:
                              above MCE_NMAX a graph is held as sorted
                              adjacency lists and enumerated by the outer
                              loop of Alg. 3 (see MCE_OUTER), which needs
                              every degree below MCE_NMAX                 */

/* ----------------------------------------------------------------------- */
/* Options                                                                   */

/* Pivot rules (Section 4.3).  GREEDY: first vertex of X in the order, else
 * first of P (GreedyBB, the paper's main variant).  GREEDY_TX: the vertex of
 * X maximising |P n N(u)|, else first of P (GreedyBBTX).  TOMITA: the vertex
 * of P u X maximising |P n N(u)| (TomitaBB).  Ties go to the vertex earliest
 * in the order. */
#define MCE_PIVOT_GREEDY     0u
#define MCE_PIVOT_GREEDY_TX  1u
#define MCE_PIVOT_TOMITA     2u
#define MCE_PIVOT_GREEDY_NX  3u  /* GreedyBBNX (Section 4.3): GreedyBBTX's
                                    pivot computed as argmin over X of
                                    |P n K(u)|, K(u) = V \ N(u), with Naude's
                                    early exit -- the same pivot as
                                    GREEDY_TX, so the same search tree     */

/* flags */
#define MCE_ORDER_IDENTITY   0x1u  /* skip the maximum-degree-first ordering
                                      (Section 4.2): the input order is the
                                      search order                            */
#define MCE_LIST             0x2u  /* also return the cliques: mce_enumerate
                                      only (device-level calls, batches and
                                      served requests: MCE_ENOTIMPL); each
                                      clique's labels ascending, cliques in
                                      no particular order                   */
#define MCE_AUTOTUNE         0x8u  /* batched form: measure the launch choice
                                      of every words-per-row class on the
                                      batch's own graphs (see
                                      mce_batch_create)                      */
#define MCE_OUTER            0x10u /* mce_enumerate: Alg. 3's outer loop (the
                                      only path for n > MCE_NMAX): for every
                                      vertex v in degeneracy order (minimum
                                      remaining degree first, smallest label
                                      on ties), the search of Alg. 4 on
                                      G[{v} u N(v)] -- ordered maximum-degree-
                                      first -- from R = {v}, P = the
                                      neighbours after v, X = those before;
                                      all subproblems run as one batch.
                                      Results equal the plain path's; node
                                      counters are this loop's (the sum of
                                      the subproblem trees).  Not with
                                      MCE_LIST.                             */
#define MCE_LIST_SORTED      0x4u  /* MCE_LIST with the cliques in
                                      lexicographic order (the problem's
                                      output, Section 2: all maximal cliques) */

typedef struct {
    uint32_t pivot_mode;        /* MCE_PIVOT_*                                */
    uint32_t flags;             /* MCE_ORDER_IDENTITY | MCE_LIST | ...        */
    uint32_t lanes_per_subtree; /* lanes of a warp that share one search
                                   subtree: 1,2,4,8,16,32; 0 = autotuned       */
    uint32_t words_per_lane;    /* 32-bit words of each set a lane holds:
                                   1,2,4; 0 = autotuned                       */
    uint32_t blocks;            /* persistent grid size; 0 = one wave         */
    uint32_t threads_per_block; /* 0 = autotuned; a multiple of 32, at most
                                   512 (else MCE_EINVAL)                      */
    uint64_t timeout_ns;        /* device-side wait budget: a search whose
                                   idle warps see no progress for this long
                                   stops with MCE_ETIMEOUT; 0 = 60 s          */
    uint32_t stack_levels;      /* explicit-stack levels per subtree before
                                   frames spill to the device work queue,
                                   1..64; 0 = 64                              */
    uint32_t queue_log2;        /* log2 of the device work-queue slots, <= 24;
                                   0 = auto (at least four times the subtree
                                   groups).  mce_enumerate retries a search
                                   that overflowed with a 16x larger queue.   */
    uint32_t split_min_p;       /* a new subtree whose candidate set P has at
                                   least this many vertices is published to
                                   the device work queue (breadth-first
                                   split of the top of the search tree) while
                                   the queue holds fewer than half its slots;
                                   0 = by edge density (about 64 expected
                                   maximal cliques in such a subtree),
                                   0xffffffff = never                      */
    uint32_t _reserved;
} mce_options;

/* Layout of the device result array d_out (uint64 words, zeroed and filled
 * by the device calls).  hist[k] is at d_out[MCE_OUT_HIST + k]. */
#define MCE_OUT_COUNT      0
#define MCE_OUT_NODES      1
#define MCE_OUT_INTERNAL   2
#define MCE_OUT_DEAD_ENDS  3
#define MCE_OUT_HASH       4
#define MCE_OUT_STATUS     5   /* 0 or a negative MCE_* code (as int64)      */
#define MCE_OUT_MAX_SIZE   6   /* size of the largest maximal clique         */
#define MCE_OUT_DONATIONS  7   /* work frames handed between warps           */
#define MCE_OUT_STEALS     8   /* frames taken from a work queue (any level) */
#define MCE_OUT_GLOBAL     9   /* ... of which from the device-wide queue    */
#define MCE_OUT_BUSY_NS   10   /* subtree-group time spent holding a frame:
                                  utilisation = busy / (groups x duration)   */
#define MCE_OUT_GROUPS    11   /* subtree groups of the launch               */
#define MCE_OUT_GPUSH     12   /* frames published to the device-wide queue  */
#define MCE_OUT_GTRY      13   /* claims of frames from it (one fetch-and-add
                                  each, for up to four frames)              */
#define MCE_OUT_CAS_FAIL  14   /* lost compare-and-swap races on ticket
                                  counters (block-private rings of the
                                  batched form; the device-wide queue
                                  takes tickets by fetch-and-add)           */
#define MCE_OUT_LANE_TASKS 15  /* subtrees handed to single lanes (frames
                                  whose P u X has at most 32 vertices,
                                  searched with 32-bit local sets)          */
#define MCE_OUT_HIST       16
#define MCE_OUT_WORDS(n)   (MCE_OUT_HIST + (uint64_t)(n) + 1)

/* ----------------------------------------------------------------------- */
/* Device-level, stream-ordered calls.  All d_* pointers are device memory
 * owned by the caller; nothing is allocated.  They are the steps of the
 * search path and may be called one by one or through
 * mce_enumerate_device. */

/* Step "input canonicalisation" from an edge list (Section 2: simple
 * undirected graph).  d_uv holds m pairs (u, v) as 2*m uint32, host order
 * irrelevant, duplicates and both orientations allowed.  Writes the
 * symmetric bitset d_rows (n * words_per_row words; it is cleared first).
 * A self-loop or an id >= n sets d_out[MCE_OUT_STATUS] = MCE_EINVAL (d_out
 * must hold MCE_OUT_WORDS(n) words; only the status word is touched). */
int mce_edges_to_rows(uint32_t n, uint64_t m, const uint32_t *d_uv,
                      uint32_t words_per_row, uint32_t *d_rows,
                      uint64_t *d_out, void *stream);

/* Step "input canonicalisation" for a bitset: checks symmetry, zero
 * diagonal and zero padding bits; on failure sets d_out[MCE_OUT_STATUS] =
 * MCE_EINVAL. */
int mce_validate_rows(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows,
                      uint64_t *d_out, void *stream);

/* Maximum-degree-first ordering (Section 4.2): d_order[0] is a vertex of
 * maximum degree in G, d_order[i] a vertex of maximum degree in the graph
 * induced by the vertices not yet placed; ties go to the smallest label.
 * d_order receives n uint32. */
int mce_order(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows,
              uint32_t *d_order, void *stream);

/* Renumbering by position (Section 4.2, "How we use the vertex ordering"):
 * d_rows_out[i] bit j = d_rows[d_order[i]] bit d_order[j], written with
 * out_words_per_row words per row (extra words and bits zero).  The order's
 * first vertex becomes bit 0, so "first in the order" is the lowest set bit
 * (the paper stores the order reversed and scans from the top; Section 4.2). */
int mce_renumber(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows,
                 const uint32_t *d_order, uint32_t out_words_per_row,
                 uint32_t *d_rows_out, void *stream);

/* Scratch bytes mce_search / mce_enumerate_device need for an n-vertex graph
 * under the given options (NULL = defaults). */
int mce_scratch_bytes(uint32_t n, const mce_options *opts, uint64_t *bytes);

/* The search (Alg. 4) on an already renumbered graph: root P = V, X = {},
 * pivot and branching by the chosen rule, per-warp explicit stacks,
 * persistent work-stealing.  d_rows_renum has mce_search_words(n, opts)
 * words per row; d_order maps position -> original label (for the hash).
 * d_out receives MCE_OUT_WORDS(n) words. */
int mce_search(uint32_t n, const uint32_t *d_rows_renum, const uint32_t *d_order,
               const mce_options *opts, void *d_scratch, uint64_t scratch_bytes,
               uint64_t *d_out, void *stream);

/* Words per renumbered row that mce_search expects for these options. */
uint32_t mce_search_words(uint32_t n, const mce_options *opts);

/* The whole path on a device bitset: validate, order (unless
 * MCE_ORDER_IDENTITY), renumber, search, reduce.  d_scratch must hold
 * mce_scratch_bytes(n, opts) bytes. */
int mce_enumerate_device(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows,
                         const mce_options *opts, void *d_scratch, uint64_t scratch_bytes,
                         uint64_t *d_out, void *stream);

/* The whole path like mce_enumerate_device, but with no scratch argument and
 * no allocation of any kind: the scratch is a fixed area of
 * MCE_STATIC_SCRATCH_BYTES of device memory inside the library (one per GPU
 * that loads it, held until the process exits).  The paper has no
 * counterpart; this exists for callers that may not allocate device memory:
 * plug-ins whose host framework owns every allocation, and request paths
 * that must not allocate per call.  The caller still owns d_rows and d_out.
 *  - Every call looks up the area's device address (cudaGetSymbolAddress,
 *    with the calling thread's current device); the first call on a device
 *    loads the library's device code there.  A device reset invalidates
 *    nothing kept by the library: the next call looks the area up again.
 *  - Every call reuses the same area; what must start from a known state is
 *    re-initialised by each call, but calls whose work overlaps on the GPU
 *    race on the area: do not issue overlapping calls (other streams, other
 *    host threads) on one device.
 *  - MCE_ENOMEM when the options need more scratch than the area holds
 *    (mce_scratch_bytes(n, opts) > MCE_STATIC_SCRATCH_BYTES).  The default
 *    work queue grows with the number of resident subtree groups, so the
 *    bound depends on the GPU: on a 152-SM GB300 the default options fit for
 *    every n <= MCE_NMAX (at most about 26 MiB, for n <= 32). */
#define MCE_STATIC_SCRATCH_BYTES (32u << 20)
int mce_enumerate_device_static(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows,
                                const mce_options *opts, uint64_t *d_out, void *stream);

/* ----------------------------------------------------------------------- */
/* Host-level API: handles, host buffers, batching and serving.             */

typedef struct mce_ctx mce_ctx;
typedef struct mce_graph mce_graph;
typedef uint64_t mce_ticket;

typedef struct {
    uint64_t count, nodes, internal_nodes, dead_ends, hash;
    uint32_t max_size;
    uint32_t status;              /* MCE_* code of this graph (batch/serve)  */
    uint64_t *hist;               /* caller-owned, hist[k] for k < hist_cap  */
    uint32_t hist_cap;
    uint32_t _pad;
    uint32_t *list_ids;           /* caller-owned host array of list_cap
                                     labels: the members of every clique    */
    uint64_t list_cap;
    uint64_t *list_off;           /* caller-owned host array of list_off_cap
                                     CSR offsets: clique i is list_ids[
                                     list_off[i] .. list_off[i+1]), count + 1
                                     entries are written                    */
    uint64_t list_off_cap;        /* (pinned buffers take one device copy;
                                     pageable ones of 32 MB and more go
                                     through two 32 MB pinned halves that the
                                     context allocates on first use)        */
    uint64_t list_ids_needed;     /* out: sum of the clique sizes           */
    double kernel_ms, total_ms;
} mce_result;

/* Create a context on `device` with a device-memory budget (0 = 90% of
 * free memory) and a stream (NULL = the library creates its own). */
int mce_ctx_create(int device, uint64_t mem_budget_bytes, void *stream, mce_ctx **out);
void mce_ctx_destroy(mce_ctx *ctx);

/* Load a graph from m host edges (2*m uint32) or from a host bitset; both
 * are copied to the device and canonicalised there (MCE_EINVAL on a
 * self-loop, id >= n, asymmetry or set padding bits). */
int mce_load_edges(mce_ctx *ctx, uint32_t n, const uint32_t *uv, uint64_t m, mce_graph **out);
int mce_load_bitset(mce_ctx *ctx, uint32_t n, const uint32_t *rows, uint32_t words_per_row,
                    mce_graph **out);
/* Release a graph.  Free every graph (and batch) of a context before
 * destroying the context; a graph must not be freed while a request or batch
 * that uses it is still running. */
void mce_graph_free(mce_graph *g);

/* Enumerate one graph (plain form).  `res` is in/out: hist and list buffers
 * are caller-owned; counters are filled.  MCE_ETRUNC if hist_cap <=
 * max_size or the listing does not fit (counters and list_ids_needed still
 * valid: a caller can ask with zero capacities, then allocate list_ids_needed
 * labels and count + 1 offsets and call again).  Listing (MCE_LIST): the
 * search records each maximal clique where Alg. 4 reports it (a node whose P
 * and X are empty); frames that move between warps carry R as a bitset; the
 * records become the CSR listing on the device before the copy to the host.
 * MCE_ENOMEM if the device records of a listing that fits the caller's
 * buffers do not fit in device memory. */
int mce_enumerate(mce_graph *g, const mce_options *opts, mce_result *res);

/* Streaming listing: every maximal clique handed to the caller's sink in
 * chunks, with no buffer sized up front (the listing output of the problem,
 * Section 2).  The call first counts (an ordinary search; the histogram gives
 * the exact number of cliques and member ids), then runs the listing search
 * with device records of exactly that size, builds the listing on the device
 * (each clique's labels ascending; with MCE_LIST_SORTED in opts->flags the
 * cliques in lexicographic order, else in no particular order), and calls
 * sink(ids, off, count, user) for consecutive chunks of up to 2^20 cliques:
 * clique i of the chunk is ids[off[i] .. off[i+1]) (original labels, uint32),
 * off has count + 1 entries and starts at 0.  The arrays live in pinned host
 * memory of the context and are valid only during the call; a non-zero return
 * from the sink stops the stream (the call still returns MCE_OK).  res gets
 * the counters (and hist, if res->hist is set) as from mce_enumerate;
 * res->list_* fields are left as the caller set them.  n = 0 gives one chunk
 * with the empty clique.  Graphs held as adjacency lists: MCE_ENOTIMPL. */
typedef int (*mce_clique_sink)(const uint32_t *ids, const uint64_t *off, uint64_t count, void *user);
int mce_enumerate_stream(mce_graph *g, const mce_options *opts, mce_clique_sink sink, void *user,
                         mce_result *res);

/* The root's children as independent subtrees (the split of one search
 * over several GPUs).  Alg. 3 (Section 3.3) splits the enumeration into
 * independent subproblems because each branch of the sequential loop gets
 * sets fixed by the branches before it; the root of Alg. 4 splits the same
 * way.  Its branching set L = V \ N(p0) (p0 the root's pivot under the
 * chosen rule) is walked in order v_1, v_2, ...; child t (0-based) is the
 * search from R = {v_t}, P = P_t n N(v_t), X = {v_1..v_{t-1}} n N(v_t),
 * P_t = V minus v_1..v_{t-1}, and it reports exactly the maximal cliques
 * that contain v_t and none of v_1..v_{t-1}.
 *
 * mce_root_children: |L| to *count and, for t < cap, sizes[t] = |P_t n
 * N(v_t)| (host array, caller-owned): the size of child t's candidate set,
 * an estimate of its subtree.  MCE_ETRUNC (with *count set) when cap < |L|.
 *
 * mce_enumerate_part: the search restricted to the children listed in
 * children[0..k) (host array, strictly increasing indices < |L|, else
 * MCE_EINVAL); the root node itself is counted only when count_root is
 * non-zero.  Over a partition of 0..|L|-1 with exactly one part counting the
 * root, count, nodes, internal, dead_ends, hash and hist add up (modulo
 * 2^64) to mce_enumerate's.  Options as for mce_enumerate (no listing, no
 * MCE_OUTER: MCE_ENOTIMPL); graphs held as adjacency lists (n > MCE_NMAX)
 * have no single root: MCE_ENOTIMPL. */
int mce_root_children(mce_graph *g, const mce_options *opts, uint32_t *sizes, uint32_t cap, uint32_t *count);
int mce_enumerate_part(mce_graph *g, const mce_options *opts, const uint32_t *children, uint32_t k,
                       int count_root, mce_result *res);

/* Batched form.  mce_batch_create plans a batch of loaded graphs once:
 * graphs are grouped by subtree shape (lanes x words: by default 512 threads
 * per block and at most two words per lane, or forced by opts, or tuned),
 * costed by the expected number of maximal cliques of G(n, m / C(n, 2)), and
 * the whole pipeline (ordering, renumbering, one persistent search launch per
 * shape, each block taking one work item at a time, most expensive first) is
 * captured into a CUDA graph.  A work item is a whole graph, or, for a graph
 * expected to cost more than half a block's fair share of its bucket, one of
 * k parts of it: part j searches the root children j, j + k, j + 2k, ... of
 * Alg. 4's root (disjoint subtrees; the root node is counted once), so that
 * the heaviest graphs spread over several blocks.  Results are the same
 * either way.
 * mce_batch_launch enqueues that graph on the context stream;
 * mce_batch_results waits and fills res[i] for graphs[i] (hist buffers
 * caller-owned as in mce_enumerate); mce_batch_run does both.  The graphs
 * must stay loaded while the batch exists.  Returns the first per-graph
 * error, with every res[i].status filled. */
typedef struct mce_batch mce_batch;
int mce_batch_create(mce_ctx *ctx, mce_graph *const *graphs, uint32_t count,
                     const mce_options *opts, mce_batch **out);

/* Autotuning (MCE_AUTOTUNE in opts->flags, with lanes_per_subtree,
 * words_per_lane, threads_per_block and split_min_p left 0): graphs are
 * classed by words per row (1, 2, 4, ..., 128).  Classes with a choice cached
 * in the context (per class and pivot rule) take it; the others, if they hold
 * at least 16 graphs of the batch, are tuned by coordinate descent in
 * decreasing order of expected work: every candidate for the class -- 1, 2
 * or 4 words per lane with the fewest lanes that hold a row, 128 / 256 / 512
 * threads per block, then the best with the breadth-first split off -- is
 * timed as one captured launch of the whole batch (up to 4096 of its graphs,
 * sampled evenly) with the other classes at their current choice, and the
 * fastest is kept and cached.  Classes with fewer graphs use the built-in
 * defaults.  Tuning runs inside mce_batch_create (seconds for thousands of
 * graphs); mce_batch_launch replays the chosen plan. */
typedef struct {
    uint32_t words_class;        /* rows of at most this many 32-bit words  */
    uint32_t graphs;             /* graphs of the batch in this bucket      */
    uint32_t lanes_per_subtree, words_per_lane, threads_per_block, blocks;
    uint32_t split_min_p;        /* 0 = by density, 0xffffffff = never      */
    uint32_t tuned;              /* 1 when the choice was measured          */
    double tuned_ms_per_graph;   /* best measured time per graph (tuning)   */
    uint32_t work_items;         /* graphs plus the extra parts of split ones */
    uint32_t split_graphs;       /* graphs split into root-child parts        */
} mce_batch_bucket;
/* The launch choice of every bucket of a batch: up to cap entries to out,
 * the number of buckets to *count. */
int mce_batch_buckets(const mce_batch *b, mce_batch_bucket *out, uint32_t cap, uint32_t *count);
int mce_batch_launch(mce_batch *b);
int mce_batch_results(mce_batch *b, mce_result *res);
int mce_batch_run(mce_batch *b, mce_result *res);
void mce_batch_destroy(mce_batch *b);

/* create + run + destroy: `count` graphs in one captured launch; res[i]
 * belongs to graphs[i]. */
int mce_enumerate_batch(mce_ctx *ctx, mce_graph *const *graphs, uint32_t count,
                        const mce_options *opts, mce_result *res);

/* Served form: requests are admitted by device memory and run with the
 * others already on the GPU; mce_poll never blocks.  While four or more
 * requests with default options wait, up to 256 of them (each expecting at
 * most 10^6 maximal cliques) run as one batched launch; otherwise an
 * admitted request runs its whole path on one of 128 streams with a grid of
 * one block per 20,000 expected maximal cliques (at most four per SM);
 * requests overlap on the device only as far as CUDA maps their streams
 * to separate hardware queues (CUDA_DEVICE_MAX_CONNECTIONS, read when a
 * context is created).  Loading the library sets it to 32 unless the process
 * set it already, so a process that loads the library before it creates its
 * CUDA context gets 32 queues; one that created its context first keeps the
 * value it had then. */
int mce_submit(mce_ctx *ctx, mce_graph *g, const mce_options *opts, mce_ticket *out);
int mce_poll(mce_ctx *ctx, mce_ticket t, mce_result *res);
int mce_wait(mce_ctx *ctx, mce_ticket t, uint64_t timeout_ns, mce_result *res);
/* Cancel a request that is still queued: it will not run, and mce_poll /
 * mce_wait deliver it with status MCE_ECANCELED.  MCE_EBUSY when it already
 * runs or has finished (it completes normally), MCE_EINVAL for an unknown
 * ticket. */
int mce_cancel(mce_ctx *ctx, mce_ticket t);

const char *mce_strerror(int code);

/* Host-side fault injection, for failure-detection tests (nothing on the GPU
 * is made to fail).  Arms `site` so that, after `skip` more passes through
 * it, the next `count` passes fail as the real failure would:
 *   MCE_FAULT_ALLOC  a device allocation of the library fails (MCE_ENOMEM;
 *                    whatever the call allocated so far is released);
 *   MCE_FAULT_COPY   a host-to-device copy of an input graph fails
 *                    (MCE_ECUDA from mce_load_edges / mce_load_bitset);
 *   MCE_FAULT_ADMIT  the served form's admission finds no memory for a
 *                    request, which stays queued and is tried again.
 * count 0 disarms the site.  Process-wide; the environment variable
 * MCE_FAULT="site:skip:count" (site = alloc, copy or admit) arms one site
 * when the library is loaded.  Returns MCE_EINVAL for an unknown site. */
#define MCE_FAULT_ALLOC 1
#define MCE_FAULT_COPY  2
#define MCE_FAULT_ADMIT 3
int mce_fault_inject(int site, uint32_t skip, uint32_t count);
/* Device memory (bytes) the context's library allocations hold now:
 * graphs, batches, request scratch (0 once everything is released). */
uint64_t mce_ctx_mem_used(const mce_ctx *ctx);

/* ----------------------------------------------------------------------- */
/* Diagnostics                                                               */

/* Per-block work timeline of the following single-graph searches on this
 * host thread's current device (NULL / 0 turns it off).  d_buf (device,
 * caller-owned, zeroed by the caller) is split evenly between the launch's
 * blocks; each block appends 16-byte records whenever it refreshes its view
 * of the device-wide queue (about every 2 us while it runs):
 *   uint64 globaltimer ns, uint16 busy groups of the block, uint16 lanes of
 *   the block holding a lane-tier subproblem (frames whose P u X has at most
 *   32 vertices), uint16 frames in the device-wide queue (saturating),
 *   uint16 starving blocks (saturating).
 * Records past a block's share are dropped. */
int mce_trace_enable(void *d_buf, uint64_t bytes);

/* Throughput of the resources that bound the search (it does no dense
 * contraction and, with the rows staged, no HBM traffic): LOP3 (the AND,
 * ANDNOT, OR of set words) and POPC lane operations per second, 128-bit
 * shared-memory load bandwidth, and the warp collectives of every node
 * (ballot, shuffle, max reduction), each measured by a microbenchmark
 * kernel with eight independent chains per thread on every SM of `device`,
 * timed with CUDA events (about 0.1 s in all).  Also the SM count and the maximum
 * SM clock from the device attributes.  Allocates a few bytes of device
 * memory; changes no clock or other device setting. */
typedef struct {
    double lop3_lane_ops_per_s;
    double popc_lane_ops_per_s;
    double lds_bytes_per_s;
    double ms_lop3, ms_popc, ms_lds;   /* per timed launch                  */
    uint32_t sm_count;
    uint32_t sm_clock_max_khz;
    /* warp collectives, in warp instructions per second (all 32 lanes):
     * __ballot_sync, __shfl_xor_sync, __reduce_max_sync (redux.sync)     */
    double ballot_warp_ops_per_s;
    double shfl_warp_ops_per_s;
    double redux_warp_ops_per_s;
} mce_peaks;
int mce_measure_peaks(int device, mce_peaks *out);

#ifdef __cplusplus
}
#endif

#endif /* MCE_H */
