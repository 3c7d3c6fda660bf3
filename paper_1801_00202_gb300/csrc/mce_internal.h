// Internal declarations shared by libmce's translation units (host launchers
// and kernels).  Not part of the public ABI (that is include/mce.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mce.h"

namespace mce {

// Words of a work frame before its P and X bitsets:
//   [0] pivot | end << 16   (branching set L = P & ~N(pivot) & [0, end))
//   [1] |R|
//   [2] S(R) low word, [3] S(R) high word   (running clique hash sum)
//   [4] graph slot (batched and served forms), [5..7] unused
// and, when cliques are listed, the bitset R after P and X.
constexpr int kFrameHdr = 8;

// Levels of the per-group explicit stack (local memory).  Deeper paths spill
// their frames to the global work queue, so this bounds nothing but
// register/local footprint.
constexpr int kStackDepth = 64;

// Global control block of one search, each counter on its own 128-byte line.
struct Ctl {
    unsigned head;     unsigned pad0[31];  // global queue consumer ticket
    unsigned tail;     unsigned pad1[31];  // global queue producer ticket
    unsigned pending;  unsigned pad2[31];  // frames in the global ring + active blocks
    unsigned starving; unsigned pad3[31];  // blocks with idle groups and no local frame
    unsigned abort;    unsigned pad4[31];  // set on error: every warp stops
};

// Per-block frame ring in shared memory (the first level of the work
// distribution): header, `slots` sequence numbers and `slots` frames, with
// slots = kLocalSlots, or kLocalSlotsSmall where halving the ring buys a
// warp of a plain search block (the planner decides).
constexpr int kLocalSlots = 32;
constexpr int kLocalSlotsSmall = 16;
struct LocalHdr {
    unsigned head, tail;  // ring tickets
    unsigned idle;        // groups of this block without a frame
    unsigned bwork;       // busy groups + frames in the ring; the block holds
                          // one unit of Ctl::pending while this is non-zero
    unsigned starving;    // this block is counted in Ctl::starving
    unsigned poller;      // a warp of this block is polling the global ring
    unsigned done;        // the search is over (1) or aborted (2)
    unsigned refreshing;  // a warp is refreshing the cached global state
    // cached global state (refreshed every few microseconds)
    unsigned g_head, g_tail, g_starving;
    unsigned spare;       // unused (keeps the stamp 8-byte aligned)
    unsigned long long stamp;
    unsigned trace_n;     // timeline records written by this block
    unsigned t2_busy;     // lanes of the block holding a lane-tier subproblem
    // work-distribution diagnostics of the block (rare events, shared-memory
    // atomics; added to the result array once the block is done)
    unsigned long long diag[8];
};
// Indices of LocalHdr::diag and the result words they are added to.
enum DiagIdx { kDiagDonations = 0, kDiagSteals, kDiagGlobal, kDiagBusyNs, kDiagGpush, kDiagGtry, kDiagCasFail,
               kDiagLaneTasks, kDiagCount };
__host__ __device__ inline size_t frame_words(uint32_t wp, bool list = false)
{
    return (8 + (list ? 3 : 2) * (size_t)wp + 3) / 4 * 4;
}
__host__ __device__ inline size_t local_queue_bytes(uint32_t wp, bool list = false, uint32_t slots = kLocalSlots)
{
    return sizeof(LocalHdr) + (size_t)slots * 4 + (size_t)slots * frame_words(wp, list) * 4;
}

// Clique listing (MCE_LIST).  Every group appends, at each maximal clique it
// reports, a record [0x80000000 | k, pos_1 .. pos_k] (positions in the search
// order) to a chunk of the record buffer it claimed; the clique's members are
// the R of the frame the group last took (its bitset in `base`, its size
// `rsb`) plus the vertices the group added on its way down (`path`, indexed
// by |R|), plus the leaf vertex.  Frames that move between groups carry R.
struct ListParams {
    uint32_t *rec;          // n_chunks * chunk_words words; null: no listing
    uint32_t *fill;         // words used in each chunk (zeroed before the search)
    unsigned *next_chunk;   // chunk claim counter (zeroed)
    unsigned *overflow;     // set when a record found no chunk (zeroed)
    uint16_t *path;         // total_groups * n entries
    uint32_t *base;         // total_groups * wp words
    uint32_t n_chunks, chunk_words;
};

// Work-distribution knobs (defaults in default_tuning(); MCE_TUNE overrides).
struct Tuning {
    uint32_t share_local;   // smallest |P| given to the block ring (0: by density)
    uint32_t share_global;  // smallest |P| given to the device-wide ring (0: by density)
    uint32_t local_check;   // busy warps: iterations between block-ring checks (a power of two)
    uint32_t global_check;  // busy warps: iterations between global checks (a power of two)
    uint32_t refresh_ns;    // age of a block's cached view of the global ring
    uint32_t serve_cpb;     // served form: expected maximal cliques per block
    uint32_t pop_tries;     // ticket attempts of one take from the device-wide ring
    uint32_t share_tail;    // smallest |P| shared once half the groups/blocks are idle
    uint32_t idle_sleep_ns; // longest back-off of an idle warp that is not polling
    uint32_t t2_p;          // lane tier: largest |P| of a subproblem handed to one lane (0: off)
    uint32_t t2_levels;     // lane tier: explicit-stack levels per lane in shared memory
    uint32_t t2_smem_rows;  // lane tier on: keep the rows in shared memory (fewer warps) when 1
    uint32_t seed;          // start from every root child as its own queued frame (1) or the root (0)
    uint32_t serve_t2;      // served requests use the lane tier too (its region beside the capped stack)
    uint32_t batch_wide;    // batched form by default: 512 threads, at most two words per lane (1), or the plain shapes (0)
    uint32_t batch_split;   // batched form: parts of about 1/(blocks * batch_split) of a bucket's cost (0: no split)
    uint32_t serve_bcost;   // served form: largest expected maximal cliques (thousands) of a micro-batched request
    uint32_t small_split;   // small graphs of density <= 0.75 split breadth first from 20 vertices (1) or by density (0)
};

// The lane tier (second search tier): a frame whose P u X has at most 32
// vertices is relabelled 0..u-1 in order and searched by one lane with 32-bit
// sets.  Per warp in shared memory: the 32 lanes' local adjacency rows
// A[row][lane] (u32), the positions of their local vertices pos[v][lane]
// (u16), and t2_levels explicit-stack levels of six words per lane
// [level][field][lane] (P, X, L, |R|, S low, S high).
// After them, for the pivot rules that score candidates (GreedyBBTX/NX,
// TomitaBB), 512 bytes of scratch for the group search's parallel pivot
// scoring (each lane's words of P'); GreedyBB needs none, so its blocks keep
// that room (on 1,000 vertices with rows in shared memory: a quarter more
// warps).
constexpr int kT2Fields = 6;
constexpr int kPivotScratchWords = 128;
__host__ __device__ inline size_t t2_warp_bytes(uint32_t levels, bool scoring)
{
    return 32 * 32 * 4 + 32 * 32 * 2 + (size_t)levels * kT2Fields * 32 * 4 + (scoring ? kPivotScratchWords * 4 : 0);
}

struct SearchParams {
    uint32_t n;             // vertices
    uint32_t wp;            // words per renumbered row (= lanes * words/lane)
    const uint32_t *rows;   // renumbered rows, n * wp words (+ pad to 16 B)
    const uint32_t *order;  // position -> original label
    Ctl *ctl;
    unsigned *seq;          // queue slot sequence numbers (qcap entries)
    uint32_t *frames;       // qcap frames of fs words
    uint32_t qcap;          // power of two
    uint32_t fs;            // frame stride in words
    uint64_t *out;          // MCE_OUT_WORDS(n) words
    uint64_t timeout_ns;
    uint32_t total_groups;
    uint32_t pivot_mode;
    uint32_t stack_levels;  // <= kStackDepth
    uint32_t split_min_p;   // publish new subtrees with |P| >= this ...
    uint32_t split_target;  // ... while the global ring holds fewer frames
    uint32_t stack_smem_levels;  // explicit-stack levels kept in shared memory
    uint32_t stack_offset;       // byte offset of the stack region in shared memory
    unsigned long long *trace;   // optional timeline (2 words per record)
    uint32_t trace_per_block;    // records per block
    Tuning tune;
    ListParams lst;              // clique listing (lst.rec null: off)
    // A part of the root's branching (the root's children are independent
    // subtrees): part (device, part_k entries, strictly increasing) lists
    // the children searched; null searches the whole tree.  The root node is
    // counted only with count_root.
    const uint32_t *part;
    uint32_t part_k;
    uint32_t count_root;
    // lane tier: byte offset of its shared-memory region (t2_warp_bytes per
    // warp), stack levels kept there, and the largest |P| handed to a lane
    // (0: the tier is off)
    uint32_t t2_offset, t2_levels, t2_max_p;
    // start from the root's children, each its own queued frame, instead of
    // the root frame (the root is still counted once)
    uint32_t seed_children;
    uint32_t local_slots;   // slots of the block ring (kLocalSlots or kLocalSlotsSmall)
};

// One graph of a batch (device table entry; pointers into library memory).
struct BatchGraph {
    const uint32_t *rows;   // validated input bitset, w words per row
    uint32_t *order;        // n entries
    uint32_t *ren;          // n * wp renumbered words (+ pad to 16 B)
    uint64_t *out;          // MCE_OUT_WORDS(n) words
    uint32_t n, w, wp, pad;
    // Subproblem of the outer loop (Alg. 3), else null / 0: label[i] is the
    // original label of local vertex i (hashes and sizes use it); root holds
    // the root's P then X as bitsets over local vertices (w words each); the
    // root's R is {rv} (a local vertex, adjacent to every other one).
    const uint32_t *label;
    const uint32_t *root;
    uint32_t rv, pad2;
};

// Outer loop of Alg. 3 (outer.cu).  CSR adjacency on the device: off[n + 1],
// adj[off[n]] with every list sorted.
cudaError_t outer_csr_from_edges_bytes(uint32_t n, uint64_t m, size_t *temp_bytes);
// Builds the CSR of the simple graph given by m edges (u, v) (duplicates and
// both orientations allowed); out[MCE_OUT_STATUS] = MCE_EINVAL on a self-loop
// or an id >= n; *adj_count (device) receives off[n].
cudaError_t outer_csr_from_edges(uint32_t n, uint64_t m, const uint32_t *d_uv, void *temp, size_t temp_bytes,
                                 uint32_t *off, uint32_t *adj, uint64_t *out, cudaStream_t s);
// CSR of an n x w bitset (off: n + 1 entries; adj: off[n] entries).
cudaError_t outer_csr_from_rows(uint32_t n, uint32_t w, const uint32_t *rows, uint32_t *off, uint32_t *adj,
                                void *temp, size_t temp_bytes, size_t *need, cudaStream_t s);
// Degeneracy order (minimum remaining degree first, smallest label on ties):
// order[i] = vertex i, pos[v] = its position.  One block; n <= 65535 and
// every degree < 65535; off/adj a symmetric adjacency.
cudaError_t outer_degeneracy(uint32_t n, const uint32_t *off, const uint32_t *adj, uint32_t *order, uint32_t *pos,
                             cudaStream_t s);
// Fill every subproblem's rows, labels, root sets and table[i].rv (one block
// each): subproblem i is vertex order[i] with its neighbourhood.
cudaError_t outer_extract(const BatchGraph *table, uint32_t count, uint32_t max_w, const uint32_t *order,
                          const uint32_t *pos, const uint32_t *off, const uint32_t *adj, cudaStream_t s);
// Sum the subproblems' results into out (MCE_OUT_WORDS(n) words, zeroed).
cudaError_t outer_reduce(const BatchGraph *table, uint32_t count, uint32_t n, uint64_t *out, cudaStream_t s);

// Most words per row of a batched graph that the batch kernel splits into
// root-child parts (its shared prefix table).
constexpr int kBatchPartWords = 128;

struct BatchParams {
    const BatchGraph *graphs;
    const uint32_t *list;   // graph indices of this bucket, most expensive first
    uint32_t count;         // entries of list
    unsigned *next;         // claim counter (zeroed before the launch)
    unsigned char *qbase;   // per-block queue regions
    size_t qstride;         // bytes per region
    uint32_t qcap, fs;      // slots per region, frame stride (words)
    uint64_t timeout_ns;
    uint32_t pivot_mode, stack_levels, groups_per_block;
    uint32_t split_min_p, split_target;
    uint32_t stack_smem_levels, stack_offset;
    Tuning tune;
    uint32_t t2_offset, t2_levels, t2_max_p;  // lane tier (as in SearchParams)
};

// Per-block queue region of the batched search: [Ctl | seq | frames]
__host__ __device__ inline size_t batch_seq_offset() { return 1024; }
__host__ __device__ inline size_t batch_frames_offset(uint32_t qcap) { return 1024 + (((size_t)qcap * 4 + 255) / 256) * 256; }
__host__ __device__ inline size_t batch_region_bytes(uint32_t qcap, uint32_t fs)
{
    return batch_frames_offset(qcap) + (((size_t)qcap * fs * 4 + 255) / 256) * 256;
}

struct LaunchShape {
    unsigned blocks, threads;
    size_t smem;
    bool rows_in_smem;
};

// One search: init kernel (root frame, queue, zeroed output) + persistent
// search kernel, and its occupancy query.  Defined per (lanes, words)
// instantiation in search_gN.cu.
struct SearchImpl {
    cudaError_t (*run)(const SearchParams &, const LaunchShape &, cudaStream_t);
    cudaError_t (*occupancy)(int threads, size_t smem, int *blocks_per_sm);
    // batched form: one graph per block at a time (kernel attributes are set
    // by batch_occupancy, so run_batch is safe inside a stream capture)
    cudaError_t (*run_batch)(const BatchParams &, const LaunchShape &, cudaStream_t);
    cudaError_t (*batch_occupancy)(int threads, size_t smem, int *blocks_per_sm);
};
SearchImpl search_impl_1_1(bool smem, int pivot);
SearchImpl search_impl_1_2(bool smem, int pivot);
SearchImpl search_impl_1_4(bool smem, int pivot);
SearchImpl search_impl_2_1(bool smem, int pivot);
SearchImpl search_impl_2_2(bool smem, int pivot);
SearchImpl search_impl_2_4(bool smem, int pivot);
SearchImpl search_impl_4_1(bool smem, int pivot);
SearchImpl search_impl_4_2(bool smem, int pivot);
SearchImpl search_impl_4_4(bool smem, int pivot);
SearchImpl search_impl_8_1(bool smem, int pivot);
SearchImpl search_impl_8_2(bool smem, int pivot);
SearchImpl search_impl_8_4(bool smem, int pivot);
SearchImpl search_impl_16_1(bool smem, int pivot);
SearchImpl search_impl_16_2(bool smem, int pivot);
SearchImpl search_impl_16_4(bool smem, int pivot);
SearchImpl search_impl_32_1(bool smem, int pivot);
SearchImpl search_impl_32_2(bool smem, int pivot);
SearchImpl search_impl_32_4(bool smem, int pivot);
// Listing variants (run/occupancy only; no batched form).
SearchImpl search_list_impl_1_1(bool smem, int pivot);
SearchImpl search_list_impl_1_2(bool smem, int pivot);
SearchImpl search_list_impl_1_4(bool smem, int pivot);
SearchImpl search_list_impl_2_1(bool smem, int pivot);
SearchImpl search_list_impl_2_2(bool smem, int pivot);
SearchImpl search_list_impl_2_4(bool smem, int pivot);
SearchImpl search_list_impl_4_1(bool smem, int pivot);
SearchImpl search_list_impl_4_2(bool smem, int pivot);
SearchImpl search_list_impl_4_4(bool smem, int pivot);
SearchImpl search_list_impl_8_1(bool smem, int pivot);
SearchImpl search_list_impl_8_2(bool smem, int pivot);
SearchImpl search_list_impl_8_4(bool smem, int pivot);
SearchImpl search_list_impl_16_1(bool smem, int pivot);
SearchImpl search_list_impl_16_2(bool smem, int pivot);
SearchImpl search_list_impl_16_4(bool smem, int pivot);
SearchImpl search_list_impl_32_1(bool smem, int pivot);
SearchImpl search_list_impl_32_2(bool smem, int pivot);
SearchImpl search_list_impl_32_4(bool smem, int pivot);


// The root's children as independent subtrees (split.cu).  The root's
// branching set is L = V \ N(p0) (p0 = root_pivot, or position 0 when null)
// over the renumbered rows; child t branches on its t-th vertex v_t with
// v_1..v_{t-1} moved from P to X.
// sizes[t] = |P_t n N(v_t)|, P_t = V minus v_1..v_{t-1}, for t < cap;
// *count = |L| (device words).
cudaError_t launch_root_children(const uint32_t *rows, uint32_t n, uint32_t wp, const unsigned *root_pivot,
                                 uint32_t *sizes, uint32_t cap, uint32_t *count, cudaStream_t s);
// Queue frame j (< prm.part_k) = child prm.part[j] (after search_init_kernel
// reserved the slots); an index beyond |L| or out of order sets MCE_EINVAL.
cudaError_t launch_part_frames(const SearchParams &prm, const unsigned *root_pivot, cudaStream_t s);
// Queue every root child as its own frame (after search_init_kernel left the
// queue empty): frame t in slot t, tail = pending = |L|.  prm.qcap >= n.
cudaError_t launch_seed_children(const SearchParams &prm, const unsigned *root_pivot, cudaStream_t s);
// TomitaBB's root pivot (the earliest vertex of maximum degree) to *dst.
cudaError_t launch_root_degree_pivot(const uint32_t *rows, uint32_t n, uint32_t wp, unsigned *dst, cudaStream_t s);

// Preprocessing kernels (prep.cu).
cudaError_t launch_edges_to_rows(uint32_t n, uint64_t m, const uint32_t *uv, uint32_t w,
                                 uint32_t *rows, uint64_t *out, cudaStream_t s);
cudaError_t launch_validate_rows(uint32_t n, uint32_t w, const uint32_t *rows, uint64_t *out,
                                 cudaStream_t s);
cudaError_t launch_order(uint32_t n, uint32_t w, const uint32_t *rows, uint32_t *order,
                         cudaStream_t s);
cudaError_t launch_identity(uint32_t n, uint32_t *order, cudaStream_t s);
cudaError_t launch_renumber(uint32_t n, uint32_t w, const uint32_t *rows, const uint32_t *order,
                            uint32_t wout, uint32_t *rows_out, cudaStream_t s);
// Batched preprocessing over a device table of graphs (max_n / max_w / max_wp
// bound every entry).  prepare_* sets kernel attributes (call before capture).
cudaError_t prepare_order_batch(uint32_t max_n, uint32_t max_w, size_t *smem);
cudaError_t launch_order_batch(const BatchGraph *graphs, uint32_t count, uint32_t max_n, size_t smem,
                               cudaStream_t s);
cudaError_t launch_renumber_batch(const BatchGraph *graphs, uint32_t count, uint32_t max_n, uint32_t max_wp,
                                  cudaStream_t s);

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Raise a kernel's dynamic shared-memory limit to the device maximum and
// prefer the largest shared-memory carveout, once per (kernel, device).  Every
// launch after that runs under the same settings, so kernels of different
// requests on different streams never wait for one another to change them.
cudaError_t kernel_smem_setup(const void *func);

// Listing post-pass (listing.cu): record chunks of a finished listing search
// -> CSR listing (off[count + 1], ids) in original labels, each clique in
// ascending order and, when `sorted`, the cliques in lexicographic order.
struct ListJob {
    const uint32_t *rec, *fill;  // record buffer and per-chunk fill (search output)
    uint32_t chunks, chunk_words;  // chunks claimed (<= n_chunks), chunk size
    const uint32_t *order;       // position -> original label
    uint32_t n, max_size;
    uint64_t count, ids;         // cliques and member ids (from the histogram)
    uint32_t *ids_out;           // device, ids entries
    uint64_t *off_out;           // device, count + 1 entries
    bool sorted;
    void *temp;                  // list_temp_bytes(count, ids, chunks, sorted) bytes
    size_t temp_bytes;
};
size_t list_temp_bytes(uint64_t count, uint64_t ids, uint32_t chunks, bool sorted);
cudaError_t list_build(const ListJob &j, cudaStream_t s);

// Tuning in effect for this process: defaults, overridden once from the
// environment variable MCE_TUNE="key=value,..." (keys as in Tuning).
Tuning default_tuning();

// Shared-memory layout of the search kernels:
//   [rows (when staged), padded to 16 B][hv: n x u64][hk: (n + 1) x u64]
//   [hist: (n + 1) x u32, padded to 16 B][local frame ring][stack]
__host__ __device__ inline size_t smem_rows_bytes(uint32_t n, uint32_t wp, bool rows_in_smem)
{
    return rows_in_smem ? ((size_t)n * wp * 4 + 15) / 16 * 16 : 0;
}
__host__ __device__ inline size_t smem_local_offset(uint32_t n, uint32_t wp, bool rows_in_smem)
{
    return smem_rows_bytes(n, wp, rows_in_smem) + (size_t)n * 8 +
           (((size_t)n + 1) * 4 + 15) / 16 * 16;
}
__host__ __device__ inline size_t search_smem_bytes(uint32_t n, uint32_t wp, bool rows_in_smem, bool list = false,
                                                   uint32_t slots = kLocalSlots)
{
    return smem_local_offset(n, wp, rows_in_smem) + local_queue_bytes(wp, list, slots);
}
// Explicit-stack words per lane per level for groups of `lanes` lanes with
// `words` words per lane: P, X and the level's scalars (one word when the
// group has four or more lanes to spread them over, else four).
__host__ __device__ inline uint32_t stack_level_words(int lanes, int words)
{
    return 2u * (uint32_t)words + (lanes >= 4 ? 1u : 4u);
}
// Most levels worth keeping in shared memory (deeper ones use local memory).
constexpr int kStackSmemMax = 24;


}  // namespace mce
