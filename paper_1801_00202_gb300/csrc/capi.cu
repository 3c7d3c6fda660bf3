// C ABI of libmce (include/mce.h): launch configuration, scratch layout,
// device-level step calls and the host-level handle API.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "mce_internal.h"

using namespace mce;

namespace {

// The served form runs each admitted request on one of many streams, and CUDA
// maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 unless
// set), read when a context is created.  A process that loads the library
// before it creates its CUDA context gets 32 unless it chose a value itself.
__attribute__((constructor)) void default_connections() { setenv("CUDA_DEVICE_MAX_CONNECTIONS", "32", 0); }

// Host-side fault injection (mce_fault_inject): per site, passes to let
// through and failures to make.  `armed` keeps the unarmed path to one
// relaxed load.
struct FaultSite {
    std::mutex mu;
    uint32_t skip = 0, count = 0;
};
FaultSite g_fault[4];
std::atomic<uint32_t> g_fault_armed{0};

bool fault_fires(int site)
{
    if (g_fault_armed.load(std::memory_order_relaxed) == 0u) return false;
    FaultSite &f = g_fault[site];
    std::lock_guard<std::mutex> lk(f.mu);
    if (f.count == 0u) return false;
    if (f.skip) {
        --f.skip;
        return false;
    }
    if (--f.count == 0u) g_fault_armed.fetch_sub(1u);
    return true;
}

int fault_arm(int site, uint32_t skip, uint32_t count)
{
    if (site < MCE_FAULT_ALLOC || site > MCE_FAULT_ADMIT) return MCE_EINVAL;
    FaultSite &f = g_fault[site];
    std::lock_guard<std::mutex> lk(f.mu);
    if (f.count) g_fault_armed.fetch_sub(1u);
    f.skip = skip;
    f.count = count;
    if (count) g_fault_armed.fetch_add(1u);
    return MCE_OK;
}

__attribute__((constructor)) void fault_from_env()
{
    const char *env = std::getenv("MCE_FAULT");
    if (!env) return;
    char site[16] = {0};
    unsigned skip = 0, count = 0;
    if (std::sscanf(env, "%15[a-z]:%u:%u", site, &skip, &count) != 3) return;
    const int s = !std::strcmp(site, "alloc") ? MCE_FAULT_ALLOC
                  : !std::strcmp(site, "copy") ? MCE_FAULT_COPY
                  : !std::strcmp(site, "admit") ? MCE_FAULT_ADMIT : 0;
    if (s) fault_arm(s, skip, count);
}

// ---------------------------------------------------------------------------
// Launch configuration

struct Config {
    int G = 32, K = 1;
    bool smem = false;
    unsigned threads = 0, blocks = 0;
    uint32_t stack_levels = 0, stack_offset = 0;
    size_t smem_bytes = 0;
    uint32_t wp = 32;
    uint32_t qcap = 1024, fs = 0;
    uint32_t total_groups = 0;
    int pivot = 0;
    bool list = false;  // frames carry R (clique listing)
    uint32_t t2_offset = 0, t2_levels = 0, t2_max_p = 0;  // lane tier (t2_max_p 0: off)
    bool seed = false;  // start from the root's children
    uint32_t local_slots = kLocalSlots;  // block ring slots
    SearchImpl impl{nullptr, nullptr, nullptr, nullptr};
};

struct Layout {
    size_t ctl = 0, order = 0, rows = 0, seq = 0, frames = 0, total = 0;
};

mce_options defaults(const mce_options *o)
{
    mce_options d{};
    if (o) d = *o;
    return d;
}

SearchImpl impl_for(int G, int K, bool smem, int pivot, bool list = false)
{
    if (pivot == MCE_PIVOT_GREEDY_NX) pivot = MCE_PIVOT_GREEDY_TX;  // the TX kernels, early exit on
#define MCE_IMPL_CASE(g, k)                                                                                \
    case g * 8 + k:                                                                                        \
        return list ? search_list_impl_##g##_##k(smem, pivot) : search_impl_##g##_##k(smem, pivot);
    switch (G * 8 + K) {
        MCE_IMPL_CASE(1, 1) MCE_IMPL_CASE(1, 2) MCE_IMPL_CASE(1, 4)
        MCE_IMPL_CASE(2, 1) MCE_IMPL_CASE(2, 2) MCE_IMPL_CASE(2, 4)
        MCE_IMPL_CASE(4, 1) MCE_IMPL_CASE(4, 2) MCE_IMPL_CASE(4, 4)
        MCE_IMPL_CASE(8, 1) MCE_IMPL_CASE(8, 2) MCE_IMPL_CASE(8, 4)
        MCE_IMPL_CASE(16, 1) MCE_IMPL_CASE(16, 2) MCE_IMPL_CASE(16, 4)
        MCE_IMPL_CASE(32, 1) MCE_IMPL_CASE(32, 2) MCE_IMPL_CASE(32, 4)
    default: return {nullptr, nullptr, nullptr, nullptr};
    }
#undef MCE_IMPL_CASE
}

uint32_t next_pow2(uint64_t x)
{
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return (uint32_t)p;
}

size_t search_smem(uint32_t n, uint32_t wp, bool rows_in_smem, bool list = false, uint32_t slots = kLocalSlots)
{
    return search_smem_bytes(n, wp, rows_in_smem, list, slots);
}

constexpr uint32_t kListFlags = MCE_LIST | MCE_LIST_SORTED;

// Shared-memory stack: as many levels (up to kStackSmemMax) as fit between
// `base` (rows, hash terms, histogram, block ring) and `limit`.
void plan_stack_for(uint32_t base, int G, int K, unsigned threads, size_t limit, uint32_t &levels, uint32_t &offset,
                    size_t &total)
{
    offset = (uint32_t)round_up(base, 16);
    const size_t per_level = (size_t)(threads / 32) * stack_level_words(G, K) * 32 * 4;
    const size_t avail = limit > offset ? limit - offset : 0;
    levels = (uint32_t)std::min<size_t>(kStackSmemMax, avail / per_level);
    total = offset + (size_t)levels * per_level;
}

// Default subtree shape (lanes G x words per lane K).  With the lane tier
// taking the small subproblems, one word per lane and as many lanes as the
// row has words won up to 24 words per row: measured on one graph of each
// size, whole path (old four-word shapes in brackets), G(45) Moon-Moser 1.33
// (1.48) ms, G(100, 0.5) 0.27 (0.29), G(128, 0.7) 1.29 (1.84), G(200, 0.55)
// 1.36 (2.10), G(256, 0.5) 1.44 (2.52), G(300, 0.5) 2.11 (2.96), G(700, 0.3)
// 1.55 (1.66) ms.  At 13-16 words two words per lane led (G(500, 0.4): 2.63
// against 2.76 with one and 3.15 with four), at 25-32 four (G(1000, 0.3):
// 7.28 against 7.96 with two and 8.97 with one: 32 one-word lanes per
// subtree leave a block too few subtrees), above 32 two (G(1500, 0.15) and
// G(2000, 0.1): 2.53 / 2.60 against 2.59 / 2.67 with four).
void default_shape(uint32_t n, int &G, int &K)
{
    const uint32_t W = std::max<uint32_t>(1, (n + 31) / 32);
    if (W <= 1) { G = 1; K = 1; }
    else if (W <= 2) { G = 2; K = 1; }
    else if (W <= 4) { G = 4; K = 1; }
    else if (W <= 8) { G = 8; K = 1; }
    else if (W <= 12) { G = 16; K = 1; }
    else if (W <= 16) { G = 8; K = 2; }
    else if (W <= 24) { G = 32; K = 1; }
    else if (W <= 32) { G = 8; K = 4; }
    else if (W <= 64) { G = 32; K = 2; }
    else { G = 32; K = 4; }
}

// Shape for n vertices under the caller's options: forced lanes/words win,
// otherwise the default.
void pick_shape(uint32_t n, const mce_options &o, int &G, int &K)
{
    const uint32_t W = std::max<uint32_t>(1, (n + 31) / 32);
    default_shape(n, G, K);
    if (o.lanes_per_subtree || o.words_per_lane) {
        if (o.lanes_per_subtree) G = (int)o.lanes_per_subtree;
        if (o.words_per_lane) K = (int)o.words_per_lane;
        else K = (int)std::max<uint32_t>(1, (W + G - 1) / G);
        if (K == 3) K = 4;
    }
}

// The search kernels are built for at most kMaxThreads threads per block
// (128 registers per thread: the group state of four-word lanes, and no
// spills for the narrower shapes), and the plain form launches that many.
// On graphs of up to 128 vertices 512 threads beat 256 wherever the search
// has real work (0.65-0.89x the time) and lost 3-9 % on the smallest,
// launch-bound ones.
constexpr unsigned kMaxThreads = 512u;

// stack_cap: most shared memory for the explicit stack per block (the served
// form keeps blocks small so that several requests share an SM).
int choose(uint32_t n, const mce_options &o, Config &c, size_t stack_cap = ~(size_t)0)
{
    if (o.pivot_mode > MCE_PIVOT_GREEDY_NX || o.stack_levels > (uint32_t)kStackDepth || o.queue_log2 > 24)
        return MCE_EINVAL;
    const uint32_t W = std::max<uint32_t>(1, (n + 31) / 32);
    int G, K;
    pick_shape(n, o, G, K);
    if ((uint32_t)(G * K) < W) return MCE_EINVAL;
    c.list = (o.flags & kListFlags) != 0u;
    c.impl = impl_for(G, K, false, (int)o.pivot_mode, c.list);
    if (!c.impl.run) return MCE_EINVAL;
    c.G = G;
    c.K = K;
    c.wp = (uint32_t)(G * K);
    c.pivot = (int)o.pivot_mode;

    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MCE_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MCE_ECUDA;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return MCE_ECUDA;
    const size_t limit = (size_t)optin - 1024;  // static shared memory + slack

    c.threads = o.threads_per_block ? o.threads_per_block : kMaxThreads;
    if (c.threads % 32 || c.threads > kMaxThreads) return MCE_EINVAL;

    // The lane tier (counting kernels, groups of two or more lanes; in the
    // served form, whose stack is capped so that requests share SMs, when
    // serve_t2 is set) needs t2_warp_bytes per warp.  Rows stay in shared
    // memory when they fit beside it; otherwise, with t2_smem_rows, the block
    // gets fewer warps so that they fit, or they are read from L2.
    const Tuning tu = default_tuning();
    const bool t2 = !c.list && G >= 2 && tu.t2_p != 0 && (stack_cap == ~(size_t)0 || tu.serve_t2);
    uint32_t t2_levels = tu.t2_levels;
    size_t t2w = t2 ? t2_warp_bytes(t2_levels, o.pivot_mode != MCE_PIVOT_GREEDY) : 0;
    auto fits = [&](bool rows_smem, unsigned threads) {
        return round_up(search_smem(n, c.wp, rows_smem, c.list, c.local_slots), 16) + (size_t)(threads / 32) * t2w <=
               limit;
    };
    c.smem = c.wp <= 32 && fits(true, c.threads);
    if (!c.smem && t2 && tu.t2_smem_rows && c.wp <= 32 && !o.threads_per_block) {
        // rows in shared memory with as many warps as fit beside them (one
        // warp at a time), with fewer lane-tier stack levels in shared memory
        // (deeper levels go to local memory) and then a half-size block ring
        // when that buys warps; G(1000, 0.3): 8 warps with four levels, 9
        // with three, 10 with two, 11 with one, 12 with one and 16 ring
        // slots (6.2 -> 5.85 ms from 11 to 12)
        auto most = [&]() {
            unsigned th = c.threads;
            while (th >= 128 && !fits(true, th)) th -= 32;
            return th >= 128 ? th : 0u;
        };
        unsigned best = 0;
        uint32_t best_levels = t2_levels, best_slots = kLocalSlots;
        for (uint32_t slots : {(uint32_t)kLocalSlots, (uint32_t)kLocalSlotsSmall}) {
            c.local_slots = slots;
            for (uint32_t lv = t2_levels; lv >= 1; --lv) {
                t2w = t2_warp_bytes(lv, o.pivot_mode != MCE_PIVOT_GREEDY);
                const unsigned th = most();
                if (th > best) {
                    best = th;
                    best_levels = lv;
                    best_slots = slots;
                }
            }
        }
        c.local_slots = best_slots;
        t2_levels = best_levels;
        t2w = t2_warp_bytes(t2_levels, o.pivot_mode != MCE_PIVOT_GREEDY);
        if (best) {
            c.threads = best;
            c.smem = true;
        }
    }
    if (t2 && !fits(c.smem, c.threads) && !o.threads_per_block)
        while (c.threads > 128 && !fits(c.smem, c.threads)) c.threads -= 64;
    const bool t2_on = t2 && fits(c.smem, c.threads);
    if (c.smem) c.impl = impl_for(G, K, true, (int)o.pivot_mode, c.list);
    if (search_smem(n, c.wp, c.smem, c.list, c.local_slots) > limit) return MCE_EINVAL;

    size_t base = search_smem(n, c.wp, c.smem, c.list, c.local_slots);
    if (t2_on) {
        c.t2_offset = (uint32_t)round_up(base, 16);
        c.t2_levels = t2_levels;
        c.t2_max_p = tu.t2_p;
        base = c.t2_offset + (size_t)(c.threads / 32) * t2w;
    }
    const size_t cap = stack_cap < limit - base ? base + stack_cap : limit;
    plan_stack_for((uint32_t)base, c.G, c.K, c.threads, cap, c.stack_levels, c.stack_offset, c.smem_bytes);
    if (o.blocks) {
        c.blocks = o.blocks;
    } else {
        int per_sm = 0;
        if (c.impl.occupancy((int)c.threads, c.smem_bytes, &per_sm) != cudaSuccess) return MCE_ECUDA;
        if (per_sm < 1) return MCE_ENOMEM;
        c.blocks = (unsigned)(per_sm * sms);
    }
    c.total_groups = c.blocks * (c.threads / 32) * (32 / G);
    c.qcap = next_pow2(std::max<uint64_t>(1024, 4ull * c.total_groups + 256));
    c.seed = tu.seed != 0;
    if (c.seed) c.qcap = std::max<uint32_t>(c.qcap, next_pow2(2ull * n + 256));  // every root child queued at once
    if (o.queue_log2) c.qcap = std::max<uint32_t>(c.qcap, 1u << o.queue_log2);
    c.fs = (uint32_t)frame_words(c.wp, c.list);
    return MCE_OK;
}

Layout layout(uint32_t n, const Config &c)
{
    Layout L;
    size_t off = 0;
    L.ctl = off;
    off += round_up(sizeof(Ctl), 256);
    L.order = off;
    off += round_up((size_t)std::max<uint32_t>(n, 1) * 4, 256);
    L.rows = off;
    off += round_up((size_t)n * c.wp * 4 + 16, 256);
    L.seq = off;
    off += round_up((size_t)c.qcap * 4, 256);
    L.frames = off;
    off += round_up((size_t)c.qcap * c.fs * 4, 256);
    L.total = off;
    return L;
}

// Smallest power of two >= v (v >= 1), capped at 2^31: the kernel tests the
// check periods with a mask.
uint32_t pow2_ceil(uint32_t v)
{
    uint32_t p = 1u;
    while (p < v && p < 0x80000000u) p <<= 1;
    return p;
}

int cuda_code(cudaError_t e) { return e == cudaSuccess ? MCE_OK : (e == cudaErrorMemoryAllocation ? MCE_ENOMEM : MCE_ECUDA); }

}  // namespace

Tuning mce::default_tuning()
{
    static const Tuning t = [] {
        // block-ring checks every 8 and device-wide checks every 16 group
        // iterations of a busy warp: with fetch-and-add ring tickets the
        // checks are cheap enough that checking more often than every 16 /
        // 64 iterations paid (G(1000, 0.3): 7.8 -> 7.4 ms; G(700, 0.3): 2.2
        // -> 1.7 ms).  Served form: a request alone gets a block per 20,000
        // expected maximal cliques, and requests expecting up to 10^6 share
        // micro-batches (on the served workload, 10,400 -> 11,300 requests/s
        // closed loop and p99 6.3 -> 3.9 ms at 0.7x that load, against one
        // block per 50,000 and micro-batches up to 10^5)
        Tuning d{0u, 0u, 8u, 16u, 2000u, 20000u, 16384u, 32u, 16384u, 32u, 4u, 1u, 1u, 1u, 1u, 4u, 1000u, 1u};  // 0: thresholds by density
        if (const char *env = std::getenv("MCE_TUNE")) {
            const char *p = env;
            while (*p) {
                char key[32] = {0};
                unsigned val = 0;
                int used = 0;
                if (std::sscanf(p, "%31[a-z0-9_]=%u%n", key, &val, &used) != 2) break;
                if (!std::strcmp(key, "share_local")) d.share_local = val;
                else if (!std::strcmp(key, "share_global")) d.share_global = val;
                else if (!std::strcmp(key, "local_check") && val) d.local_check = pow2_ceil(val);
                else if (!std::strcmp(key, "global_check") && val) d.global_check = pow2_ceil(val);
                else if (!std::strcmp(key, "refresh_ns")) d.refresh_ns = val;
                else if (!std::strcmp(key, "serve_cpb") && val) d.serve_cpb = val;
                else if (!std::strcmp(key, "pop_tries") && val) d.pop_tries = val;
                else if (!std::strcmp(key, "share_tail") && val) d.share_tail = val;
                else if (!std::strcmp(key, "idle_sleep_ns") && val) d.idle_sleep_ns = val;
                else if (!std::strcmp(key, "t2_p")) d.t2_p = std::min(val, 32u);
                else if (!std::strcmp(key, "t2_levels")) d.t2_levels = std::min(val, 31u);
                else if (!std::strcmp(key, "t2_smem_rows")) d.t2_smem_rows = val;
                else if (!std::strcmp(key, "seed")) d.seed = val;
                else if (!std::strcmp(key, "serve_t2")) d.serve_t2 = val;
                else if (!std::strcmp(key, "batch_wide")) d.batch_wide = val;
                else if (!std::strcmp(key, "batch_split")) d.batch_split = val;
                else if (!std::strcmp(key, "serve_bcost")) d.serve_bcost = val;
                else if (!std::strcmp(key, "small_split")) d.small_split = val;
                p += used;
                if (*p == ',') ++p;
            }
        }
        return d;
    }();
    return t;
}

namespace {

thread_local void *g_trace = nullptr;
thread_local uint64_t g_trace_bytes = 0;

SearchParams params(uint32_t n, const Config &c, const Layout &L, unsigned char *scratch, const uint32_t *rows,
                    const uint32_t *order, uint64_t *out, const mce_options &o, const ListParams *lp)
{
    SearchParams p{};
    p.n = n;
    p.wp = c.wp;
    p.rows = rows;
    p.order = order;
    p.ctl = reinterpret_cast<Ctl *>(scratch + L.ctl);
    p.seq = reinterpret_cast<unsigned *>(scratch + L.seq);
    p.frames = reinterpret_cast<uint32_t *>(scratch + L.frames);
    p.qcap = c.qcap;
    p.fs = c.fs;
    p.out = out;
    p.timeout_ns = o.timeout_ns ? o.timeout_ns : 60ull * 1000000000ull;
    p.total_groups = c.total_groups;
    p.pivot_mode = (uint32_t)c.pivot;
    p.stack_levels = o.stack_levels ? std::min<uint32_t>(o.stack_levels, kStackDepth) : kStackDepth;
    p.split_min_p = o.split_min_p;  // 0: by density
    p.split_target = c.qcap / 2;
    p.stack_smem_levels = c.stack_levels;
    p.stack_offset = c.stack_offset;
    p.tune = default_tuning();
    // the breadth-first split of small graphs from 20 vertices pays in a
    // full-wave launch of one graph; a grid sized for one served request
    // (o.blocks) ran slower with it (10,800 -> 10,300 requests/s)
    if (o.blocks) p.tune.small_split = 0u;
    p.trace = nullptr;
    p.trace_per_block = 0;
    if (g_trace && c.blocks) {
        p.trace = static_cast<unsigned long long *>(g_trace);
        p.trace_per_block = (uint32_t)std::min<uint64_t>(g_trace_bytes / 16 / c.blocks, 0xffffffffu);
    }
    p.lst = lp ? *lp : ListParams{};
    p.part = nullptr;
    p.part_k = 0;
    p.count_root = 1;
    p.t2_offset = c.t2_offset;
    p.t2_levels = c.t2_levels;
    p.t2_max_p = c.t2_max_p;
    p.seed_children = c.seed ? 1u : 0u;
    p.local_slots = c.local_slots;
    return p;
}

// A part of the root's branching: d_children (device) lists k root-child
// indices, strictly increasing.
struct PartSpec {
    const uint32_t *d_children;
    uint32_t k;
    uint32_t count_root;
};

int run_search(uint32_t n, const Config &c, const Layout &L, unsigned char *scratch, const uint32_t *rows,
               const uint32_t *order, uint64_t *out, const mce_options &o, cudaStream_t s,
               const ListParams *lp = nullptr, const PartSpec *part = nullptr)
{
    SearchParams p = params(n, c, L, scratch, rows, order, out, o, lp);
    if (part) {
        p.part = part->d_children;
        p.part_k = part->k;
        p.count_root = part->count_root;
    }
    LaunchShape sh{c.blocks, c.threads, c.smem_bytes, c.smem};
    return cuda_code(c.impl.run(p, sh, s));
}

}  // namespace

// ---------------------------------------------------------------------------
// Device-level calls

extern "C" int mce_edges_to_rows(uint32_t n, uint64_t m, const uint32_t *d_uv, uint32_t words_per_row,
                                 uint32_t *d_rows, uint64_t *d_out, void *stream)
{
    if (n > MCE_NMAX || !d_out || (m && !d_uv) || (n && !d_rows) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    return cuda_code(launch_edges_to_rows(n, m, d_uv, words_per_row, d_rows, d_out, (cudaStream_t)stream));
}

extern "C" int mce_validate_rows(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows, uint64_t *d_out,
                                 void *stream)
{
    if (n > MCE_NMAX || !d_out || (n && !d_rows) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    return cuda_code(launch_validate_rows(n, words_per_row, d_rows, d_out, (cudaStream_t)stream));
}

extern "C" int mce_order(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows, uint32_t *d_order, void *stream)
{
    if (n > MCE_NMAX || (n && (!d_rows || !d_order)) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    return cuda_code(launch_order(n, words_per_row, d_rows, d_order, (cudaStream_t)stream));
}

extern "C" int mce_renumber(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows, const uint32_t *d_order,
                            uint32_t out_words_per_row, uint32_t *d_rows_out, void *stream)
{
    if (n > MCE_NMAX || (n && (!d_rows || !d_order || !d_rows_out)) || words_per_row < (n + 31) / 32 ||
        out_words_per_row < (n + 31) / 32)
        return MCE_EINVAL;
    return cuda_code(launch_renumber(n, words_per_row, d_rows, d_order, out_words_per_row, d_rows_out,
                                     (cudaStream_t)stream));
}

extern "C" uint32_t mce_search_words(uint32_t n, const mce_options *opts)
{
    Config c;
    const mce_options o = defaults(opts);
    if (n > MCE_NMAX || (o.flags & kListFlags) || choose(n, o, c) != MCE_OK) return 0;
    return c.wp;
}

extern "C" int mce_scratch_bytes(uint32_t n, const mce_options *opts, uint64_t *bytes)
{
    if (!bytes || n > MCE_NMAX) return MCE_EINVAL;
    const mce_options o = defaults(opts);
    if (o.flags & kListFlags) return MCE_ENOTIMPL;  // listing: host API only
    Config c;
    int rc = choose(n, o, c);
    if (rc) return rc;
    *bytes = layout(n, c).total;
    return MCE_OK;
}

extern "C" int mce_search(uint32_t n, const uint32_t *d_rows_renum, const uint32_t *d_order, const mce_options *opts,
                          void *d_scratch, uint64_t scratch_bytes, uint64_t *d_out, void *stream)
{
    if (n > MCE_NMAX || !d_out || !d_scratch || (n && (!d_rows_renum || !d_order))) return MCE_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_scratch) % 256 || reinterpret_cast<uintptr_t>(d_rows_renum) % 16)
        return MCE_EINVAL;
    const mce_options o = defaults(opts);
    if (o.flags & kListFlags) return MCE_ENOTIMPL;  // listing: host API only
    Config c;
    int rc = choose(n, o, c);
    if (rc) return rc;
    const Layout L = layout(n, c);
    if (scratch_bytes < L.total) return MCE_ENOMEM;
    return run_search(n, c, L, static_cast<unsigned char *>(d_scratch), d_rows_renum, d_order, d_out, o,
                      (cudaStream_t)stream);
}

namespace {

// The whole path (validate, order, renumber, search) for a chosen
// configuration; lp non-null lists the cliques (host API).
int enumerate_device_impl(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows, const mce_options &o,
                          const Config &c, const Layout &L, unsigned char *scr, uint64_t *d_out, cudaStream_t s,
                          const ListParams *lp, const PartSpec *part = nullptr)
{
    uint32_t *order = reinterpret_cast<uint32_t *>(scr + L.order);
    uint32_t *rows = reinterpret_cast<uint32_t *>(scr + L.rows);
    cudaError_t e = cudaMemsetAsync(d_out + MCE_OUT_STATUS, 0, sizeof(uint64_t), s);
    if (e == cudaSuccess) e = launch_validate_rows(n, words_per_row, d_rows, d_out, s);
    if (e == cudaSuccess)
        e = (o.flags & MCE_ORDER_IDENTITY) ? launch_identity(n, order, s) : launch_order(n, words_per_row, d_rows, order, s);
    if (e == cudaSuccess) e = launch_renumber(n, words_per_row, d_rows, order, c.wp, rows, s);
    if (e != cudaSuccess) return cuda_code(e);
    return run_search(n, c, L, scr, rows, order, d_out, o, s, lp, part);
}

}  // namespace

extern "C" int mce_enumerate_device(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows,
                                    const mce_options *opts, void *d_scratch, uint64_t scratch_bytes,
                                    uint64_t *d_out, void *stream)
{
    if (n > MCE_NMAX || !d_out || !d_scratch || (n && !d_rows) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_scratch) % 256) return MCE_EINVAL;
    const mce_options o = defaults(opts);
    if (o.flags & kListFlags) return MCE_ENOTIMPL;  // listing: host API only
    Config c;
    int rc = choose(n, o, c);
    if (rc) return rc;
    const Layout L = layout(n, c);
    if (scratch_bytes < L.total) return MCE_ENOMEM;
    return enumerate_device_impl(n, words_per_row, d_rows, o, c, L, static_cast<unsigned char *>(d_scratch), d_out,
                                 (cudaStream_t)stream, nullptr);
}

// ---------------------------------------------------------------------------
// Host-level API

struct Server;

// A batch bucket's launch choice: subtree shape, block size, split threshold.
struct TuneChoice {
    int G = 0, K = 0;
    unsigned threads = 0;
    uint32_t split = 0;
    bool tuned = false;
    double ms_per_graph = 0.0;
};

struct mce_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;
    uint64_t budget = 0;
    std::atomic<uint64_t> used{0};
    Server *server = nullptr;  // started by the first mce_submit
    std::mutex tune_mu;        // autotuned batch choices by (words class, pivot)
    std::map<uint32_t, TuneChoice> tuned;
    std::mutex stage_mu;       // two pinned halves for copies to pageable host memory
    void *stage[2] = {nullptr, nullptr};
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
};

struct mce_graph {
    mce_ctx *ctx = nullptr;
    uint32_t n = 0, w = 0;
    uint32_t *d_rows = nullptr;  // bitset (null for a graph held only as CSR)
    uint64_t bytes = 0;
    uint64_t m = 0;  // edges (as given: an estimate when duplicates were passed)
    // CSR (sorted lists) for the outer loop of Alg. 3: built at load for
    // n > MCE_NMAX, else on first use
    uint32_t *d_off = nullptr, *d_adj = nullptr;
    uint64_t csr_bytes = 0;
    // a subproblem of the outer loop (library-internal graphs only)
    const uint32_t *label = nullptr, *root = nullptr;
    uint32_t rv = 0;
    double cost_hint = 0.0;
};

namespace {

struct DevicePick {
    int prev = -1;
    explicit DevicePick(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevicePick()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int dalloc(mce_ctx *ctx, void **p, size_t bytes, cudaStream_t s = nullptr)
{
    *p = nullptr;
    if (fault_fires(MCE_FAULT_ALLOC)) return MCE_ENOMEM;
    if (bytes == 0) bytes = 256;
    if (ctx->budget && ctx->used.fetch_add(bytes) + bytes > ctx->budget) {
        ctx->used.fetch_sub(bytes);
        return MCE_ENOMEM;
    }
    if (!ctx->budget) ctx->used.fetch_add(bytes);
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, s ? s : ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->used.fetch_sub(bytes);
        return MCE_ENOMEM;
    }
    return MCE_OK;
}

void dfree(mce_ctx *ctx, void *p, size_t bytes, cudaStream_t s = nullptr)
{
    if (!p) return;
    cudaFreeAsync(p, s ? s : ctx->stream);
    if (bytes == 0) bytes = 256;
    ctx->used.fetch_sub(bytes);
}

double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" int mce_ctx_create(int device, uint64_t mem_budget_bytes, void *stream, mce_ctx **out)
{
    if (!out) return MCE_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return device < 0 ? MCE_EINVAL : MCE_ECUDA;
    }
    mce_ctx *c = new (std::nothrow) mce_ctx;
    if (!c) return MCE_ENOMEM;
    DevicePick pick(device);
    c->device = device;
    cudaError_t e = cudaSuccess;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = true;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&c->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = ~0ull;  // keep freed blocks for reuse
        e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    size_t fr = 0, tot = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
        if (c->pool) cudaMemPoolDestroy(c->pool);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return MCE_ECUDA;
    }
    c->budget = mem_budget_bytes ? mem_budget_bytes : (uint64_t)(fr * 0.9);
    *out = c;
    return MCE_OK;
}

void server_stop(mce_ctx *ctx);

extern "C" void mce_ctx_destroy(mce_ctx *ctx)
{
    if (!ctx) return;
    {
        DevicePick pick(ctx->device);
        server_stop(ctx);
        cudaStreamSynchronize(ctx->stream);
        for (int i = 0; i < 2; ++i) {
            if (ctx->stage[i]) cudaFreeHost(ctx->stage[i]);
            if (ctx->stage_ev[i]) cudaEventDestroy(ctx->stage_ev[i]);
        }
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
}

namespace {

int finish_load(mce_ctx *ctx, mce_graph *g, uint64_t *d_status, mce_graph **out)
{
    uint64_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, d_status + MCE_OUT_STATUS, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, d_status, 64);
    if (e != cudaSuccess || st != 0) {
        dfree(ctx, g->d_rows, g->bytes);
        cudaStreamSynchronize(ctx->stream);
        delete g;
        return e != cudaSuccess ? MCE_ECUDA : (int)(int64_t)st;
    }
    *out = g;
    return MCE_OK;
}

}  // namespace

namespace {

// A graph beyond the bitset path: CSR only (Alg. 3's outer loop).
int load_edges_csr(mce_ctx *ctx, uint32_t n, const uint32_t *uv, uint64_t m, mce_graph **out)
{
    mce_graph *g = new (std::nothrow) mce_graph;
    if (!g) return MCE_ENOMEM;
    g->ctx = ctx;
    g->n = n;
    g->w = (n + 31) / 32;
    g->m = m;
    size_t tb = 0;
    outer_csr_from_edges_bytes(n, m, &tb);
    uint32_t *d_uv = nullptr;
    uint64_t *d_status = nullptr;
    void *temp = nullptr;
    g->csr_bytes = round_up(((uint64_t)n + 1) * 4, 256) + round_up(std::max<uint64_t>(2 * m, 1) * 4, 256);
    int rc = dalloc(ctx, (void **)&g->d_off, g->csr_bytes);
    if (rc == MCE_OK) rc = dalloc(ctx, (void **)&d_status, 64);
    if (rc == MCE_OK && m) rc = dalloc(ctx, (void **)&d_uv, m * 8);
    if (rc == MCE_OK) rc = dalloc(ctx, &temp, tb);
    cudaError_t e = cudaSuccess;
    if (rc == MCE_OK) {
        g->d_adj = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(g->d_off) +
                                                round_up(((uint64_t)n + 1) * 4, 256));
        e = cudaMemsetAsync(d_status, 0, 64, ctx->stream);
        if (e == cudaSuccess && m)
            e = fault_fires(MCE_FAULT_COPY) ? cudaErrorInvalidValue
                                            : cudaMemcpyAsync(d_uv, uv, m * 8, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = outer_csr_from_edges(n, m, d_uv, temp, tb, g->d_off, g->d_adj, d_status, ctx->stream);
        if (e != cudaSuccess) rc = MCE_ECUDA;
    }
    dfree(ctx, temp, tb);
    dfree(ctx, d_uv, m * 8);
    uint64_t st = 0;
    if (rc == MCE_OK) {
        e = cudaMemcpyAsync(&st, d_status + MCE_OUT_STATUS, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = MCE_ECUDA;
        else if (st) rc = (int)(int64_t)st;
    }
    dfree(ctx, d_status, 64);
    if (rc != MCE_OK) {
        dfree(ctx, g->d_off, g->csr_bytes);
        cudaStreamSynchronize(ctx->stream);
        delete g;
        return rc;
    }
    *out = g;
    return MCE_OK;
}

}  // namespace

extern "C" int mce_load_edges(mce_ctx *ctx, uint32_t n, const uint32_t *uv, uint64_t m, mce_graph **out)
{
    if (!ctx || !out || n > MCE_NMAX_SPARSE || (m && !uv)) return MCE_EINVAL;
    *out = nullptr;
    DevicePick pick(ctx->device);
    if (n > MCE_NMAX) return load_edges_csr(ctx, n, uv, m, out);
    mce_graph *g = new (std::nothrow) mce_graph;
    if (!g) return MCE_ENOMEM;
    g->ctx = ctx;
    g->n = n;
    g->w = std::max<uint32_t>(1, (n + 31) / 32);
    g->bytes = (uint64_t)std::max<uint32_t>(n, 1) * g->w * 4;
    g->m = m;
    uint32_t *d_uv = nullptr;
    uint64_t *d_status = nullptr;
    int rc = dalloc(ctx, (void **)&g->d_rows, g->bytes);
    if (rc == MCE_OK) rc = dalloc(ctx, (void **)&d_status, 64);
    if (rc == MCE_OK && m) rc = dalloc(ctx, (void **)&d_uv, m * 8);
    cudaError_t e = cudaSuccess;
    if (rc == MCE_OK) {
        e = cudaMemsetAsync(d_status, 0, 64, ctx->stream);
        if (e == cudaSuccess && m)
            e = fault_fires(MCE_FAULT_COPY) ? cudaErrorInvalidValue
                                            : cudaMemcpyAsync(d_uv, uv, m * 8, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = launch_edges_to_rows(n, m, d_uv, g->w, g->d_rows, d_status, ctx->stream);
        if (e != cudaSuccess) rc = MCE_ECUDA;
    }
    dfree(ctx, d_uv, m * 8);
    if (rc != MCE_OK) {
        dfree(ctx, d_status, 64);
        dfree(ctx, g->d_rows, g->bytes);
        cudaStreamSynchronize(ctx->stream);
        delete g;
        return rc;
    }
    return finish_load(ctx, g, d_status, out);
}

extern "C" int mce_load_bitset(mce_ctx *ctx, uint32_t n, const uint32_t *rows, uint32_t words_per_row,
                               mce_graph **out)
{
    if (!ctx || !out || n > MCE_NMAX || (n && !rows) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    *out = nullptr;
    DevicePick pick(ctx->device);
    mce_graph *g = new (std::nothrow) mce_graph;
    if (!g) return MCE_ENOMEM;
    g->ctx = ctx;
    g->n = n;
    g->w = std::max<uint32_t>(1, words_per_row);
    g->bytes = (uint64_t)std::max<uint32_t>(n, 1) * g->w * 4;
    for (uint64_t i = 0; i < (uint64_t)n * words_per_row; ++i) g->m += (uint64_t)__builtin_popcount(rows[i]);
    g->m /= 2;
    uint64_t *d_status = nullptr;
    int rc = dalloc(ctx, (void **)&g->d_rows, g->bytes);
    if (rc == MCE_OK) rc = dalloc(ctx, (void **)&d_status, 64);
    cudaError_t e = cudaSuccess;
    if (rc == MCE_OK) {
        e = cudaMemsetAsync(d_status, 0, 64, ctx->stream);
        if (e == cudaSuccess && n)
            e = fault_fires(MCE_FAULT_COPY)
                    ? cudaErrorInvalidValue
                    : cudaMemcpyAsync(g->d_rows, rows, (size_t)n * words_per_row * 4, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = launch_validate_rows(n, g->w, g->d_rows, d_status, ctx->stream);
        if (e != cudaSuccess) rc = MCE_ECUDA;
    }
    if (rc != MCE_OK) {
        dfree(ctx, d_status, 64);
        dfree(ctx, g->d_rows, g->bytes);
        cudaStreamSynchronize(ctx->stream);
        delete g;
        return rc;
    }
    return finish_load(ctx, g, d_status, out);
}

extern "C" void mce_graph_free(mce_graph *g)
{
    if (!g) return;
    DevicePick pick(g->ctx->device);
    dfree(g->ctx, g->d_rows, g->bytes);
    dfree(g->ctx, g->d_off, g->csr_bytes);
    cudaStreamSynchronize(g->ctx->stream);
    delete g;
}

namespace {

int fill_result(const std::vector<uint64_t> &h, uint32_t n, mce_result *res)
{
    res->count = h[MCE_OUT_COUNT];
    res->nodes = h[MCE_OUT_NODES];
    res->internal_nodes = h[MCE_OUT_INTERNAL];
    res->dead_ends = h[MCE_OUT_DEAD_ENDS];
    res->hash = h[MCE_OUT_HASH];
    res->max_size = (uint32_t)h[MCE_OUT_MAX_SIZE];
    const int st = (int)(int64_t)h[MCE_OUT_STATUS];
    res->status = (uint32_t)st;
    if (st) return st;
    if (res->hist) {
        const uint32_t k = std::min<uint32_t>(res->hist_cap, n + 1);
        for (uint32_t i = 0; i < k; ++i) res->hist[i] = h[MCE_OUT_HIST + i];
        for (uint32_t i = k; i < res->hist_cap; ++i) res->hist[i] = 0;
        if (res->hist_cap <= res->max_size && res->count) return MCE_ETRUNC;
    }
    return MCE_OK;
}

}  // namespace

namespace {
// children / k / count_root: a part of the root's branching (children null:
// the whole search).
struct Sink;
int enumerate_once(mce_graph *g, const mce_options &o, mce_result *res, std::chrono::steady_clock::time_point t0,
                   const uint32_t *children = nullptr, uint32_t k = 0, uint32_t count_root = 1,
                   const Sink *sink = nullptr);
}

namespace {
int enumerate_outer(mce_graph *g, const mce_options &o, mce_result *res, std::chrono::steady_clock::time_point t0);
}

extern "C" int mce_enumerate(mce_graph *g, const mce_options *opts, mce_result *res)
{
    if (!g || !res) return MCE_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    DevicePick pick(g->ctx->device);
    mce_options o = defaults(opts);
    if (!g->d_rows || ((o.flags & MCE_OUTER) && g->n > 0)) {
        if (o.flags & kListFlags) return MCE_ENOTIMPL;
        if (o.pivot_mode > MCE_PIVOT_GREEDY_NX) return MCE_EINVAL;
        return enumerate_outer(g, o, res, t0);
    }
    int rc = enumerate_once(g, o, res, t0);
    // a queue overflow leaves no partial state behind: retry with 16x the slots
    for (int tries = 0; rc == MCE_EOVERFLOW && tries < 2; ++tries) {
        Config c;
        if (choose(g->n, o, c) != MCE_OK) break;
        uint32_t lg = 0;
        while ((1u << lg) < c.qcap) ++lg;
        if (lg + 4 > 24) break;
        o.queue_log2 = lg + 4;
        rc = enumerate_once(g, o, res, t0);
    }
    return rc;
}

extern "C" int mce_root_children(mce_graph *g, const mce_options *opts, uint32_t *sizes, uint32_t cap,
                                 uint32_t *count)
{
    if (!g || !count || (cap && !sizes)) return MCE_EINVAL;
    if (!g->d_rows) return MCE_ENOTIMPL;  // sparse graphs: the outer loop has no single root
    DevicePick pick(g->ctx->device);
    mce_ctx *ctx = g->ctx;
    const mce_options o = defaults(opts);
    if (o.flags & (kListFlags | MCE_OUTER)) return MCE_ENOTIMPL;
    Config c;
    int rc = choose(g->n, o, c);
    if (rc) return rc;
    const Layout L = layout(g->n, c);
    const uint32_t n = g->n;
    // order | renumbered rows (scratch layout) | status words | pivot, count | sizes
    const size_t o_stat = L.rows + round_up((size_t)n * c.wp * 4 + 16, 256);
    const size_t o_piv = o_stat + 256, o_sizes = o_piv + 256;
    const size_t bytes = o_sizes + round_up((size_t)std::max<uint32_t>(n, 1) * 4, 256);
    void *mem = nullptr;
    rc = dalloc(ctx, &mem, bytes);
    if (rc != MCE_OK) return rc;
    unsigned char *m = static_cast<unsigned char *>(mem);
    uint32_t *order = reinterpret_cast<uint32_t *>(m + L.order);
    uint32_t *rows = reinterpret_cast<uint32_t *>(m + L.rows);
    uint64_t *stat = reinterpret_cast<uint64_t *>(m + o_stat);
    unsigned *piv = reinterpret_cast<unsigned *>(m + o_piv);
    uint32_t *d_count = piv + 1;
    uint32_t *d_sizes = reinterpret_cast<uint32_t *>(m + o_sizes);
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemsetAsync(stat, 0, 64, s);
    if (e == cudaSuccess) e = launch_validate_rows(n, g->w, g->d_rows, stat, s);  // status at stat[MCE_OUT_STATUS]
    if (e == cudaSuccess)
        e = (o.flags & MCE_ORDER_IDENTITY) ? launch_identity(n, order, s) : launch_order(n, g->w, g->d_rows, order, s);
    if (e == cudaSuccess) e = launch_renumber(n, g->w, g->d_rows, order, c.wp, rows, s);
    const bool tomita = o.pivot_mode == MCE_PIVOT_TOMITA;
    if (e == cudaSuccess && tomita) e = launch_root_degree_pivot(rows, n, c.wp, piv, s);
    if (e == cudaSuccess) e = launch_root_children(rows, n, c.wp, tomita ? piv : nullptr, d_sizes, n, d_count, s);
    uint64_t st[MCE_OUT_STATUS + 1] = {0};
    uint32_t cnt = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(st, stat, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, d_count, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && st[MCE_OUT_STATUS] == 0 && cnt && cap) {
        e = cudaMemcpyAsync(sizes, d_sizes, (size_t)std::min(cap, cnt) * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    dfree(ctx, mem, bytes, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        return MCE_ECUDA;
    }
    if (st[MCE_OUT_STATUS]) return (int)(int64_t)st[MCE_OUT_STATUS];
    *count = cnt;
    return cnt > cap ? MCE_ETRUNC : MCE_OK;
}

extern "C" int mce_enumerate_part(mce_graph *g, const mce_options *opts, const uint32_t *children, uint32_t k,
                                  int count_root, mce_result *res)
{
    if (!g || !res || (k && !children)) return MCE_EINVAL;
    if (!g->d_rows) return MCE_ENOTIMPL;
    for (uint32_t j = 1; j < k; ++j)
        if (children[j] <= children[j - 1]) return MCE_EINVAL;
    if (k && children[k - 1] >= g->n) return MCE_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    DevicePick pick(g->ctx->device);
    mce_options o = defaults(opts);
    if (o.flags & (kListFlags | MCE_OUTER)) return MCE_ENOTIMPL;
    static const uint32_t none = 0;
    const uint32_t *ch = k ? children : &none;  // non-null marks a part
    int rc = enumerate_once(g, o, res, t0, ch, k, count_root ? 1u : 0u);
    for (int tries = 0; rc == MCE_EOVERFLOW && tries < 2; ++tries) {
        Config c;
        if (choose(g->n, o, c) != MCE_OK) break;
        uint32_t lg = 0;
        while ((1u << lg) < std::max<uint32_t>(c.qcap, 2u * k)) ++lg;
        if (lg + 4 > 24) break;
        o.queue_log2 = lg + 4;
        rc = enumerate_once(g, o, res, t0, ch, k, count_root ? 1u : 0u);
    }
    return rc;
}

namespace {

// Device memory of one listing search: control words, chunk fill counts,
// per-group path and base R, and the record chunks.
struct ListArea {
    void *mem = nullptr;
    size_t bytes = 0;
    ListParams prm{};
};

int list_alloc(mce_ctx *ctx, uint32_t n, const Config &c, const mce_result *res, ListArea &la, cudaStream_t s)
{
    const uint64_t groups = c.total_groups;
    const uint32_t cw = std::max<uint32_t>(2048u, 2u * next_pow2((uint64_t)n + 2u));
    // room for the caller's capacity twice over (chunk tails stay unused) plus
    // one chunk in every group's hands, within 2^32 words and a third of the
    // free memory
    auto sat_add = [](uint64_t x, uint64_t y) { return x + y < x ? ~0ull : x + y; };
    uint64_t want = sat_add(res->list_cap, res->list_off_cap);
    want = sat_add(want, want);
    want = sat_add(want, groups * cw);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return MCE_ECUDA;
    uint64_t cap_words = std::min<uint64_t>((1ull << 32) - cw, free_b / 3 / 4);
    if (ctx->budget) {
        const uint64_t used = ctx->used.load();
        cap_words = std::min<uint64_t>(cap_words, used < ctx->budget ? (ctx->budget - used) / 2 / 4 : 0);
    }
    const uint64_t chunks = std::max<uint64_t>(1, std::min(want, cap_words) / cw);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = round_up(off, 256);
        const size_t at = off;
        off += bytes;
        return at;
    };
    const size_t o_ctl = take(256), o_fill = take(chunks * 4), o_path = take(groups * n * 2 + 2),
                 o_base = take(groups * c.wp * 4), o_rec = take(chunks * (uint64_t)cw * 4);
    la.bytes = round_up(off, 256);
    int rc = dalloc(ctx, &la.mem, la.bytes, s);
    if (rc != MCE_OK) return rc;
    unsigned char *m = static_cast<unsigned char *>(la.mem);
    la.prm.next_chunk = reinterpret_cast<unsigned *>(m + o_ctl);
    la.prm.overflow = reinterpret_cast<unsigned *>(m + o_ctl + 128);
    la.prm.fill = reinterpret_cast<uint32_t *>(m + o_fill);
    la.prm.path = reinterpret_cast<uint16_t *>(m + o_path);
    la.prm.base = reinterpret_cast<uint32_t *>(m + o_base);
    la.prm.rec = reinterpret_cast<uint32_t *>(m + o_rec);
    la.prm.n_chunks = (uint32_t)chunks;
    la.prm.chunk_words = cw;
    return cuda_code(cudaMemsetAsync(m, 0, o_path, s));  // control words and fill counts
}

constexpr size_t kStageBytes = 32u << 20;  // one pinned staging half

// memcpy split over up to 8 host threads (a pageable destination is written
// at the speed of the threads that touch it); a part whose thread cannot be
// started is copied by the caller.
void host_copy(unsigned char *dst, const unsigned char *src, size_t bytes)
{
    const unsigned t = (unsigned)std::min<size_t>(8, std::max<size_t>(1, bytes >> 22));
    const size_t part = (bytes + t - 1) / t;
    std::vector<std::thread> th;
    th.reserve(t);
    for (unsigned i = 1; i < t; ++i) {
        const size_t b = i * part, e = std::min(bytes, b + part);
        if (b >= e) continue;
        try {
            th.emplace_back([=] { std::memcpy(dst + b, src + b, e - b); });
        } catch (...) {
            std::memcpy(dst + b, src + b, e - b);
        }
    }
    std::memcpy(dst, src, std::min(bytes, part));
    for (auto &x : th) x.join();
}

// Device-to-host copy, complete on return.  A pinned or registered
// destination takes one copy; a large pageable one goes through the
// context's two pinned staging halves, the device copy of each chunk
// overlapping the host copy of the one before.
cudaError_t copy_to_host(mce_ctx *ctx, void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    cudaPointerAttributes at{};
    const bool pinned = cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeHost;
    cudaGetLastError();
    if (pinned || bytes < kStageBytes) {
        const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
        return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
    }
    std::lock_guard<std::mutex> lk(ctx->stage_mu);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        if (!ctx->stage[i]) e = cudaHostAlloc(&ctx->stage[i], kStageBytes, cudaHostAllocDefault);
        if (e == cudaSuccess && !ctx->stage_ev[i])
            e = cudaEventCreateWithFlags(&ctx->stage_ev[i], cudaEventDisableTiming);
    }
    unsigned char *d = static_cast<unsigned char *>(dst);
    const unsigned char *sp = static_cast<const unsigned char *>(src);
    const size_t chunks = (bytes + kStageBytes - 1) / kStageBytes;
    for (size_t i = 0; i <= chunks && e == cudaSuccess; ++i) {
        if (i < chunks) {  // half i & 1 was emptied by the host copy of chunk i - 2
            const size_t off = i * kStageBytes;
            e = cudaMemcpyAsync(ctx->stage[i & 1], sp + off, std::min(kStageBytes, bytes - off),
                                cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->stage_ev[i & 1], s);
        }
        if (e == cudaSuccess && i > 0) {
            const size_t j = i - 1, off = j * kStageBytes;
            e = cudaEventSynchronize(ctx->stage_ev[j & 1]);
            if (e == cudaSuccess)
                host_copy(d + off, static_cast<const unsigned char *>(ctx->stage[j & 1]),
                          std::min(kStageBytes, bytes - off));
        }
    }
    if (e != cudaSuccess) cudaStreamSynchronize(s);  // no copy into a staging half stays in flight
    return e;
}

// CSR listing from a finished listing search (result words h) into the
// caller's host buffers.
// A caller's sink of listed cliques (mce_enumerate_stream), or none.
struct Sink {
    mce_clique_sink fn = nullptr;
    void *user = nullptr;
};

// The device CSR (ids, off; count cliques) to the sink in chunks that fit
// the context's pinned staging halves: offsets of up to 2^20 cliques in one
// half, their member ids in the other; the offsets handed over are rebased
// to the chunk.  A non-zero return of the sink stops the stream.
int stream_to_sink(mce_ctx *ctx, const uint32_t *d_ids, const uint64_t *d_off, uint64_t count, const Sink &sk,
                   cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(ctx->stage_mu);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        if (!ctx->stage[i]) e = cudaHostAlloc(&ctx->stage[i], kStageBytes, cudaHostAllocDefault);
    if (e != cudaSuccess) return MCE_ENOMEM;
    uint64_t *hoff = static_cast<uint64_t *>(ctx->stage[0]);
    uint32_t *hids = static_cast<uint32_t *>(ctx->stage[1]);
    const uint64_t max_cliques = std::min<uint64_t>(1u << 20, kStageBytes / 8 - 1);
    for (uint64_t c0 = 0; c0 < count;) {
        uint64_t k = std::min<uint64_t>(count - c0, max_cliques);
        e = cudaMemcpyAsync(hoff, d_off + c0, (k + 1) * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return MCE_ECUDA;
        const uint64_t base = hoff[0];
        while (k > 1 && (hoff[k] - base) * 4 > kStageBytes) k = (k + 1) / 2;  // members must fit one half
        const uint64_t nid = hoff[k] - base;
        if (nid * 4 > kStageBytes) return MCE_ENOMEM;  // one clique larger than a staging half
        e = cudaMemcpyAsync(hids, d_ids + base, nid * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return MCE_ECUDA;
        for (uint64_t i = 0; i <= k; ++i) hoff[i] -= base;
        if (sk.fn(hids, hoff, k, sk.user) != 0) break;
        c0 += k;
    }
    return MCE_OK;
}

int list_deliver(mce_ctx *ctx, uint32_t n, const ListArea &la, const uint32_t *d_order,
                 const std::vector<uint64_t> &h, bool sorted, mce_result *res, cudaStream_t s,
                 const Sink &sk = Sink{})
{
    const uint64_t count = h[MCE_OUT_COUNT];
    uint64_t ids = 0;
    for (uint32_t k = 0; k <= n; ++k) ids += (uint64_t)k * h[MCE_OUT_HIST + k];
    res->list_ids_needed = ids;
    unsigned ctl[2] = {0u, 0u};
    cudaError_t e = cudaMemcpyAsync(&ctl[0], la.prm.next_chunk, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl[1], la.prm.overflow, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return MCE_ECUDA;
    const bool fits = sk.fn || (res->list_off && res->list_off_cap >= count + 1 &&
                                (ids == 0 || (res->list_ids && res->list_cap >= ids)));
    if (!fits) return MCE_ETRUNC;
    if (ctl[1]) return MCE_ENOMEM;  // the caller's buffers fit, the device records did not
    if (n == 0) {                   // the empty set, reported by the root
        uint64_t off[2] = {0, 0};
        if (sk.fn) sk.fn(nullptr, off, 1, sk.user);
        else res->list_off[0] = res->list_off[1] = 0;
        return MCE_OK;
    }
    ListJob j{};
    j.rec = la.prm.rec;
    j.fill = la.prm.fill;
    j.chunks = std::min<uint32_t>(ctl[0], la.prm.n_chunks);
    j.chunk_words = la.prm.chunk_words;
    j.order = d_order;
    j.n = n;
    j.max_size = (uint32_t)h[MCE_OUT_MAX_SIZE];
    j.count = count;
    j.ids = ids;
    j.sorted = sorted;
    if (sorted && count > 0xffffffffull) return MCE_ENOTIMPL;
    const size_t tb = list_temp_bytes(count, ids, j.chunks, sorted);
    const size_t ib = round_up(std::max<uint64_t>(ids, 1) * 4, 256), ob = round_up((count + 1) * 8, 256);
    void *mem = nullptr;
    int rc = dalloc(ctx, &mem, ib + ob + tb, s);
    if (rc != MCE_OK) return rc;
    unsigned char *m = static_cast<unsigned char *>(mem);
    j.ids_out = reinterpret_cast<uint32_t *>(m);
    j.off_out = reinterpret_cast<uint64_t *>(m + ib);
    j.temp = m + ib + ob;
    j.temp_bytes = tb;
    e = list_build(j, s);
    if (sk.fn) {
        rc = e == cudaSuccess ? stream_to_sink(ctx, j.ids_out, j.off_out, count, sk, s) : MCE_ECUDA;
        dfree(ctx, mem, ib + ob + tb, s);
        return rc;
    }
    if (e == cudaSuccess) e = copy_to_host(ctx, res->list_ids, j.ids_out, ids * 4, s);
    if (e == cudaSuccess) e = copy_to_host(ctx, res->list_off, j.off_out, (count + 1) * 8, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(ctx, mem, ib + ob + tb, s);
    return e == cudaSuccess ? MCE_OK : MCE_ECUDA;
}

int enumerate_once(mce_graph *g, const mce_options &o, mce_result *res, std::chrono::steady_clock::time_point t0,
                   const uint32_t *children, uint32_t k, uint32_t count_root, const Sink *sink)
{
    mce_ctx *ctx = g->ctx;
    const bool listing = (o.flags & kListFlags) != 0u;
    Config c;
    int rc = choose(g->n, o, c);
    if (rc) return rc;
    if (children && c.qcap < 2u * k) c.qcap = next_pow2(2ull * k);  // every child frame queued at once
    const Layout L = layout(g->n, c);
    const uint64_t sbytes = L.total + (children ? round_up((size_t)k * 4 + 4, 256) : 0);
    const size_t obytes = MCE_OUT_WORDS(g->n) * 8;
    void *scr = nullptr;
    uint64_t *d_out = nullptr;
    ListArea la;
    PartSpec part{nullptr, k, count_root};
    rc = dalloc(ctx, &scr, sbytes);
    if (rc == MCE_OK && children) {
        uint32_t *dc = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(scr) + L.total);
        part.d_children = dc;
        if (k && cudaMemcpyAsync(dc, children, (size_t)k * 4, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
            rc = MCE_ECUDA;
    }
    if (rc == MCE_OK) rc = dalloc(ctx, (void **)&d_out, obytes);
    if (rc == MCE_OK && listing) rc = list_alloc(ctx, g->n, c, res, la, ctx->stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<uint64_t> h(MCE_OUT_WORDS(g->n), 0);
    if (rc == MCE_OK) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, ctx->stream);
        rc = enumerate_device_impl(g->n, g->w, g->d_rows, o, c, L, static_cast<unsigned char *>(scr), d_out, ctx->stream,
                                   listing ? &la.prm : nullptr, children ? &part : nullptr);
        cudaEventRecord(e1, ctx->stream);
        if (rc == MCE_OK) {
            cudaError_t e = cudaMemcpyAsync(h.data(), d_out, obytes, cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) rc = MCE_ECUDA;
        }
    }
    float kms = 0.f;
    if (rc == MCE_OK && e0 && e1) cudaEventElapsedTime(&kms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const bool ran = rc == MCE_OK;
    if (ran) {
        rc = fill_result(h, g->n, res);
        res->kernel_ms = kms;
        if (listing && rc == MCE_OK) {
            const uint32_t *d_order = reinterpret_cast<const uint32_t *>(static_cast<unsigned char *>(scr) + L.order);
            rc = list_deliver(ctx, g->n, la, d_order, h, (o.flags & MCE_LIST_SORTED) != 0u, res, ctx->stream,
                              sink ? *sink : Sink{});
        }
    }
    if (la.mem) dfree(ctx, la.mem, la.bytes, ctx->stream);
    dfree(ctx, d_out, obytes);
    dfree(ctx, scr, sbytes);
    if (!ran) {
        cudaStreamSynchronize(ctx->stream);
        return rc;
    }
    res->total_ms = ms_since(t0);
    return rc;
}
}  // namespace

extern "C" int mce_enumerate_stream(mce_graph *g, const mce_options *opts, mce_clique_sink sink, void *user,
                                    mce_result *res)
{
    if (!g || !sink || !res) return MCE_EINVAL;
    if (!g->d_rows) return MCE_ENOTIMPL;
    const auto t0 = std::chrono::steady_clock::now();
    DevicePick pick(g->ctx->device);
    mce_options o = defaults(opts);
    if (o.flags & MCE_OUTER) return MCE_ENOTIMPL;
    if (!(o.flags & kListFlags)) o.flags |= MCE_LIST;
    // a counting search first: the listing search's device records are then
    // sized exactly (count cliques, sum of sizes member ids)
    mce_options oc = o;
    oc.flags &= ~kListFlags;
    std::vector<uint64_t> hist((size_t)g->n + 1, 0);
    mce_result r0{};
    r0.hist = hist.data();
    r0.hist_cap = g->n + 1;
    int rc = mce_enumerate(g, &oc, &r0);
    if (rc != MCE_OK) return rc;
    uint64_t ids = 0;
    for (uint32_t k = 0; k <= g->n; ++k) ids += (uint64_t)k * hist[k];
    mce_result rl = *res;
    rl.list_ids = nullptr;
    rl.list_cap = ids;
    rl.list_off = nullptr;
    rl.list_off_cap = r0.count + 1;
    const Sink sk{sink, user};
    rc = enumerate_once(g, o, &rl, t0, nullptr, 0, 1, &sk);
    for (int tries = 0; rc == MCE_EOVERFLOW && tries < 2; ++tries) {
        Config c;
        if (choose(g->n, o, c) != MCE_OK) break;
        uint32_t lg = 0;
        while ((1u << lg) < c.qcap) ++lg;
        if (lg + 4 > 24) break;
        o.queue_log2 = lg + 4;
        rc = enumerate_once(g, o, &rl, t0, nullptr, 0, 1, &sk);
    }
    rl.list_ids = res->list_ids;
    rl.list_cap = res->list_cap;
    rl.list_off = res->list_off;
    rl.list_off_cap = res->list_off_cap;
    *res = rl;
    return rc;
}

// ---------------------------------------------------------------------------
// Batched form

struct mce_batch {
    mce_ctx *ctx = nullptr;
    uint32_t count = 0;
    std::vector<uint32_t> n;
    std::vector<size_t> out_off;  // words into d_out
    size_t out_words = 0;
    void *dmem = nullptr;
    size_t dbytes = 0;
    uint64_t *d_out = nullptr;
    std::vector<uint64_t> h_out;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> events;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    std::vector<mce_batch_bucket> info;  // launch choice of every bucket
    const BatchGraph *d_table = nullptr;
    cudaStream_t stream = nullptr;       // where it is planned and launched
};

namespace {

// Expected number of maximal cliques of G(n, p) (sum over clique sizes k of
// C(n,k) p^C(k,2) (1 - p^k)^(n-k)): the cost key that orders a batch.
double expected_cliques(uint32_t n, uint64_t m)
{
    if (n < 2) return 1.0;
    const double p = std::min(1.0, (double)m / (0.5 * n * (n - 1.0)));
    if (p <= 0.0) return n;
    if (p >= 1.0) return 1.0;
    double total = 0.0;
    const double ln = std::lgamma(n + 1.0), lp = std::log(p);
    for (uint32_t k = 1; k <= n; ++k) {
        const double t = ln - std::lgamma(k + 1.0) - std::lgamma(n - k + 1.0) + 0.5 * k * (k - 1.0) * lp +
                         (n - k) * std::log1p(-std::pow(p, (double)k));
        total += std::exp(t);
    }
    return total + n;
}

struct Bucket {
    int G = 0, K = 0;
    unsigned threads = 0;
    uint32_t split = 0, wclass = 0;
    bool tuned = false;
    double tuned_ms = 0.0;
    bool smem = false;
    std::vector<uint32_t> graphs;
    std::vector<uint32_t> items;  // work items: graph | part << 16 | parts << 24
    uint32_t split_graphs = 0;
    SearchImpl impl{nullptr, nullptr, nullptr, nullptr};
    LaunchShape shape{};
    uint32_t qcap = 0, fs = 0, groups = 0;
    uint32_t stack_levels = 0, stack_offset = 0;
    uint32_t t2_offset = 0, t2_levels = 0, t2_max_p = 0;  // lane tier (t2_max_p 0: off)
    size_t qstride = 0, list_off = 0, region_off = 0, next_off = 0;
};

void batch_free(mce_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    if (b->dmem) dfree(b->ctx, b->dmem, b->dbytes, b->stream);
    cudaStreamSynchronize(b->stream);
    delete b;
}

}  // namespace

namespace {

// Words-per-row class of n vertices: the smallest c with W <= 2^c.
uint32_t words_class(uint32_t n)
{
    const uint32_t W = std::max<uint32_t>(1, (n + 31) / 32);
    uint32_t c = 0;
    while ((1u << c) < W) ++c;
    return c;
}

// Work items of a bucket whose graphs are sorted most expensive first.  With
// target = the bucket's expected cost / (blocks * div), a graph expected to
// cost more than twice the target (with div = 4: half a block's fair share)
// is split into k parts of about the target: part j searches the root's children j, j + k, j + 2k, ... (disjoint
// subtrees of Alg. 4's root), so the heaviest graphs of a batch no longer run
// on one block while the others idle.  k is capped by about half the
// expected number of root children (|P \ N(pivot)| ~ n(1 - p)), by
// kBatchMaxParts and by the kernel's prefix table (kBatchPartWords words per
// row); subproblems of the outer loop are never split.  Items are sorted by
// expected cost, largest first.  Returns the most child frames one part
// queues at its start (0 when nothing is split), which the ring must hold.
constexpr uint32_t kBatchMaxParts = 64;

uint32_t plan_items(Bucket &bk, mce_graph *const *graphs, const std::vector<double> &cost,
                    const std::vector<uint32_t> &wp_of, unsigned blocks, uint32_t div)
{
    double total = 0.0;
    for (uint32_t i : bk.graphs) total += cost[i];
    const double target = blocks && div ? total / ((double)div * blocks) : 0.0;
    std::vector<std::pair<double, uint32_t>> items;
    uint32_t frames = 0;
    for (uint32_t i : bk.graphs) {
        const mce_graph *g = graphs[i];
        uint32_t k = 1;
        if (!g->root && target > 0.0 && cost[i] > 2.0 * target && wp_of[i] <= (uint32_t)kBatchPartWords && g->n > 1) {
            const double p = std::min(1.0, 2.0 * (double)g->m / ((double)g->n * (g->n - 1.0)));
            const double children = 0.5 * g->n * (1.0 - p);
            const double cap = std::min<double>(kBatchMaxParts, std::max(1.0, children));
            k = (uint32_t)std::min(cap, std::ceil(cost[i] / target));
        }
        for (uint32_t j = 0; j < k; ++j) items.push_back({cost[i] / k, i | (j << 16) | (k << 24)});
        if (k >= 2) {
            frames = std::max(frames, (g->n + k - 1) / k + 1);
            ++bk.split_graphs;
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, uint32_t> &a, const std::pair<double, uint32_t> &c) {
                         return a.first > c.first;
                     });
    bk.items.clear();
    for (auto &it : items) bk.items.push_back(it.second);
    return frames;
}

// Launch choice of a batched graph without a tuned one: forced shapes as
// given; otherwise 512 threads and subtrees of at most two words per lane
// (one up to 128 vertices), the pattern the autotuner settled on for every
// words class of the mixed 4,096-graph workload (more, narrower subtrees per
// block than the plain form's shapes: a batched graph has no device-wide ring
// to spread its work, so a block needs many subtrees of its own).
TuneChoice default_choice(uint32_t n, const mce_options &o, bool wide)
{
    TuneChoice t;
    pick_shape(n, o, t.G, t.K);
    t.threads = o.threads_per_block ? o.threads_per_block : 256u;
    if (wide && default_tuning().batch_wide && !o.lanes_per_subtree && !o.words_per_lane) {
        const uint32_t W = std::max<uint32_t>(1, (n + 31) / 32);
        t.K = W <= 4 ? 1 : (W <= 64 ? 2 : 4);
        t.G = 1;
        while ((uint32_t)(t.G * t.K) < W) t.G <<= 1;
        if (!o.threads_per_block) t.threads = kMaxThreads;
    }
    t.split = o.split_min_p;
    return t;
}

// Plan and capture a batch with the launch choice of every words class
// given in `choice` (classes not in it: the defaults).
// subproblems: a batch of the outer loop's many small subproblems (Alg. 3):
// untuned graphs take the plain form's shapes instead of default_choice's
// wide ones, and no lane tier (on G(10000, p) with p = 0.01 / 0.03 the lane
// tier made the batch 5.8 / 19.5 ms against 3.9 / 17.1 ms without it: a
// subproblem's frames are small from the start, and the tier's region costs
// the block its stack levels in shared memory).
int batch_create_impl(mce_ctx *ctx, mce_graph *const *graphs, uint32_t count, const mce_options &o,
                      const std::map<uint32_t, TuneChoice> &choice, mce_batch **out,
                      cudaStream_t stream = nullptr, bool subproblems = false);

// Milliseconds of one launch of a batch planned with `choice` (the second of
// two launches), or a negative value if it cannot run.
double time_choices(mce_ctx *ctx, const std::vector<mce_graph *> &graphs, const mce_options &o,
                    const std::map<uint32_t, TuneChoice> &choice)
{
    mce_batch *b = nullptr;
    if (batch_create_impl(ctx, graphs.data(), (uint32_t)graphs.size(), o, choice, &b) != MCE_OK) return -1.0;
    double ms = -1.0;
    if (mce_batch_run(b, nullptr) == MCE_OK && mce_batch_run(b, nullptr) == MCE_OK) {
        float f = 0.f;
        if (cudaEventElapsedTime(&f, b->t0, b->t1) == cudaSuccess) ms = f;
    }
    mce_batch_destroy(b);
    return ms;
}

// Coordinate descent over the words classes that have no cached choice:
// classes in decreasing order of expected work; for each, every candidate
// (1, 2 or 4 words per lane with the fewest lanes that hold a row; 128, 256
// or 512 threads; then the best with breadth-first split off) is timed on
// the whole batch (up to 4096 of its graphs, sampled evenly) with the other
// classes at their current choice, and the fastest is kept.
void tune_batch(mce_ctx *ctx, mce_graph *const *graphs, uint32_t count, const mce_options &o,
                const std::vector<double> &cost, std::map<uint32_t, TuneChoice> &choice)
{
    std::map<uint32_t, double> work;
    std::map<uint32_t, uint32_t> members;
    for (uint32_t i = 0; i < count; ++i) {
        const uint32_t c = words_class(graphs[i]->n);
        work[c] += cost[i];
        ++members[c];
    }
    std::vector<mce_graph *> sample;
    const uint32_t take = std::min<uint32_t>(count, 4096);
    for (uint32_t j = 0; j < take; ++j) sample.push_back(graphs[(uint64_t)j * count / take]);
    std::vector<std::pair<double, uint32_t>> order;
    for (auto &kv : work)
        if (!choice.count(kv.first) && members[kv.first] >= 16) order.push_back({kv.second, kv.first});
    std::sort(order.rbegin(), order.rend());
    for (auto &oc : order) {
        const uint32_t c = oc.second, W = 1u << c;
        TuneChoice best;
        double best_ms = -1.0;
        auto consider = [&](TuneChoice t) {
            auto trial = choice;
            trial[c] = t;
            const double ms = time_choices(ctx, sample, o, trial);
            if (ms >= 0.0 && (best_ms < 0.0 || ms < best_ms)) {
                best_ms = ms;
                best = t;
            }
        };
        for (int K : {1, 2, 4}) {
            uint32_t G = 1;
            while (G * (uint32_t)K < W) G <<= 1;
            if (G > 32) continue;
            for (unsigned threads : {128u, 256u, 512u}) {
                TuneChoice t;
                t.G = (int)G;
                t.K = K;
                t.threads = threads;
                t.split = o.split_min_p;
                consider(t);
            }
        }
        if (best_ms < 0.0) continue;
        TuneChoice t = best;
        t.split = 0xffffffffu;
        consider(t);
        best.tuned = true;
        best.ms_per_graph = best_ms / (double)sample.size();
        choice[c] = best;
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        ctx->tuned[c * 4u + o.pivot_mode] = best;
    }
}

}  // namespace

extern "C" int mce_batch_buckets(const mce_batch *b, mce_batch_bucket *out, uint32_t cap, uint32_t *count)
{
    if (!b || !count || (cap && !out)) return MCE_EINVAL;
    *count = (uint32_t)b->info.size();
    for (uint32_t i = 0; i < cap && i < b->info.size(); ++i) out[i] = b->info[i];
    return MCE_OK;
}

extern "C" int mce_batch_create(mce_ctx *ctx, mce_graph *const *graphs, uint32_t count, const mce_options *opts,
                                mce_batch **out)
{
    if (!ctx || !out || (count && !graphs) || count > 65535u) return MCE_EINVAL;
    *out = nullptr;
    DevicePick pick(ctx->device);
    const mce_options o = defaults(opts);
    if (o.pivot_mode > MCE_PIVOT_GREEDY_NX || o.stack_levels > (uint32_t)kStackDepth || o.queue_log2 > 24)
        return MCE_EINVAL;
    if (o.flags & (MCE_LIST | MCE_LIST_SORTED)) return MCE_ENOTIMPL;
    for (uint32_t i = 0; i < count; ++i)
        if (!graphs[i] || graphs[i]->ctx != ctx || !graphs[i]->d_rows) return MCE_EINVAL;
    // autotuning: cached choices first, the rest measured on this batch
    std::map<uint32_t, TuneChoice> choice;
    const bool forced = o.lanes_per_subtree || o.words_per_lane || o.threads_per_block || o.split_min_p;
    if ((o.flags & MCE_AUTOTUNE) && !forced) {
        std::vector<double> cost(count);
        for (uint32_t i = 0; i < count; ++i) {
            cost[i] = expected_cliques(graphs[i]->n, graphs[i]->m);
            const uint32_t key = words_class(graphs[i]->n) * 4u + o.pivot_mode;
            std::lock_guard<std::mutex> lk(ctx->tune_mu);
            auto it = ctx->tuned.find(key);
            if (it != ctx->tuned.end()) choice[words_class(graphs[i]->n)] = it->second;
        }
        tune_batch(ctx, graphs, count, o, cost, choice);
    }
    return batch_create_impl(ctx, graphs, count, o, choice, out);
}

namespace {

int batch_create_impl(mce_ctx *ctx, mce_graph *const *graphs, uint32_t count, const mce_options &o,
                      const std::map<uint32_t, TuneChoice> &choice, mce_batch **out, cudaStream_t stream,
                      bool subproblems)
{
    *out = nullptr;
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))
        return MCE_ECUDA;
    const size_t slimit = (size_t)optin - 1024;

    mce_batch *b = new (std::nothrow) mce_batch;
    if (!b) return MCE_ENOMEM;
    b->ctx = ctx;
    b->stream = stream ? stream : ctx->stream;
    b->count = count;
    b->n.resize(count);

    // ---- plan: a launch choice per graph (given per words class, else the
    // defaults), buckets of equal choice, most expensive first
    std::vector<Bucket> buckets;
    std::vector<double> cost(count);
    uint32_t max_n = 0, max_w = 0, max_wp = 0;
    std::vector<uint32_t> wp_of(count);
    for (uint32_t i = 0; i < count; ++i) {
        const mce_graph *g = graphs[i];
        if (!g || g->ctx != ctx || !g->d_rows) { delete b; return MCE_EINVAL; }
        cost[i] = g->cost_hint > 0.0 ? g->cost_hint : expected_cliques(g->n, g->m);
    }
    for (uint32_t i = 0; i < count; ++i) {
        const mce_graph *g = graphs[i];
        b->n[i] = g->n;
        const uint32_t W = std::max<uint32_t>(1, (g->n + 31) / 32);
        const uint32_t wc = words_class(g->n);
        auto it = choice.find(wc);
        const TuneChoice t = it != choice.end() ? it->second : default_choice(g->n, o, !subproblems);
        const int G = t.G, K = t.K;
        if ((uint32_t)(G * K) < W || !impl_for(G, K, false, (int)o.pivot_mode).run) { delete b; return MCE_EINVAL; }
        size_t bi = 0;
        while (bi < buckets.size() && !(buckets[bi].G == G && buckets[bi].K == K && buckets[bi].threads == t.threads &&
                                        buckets[bi].split == t.split))
            ++bi;
        if (bi == buckets.size()) {
            Bucket nb;
            nb.G = G;
            nb.K = K;
            nb.threads = t.threads;
            nb.split = t.split;
            nb.wclass = wc;
            nb.tuned = t.tuned;
            nb.tuned_ms = t.ms_per_graph;
            nb.smem = G * K <= 32;
            buckets.push_back(nb);
        }
        buckets[bi].wclass = std::max(buckets[bi].wclass, wc);
        buckets[bi].graphs.push_back(i);
        wp_of[i] = (uint32_t)(G * K);
        max_n = std::max(max_n, g->n);
        max_w = std::max(max_w, g->w);
        max_wp = std::max(max_wp, wp_of[i]);
    }

    // ---- launch shapes and the device memory layout
    size_t off = 0;
    auto take = [&](size_t bytes, size_t align) {
        off = round_up(off, align);
        const size_t at = off;
        off += bytes;
        return at;
    };
    const size_t table_off = take(sizeof(BatchGraph) * std::max<uint32_t>(count, 1), 256);
    std::vector<size_t> order_off(count), ren_off(count);
    b->out_off.resize(count);
    for (uint32_t i = 0; i < count; ++i) order_off[i] = take((size_t)std::max<uint32_t>(b->n[i], 1) * 4, 16);
    for (uint32_t i = 0; i < count; ++i) ren_off[i] = take((size_t)b->n[i] * wp_of[i] * 4 + 16, 256);
    const size_t out_at = take(0, 256);
    for (uint32_t i = 0; i < count; ++i) {
        b->out_off[i] = b->out_words;
        b->out_words += MCE_OUT_WORDS(b->n[i]);
    }
    off += b->out_words * 8;
    int rc = MCE_OK;
    for (Bucket &bk : buckets) {
        std::stable_sort(bk.graphs.begin(), bk.graphs.end(), [&](uint32_t a, uint32_t c2) { return cost[a] > cost[c2]; });
        bk.impl = impl_for(bk.G, bk.K, bk.smem, (int)o.pivot_mode);
        size_t base = 0;
        for (uint32_t i : bk.graphs) base = std::max(base, search_smem(b->n[i], (uint32_t)(bk.G * bk.K), bk.smem));
        const unsigned threads = bk.threads;
        if (threads % 32 || threads > kMaxThreads) { rc = MCE_EINVAL; break; }
        // the lane tier's region (groups of two or more lanes) when it fits,
        // then at most 56 KB of stack per block, so that several blocks share
        // an SM
        const Tuning tu = default_tuning();
        if (bk.G >= 2 && tu.t2_p != 0u && !subproblems) {
            const size_t off = round_up(base, 16), t2b = (size_t)(threads / 32) * t2_warp_bytes(tu.t2_levels, o.pivot_mode != MCE_PIVOT_GREEDY);
            if (off + t2b <= slimit) {
                bk.t2_offset = (uint32_t)off;
                bk.t2_levels = tu.t2_levels;
                bk.t2_max_p = tu.t2_p;
                base = off + t2b;
            }
        }
        size_t smem = 0;
        plan_stack_for((uint32_t)base, bk.G, bk.K, threads, std::min<size_t>(slimit, base + 56 * 1024),
                       bk.stack_levels, bk.stack_offset, smem);
        int per_sm = 0;
        if (bk.impl.batch_occupancy((int)threads, smem, &per_sm) != cudaSuccess || per_sm < 1) { rc = MCE_EINVAL; break; }
        unsigned blocks = o.blocks ? o.blocks : (unsigned)(per_sm * sms);
        const uint32_t part_frames = plan_items(bk, graphs, cost, wp_of, blocks, default_tuning().batch_split);
        blocks = std::min<unsigned>(blocks, (unsigned)bk.items.size());
        bk.shape = LaunchShape{blocks, threads, smem, bk.smem};
        bk.groups = threads / 32 * (32 / bk.G);
        bk.qcap = next_pow2(std::max<uint64_t>(256, 4ull * bk.groups + 64 + part_frames));
        if (o.queue_log2) bk.qcap = std::max<uint32_t>(bk.qcap, 1u << o.queue_log2);
        bk.fs = (uint32_t)frame_words((uint32_t)(bk.G * bk.K));
        bk.qstride = batch_region_bytes(bk.qcap, bk.fs);
        bk.list_off = take(bk.items.size() * 4, 16);
        bk.next_off = take(4, 128);
        bk.region_off = take(bk.qstride * blocks, 256);
    }
    if (rc != MCE_OK) { delete b; return rc; }
    for (const Bucket &bk : buckets) {
        mce_batch_bucket bi{};
        bi.words_class = 1u << bk.wclass;
        bi.graphs = (uint32_t)bk.graphs.size();
        bi.lanes_per_subtree = (uint32_t)bk.G;
        bi.words_per_lane = (uint32_t)bk.K;
        bi.threads_per_block = bk.threads;
        bi.blocks = bk.shape.blocks;
        bi.split_min_p = bk.split;
        bi.tuned = bk.tuned ? 1u : 0u;
        bi.tuned_ms_per_graph = bk.tuned_ms;
        bi.work_items = (uint32_t)bk.items.size();
        bi.split_graphs = bk.split_graphs;
        b->info.push_back(bi);
    }
    b->dbytes = round_up(off, 256);
    rc = dalloc(ctx, &b->dmem, b->dbytes, b->stream);
    if (rc != MCE_OK) { delete b; return rc; }
    unsigned char *base = static_cast<unsigned char *>(b->dmem);
    b->d_out = reinterpret_cast<uint64_t *>(base + out_at);

    // ---- tables
    std::vector<BatchGraph> table(count);
    for (uint32_t i = 0; i < count; ++i) {
        BatchGraph &t = table[i];
        t.rows = graphs[i]->d_rows;
        t.order = reinterpret_cast<uint32_t *>(base + order_off[i]);
        t.ren = reinterpret_cast<uint32_t *>(base + ren_off[i]);
        t.out = b->d_out + b->out_off[i];
        t.n = b->n[i];
        t.w = graphs[i]->w;
        t.wp = wp_of[i];
        t.pad = 0;
        t.label = graphs[i]->label;
        t.root = graphs[i]->root;
        t.rv = graphs[i]->rv;
        t.pad2 = 0;
    }
    cudaStream_t s = b->stream;
    cudaError_t e = cudaSuccess;
    if (count) e = cudaMemcpyAsync(base + table_off, table.data(), sizeof(BatchGraph) * count, cudaMemcpyHostToDevice, s);
    for (const Bucket &bk : buckets)
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + bk.list_off, bk.items.data(), bk.items.size() * 4, cudaMemcpyHostToDevice, s);
    size_t order_smem = 0;
    if (e == cudaSuccess) e = prepare_order_batch(max_n, max_w, &order_smem);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t i = 0; e == cudaSuccess && i < buckets.size(); ++i) {
        cudaStream_t ss = nullptr;
        e = cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->side.push_back(ss);
    }
    for (size_t i = 0; e == cudaSuccess && i < buckets.size() + 1; ++i) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->events.push_back(ev);
    }
    if (e == cudaSuccess) e = cudaEventCreate(&b->t0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t1);

    // ---- capture: clear results, order, renumber, then one persistent
    // search launch per shape, forked so their tails overlap
    const BatchGraph *d_table = reinterpret_cast<const BatchGraph *>(base + table_off);
    b->d_table = d_table;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t ce = cudaMemsetAsync(b->d_out, 0, b->out_words * 8, s);
        for (const Bucket &bk : buckets)
            if (ce == cudaSuccess) ce = cudaMemsetAsync(base + bk.next_off, 0, 4, s);
        if (ce == cudaSuccess) ce = launch_order_batch(d_table, count, max_n, order_smem, s);
        if (ce == cudaSuccess) ce = launch_renumber_batch(d_table, count, max_n, max_wp, s);
        if (ce == cudaSuccess) ce = cudaEventRecord(b->events[0], s);
        for (size_t i = 0; ce == cudaSuccess && i < buckets.size(); ++i) {
            const Bucket &bk = buckets[i];
            BatchParams bp{};
            bp.graphs = d_table;
            bp.list = reinterpret_cast<const uint32_t *>(base + bk.list_off);
            bp.count = (uint32_t)bk.items.size();
            bp.next = reinterpret_cast<unsigned *>(base + bk.next_off);
            bp.qbase = base + bk.region_off;
            bp.qstride = bk.qstride;
            bp.qcap = bk.qcap;
            bp.fs = bk.fs;
            bp.timeout_ns = o.timeout_ns ? o.timeout_ns : 60ull * 1000000000ull;
            bp.pivot_mode = o.pivot_mode;
            bp.stack_levels = o.stack_levels ? std::min<uint32_t>(o.stack_levels, kStackDepth) : kStackDepth;
            bp.groups_per_block = bk.groups;
            bp.split_min_p = bk.split;
            bp.split_target = bk.qcap / 2;
            bp.stack_smem_levels = bk.stack_levels;
            bp.stack_offset = bk.stack_offset;
            bp.tune = default_tuning();
            bp.tune.small_split = 0u;  // the batched form ran 6 % slower with it
            bp.t2_offset = bk.t2_offset;
            bp.t2_levels = bk.t2_levels;
            bp.t2_max_p = bk.t2_max_p;
            ce = cudaStreamWaitEvent(b->side[i], b->events[0], 0);
            if (ce == cudaSuccess) ce = bk.impl.run_batch(bp, bk.shape, b->side[i]);
            if (ce == cudaSuccess) ce = cudaEventRecord(b->events[i + 1], b->side[i]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, b->events[i + 1], 0);
        }
        cudaGraph_t gr = nullptr;
        e = cudaStreamEndCapture(s, &gr);
        if (e == cudaSuccess) e = ce;
        b->graph = gr;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return MCE_ECUDA;
    }
    *out = b;
    return MCE_OK;
}

}  // namespace

namespace {

// Alg. 3's outer loop: CSR, degeneracy order, one subproblem per vertex
// (rows, labels and root sets extracted on the device), all subproblems
// searched as one batch, their results summed.
int enumerate_outer(mce_graph *g, const mce_options &o, mce_result *res, std::chrono::steady_clock::time_point t0)
{
    mce_ctx *ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    const uint32_t n = g->n;
    int rc = MCE_OK;
    cudaError_t e = cudaSuccess;
    if (!g->d_off) {  // bitset graph: CSR built once from its rows
        size_t need = 0;
        outer_csr_from_rows(n, g->w, g->d_rows, nullptr, nullptr, nullptr, 0, &need, s);
        void *temp = nullptr;
        uint32_t *off = nullptr;
        const uint64_t offb = round_up(((uint64_t)n + 1) * 4, 256);
        rc = dalloc(ctx, &temp, need);
        if (rc == MCE_OK) rc = dalloc(ctx, (void **)&off, offb);
        if (rc == MCE_OK) e = outer_csr_from_rows(n, g->w, g->d_rows, off, nullptr, temp, need, nullptr, s);
        uint32_t total = 0;
        if (rc == MCE_OK && e == cudaSuccess) e = cudaMemcpyAsync(&total, off + n, 4, cudaMemcpyDeviceToHost, s);
        if (rc == MCE_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (rc == MCE_OK && e == cudaSuccess) {
            g->csr_bytes = offb + round_up(std::max<uint64_t>(total, 1) * 4, 256);
            rc = dalloc(ctx, (void **)&g->d_off, g->csr_bytes);
            if (rc == MCE_OK) {
                g->d_adj = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(g->d_off) + offb);
                e = outer_csr_from_rows(n, g->w, g->d_rows, g->d_off, g->d_adj, temp, need, nullptr, s);
            } else {
                g->d_off = nullptr;
            }
        }
        dfree(ctx, off, offb, s);
        dfree(ctx, temp, need, s);
        if (rc == MCE_OK && e != cudaSuccess) rc = MCE_ECUDA;
        if (rc != MCE_OK) {
            cudaStreamSynchronize(s);
            return rc;
        }
    }
    // degrees (host copy of the offsets) and the degeneracy order
    std::vector<uint32_t> off(n + 1), order(n);
    e = cudaMemcpyAsync(off.data(), g->d_off, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return MCE_ECUDA;
    uint32_t maxd = 0;
    for (uint32_t v = 0; v < n; ++v) maxd = std::max(maxd, off[v + 1] - off[v]);
    if (maxd + 1 > MCE_NMAX) return MCE_ENOTIMPL;  // a subproblem beyond the bitset path
    uint32_t *d_ord = nullptr;
    rc = dalloc(ctx, (void **)&d_ord, ((size_t)n * 2 + 64) * 4, s);
    if (rc != MCE_OK) return rc;
    uint32_t *d_pos = d_ord + n + 32;
    e = outer_degeneracy(n, g->d_off, g->d_adj, d_ord, d_pos, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(order.data(), d_ord, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        dfree(ctx, d_ord, ((size_t)n * 2 + 64) * 4, s);
        return MCE_ECUDA;
    }
    // subproblem i: vertex order[i] with its neighbourhood; arena layout
    std::vector<mce_graph> sub(n);
    std::vector<size_t> rows_at(n), label_at(n), root_at(n);
    size_t bytes = 0;
    auto take = [&](size_t b) {
        bytes = round_up(bytes, 256);
        const size_t at = bytes;
        bytes += b;
        return at;
    };
    uint32_t max_w = 1;
    for (uint32_t i = 0; i < n; ++i) {
        const uint32_t v = order[i], h = off[v + 1] - off[v] + 1, wl = (h + 31) / 32;
        max_w = std::max(max_w, wl);
        rows_at[i] = take((size_t)h * wl * 4);
        label_at[i] = take((size_t)h * 4);
        root_at[i] = take((size_t)2 * wl * 4);
        sub[i].ctx = ctx;
        sub[i].n = h;
        sub[i].w = wl;
        sub[i].m = (uint64_t)h * h / 4;
        sub[i].cost_hint = (double)h * h;
    }
    void *arena = nullptr;
    const size_t arena_bytes = std::max<size_t>(round_up(bytes, 256), 256);
    rc = dalloc(ctx, &arena, arena_bytes, s);
    if (rc != MCE_OK) {
        dfree(ctx, d_ord, ((size_t)n * 2 + 64) * 4, s);
        return rc;
    }
    unsigned char *a = static_cast<unsigned char *>(arena);
    std::vector<mce_graph *> ptrs(n);
    for (uint32_t i = 0; i < n; ++i) {
        sub[i].d_rows = reinterpret_cast<uint32_t *>(a + rows_at[i]);
        sub[i].label = reinterpret_cast<uint32_t *>(a + label_at[i]);
        sub[i].root = reinterpret_cast<uint32_t *>(a + root_at[i]);
        sub[i].rv = 0;  // v's local index: set on the device by the extraction
        ptrs[i] = &sub[i];
    }
    mce_batch *b = nullptr;
    mce_options bo = o;
    bo.flags &= ~(MCE_OUTER | MCE_AUTOTUNE | MCE_ORDER_IDENTITY);
    if (e == cudaSuccess)
        rc = batch_create_impl(ctx, ptrs.data(), n, bo, std::map<uint32_t, TuneChoice>{}, &b, nullptr, true);
    uint64_t *d_out = nullptr;
    const size_t obytes = MCE_OUT_WORDS(n) * 8;
    if (e == cudaSuccess && rc == MCE_OK) rc = dalloc(ctx, (void **)&d_out, obytes, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<uint64_t> h(MCE_OUT_WORDS(n), 0);
    if (e == cudaSuccess && rc == MCE_OK) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
        e = outer_extract(b->d_table, n, max_w, d_ord, d_pos, g->d_off, g->d_adj, s);
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_out, 0, obytes, s);
        if (e == cudaSuccess) e = outer_reduce(b->d_table, n, n, d_out, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_out, obytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    float kms = 0.f;
    if (e == cudaSuccess && rc == MCE_OK && e0 && e1) cudaEventElapsedTime(&kms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (b) mce_batch_destroy(b);
    dfree(ctx, d_out, obytes, s);
    dfree(ctx, arena, arena_bytes, s);
    dfree(ctx, d_ord, ((size_t)n * 2 + 64) * 4, s);
    if (rc == MCE_OK && e != cudaSuccess) rc = MCE_ECUDA;
    if (rc != MCE_OK) {
        cudaStreamSynchronize(s);
        return rc;
    }
    rc = fill_result(h, n, res);
    res->kernel_ms = kms;
    res->total_ms = ms_since(t0);
    return rc;
}

}  // namespace

extern "C" int mce_batch_launch(mce_batch *b)
{
    if (!b) return MCE_EINVAL;
    DevicePick pick(b->ctx->device);
    cudaError_t e = cudaEventRecord(b->t0, b->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->t1, b->stream);
    return cuda_code(e);
}

extern "C" int mce_batch_results(mce_batch *b, mce_result *res)
{
    if (!b) return MCE_EINVAL;
    DevicePick pick(b->ctx->device);
    if (b->h_out.size() != b->out_words) b->h_out.assign(b->out_words, 0);  // first results call
    cudaError_t e = cudaMemcpyAsync(b->h_out.data(), b->d_out, b->out_words * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return MCE_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->t0, b->t1);
    int first = MCE_OK;
    for (uint32_t i = 0; i < b->count; ++i) {
        std::vector<uint64_t> h(b->h_out.begin() + (long)b->out_off[i],
                                b->h_out.begin() + (long)(b->out_off[i] + MCE_OUT_WORDS(b->n[i])));
        int rc = MCE_OK;
        if (res) {
            rc = fill_result(h, b->n[i], &res[i]);
            res[i].kernel_ms = ms;
            res[i].total_ms = ms;
        } else {
            rc = (int)(int64_t)h[MCE_OUT_STATUS];
        }
        if (rc != MCE_OK && first == MCE_OK) first = rc;
    }
    return first;
}

extern "C" int mce_batch_run(mce_batch *b, mce_result *res)
{
    int rc = mce_batch_launch(b);
    return rc != MCE_OK ? rc : mce_batch_results(b, res);
}

extern "C" void mce_batch_destroy(mce_batch *b)
{
    if (!b) return;
    DevicePick pick(b->ctx->device);
    batch_free(b);
}

extern "C" int mce_enumerate_batch(mce_ctx *ctx, mce_graph *const *graphs, uint32_t count, const mce_options *opts,
                                   mce_result *res)
{
    mce_batch *b = nullptr;
    int rc = mce_batch_create(ctx, graphs, count, opts, &b);
    if (rc != MCE_OK) return rc;
    rc = mce_batch_run(b, res);
    mce_batch_destroy(b);
    return rc;
}

// ---------------------------------------------------------------------------
// Served form: continuous batching.  A scheduler thread per context admits
// submitted requests in arrival order while device memory (rows already
// resident + scratch: work queue and stack space + result) fits the
// context's budget and a stream slot is free, launches each admitted request's
// whole path on its own stream with a grid sized by its expected cost, so
// requests that arrive while others run overlap with them on the device, and
// retires them as their completion events fire.

namespace {

constexpr int kServeSlots = 128;
constexpr size_t kServeStackBytes = 56 * 1024;  // shared-memory stack per block
// Micro-batches: while at least kBatchMin requests that can share a launch
// wait, up to kBatchMax of them (each expecting at most serve_bcost
// thousand maximal cliques) run as one batched launch on one stream slot.
constexpr size_t kBatchMin = 4, kBatchMax = 256;

struct MicroBatch;

struct Request {
    mce_ticket id = 0;
    mce_graph *g = nullptr;
    mce_options o{};
    bool batchable = false;  // default launch options and a small expected cost
    MicroBatch *mb = nullptr;
    uint32_t mb_index = 0;
    Config c;
    Layout L;
    uint64_t scratch_bytes = 0, out_bytes = 0, need = 0;
    void *scratch = nullptr;
    uint64_t *d_out = nullptr;
    int slot = -1;
    int state = 0;  // 0 queued, 1 running, 2 done
    int rc = MCE_OK;
    std::vector<uint64_t> words;
    std::chrono::steady_clock::time_point t_submit, t_done;
    float kernel_ms = 0.f;
};

struct MicroBatch {
    mce_batch *b = nullptr;
    int slot = -1;
    std::vector<Request *> reqs;
};

}  // namespace

struct Server {
    mce_ctx *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Request *> pending;
    std::vector<Request *> running;
    std::vector<MicroBatch *> batches;  // micro-batches on the device
    std::unordered_map<mce_ticket, Request *> all;
    std::thread th;
    bool stop = false;
    mce_ticket next = 1;
    uint64_t in_use = 0;
    int sms = 1;
    cudaStream_t streams[kServeSlots] = {};
    cudaEvent_t ev0[kServeSlots] = {}, ev1[kServeSlots] = {};
    uint64_t *pinned[kServeSlots] = {};
    bool busy[kServeSlots] = {};
};

namespace {

void retire(Server *sv, Request *r, int rc)
{
    const int i = r->slot;
    if (rc == MCE_OK) {
        r->words.assign(sv->pinned[i], sv->pinned[i] + MCE_OUT_WORDS(r->g->n));
        cudaEventElapsedTime(&r->kernel_ms, sv->ev0[i], sv->ev1[i]);
    }
    r->rc = rc;
    dfree(sv->ctx, r->scratch, r->scratch_bytes, sv->streams[i]);
    dfree(sv->ctx, r->d_out, r->out_bytes, sv->streams[i]);
    sv->in_use -= r->need;
    sv->busy[i] = false;
    r->slot = -1;
    r->state = 2;
    r->t_done = std::chrono::steady_clock::now();
}

// Launch one request on a free slot; false when it must wait.
bool admit(Server *sv, Request *r)
{
    if (fault_fires(MCE_FAULT_ADMIT)) return false;  // as if out of memory: stays queued
    int slot = -1;
    for (int i = 0; i < kServeSlots; ++i)
        if (!sv->busy[i]) { slot = i; break; }
    if (slot < 0) return false;
    if (sv->ctx->budget && sv->in_use + r->need > sv->ctx->budget) return false;
    cudaStream_t s = sv->streams[slot];
    int rc = dalloc(sv->ctx, &r->scratch, r->scratch_bytes, s);
    if (rc == MCE_OK) rc = dalloc(sv->ctx, (void **)&r->d_out, r->out_bytes, s);
    if (rc == MCE_ENOMEM) {
        dfree(sv->ctx, r->scratch, r->scratch_bytes, s);
        r->scratch = nullptr;
        return false;  // retry once others have retired
    }
    sv->busy[slot] = true;
    r->slot = slot;
    sv->in_use += r->need;
    cudaError_t e = cudaEventRecord(sv->ev0[slot], s);
    if (e == cudaSuccess) {
        rc = enumerate_device_impl(r->g->n, r->g->w, r->g->d_rows, r->o, r->c, r->L,
                                   static_cast<unsigned char *>(r->scratch), r->d_out, s, nullptr);
        if (rc == MCE_OK)
            e = cudaMemcpyAsync(sv->pinned[slot], r->d_out, r->out_bytes, cudaMemcpyDeviceToHost, s);
        if (rc == MCE_OK && e == cudaSuccess) e = cudaEventRecord(sv->ev1[slot], s);
    }
    if (rc == MCE_OK && e != cudaSuccess) rc = MCE_ECUDA;
    r->state = 1;
    if (rc != MCE_OK) {
        cudaStreamSynchronize(s);
        retire(sv, r, rc);
        sv->done_cv.notify_all();
        return true;
    }
    sv->running.push_back(r);
    return true;
}

// Run batchable requests with the pivot rule of the front one, gathered in
// arrival order from the first kBatchScan queued, as one batched launch on a
// free slot; false when none was formed.
constexpr size_t kBatchScan = 4096;

bool admit_batch(Server *sv)
{
    const uint32_t pivot = sv->pending.front()->o.pivot_mode;
    std::vector<size_t> pick;
    for (size_t i = 0; i < sv->pending.size() && i < kBatchScan && pick.size() < kBatchMax; ++i)
        if (sv->pending[i]->batchable && sv->pending[i]->o.pivot_mode == pivot) pick.push_back(i);
    const size_t k = pick.size();
    if (k < kBatchMin) return false;
    int slot = -1;
    for (int i = 0; i < kServeSlots; ++i)
        if (!sv->busy[i]) { slot = i; break; }
    if (slot < 0) return false;
    std::vector<mce_graph *> graphs(k);
    for (size_t i = 0; i < k; ++i) graphs[i] = sv->pending[pick[i]]->g;
    mce_options o{};
    o.pivot_mode = pivot;
    mce_batch *b = nullptr;
    if (batch_create_impl(sv->ctx, graphs.data(), (uint32_t)k, o, std::map<uint32_t, TuneChoice>{}, &b,
                          sv->streams[slot]) != MCE_OK)
        return false;  // e.g. memory: the requests go one by one
    cudaStream_t s = sv->streams[slot];
    cudaError_t e = cudaEventRecord(sv->ev0[slot], s);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(sv->ev1[slot], s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        mce_batch_destroy(b);
        return false;
    }
    MicroBatch *mb = new (std::nothrow) MicroBatch;
    if (!mb) {
        cudaStreamSynchronize(s);
        mce_batch_destroy(b);
        return false;
    }
    mb->b = b;
    mb->slot = slot;
    sv->busy[slot] = true;
    std::vector<Request *> taken(k);
    for (size_t i = 0; i < k; ++i) taken[i] = sv->pending[pick[i]];
    for (size_t i = k; i-- > 0;) sv->pending.erase(sv->pending.begin() + (long)pick[i]);
    for (size_t i = 0; i < k; ++i) {
        Request *r = taken[i];
        r->mb = mb;
        r->mb_index = (uint32_t)i;
        r->slot = slot;
        r->state = 1;
        mb->reqs.push_back(r);
    }
    sv->batches.push_back(mb);
    return true;
}

// A finished micro-batch: results to its requests, launch resources freed.
void retire_batch(Server *sv, MicroBatch *mb, bool ok)
{
    mce_batch *b = mb->b;
    std::vector<uint64_t> h;
    float ms = 0.f;
    if (ok) {  // on the slot's own stream: no wait on other streams' work
        h.resize(b->out_words);
        cudaStream_t s = sv->streams[mb->slot];
        ok = cudaMemcpyAsync(h.data(), b->d_out, b->out_words * 8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
             cudaStreamSynchronize(s) == cudaSuccess;
        cudaEventElapsedTime(&ms, sv->ev0[mb->slot], sv->ev1[mb->slot]);
    }
    const auto now = std::chrono::steady_clock::now();
    for (Request *r : mb->reqs) {
        if (ok) {
            const size_t at = b->out_off[r->mb_index];
            r->words.assign(h.begin() + (long)at, h.begin() + (long)(at + MCE_OUT_WORDS(r->g->n)));
            r->rc = (int)(int64_t)r->words[MCE_OUT_STATUS];
            if (r->rc > 0) r->rc = MCE_OK;
            r->kernel_ms = ms;
        } else {
            r->rc = MCE_ECUDA;
        }
        r->mb = nullptr;
        r->slot = -1;
        r->state = 2;
        r->t_done = now;
    }
    sv->busy[mb->slot] = false;
    mce_batch_destroy(b);
    delete mb;
}

void serve_loop(Server *sv)
{
    DevicePick pick(sv->ctx->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        bool changed = false;
        for (size_t k = 0; k < sv->running.size();) {
            Request *r = sv->running[k];
            const cudaError_t q = cudaEventQuery(sv->ev1[r->slot]);
            if (q == cudaErrorNotReady) { ++k; continue; }
            retire(sv, r, q == cudaSuccess ? MCE_OK : MCE_ECUDA);
            sv->running[k] = sv->running.back();
            sv->running.pop_back();
            changed = true;
        }
        for (size_t k = 0; k < sv->batches.size();) {
            MicroBatch *mb = sv->batches[k];
            const cudaError_t q = cudaEventQuery(sv->ev1[mb->slot]);
            if (q == cudaErrorNotReady) { ++k; continue; }
            retire_batch(sv, mb, q == cudaSuccess);
            sv->batches[k] = sv->batches.back();
            sv->batches.pop_back();
            changed = true;
        }
        while (!sv->pending.empty()) {
            Request *r = sv->pending.front();
            if (r->need > sv->ctx->budget && sv->ctx->budget) {  // can never fit
                sv->pending.pop_front();
                r->rc = MCE_ENOMEM;
                r->state = 2;
                r->t_done = std::chrono::steady_clock::now();
                changed = true;
                continue;
            }
            if (sv->pending.size() >= kBatchMin && admit_batch(sv)) {
                changed = true;
                continue;
            }
            if (!admit(sv, r)) break;
            sv->pending.pop_front();
            changed = true;
        }
        if (changed) sv->done_cv.notify_all();
        if (sv->running.empty() && sv->batches.empty() && sv->pending.empty()) {
            sv->cv.wait(lk);
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

int server_start(mce_ctx *ctx)
{
    Server *sv = new (std::nothrow) Server;
    if (!sv) return MCE_ENOMEM;
    sv->ctx = ctx;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sv->sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kServeSlots && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&sv->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&sv->ev0[i]);
        if (e == cudaSuccess) e = cudaEventCreate(&sv->ev1[i]);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sv->pinned[i], MCE_OUT_WORDS(MCE_NMAX) * 8);
    }
    if (e != cudaSuccess) {
        for (int i = 0; i < kServeSlots; ++i) {
            if (sv->streams[i]) cudaStreamDestroy(sv->streams[i]);
            if (sv->ev0[i]) cudaEventDestroy(sv->ev0[i]);
            if (sv->ev1[i]) cudaEventDestroy(sv->ev1[i]);
            if (sv->pinned[i]) cudaFreeHost(sv->pinned[i]);
        }
        delete sv;
        return MCE_ECUDA;
    }
    sv->th = std::thread(serve_loop, sv);
    ctx->server = sv;
    return MCE_OK;
}

}  // namespace

void server_stop(mce_ctx *ctx)
{
    Server *sv = ctx->server;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    sv->th.join();
    for (int i = 0; i < kServeSlots; ++i) cudaStreamSynchronize(sv->streams[i]);
    for (Request *r : sv->running) retire(sv, r, MCE_ECUDA);
    for (MicroBatch *mb : sv->batches) retire_batch(sv, mb, false);
    sv->batches.clear();
    for (auto &kv : sv->all) delete kv.second;
    for (int i = 0; i < kServeSlots; ++i) {
        cudaStreamDestroy(sv->streams[i]);
        cudaEventDestroy(sv->ev0[i]);
        cudaEventDestroy(sv->ev1[i]);
        cudaFreeHost(sv->pinned[i]);
    }
    delete sv;
    ctx->server = nullptr;
}

extern "C" int mce_submit(mce_ctx *ctx, mce_graph *g, const mce_options *opts, mce_ticket *out)
{
    if (!ctx || !g || !out || g->ctx != ctx || !g->d_rows) return MCE_EINVAL;
    DevicePick pick(ctx->device);
    mce_options o = defaults(opts);
    if (o.flags & (MCE_LIST | MCE_LIST_SORTED)) return MCE_ENOTIMPL;
    if (!ctx->server) {
        int rc = server_start(ctx);
        if (rc) return rc;
    }
    Server *sv = ctx->server;
    const double cost = expected_cliques(g->n, g->m);
    // default launch options and a small expected cost: may share a launch
    const bool batchable = !o.lanes_per_subtree && !o.words_per_lane && !o.threads_per_block && !o.blocks &&
                           !o.split_min_p && !o.stack_levels && !o.queue_log2 && !o.flags && !o.timeout_ns &&
                           cost <= 1e3 * default_tuning().serve_bcost;
    if (!o.threads_per_block) o.threads_per_block = 256;
    if (!o.blocks) {
        const double per_block = default_tuning().serve_cpb;
        o.blocks = (uint32_t)std::min<double>(std::max(1.0, std::ceil(cost / per_block)), 4.0 * sv->sms);
    }
    Request *r = new (std::nothrow) Request;
    if (!r) return MCE_ENOMEM;
    r->g = g;
    r->o = o;
    r->batchable = batchable;
    int rc = g->n > MCE_NMAX ? MCE_EINVAL : choose(g->n, o, r->c, kServeStackBytes);
    if (rc) { delete r; return rc; }
    r->L = layout(g->n, r->c);
    r->scratch_bytes = r->L.total;
    r->out_bytes = MCE_OUT_WORDS(g->n) * 8;
    r->need = r->scratch_bytes + r->out_bytes;
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->id = sv->next++;
        sv->all[r->id] = r;
        sv->pending.push_back(r);
    }
    sv->cv.notify_all();
    *out = r->id;
    return MCE_OK;
}

namespace {

// Caller holds the lock; the request is done.  Fills res and forgets it.
int deliver(Server *sv, Request *r, mce_result *res)
{
    int rc = r->rc;
    if (rc == MCE_OK) {
        rc = fill_result(r->words, r->g->n, res);
        res->kernel_ms = r->kernel_ms;
    } else {
        res->status = (uint32_t)rc;
    }
    res->total_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    sv->all.erase(r->id);
    delete r;
    return rc;
}

}  // namespace

extern "C" int mce_poll(mce_ctx *ctx, mce_ticket t, mce_result *res)
{
    if (!ctx || !res || !ctx->server) return MCE_EINVAL;
    Server *sv = ctx->server;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(t);
    if (it == sv->all.end()) return MCE_EINVAL;
    if (it->second->state != 2) return MCE_PENDING;
    return deliver(sv, it->second, res);
}

extern "C" int mce_wait(mce_ctx *ctx, mce_ticket t, uint64_t timeout_ns, mce_result *res)
{
    if (!ctx || !res || !ctx->server) return MCE_EINVAL;
    Server *sv = ctx->server;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(t);
    if (it == sv->all.end()) return MCE_EINVAL;
    Request *r = it->second;
    const auto limit = std::chrono::nanoseconds(timeout_ns ? timeout_ns : 3600ull * 1000000000ull);
    if (!sv->done_cv.wait_for(lk, limit, [&] { return r->state == 2; })) return MCE_ETIMEOUT;
    return deliver(sv, r, res);
}

extern "C" int mce_cancel(mce_ctx *ctx, mce_ticket t)
{
    if (!ctx || !ctx->server) return MCE_EINVAL;
    Server *sv = ctx->server;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->all.find(t);
        if (it == sv->all.end()) return MCE_EINVAL;
        Request *r = it->second;
        if (r->state != 0) return MCE_EBUSY;
        auto q = std::find(sv->pending.begin(), sv->pending.end(), r);
        if (q == sv->pending.end()) return MCE_EBUSY;
        sv->pending.erase(q);
        r->rc = MCE_ECANCELED;
        r->state = 2;
        r->t_done = std::chrono::steady_clock::now();
    }
    sv->done_cv.notify_all();
    return MCE_OK;
}

extern "C" int mce_fault_inject(int site, uint32_t skip, uint32_t count) { return fault_arm(site, skip, count); }

extern "C" uint64_t mce_ctx_mem_used(const mce_ctx *ctx) { return ctx ? ctx->used.load() : 0ull; }

extern "C" int mce_trace_enable(void *d_buf, uint64_t bytes)
{
    g_trace = bytes >= 16 ? d_buf : nullptr;
    g_trace_bytes = g_trace ? bytes : 0;
    return MCE_OK;
}

extern "C" const char *mce_strerror(int code)
{
    switch (code) {
    case MCE_OK: return "ok";
    case MCE_PENDING: return "pending";
    case MCE_EINVAL: return "invalid argument or graph";
    case MCE_ENOMEM: return "out of memory";
    case MCE_ECUDA: return "CUDA error";
    case MCE_ETRUNC: return "output buffer too small";
    case MCE_ETIMEOUT: return "timed out";
    case MCE_EOVERFLOW: return "work queue overflow";
    case MCE_ENOTIMPL: return "not implemented";
    case MCE_ECANCELED: return "cancelled";
    case MCE_EBUSY: return "already running";
    default: return "unknown error";
    }
}
