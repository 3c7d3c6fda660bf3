// Bit-parallel Bron-Kerbosch search (Alg. 4, BKPivotOrdered with
// ChoosePivotOrdered) as a persistent, work-stealing CUDA kernel for sm_103a.
//
// Mapping (Section 4.1 describes the CPU bitset encoding this replaces):
//  * A *group* of G lanes of one warp owns one search subtree.  Lane l of the
//    group holds words [l*K, l*K + K) of every set, so a set of n vertices
//    takes WP = G*K 32-bit words spread over the group.  32/G groups share a
//    warp and advance in lock step: every warp-wide collective (ballot,
//    shuffle) is executed by all 32 lanes, and group-specific decisions are
//    data predicates.
//  * The renumbered adjacency (Section 4.2) is staged in shared memory by a
//    1-D bulk-copy (TMA) when it fits, else read from L2 through the
//    read-only path with 64/128-bit loads.
//  * A frame (P, X, pivot, end, |R|, S(R)) stands for "expand the children
//    v in L = P & ~N(pivot) & [0, end) in increasing position": the current
//    frame lives in registers, its ancestors on a per-group explicit stack in
//    local memory (no recursion).  A frame is pushed only while it has
//    children left, so single-child chains (e.g. a complete graph) do not
//    grow the stack.
//  * Work moves at two levels.  Idle groups take frames from their block's
//    ring in shared memory, which busy groups of the block refill by giving
//    away the front half of their shallowest branching set; blocks whose
//    groups are idle with an empty ring count as starving, one idle warp per
//    block polls the global ring (a bounded MPMC ring in global memory whose
//    tickets are taken by fetch-and-add at both ends, never by a contended
//    compare-and-swap), and busy groups feed that ring while starving blocks
//    outnumber its frames.
//    Cutting a branching set L into a front part L1 (given) and the rest as
//    (P, X, end = first kept element) and (P \ L1, X u L1, end) reproduces
//    exactly the sequential P/X updates of Alg. 4, so node counts do not
//    depend on how the work was split.
//  * Leaves update per-group register counters; sizes go to a shared-memory
//    histogram; everything is integer arithmetic modulo 2^64, so the
//    reduction order does not matter and results are bit-exact.
//
// Every spin (queue tickets, idle wait, the bulk-copy barrier) is bounded and
// ends in an error status plus a global abort flag, never a hang or a trap.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mce_internal.h"

namespace mce {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned kCasTries = 1u << 14; // bound of one queue ticket loop

// Work-distribution thresholds by edge density p = i/40 (i = 1..39): the
// smallest candidate-set size k whose random subgraph G(k, p) has at least
// 256, 2048 or 16384 maximal cliques in expectation
// (sum_j C(k,j) p^C(j,2) (1-p^j)^(k-j)).  A frame is given to the block ring
// when its candidate set reaches the first, to the device-wide ring when it
// reaches the second, and a new subtree is published breadth-first when it
// reaches the third: what moves must carry enough work to pay for the move,
// and the further it moves the more work that takes.  The two sharing
// thresholds are capped by a fraction of n (see density_thresholds).
__constant__ unsigned short kShareLocalByDensity[39] = {147, 111, 96, 87, 80, 73, 68, 63, 58, 55, 52, 49, 47,
                                                        44,  42,  41, 39, 37, 36, 35, 33, 32, 31, 30, 29, 29,
                                                        28,  27,  26, 26, 25, 25, 25, 25, 25, 25, 26, 28, 34};
__constant__ unsigned short kShareGlobalByDensity[39] = {440, 343, 283, 234, 199, 174, 155, 141, 129, 119, 110,
                                                         102, 94,  88,  82,  77,  73,  69,  65,  62,  58,  55,
                                                         53,  50,  48,  46,  44,  42,  41,  39,  38,  37,  36,
                                                         35,  34,  34,  35,  36,  42};
__constant__ unsigned short kSplitByDensity[39] = {1363, 907, 651, 515, 433, 376, 329, 290, 257, 230, 208, 189, 173,
                                                   159,  146, 135, 125, 116, 108, 101, 94,  88,  83,  78,  73,  69,
                                                   65,   61,  58,  55,  52,  50,  48,  46,  45,  44,  43,  45,  51};

struct Thresholds {
    unsigned share_local, share_global, split;
};

// Thresholds for a block's graph from the density of its rows; non-zero
// caller values win.  Whole block (barriers inside); every thread gets the
// same values.
__device__ __forceinline__ Thresholds density_thresholds(const uint32_t *rows, uint32_t n, uint32_t wp,
                                                         unsigned fixed_local, unsigned fixed_global,
                                                         unsigned fixed_split, unsigned *scratch_u32,
                                                         bool small_split)
{
    if (threadIdx.x == 0) *scratch_u32 = 0u;
    __syncthreads();
    unsigned mine = 0;
    for (uint32_t i = threadIdx.x; i < n * wp; i += blockDim.x) mine += __popc(rows[i]);
    atomicAdd(scratch_u32, mine);
    __syncthreads();
    const unsigned deg_sum = *scratch_u32;
    __syncthreads();
    Thresholds t{0xffffffffu, 0xffffffffu, 0xffffffffu};
    if (n >= 2) {
        const double pd = (double)deg_sum / ((double)n * (double)(n - 1));
        int i = (int)(pd * 40.0 + 0.5);
        i = i < 1 ? 1 : (i > 39 ? 39 : i);
        // The tables assume random graphs; a structured graph (Moon-Moser:
        // every branching set has three vertices) keeps big subtrees at
        // much smaller |P|, so a candidate set holding a good share of the
        // graph also counts as big.
        t.share_local = min((unsigned)kShareLocalByDensity[i - 1], max(16u, n / 8u));
        t.share_global = min((unsigned)kShareGlobalByDensity[i - 1], max(20u, n / 4u));
        // dense structured graphs (Moon-Moser: every child keeps all but three
        // vertices) would never reach the density's split size; cap it at
        // half of n (Moon-Moser 45: 1.37 -> 0.90 ms against two thirds).
        // With small_split (full-wave launches of one graph), small graphs
        // of density up to 0.75 split from 20 vertices: their whole tree is
        // too small for the density's split size, and only frames that move
        // keep the GPU busy (measured, whole path: G(100, 0.5) 0.28 -> 0.21
        // ms, G(100, 0.7) 0.95 -> 0.50, G(128, 0.5) 0.36 -> 0.24, G(200,
        // 0.5) 0.83 -> 0.54, G(256, 0.4) 0.72 -> 0.51; G(100, 0.8) would
        // lose: 1.27 -> 2.2 ms)
        t.split = min((unsigned)kSplitByDensity[i - 1], max(20u, n / 2u));
        if (small_split && n <= 256u && i <= 30) t.split = min(t.split, 20u);
    }
    if (fixed_local) t.share_local = fixed_local;
    if (fixed_global) t.share_global = fixed_global;
    if (fixed_split) t.split = fixed_split;
    return t;
}

// SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014), the mixing step
// of the clique hash h(K) = mix64(S(K) ^ mix64(|K|)).
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void set_status(uint64_t *out, Ctl *ctl, int code)
{
    atomicCAS(reinterpret_cast<unsigned long long *>(out + MCE_OUT_STATUS), 0ull,
              static_cast<unsigned long long>(static_cast<long long>(code)));
    atomicExch(&ctl->abort, 1u);
}

// ---------------------------------------------------------------------------
// Bounded MPMC ring of frames (per-slot sequence numbers: a slot with
// seq == ticket is free for producer `ticket`, seq == ticket + 1 holds the
// frame for consumer `ticket`).

// Reserve a producer ticket: check the room left -- producer tickets at
// most qcap - margin ahead of the consumers', margin = the groups that can
// reserve at once (one ticket each) -- and take the ticket with one
// fetch-and-add, so producers race no compare-and-swap either.  The room
// check puts the ticket's slot behind a consumer ticket already claimed, so
// the slot is free as soon as that frame has been taken (microseconds;
// waited for, with a bound).  On false the caller keeps its frame; a ticket
// taken but never filled (the bounded wait ran out, or the search aborted)
// only leaves its consumer idle.
__device__ __forceinline__ bool q_reserve_push(Ctl *ctl, unsigned *seq, unsigned mask, unsigned &ticket,
                                               unsigned margin)
{
    const unsigned hd = ld_relaxed(&ctl->head), tl = ld_relaxed(&ctl->tail);
    if ((int)(tl - hd) >= (int)(mask + 1u) - (int)margin) return false;
    const unsigned tk = atomicAdd(&ctl->tail, 1u);
    for (unsigned t = 0; ld_acquire(&seq[tk & mask]) != tk; ++t) {
        if (t >= (kCasTries << 8) || ld_relaxed(&ctl->abort)) return false;
        __nanosleep(32);
    }
    ticket = tk;
    return true;
}

// Take the oldest published frame of a block-private ring (batched form:
// the only contenders are the block's own groups, so a compare-and-swap on
// the head is cheap there).
__device__ __forceinline__ bool q_reserve_pop(Ctl *ctl, unsigned *seq, unsigned mask, unsigned &ticket,
                                              unsigned long long *fails, unsigned tries = kCasTries)
{
    unsigned pos = ld_relaxed(&ctl->head);
    for (unsigned t = 0; t < tries; ++t) {
        unsigned s = ld_acquire(&seq[pos & mask]);
        int dif = (int)(s - (pos + 1));
        if (dif == 0) {
            unsigned prev = atomicCAS(&ctl->head, pos, pos + 1);
            if (prev == pos) { ticket = pos; return true; }
            atomicAdd(fails, 1ull);
            pos = prev;
        } else if (dif < 0) {
            return false;  // empty
        } else {
            pos = ld_relaxed(&ctl->head);
        }
    }
    return false;
}

// Room kept free in a frame ring for producers that reserve at once: every
// group of the launch on the device-wide ring (the plain form sizes the ring
// at four frames per group and more), the block's groups on a block-private
// ring (batched form).
template <int G>
__device__ __forceinline__ unsigned push_margin(const SearchParams &prm)
{
    const unsigned block_groups = (blockDim.x >> 5) * (32u / G);
    return (prm.total_groups > block_groups ? prm.total_groups : block_groups) + 32u;
}

// Claim up to `want` consecutive consumer tickets of the device-wide ring
// with one fetch-and-add: first .. first + k - 1.  Only frames seen in the
// ring are claimed, so claimers never race a compare-and-swap on the head
// (under a compare-and-swap, most of the idle blocks' attempts failed and
// were retried, and the ring's head was the search's bottleneck); two
// claimers that saw the same frames can take tickets past the producers'.
// A claimed ticket is the claimer's alone: its frame is taken once the
// producer has published it (seq == ticket + 1), or never if the search ends
// first -- the search ends only when no frame is queued or held anywhere
// (pending == 0), so no published frame is ever left behind.  Returns k.
__device__ __forceinline__ unsigned q_claim(Ctl *ctl, unsigned want, unsigned &first)
{
    const unsigned h = ld_relaxed(&ctl->head), t = ld_relaxed(&ctl->tail);
    const int avail = (int)(t - h);
    if (avail <= 0) return 0u;
    const unsigned k = min(want, (unsigned)avail);
    first = atomicAdd(&ctl->head, k);
    return k;
}

// ---------------------------------------------------------------------------
// Group-wide set primitives.  All collectives use the full warp mask and must
// be reached by all 32 lanes: call them only as standalone statements in
// warp-uniform code, never behind a short-circuit && / || or a ?: whose
// condition differs between lanes.

template <int G, int K>
struct Grp {
    static constexpr int WP = G * K;
    unsigned lane, gl, gbase, gmask;

    __device__ __forceinline__ void init()
    {
        lane = threadIdx.x & 31u;
        gl = lane & (unsigned)(G - 1);
        gbase = lane - gl;
        gmask = (G == 32) ? FULL : (((1u << G) - 1u) << gbase);
    }
    __device__ __forceinline__ bool leader() const { return gl == 0; }

    __device__ __forceinline__ bool anyp(bool p) const
    {
        if (G == 1) return p;
        return (__ballot_sync(FULL, p) & gmask) != 0u;
    }
    __device__ __forceinline__ bool any(const uint32_t (&s)[K]) const
    {
        uint32_t o = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) o |= s[k];
        return anyp(o != 0u);
    }
    // Position of the lowest set bit of the group's set (= the vertex first
    // in the order), or -1 if the set is empty.  A whole-warp group takes
    // one min-reduction; narrower groups a ballot and a shuffle.
    __device__ __forceinline__ int first(const uint32_t (&s)[K]) const
    {
        int loc = -1;
#pragma unroll
        for (int k = K - 1; k >= 0; --k)
            if (s[k]) loc = (int)((gl * K + k) * 32u) + __ffs(s[k]) - 1;
        if (G == 1) return loc;
        if (G == 32) return (int)__reduce_min_sync(FULL, (unsigned)loc);
        unsigned b = __ballot_sync(FULL, loc >= 0) & gmask;
        int src = b ? (__ffs(b) - 1) : (int)lane;
        int r = __shfl_sync(FULL, loc, src);
        return b ? r : -1;
    }
    // Emptiness of sets a and b, and the first element of a when a is
    // non-empty, else of b (-1 when both are empty).
    __device__ __forceinline__ int first_either(const uint32_t (&a)[K], const uint32_t (&b)[K], bool &na,
                                                bool &nb) const
    {
        uint32_t oa = 0, ob = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            oa |= a[k];
            ob |= b[k];
        }
        unsigned ba = 0u, bb = 0u;
        if (G == 1) {
            na = oa != 0u;
            nb = ob != 0u;
        } else {
            ba = __ballot_sync(FULL, oa != 0u) & gmask;
            bb = __ballot_sync(FULL, ob != 0u) & gmask;
            na = ba != 0u;
            nb = bb != 0u;
        }
        int loc = -1;
#pragma unroll
        for (int k = K - 1; k >= 0; --k) {
            const uint32_t w = na ? a[k] : b[k];
            if (w) loc = (int)((gl * K + k) * 32u) + __ffs(w) - 1;
        }
        if (G == 1) return loc;
        if (G == 32) return (int)__reduce_min_sync(FULL, (unsigned)loc);
        const unsigned m = na ? ba : bb;
        const int src = m ? (__ffs(m) - 1) : (int)lane;
        const int r = __shfl_sync(FULL, loc, src);
        return m ? r : -1;
    }
    // Emptiness of two sets at once.
    __device__ __forceinline__ void any2(const uint32_t (&a)[K], const uint32_t (&b)[K], bool &ra, bool &rb) const
    {
        uint32_t oa = 0, ob = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            oa |= a[k];
            ob |= b[k];
        }
        if (G == 1) {
            ra = oa != 0u;
            rb = ob != 0u;
        } else if (G == 32) {
            const unsigned m = __reduce_or_sync(FULL, (oa != 0u ? 1u : 0u) | (ob != 0u ? 2u : 0u));
            ra = (m & 1u) != 0u;
            rb = (m & 2u) != 0u;
        } else {
            const unsigned ba = __ballot_sync(FULL, oa != 0u), bb = __ballot_sync(FULL, ob != 0u);
            ra = (ba & gmask) != 0u;
            rb = (bb & gmask) != 0u;
        }
    }
    __device__ __forceinline__ int sum(int x) const
    {
        if (G == 32) return (int)__reduce_add_sync(FULL, (unsigned)x);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
        return x;
    }
    __device__ __forceinline__ int excl_scan(int x) const
    {
        int incl = x;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            int y = __shfl_up_sync(FULL, incl, o, G);
            if ((int)gl >= o) incl += y;
        }
        return incl - x;
    }
    __device__ __forceinline__ unsigned from_leader(unsigned x) const
    {
        if (G == 1) return x;
        return __shfl_sync(FULL, x, gbase);
    }
    // Bits [0, end) of this lane's k-th word.
    __device__ __forceinline__ uint32_t below(int k, unsigned end) const
    {
        unsigned base = (gl * K + k) * 32u;
        if (end >= base + 32u) return FULL;
        if (end <= base) return 0u;
        return (1u << (end - base)) - 1u;
    }
    __device__ __forceinline__ void clear(uint32_t (&s)[K], int v) const
    {
        unsigned w = (unsigned)v >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (w == gl * K + k) s[k] &= ~(1u << (v & 31));
    }
    __device__ __forceinline__ void set(uint32_t (&s)[K], int v) const
    {
        unsigned w = (unsigned)v >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (w == gl * K + k) s[k] |= 1u << (v & 31);
    }
};

template <int K, bool SMEM>
__device__ __forceinline__ void load_row(uint32_t (&r)[K], const uint32_t *p)
{
    if (K == 1) {
        r[0] = SMEM ? p[0] : __ldg(p);
    } else if (K == 2) {
        uint2 t = SMEM ? *reinterpret_cast<const uint2 *>(p) : __ldg(reinterpret_cast<const uint2 *>(p));
        r[0] = t.x;
        r[1] = t.y;
    } else {
        uint4 t = SMEM ? *reinterpret_cast<const uint4 *>(p) : __ldg(reinterpret_cast<const uint4 *>(p));
        r[0] = t.x;
        r[1] = t.y;
        r[2] = t.z;
        r[3] = t.w;
    }
}

// ---------------------------------------------------------------------------
// Block-local frame ring (shared memory): the same per-slot sequence-number
// protocol as the global ring, with block-scope atomics.

__device__ __forceinline__ unsigned vld(const unsigned *p) { return *reinterpret_cast<const volatile unsigned *>(p); }
__device__ __forceinline__ void vst(unsigned *p, unsigned v) { *reinterpret_cast<volatile unsigned *>(p) = v; }

__device__ __forceinline__ bool lq_reserve_push(LocalHdr *h, unsigned *seq, unsigned mask, unsigned &ticket)
{
    unsigned pos = vld(&h->tail);
    for (unsigned t = 0; t < 256; ++t) {
        const unsigned s = vld(&seq[pos & mask]);
        const int dif = (int)(s - pos);
        if (dif == 0) {
            const unsigned prev = atomicCAS(&h->tail, pos, pos + 1);
            if (prev == pos) { ticket = pos; return true; }
            pos = prev;
        } else if (dif < 0) {
            return false;
        } else {
            pos = vld(&h->tail);
        }
    }
    return false;
}

__device__ __forceinline__ bool lq_reserve_pop(LocalHdr *h, unsigned *seq, unsigned mask, unsigned &ticket)
{
    unsigned pos = vld(&h->head);
    for (unsigned t = 0; t < 256; ++t) {
        const unsigned s = vld(&seq[pos & mask]);
        const int dif = (int)(s - (pos + 1));
        if (dif == 0) {
            const unsigned prev = atomicCAS(&h->head, pos, pos + 1);
            if (prev == pos) { ticket = pos; return true; }
            pos = prev;
        } else if (dif < 0) {
            return false;
        } else {
            pos = vld(&h->head);
        }
    }
    return false;
}

struct LocalQ {
    LocalHdr *h;
    unsigned *seq;
    uint32_t *frames;
    unsigned mask;  // slots - 1
};

__device__ __forceinline__ LocalQ local_queue_at(unsigned char *base, uint32_t wp, uint32_t slots = kLocalSlots)
{
    LocalQ q;
    q.h = reinterpret_cast<LocalHdr *>(base);
    q.seq = reinterpret_cast<unsigned *>(base + sizeof(LocalHdr));
    q.frames = reinterpret_cast<uint32_t *>(base + sizeof(LocalHdr) + (size_t)slots * 4);
    q.mask = slots - 1u;
    (void)wp;
    return q;
}

// Reset the block's ring (whole block; a barrier must follow).
__device__ __forceinline__ void local_queue_reset(const LocalQ &q, unsigned groups)
{
    for (unsigned i = threadIdx.x; i <= q.mask; i += blockDim.x) q.seq[i] = i;
    if (threadIdx.x == 0) {
        q.h->head = 0u;
        q.h->tail = 0u;
        q.h->idle = groups;
        q.h->bwork = 0u;
        q.h->starving = 0u;
        q.h->poller = 0u;
        q.h->done = 0u;
        q.h->refreshing = 0u;
        q.h->g_head = 0u;
        q.h->g_tail = 0u;
        q.h->g_starving = 0u;
        q.h->stamp = 0ull;
        q.h->trace_n = 0u;
        q.h->t2_busy = 0u;
        for (int i = 0; i < kDiagCount; ++i) q.h->diag[i] = 0ull;
    }
}

// Per-lane result counters (summed over the warp at the end; nodes is formed
// at the flush as leaves + dead ends + internal nodes).  The block's
// work-distribution diagnostics live in shared memory (diag).
struct Counters {
    uint64_t cnt = 0, nodes = 0, intl = 0, dead = 0, hash = 0;
    unsigned max = 0;
    unsigned long long *diag = nullptr;
    __device__ __forceinline__ void note(int i, unsigned long long v = 1ull) const { atomicAdd(diag + i, v); }
};

// ---------------------------------------------------------------------------
// Give away the front of a frame's branching set L (c elements, in order).
// The taker gets L1 = the first `give` elements as the frame
// (P, X, pivot, end = first kept element); the giver keeps the rest as
// (P \ L1, X u L1, pivot, end).  Walking L1 then the rest is exactly the
// sequential loop of Alg. 4 (each child sees P minus, and X plus, every
// earlier sibling), so the search tree is the same however often it is cut.
// give = floor(c/2) for c >= 2; with c == 1 the whole frame goes only when
// `allow_whole`.  A frame whose candidate set has fewer than `min_p` vertices
// is kept.  Returns true when a frame was handed over; the giver then applies
// (P, X, L) &= ~L1 / |= L1 through the returned mask l1 (its own words).

template <int G, int K, bool LOCAL>
__device__ __forceinline__ bool donate_front(const Grp<G, K> &g, const SearchParams &prm, const LocalQ &lq,
                                             bool pred, bool allow_whole, int min_p, const uint32_t (&P)[K],
                                             const uint32_t (&X)[K], const uint32_t (&L)[K], unsigned pe,
                                             unsigned rs, uint64_t S, bool list, const uint32_t (&R)[K],
                                             uint32_t (&l1)[K], bool &whole, Counters &cn)
{
    constexpr int WP = G * K;
    int cl = 0, cp = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        cl += __popc(L[k]);
        cp += __popc(P[k]);
    }
    const int c = g.sum(cl);
    const int np = g.sum(cp);
    const int give = (c >= 2) ? c / 2 : ((c == 1 && allow_whole) ? 1 : 0);
    const bool ok = pred && give > 0 && np >= min_p;
    // split = position of element #give of L (the first one kept), or the
    // frame's end when everything goes
    const int pre = g.excl_scan(cl);
    int pos = -1;
    if (ok && give < c && pre <= give && give < pre + cl) {
        int r = give - pre;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int cw = __popc(L[k]);
            if (pos < 0) {
                if (r < cw) {
                    uint32_t w = L[k];
                    for (int j = 0; j < r; ++j) w &= w - 1u;
                    pos = (int)((g.gl * K + k) * 32u) + __ffs(w) - 1;
                } else {
                    r -= cw;
                }
            }
        }
    }
    int split = pos;
    if (G > 1) {
        const unsigned b = __ballot_sync(FULL, pos >= 0) & g.gmask;
        split = __shfl_sync(FULL, pos, b ? (__ffs(b) - 1) : (int)g.lane);
    }
    if (give >= c) split = (int)(pe >> 16);

    // A frame in the block ring is block work (the giver keeps the block
    // active); a frame in the global ring is one unit of global pending.
    unsigned ticket = 0, got = 0;
    if (ok && g.leader()) {
        if (LOCAL) {
            atomicAdd(&lq.h->bwork, 1u);
            got = lq_reserve_push(lq.h, lq.seq, lq.mask, ticket) ? 1u : 0u;
            if (!got) atomicSub(&lq.h->bwork, 1u);
        } else {
            atomicAdd(&prm.ctl->pending, 1u);
            got = q_reserve_push(prm.ctl, prm.seq, prm.qcap - 1u, ticket, push_margin<G>(prm)) ? 1u : 0u;
            if (got) cn.note(kDiagGpush);
            if (!got) atomicSub(&prm.ctl->pending, 1u);
        }
    }
    got = g.from_leader(got);
    ticket = g.from_leader(ticket);
    const unsigned npe = (pe & 0xffffu) | ((unsigned)split << 16);
#pragma unroll
    for (int k = 0; k < K; ++k) l1[k] = got ? (L[k] & g.below(k, (unsigned)split)) : 0u;
    if (got) {
        if (LOCAL) {
            volatile uint32_t *fr = lq.frames + (size_t)(ticket & lq.mask) * frame_words(WP, list);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                fr[kFrameHdr + g.gl * K + k] = P[k];
                fr[kFrameHdr + WP + g.gl * K + k] = X[k];
                if (list) fr[kFrameHdr + 2 * WP + g.gl * K + k] = R[k];
            }
            if (g.leader()) {
                fr[0] = npe;
                fr[1] = rs;
                fr[2] = (uint32_t)S;
                fr[3] = (uint32_t)(S >> 32);
            }
            __threadfence_block();
        } else {
            uint32_t *fr = prm.frames + (size_t)(ticket & (prm.qcap - 1u)) * prm.fs;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                __stcg(fr + kFrameHdr + g.gl * K + k, P[k]);
                __stcg(fr + kFrameHdr + WP + g.gl * K + k, X[k]);
                if (list) __stcg(fr + kFrameHdr + 2 * WP + g.gl * K + k, R[k]);
            }
            if (g.leader()) {
                __stcg(fr + 0, npe);
                __stcg(fr + 1, rs);
                __stcg(fr + 2, (uint32_t)S);
                __stcg(fr + 3, (uint32_t)(S >> 32));
            }
            __threadfence();
        }
    }
    __syncwarp();
    if (got && g.leader()) {
        if (LOCAL) {
            __threadfence_block();
            vst(&lq.seq[ticket & lq.mask], ticket + 1u);
        } else {
            st_release(&prm.seq[ticket & (prm.qcap - 1u)], ticket + 1u);
        }
        cn.note(kDiagDonations);
    }
    whole = give >= c;
    return got != 0u;
}

// Warp-reduce the counters and add them to out[] (one atomic per counter per
// warp).  Called by all 32 lanes.
__device__ __forceinline__ void flush_counters(Counters &c, uint64_t *out)
{
    c.nodes = c.cnt + c.dead + c.intl;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c.cnt += __shfl_xor_sync(FULL, c.cnt, o);
        c.nodes += __shfl_xor_sync(FULL, c.nodes, o);
        c.intl += __shfl_xor_sync(FULL, c.intl, o);
        c.dead += __shfl_xor_sync(FULL, c.dead, o);
        c.hash += __shfl_xor_sync(FULL, c.hash, o);
        c.max = max(c.max, __shfl_xor_sync(FULL, c.max, o));
    }
    if ((threadIdx.x & 31u) == 0) {
        unsigned long long *o = reinterpret_cast<unsigned long long *>(out);
        if (c.cnt) atomicAdd(o + MCE_OUT_COUNT, c.cnt);
        if (c.nodes) atomicAdd(o + MCE_OUT_NODES, c.nodes);
        if (c.intl) atomicAdd(o + MCE_OUT_INTERNAL, c.intl);
        if (c.dead) atomicAdd(o + MCE_OUT_DEAD_ENDS, c.dead);
        if (c.hash) atomicAdd(o + MCE_OUT_HASH, c.hash);
        if (c.max) atomicMax(o + MCE_OUT_MAX_SIZE, (unsigned long long)c.max);
    }
}

// The block's diagnostics to out[] (one thread, after the block's warps are
// done).
__device__ __forceinline__ void flush_diag(const unsigned long long *diag, uint64_t *out)
{
    unsigned long long *o = reinterpret_cast<unsigned long long *>(out);
    const int word[kDiagCount] = {MCE_OUT_DONATIONS, MCE_OUT_STEALS,   MCE_OUT_GLOBAL,    MCE_OUT_BUSY_NS,
                                  MCE_OUT_GPUSH,     MCE_OUT_GTRY,     MCE_OUT_CAS_FAIL,  MCE_OUT_LANE_TASKS};
#pragma unroll
    for (int i = 0; i < kDiagCount; ++i)
        if (diag[i]) atomicAdd(o + word[i], diag[i]);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mb, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of the barrier at mb: ~2 s, then false.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mb, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    for (unsigned t = 0;; ++t) {
        if (mbar_try_wait(mb, parity)) return true;
        if ((t & 63u) == 63u && global_ns() - t0 > 2000000000ull) return false;
    }
}

// Stage `bytes` (multiple of 16, 16-byte aligned ends) of rows from global to
// shared memory with 1-D bulk copies completing on the barrier at mb.  Thread 0
// issues; every thread waits (bounded) for phase `parity`.  Returns false on a
// timeout, after a second bounded wait that lets copies in flight land before
// the shared memory can be reused.  Must be called by the whole block.
__device__ __forceinline__ bool stage_rows(uint32_t *sdst, const uint32_t *gsrc, uint32_t bytes, uint32_t mb,
                                           uint32_t parity)
{
    if (threadIdx.x == 0) {
        // order earlier generic-proxy reads of this shared memory before the
        // async-proxy writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
        const uint32_t dst0 = (uint32_t)__cvta_generic_to_shared(sdst);
        for (uint32_t off = 0; off < bytes; off += 65536u) {
            const uint32_t len = (bytes - off) < 65536u ? (bytes - off) : 65536u;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    dst0 + off),
                "l"(reinterpret_cast<const unsigned char *>(gsrc) + off), "r"(len), "r"(mb)
                : "memory");
        }
    }
    if (mbar_wait_bounded(mb, parity)) return true;
    mbar_wait_bounded(mb, parity);
    return false;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Explicit per-group stack of frames.  Levels [0, SL) live in this warp's
// slice of shared memory, laid out [level][word][lane] so every lane has its
// own bank; deeper levels live in local memory.  Per level a lane keeps its
// K words of P and of X plus M "meta" words: with four or more lanes per
// group, lane j < 4 of the group keeps field j of (pivot|end, |R|, S low,
// S high) and the fields come back by shuffles; narrower groups keep all
// four fields in every lane.  |R| and S are the same in every lane.
template <int G, int K>
struct Stack {
    static constexpr int M = (G >= 4) ? 1 : 4;
    static constexpr int LW = 2 * K + M;
    uint32_t *sm;  // the warp's slice of shared memory (kept in a register)
    unsigned ln;   // this lane
    int SL;
    uint32_t (*lw)[LW];  // local-memory levels, indexed by the absolute level

    __device__ __forceinline__ static uint32_t pick(unsigned pe, unsigned rs, uint64_t S, unsigned j)
    {
        return j == 0u ? pe : (j == 1u ? rs : (j == 2u ? (uint32_t)S : (uint32_t)(S >> 32)));
    }
    // A shared-memory level: P of all 32 lanes (K words each, lane-major, so
    // one vector access per lane), then X likewise, then M meta words per
    // lane (word-major).  The region starts 16-byte aligned and a level is
    // 128 * LW bytes, so every vector is aligned.
    __device__ __forceinline__ static void st_vec(uint32_t *p, const uint32_t (&v)[K])
    {
        if (K == 1) {
            p[0] = v[0];
        } else if (K == 2) {
            *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], v[1]);
        } else {
            *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1], v[2], v[3]);
        }
    }
    __device__ __forceinline__ static void ld_vec(const uint32_t *p, uint32_t (&v)[K])
    {
        if (K == 1) {
            v[0] = p[0];
        } else if (K == 2) {
            const uint2 t = *reinterpret_cast<const uint2 *>(p);
            v[0] = t.x;
            v[1] = t.y;
        } else {
            const uint4 t = *reinterpret_cast<const uint4 *>(p);
            v[0] = t.x;
            v[1] = t.y;
            v[2] = t.z;
            v[3] = t.w;
        }
    }
    __device__ __forceinline__ void put(int d, unsigned gl, const uint32_t (&P)[K], const uint32_t (&X)[K],
                                        unsigned pe, unsigned rs, uint64_t S)
    {
        if (d < SL) {
            uint32_t *w = sm + (size_t)d * LW * 32;
            st_vec(w + ln * K, P);
            st_vec(w + 32 * K + ln * K, X);
            if (M == 1) {
                if (gl < 4u) w[2 * K * 32 + ln] = pick(pe, rs, S, gl);
            } else {
#pragma unroll
                for (int j = 0; j < M; ++j) w[(2 * K + j) * 32 + ln] = pick(pe, rs, S, (unsigned)j);
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                lw[d][k] = P[k];
                lw[d][K + k] = X[k];
            }
            if (M == 1) {
                lw[d][2 * K] = pick(pe, rs, S, gl < 4u ? gl : 0u);
            } else {
#pragma unroll
                for (int j = 0; j < M; ++j) lw[d][2 * K + j] = pick(pe, rs, S, (unsigned)j);
            }
        }
    }
    __device__ __forceinline__ void put_px(int d, const uint32_t (&P)[K], const uint32_t (&X)[K])
    {
        if (d < SL) {
            uint32_t *w = sm + (size_t)d * LW * 32;
            st_vec(w + ln * K, P);
            st_vec(w + 32 * K + ln * K, X);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                lw[d][k] = P[k];
                lw[d][K + k] = X[k];
            }
        }
    }
    __device__ __forceinline__ void get(int d, uint32_t (&P)[K], uint32_t (&X)[K], uint32_t (&mr)[M])
    {
        if (d < SL) {
            const uint32_t *w = sm + (size_t)d * LW * 32;
            ld_vec(w + ln * K, P);
            ld_vec(w + 32 * K + ln * K, X);
#pragma unroll
            for (int j = 0; j < M; ++j) mr[j] = w[(2 * K + j) * 32 + ln];
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                P[k] = lw[d][k];
                X[k] = lw[d][K + k];
            }
#pragma unroll
            for (int j = 0; j < M; ++j) mr[j] = lw[d][2 * K + j];
        }
    }
};

// Fields of a stack level from the meta words get() returned.  Warp-uniform
// call (shuffles when the fields are spread over the group's lanes).
template <int G, int K>
__device__ __forceinline__ void meta_unpack(const Grp<G, K> &g, const uint32_t (&mr)[Stack<G, K>::M], unsigned &pe,
                                            unsigned &rs, uint64_t &S)
{
    if (Stack<G, K>::M == 1) {
        pe = __shfl_sync(FULL, mr[0], (int)g.gbase);
        rs = __shfl_sync(FULL, mr[0], (int)g.gbase + 1);
        const uint32_t lo = __shfl_sync(FULL, mr[0], (int)g.gbase + 2);
        const uint32_t hi = __shfl_sync(FULL, mr[0], (int)g.gbase + 3);
        S = (uint64_t)lo | ((uint64_t)hi << 32);
    } else {
        pe = mr[0];
        rs = mr[Stack<G, K>::M > 1 ? 1 : 0];
        S = (uint64_t)mr[Stack<G, K>::M > 2 ? 2 : 0] | ((uint64_t)mr[Stack<G, K>::M > 3 ? 3 : 0] << 32);
    }
}

// Publish a frame (P, X, pivot|end, |R|, S, and R itself when listing) as it
// stands to the global ring (one unit of global pending).  Warp-uniform call;
// true where it went.
template <int G, int K>
__device__ __forceinline__ bool push_global(const Grp<G, K> &g, const SearchParams &prm, bool pred,
                                            const uint32_t (&P)[K], const uint32_t (&X)[K], unsigned pe, unsigned rs,
                                            uint64_t S, bool list, const uint32_t (&R)[K], Counters &cn)
{
    constexpr int WP = G * K;
    const unsigned qmask = prm.qcap - 1u;
    unsigned ticket = 0, got = 0;
    if (pred && g.leader()) {
        atomicAdd(&prm.ctl->pending, 1u);
        got = q_reserve_push(prm.ctl, prm.seq, qmask, ticket, push_margin<G>(prm)) ? 1u : 0u;
        if (got) cn.note(kDiagGpush);
        if (!got) atomicSub(&prm.ctl->pending, 1u);
    }
    got = g.from_leader(got);
    ticket = g.from_leader(ticket);
    if (got) {
        uint32_t *fr = prm.frames + (size_t)(ticket & qmask) * prm.fs;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            __stcg(fr + kFrameHdr + g.gl * K + k, P[k]);
            __stcg(fr + kFrameHdr + WP + g.gl * K + k, X[k]);
            if (list) __stcg(fr + kFrameHdr + 2 * WP + g.gl * K + k, R[k]);
        }
        if (g.leader()) {
            __stcg(fr + 0, pe);
            __stcg(fr + 1, rs);
            __stcg(fr + 2, (uint32_t)S);
            __stcg(fr + 3, (uint32_t)(S >> 32));
        }
        __threadfence();
    }
    __syncwarp();
    if (got && g.leader()) st_release(&prm.seq[ticket & qmask], ticket + 1u);
    return got != 0u;
}

// ---------------------------------------------------------------------------
// The lane tier.  Most nodes of the search tree lie where few vertices are
// left: once a frame's P u X has at most 32 vertices, nothing outside that
// set can ever enter a descendant's P or X (Alg. 4 only intersects them with
// rows of vertices of P).  Such a frame is compressed: U = P u X in
// increasing position is relabelled 0..u-1 -- order-preserving, so "first in
// the order" is still the lowest set bit and every pivot rule (first of X or
// P; the TX / TomitaBB argmax with ties to the earliest) picks the same
// vertex -- its induced adjacency becomes u rows of 32 bits, and one lane
// runs Alg. 4 on it alone with single-word sets, next to 31 other lanes doing
// the same on their own subproblems.  The tree, the leaves and the hash terms
// (through the positions of the local vertices) are exactly those of the
// group search.

struct T2Lane {
    uint32_t P = 0, X = 0, L = 0, rs = 0;  // local sets of the current frame, |R|
    uint64_t S = 0;                        // S(R)
    int d = 0;                             // explicit-stack depth
    bool busy = false;
};

struct T2Warp {
    uint32_t *A;    // [32 local rows][32 lanes]
    uint16_t *pos;  // [32 local vertices][32 lanes]: position in the order
    uint32_t *stk;  // [levels][kT2Fields][32 lanes]
    uint32_t *piv;  // kPivotScratchWords: the lanes' words of P' (pivot scoring)
    int levels;
};

// One node of every busy lane's subproblem: the child v = first of L of the
// lane's current frame (the same step as the group search's section C, on
// 32-bit sets).  Divergent by design: no warp collectives inside.
template <int PIVOT>
__device__ __forceinline__ void t2_step(T2Lane &t, const T2Warp &m, unsigned lane, const uint64_t *hv,
                                        uint32_t *hist, uint64_t *out, uint32_t pivot_mode,
                                        uint32_t (&spill)[32][kT2Fields], Counters &cn, unsigned *busy_lanes)
{
    if (!t.busy) return;
    const int v = __ffs(t.L) - 1;
    t.L &= t.L - 1u;
    const uint32_t *A = m.A + lane;
    const uint32_t a = A[v * 32];
    const uint32_t Pc = t.P & a, Xc = t.X & a;  // P n N(v), X n N(v)
    t.P &= ~(1u << v);                           // P <- P \ {v}
    t.X |= 1u << v;                              // X <- X u {v}
    const uint64_t Sc = t.S + hv[m.pos[v * 32 + lane]];
    const unsigned k = t.rs + 1u;
    if (Pc == 0u) {
        if (Xc == 0u) {  // P u X empty: R u {v} is a maximal clique
            ++cn.cnt;
            cn.hash += mix64(Sc ^ mix64((uint64_t)k));
            cn.max = k > cn.max ? k : cn.max;
            const unsigned old = atomicAdd(&hist[k], 1u);
            if (old == 0xffffffffu)
                atomicAdd(reinterpret_cast<unsigned long long *>(out + MCE_OUT_HIST + k), 1ull << 32);
        } else {
            ++cn.dead;
        }
    } else {
        ++cn.intl;
    }
    uint32_t Lc = 0u;
    if (Pc != 0u) {
        int p;
        if (PIVOT == MCE_PIVOT_GREEDY) {
            p = __ffs(Xc != 0u ? Xc : Pc) - 1;
        } else {
            // argmax |P' n N(u)| over X' (TX, NX) or P' u X' (TomitaBB),
            // candidates in increasing position with '>' keeping the earliest
            uint32_t cand = (PIVOT == MCE_PIVOT_GREEDY_TX) ? Xc : (Pc | Xc);
            p = __ffs(Pc) - 1;  // TX with X' empty: first of P'
            int best = -1;
            const int all = __popc(Pc);
            const bool nx = PIVOT == MCE_PIVOT_GREEDY_TX && pivot_mode == MCE_PIVOT_GREEDY_NX;
            while (cand) {
                const int u = __ffs(cand) - 1;
                cand &= cand - 1u;
                const int c = __popc(Pc & A[u * 32]);
                if (c > best) {
                    best = c;
                    p = u;
                }
                if (nx && best == all) break;  // Naude's early exit: nothing later can beat it
            }
        }
        Lc = Pc & ~A[p * 32];  // L' = P' \ N(p)
    }
    if (Lc != 0u) {
        if (t.L != 0u) {  // the frame keeps children: push it
            const uint32_t f[kT2Fields] = {t.P, t.X, t.L, t.rs, (uint32_t)t.S, (uint32_t)(t.S >> 32)};
            if (t.d < m.levels) {
                uint32_t *w = m.stk + (size_t)t.d * kT2Fields * 32 + lane;
#pragma unroll
                for (int i = 0; i < kT2Fields; ++i) w[i * 32] = f[i];
            } else {
#pragma unroll
                for (int i = 0; i < kT2Fields; ++i) spill[t.d][i] = f[i];
            }
            ++t.d;
        }
        t.P = Pc;
        t.X = Xc;
        t.L = Lc;
        t.rs = k;
        t.S = Sc;
    } else if (t.L == 0u) {  // the frame is exhausted: back to its parent
        if (t.d == 0) {
            t.busy = false;
            atomicSub(busy_lanes, 1u);
        } else {
            --t.d;
            uint32_t f[kT2Fields];
            if (t.d < m.levels) {
                const uint32_t *w = m.stk + (size_t)t.d * kT2Fields * 32 + lane;
#pragma unroll
                for (int i = 0; i < kT2Fields; ++i) f[i] = w[i * 32];
            } else {
#pragma unroll
                for (int i = 0; i < kT2Fields; ++i) f[i] = spill[t.d][i];
            }
            t.P = f[0];
            t.X = f[1];
            t.L = f[2];
            t.rs = f[3];
            t.S = (uint64_t)f[4] | ((uint64_t)f[5] << 32);
        }
    }
}

// The search proper: the groups of this warp expand frames until the search
// is over or aborts.  Work moves at two levels: idle groups take frames from
// the block's shared-memory ring, which busy groups of the block refill by
// giving away the front of their shallowest branching set; a block with idle
// groups and an empty ring counts itself as starving, one of its idle warps
// polls the global ring, and busy groups feed the global ring while starving
// blocks outnumber its frames.  rows, hv, hist, lq are this block's staged
// rows (or global rows), vertex hash terms, clique-size histogram and ring.
// Called by all 32 lanes of every warp.
template <int G, int K, bool SMEM, int PIVOT, bool LIST>
__device__ __forceinline__ void search_loop(const SearchParams &prm, const uint32_t *rows, const uint64_t *hv,
                                            uint32_t *hist, const LocalQ &lq, const Thresholds th,
                                            uint32_t *stack_smem, int stack_smem_levels, unsigned char *t2_smem,
                                            Counters &cn)
{
    using Gp = Grp<G, K>;
    constexpr int WP = G * K;
    // the lane tier serves the counting kernels of groups of two or more
    // lanes (one-lane groups already search with one or two words per lane)
    constexpr bool T2 = !LIST && G >= 2;
    constexpr unsigned GPW = 32u / G;  // groups per warp
    const uint32_t n = prm.n;
    Ctl *ctl = prm.ctl;
    Gp g;
    g.init();
    uint32_t P[K], X[K], L[K];
#pragma unroll
    for (int k = 0; k < K; ++k) P[k] = X[k] = L[k] = 0u;
    unsigned pe = 0, rs = 0;
    uint64_t S = 0;
    int d = 0, dbase = 0;
    bool work = false;
    bool lempty = true;  // the current frame's branching set is exhausted
    bool poller = false;
    unsigned gq = 0;  // global ring length last seen
    // a claimed ticket of the device-wide ring whose frame this (idle) group
    // takes once it is published
    bool held = false;
    unsigned hticket = 0;
    // Clique listing (ListParams): this group's index, the |R| of the frame
    // it took last, and (leader) the chunk it appends records to.
    constexpr bool list = LIST;
    const unsigned gidx = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32u / G) + g.lane / G;
    unsigned rsb = 0, cpos = 0, cend = 0;
    bool cfull = false;

    using Stk = Stack<G, K>;
    uint32_t stack_local[kStackDepth][Stk::LW];
    Stk stk;
    stk.SL = stack_smem_levels;
    stk.sm = stack_smem + (size_t)(threadIdx.x >> 5) * (size_t)stack_smem_levels * Stk::LW * 32;
    stk.ln = g.lane;
    stk.lw = stack_local;

    // lane tier: this lane's subproblem and the warp's region
    T2Lane t2;
    T2Warp t2m;
    uint32_t t2_spill[32][kT2Fields];
    const unsigned t2p = T2 ? min(prm.t2_max_p, th.share_local) : 0u;
    {
        unsigned char *wb = t2_smem + (size_t)(threadIdx.x >> 5) * t2_warp_bytes(prm.t2_levels, PIVOT != MCE_PIVOT_GREEDY);
        t2m.A = reinterpret_cast<uint32_t *>(wb);
        t2m.pos = reinterpret_cast<uint16_t *>(wb + 32 * 32 * 4);
        t2m.stk = reinterpret_cast<uint32_t *>(wb + 32 * 32 * 4 + 32 * 32 * 2);
        t2m.piv = t2m.stk + (size_t)prm.t2_levels * kT2Fields * 32;
        t2m.levels = (int)prm.t2_levels;
    }
    unsigned t2it = 0;

    uint64_t quiet_since = 0;
    const uint64_t t_start = global_ns();
    unsigned last_pend = 0xffffffffu, last_head = 0xffffffffu;
    unsigned backoff = 32;
    const unsigned qmask = prm.qcap - 1u;
    const size_t lfs = frame_words(WP, list);

    auto rowp = [&](int v) -> const uint32_t * { return rows + (size_t)v * WP + g.gl * K; };

    // This lane's words of R for a frame of this group with |R| = r, plus
    // vertex `extra` when it is >= 0 (listing only).
    auto r_bits = [&](unsigned r, int extra, uint32_t (&out)[K]) {
        const uint32_t *b = prm.lst.base + (size_t)gidx * WP + g.gl * K;
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = b[k];
        const uint16_t *pp = prm.lst.path + (size_t)gidx * n;
        for (unsigned j = rsb; j < r; ++j) g.set(out, (int)pp[j]);
        if (extra >= 0) g.set(out, extra);
    };

    // Append the maximal clique R u {v} (|R| = rs) as a record to this
    // group's chunk.  Warp-uniform call; `emit` marks the groups reporting.
    auto emit_clique = [&](bool emit, int v) {
        const unsigned k = rs + 1u;
        unsigned ok = 0u, wpos = 0u;
        if (emit && g.leader()) {
            const unsigned need = k + 1u, CW = prm.lst.chunk_words;
            if (cpos + need > cend && !cfull) {
                if (cend) prm.lst.fill[cend / CW - 1u] = cpos - (cend - CW);  // retire the chunk
                const unsigned c = atomicAdd(prm.lst.next_chunk, 1u);
                if (c < prm.lst.n_chunks) {
                    cpos = c * CW;
                    cend = cpos + CW;
                } else {
                    cpos = cend = 0u;
                    cfull = true;
                    atomicExch(prm.lst.overflow, 1u);
                }
            }
            if (!cfull && cpos + need <= cend) {
                ok = 1u;
                wpos = cpos;
                cpos += need;
            }
        }
        ok = g.from_leader(ok);
        wpos = g.from_leader(wpos);
        uint32_t rb[K];
        const uint32_t *b = prm.lst.base + (size_t)gidx * WP + g.gl * K;
#pragma unroll
        for (int kk = 0; kk < K; ++kk) rb[kk] = (emit && ok) ? b[kk] : 0u;
        int c = 0;
#pragma unroll
        for (int kk = 0; kk < K; ++kk) c += __popc(rb[kk]);
        int o = g.excl_scan(c);
        if (emit && ok) {
            // R of the taken frame fills slots [0, rsb), the path [rsb, rs),
            // the leaf vertex slot rs
            uint32_t *rec = prm.lst.rec + wpos + 1u;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                uint32_t w = rb[kk];
                while (w) {
                    if (o < (int)rsb) rec[o] = (g.gl * K + kk) * 32u + (unsigned)(__ffs(w) - 1);
                    ++o;
                    w &= w - 1u;
                }
            }
            const uint16_t *pp = prm.lst.path + (size_t)gidx * n;
            for (unsigned j = rsb + g.gl; j < rs; j += G) rec[j] = pp[j];
            if (g.leader()) {
                rec[rs] = (uint32_t)v;
                prm.lst.rec[wpos] = 0x80000000u | k;
            }
        }
    };

    // Take (P, X, pivot|end, |R|, S) as this group's frame.
    uint64_t t_busy = 0;
    auto start_frame = [&]() {
        work = true;
        lempty = false;
        rsb = rs;
        if (g.leader()) t_busy = global_ns();
        d = dbase = 0;
        uint32_t rp[K];
        load_row<K, SMEM>(rp, rowp((int)(pe & 0xffffu)));
#pragma unroll
        for (int k = 0; k < K; ++k) L[k] = P[k] & ~rp[k] & g.below(k, pe >> 16);
    };

    // Share the shallowest frame this group owns (the stack bottom, else the
    // current frame) through level LOCAL (true: block ring, false: global).
    auto share = [&](bool want, bool local, int min_p) {
        const bool from_stack = want && d > dbase;
        uint32_t sP[K], sX[K], sL[K], l1[K];
        uint32_t mr[Stk::M];
#pragma unroll
        for (int j = 0; j < Stk::M; ++j) mr[j] = 0u;
        unsigned spe = pe, srs = rs;
        uint64_t sS = S;
        if (from_stack) stk.get(dbase, sP, sX, mr);
        {
            unsigned pe2, rs2;
            uint64_t S2;
            meta_unpack<G, K>(g, mr, pe2, rs2, S2);
            if (from_stack) {
                spe = pe2;
                srs = rs2;
                sS = S2;
            }
        }
        if (from_stack) {
            uint32_t rp[K];
            load_row<K, SMEM>(rp, rowp((int)(spe & 0xffffu)));
#pragma unroll
            for (int k = 0; k < K; ++k) sL[k] = sP[k] & ~rp[k] & g.below(k, spe >> 16);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                sP[k] = P[k];
                sX[k] = X[k];
                sL[k] = L[k];
            }
        }
        uint32_t sR[K];
#pragma unroll
        for (int k = 0; k < K; ++k) sR[k] = 0u;
        if (list && want) r_bits(srs, -1, sR);
        bool whole = false, gave;
        if (local)
            gave = donate_front<G, K, true>(g, prm, lq, want, from_stack, min_p, sP, sX, sL, spe, srs, sS,
                                            list, sR, l1, whole, cn);
        else
            gave = donate_front<G, K, false>(g, prm, lq, want, from_stack, min_p, sP, sX, sL, spe, srs, sS,
                                             list, sR, l1, whole, cn);
        if (gave) {
            if (from_stack) {
                if (whole) {
                    ++dbase;
                } else {
                    uint32_t nP[K], nX[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        nP[k] = sP[k] & ~l1[k];
                        nX[k] = sX[k] | l1[k];
                    }
                    stk.put_px(dbase, nP, nX);
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    P[k] &= ~l1[k];
                    X[k] |= l1[k];
                    L[k] &= ~l1[k];
                }
            }
        }
    };

    // Hand the child frames (Pc, Xc, Lc, |R| = rs1, S = Sc) of the groups
    // with `comp` to free lanes of this warp as lane-tier subproblems (the
    // first groups in lane order, as many as lanes are free).  Per group: the
    // group's lanes list U = Pc u Xc in order into the slot's position column
    // and form the local P, X, L words; then the whole warp builds the local
    // rows, one ballot per row (lane i tests whether U[i] is adjacent to
    // U[j]).  Warp-uniform call; true in the groups whose frame was taken.
    auto t2_take = [&](bool comp, const uint32_t (&Pc)[K], const uint32_t (&Xc)[K], const uint32_t (&Lc)[K],
                       unsigned rs1, uint64_t Sc) -> bool {
        const unsigned freem = ~__ballot_sync(FULL, t2.busy);
        const unsigned leads = __ballot_sync(FULL, comp && g.leader());
        const unsigned rank = (unsigned)__popc(leads & ((1u << g.gbase) - 1u));
        const bool ok = comp && rank < (unsigned)__popc(freem);
        const unsigned okl = __ballot_sync(FULL, ok && g.leader());
        if (okl == 0u) return false;
        unsigned f = freem;
        for (unsigned r = 0; r < rank && f; ++r) f &= f - 1u;
        const unsigned slot = (ok && f) ? (unsigned)(__ffs(f) - 1) : 0u;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) cnt += ok ? __popc(Pc[k] | Xc[k]) : 0;
        const int off = g.excl_scan(cnt);
        const int u_grp = g.sum(cnt);
        uint32_t lp = 0u, lx = 0u, ll = 0u;
        if (ok) {
            unsigned i = (unsigned)off;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                uint32_t w = Pc[k] | Xc[k];
                while (w) {
                    const unsigned b = (unsigned)(__ffs(w) - 1);
                    w &= w - 1u;
                    t2m.pos[i * 32 + slot] = (uint16_t)((g.gl * K + k) * 32u + b);
                    lp |= ((Pc[k] >> b) & 1u) << i;
                    lx |= ((Xc[k] >> b) & 1u) << i;
                    ll |= ((Lc[k] >> b) & 1u) << i;
                    ++i;
                }
            }
        }
        if (G > 1) {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                lp |= __shfl_xor_sync(FULL, lp, o);
                lx |= __shfl_xor_sync(FULL, lx, o);
                ll |= __shfl_xor_sync(FULL, ll, o);
            }
        }
        __syncwarp();
        unsigned todo = okl;
        while (todo) {
            const int gb = __ffs(todo) - 1;
            todo &= todo - 1u;
            const unsigned s = __shfl_sync(FULL, slot, gb);
            const unsigned u = (unsigned)__shfl_sync(FULL, u_grp, gb);
            const uint32_t P0 = __shfl_sync(FULL, lp, gb), X0 = __shfl_sync(FULL, lx, gb);
            const uint32_t L0 = __shfl_sync(FULL, ll, gb), r0 = __shfl_sync(FULL, rs1, gb);
            const uint32_t s_lo = __shfl_sync(FULL, (uint32_t)Sc, gb), s_hi = __shfl_sync(FULL, (uint32_t)(Sc >> 32), gb);
            const unsigned q = g.lane < u ? (unsigned)t2m.pos[g.lane * 32 + s] : 0u;
            const uint32_t *rq = rows + (q >> 5);
            const unsigned qb = q & 31u;
            uint32_t row = 0u;
#pragma unroll 4
            for (unsigned j = 0; j < u; ++j) {
                const unsigned qj = (unsigned)__shfl_sync(FULL, q, (int)j);
                uint32_t w = 0u;
                if (g.lane < u) w = SMEM ? rq[(size_t)qj * WP] : __ldg(rq + (size_t)qj * WP);
                const unsigned b = __ballot_sync(FULL, (w >> qb) & 1u);
                if (g.lane == j) row = b;
            }
            if (g.lane < u) t2m.A[g.lane * 32 + s] = row;
            if (g.lane == s) {
                t2.P = P0;
                t2.X = X0;
                t2.L = L0;
                t2.rs = r0;
                t2.S = (uint64_t)s_lo | ((uint64_t)s_hi << 32);
                t2.d = 0;
                t2.busy = true;
            }
        }
        __syncwarp();
        if (g.lane == 0) {
            cn.note(kDiagLaneTasks, (unsigned long long)__popc(okl));
            atomicAdd(&lq.h->t2_busy, (unsigned)__popc(okl));
        }
        return ok;
    };

    for (unsigned it = 0;;) {
        // ---- T: the lane tier.  While this warp's lanes hold subproblems,
        // a lane step advances every one of them by a node.  It runs when
        // fewer lanes are free than the warp has groups (room is made before
        // the groups may hand over more), and when no group of the warp has a
        // frame -- then every 4th iteration still goes through A and B so
        // idle groups can take frames.
        bool t2any = false;
        if (T2) {
            const unsigned busym = __ballot_sync(FULL, t2.busy);
            t2any = busym != 0u;
            if (t2any) {
                const unsigned g1 = __ballot_sync(FULL, work);
                if (32u - (unsigned)__popc(busym) < GPW || (g1 == 0u && (++t2it & 3u) != 0u)) {
                    t2_step<PIVOT>(t2, t2m, g.lane, hv, hist, prm.out, prm.pivot_mode, t2_spill, cn,
                                   &lq.h->t2_busy);
                    continue;
                }
            }
        }
        ++it;  // group-search iterations: the periodic ring checks below count these
        // ---- A: a frame whose branching set is exhausted returns to its
        // parent (a stacked level always has children left), or the group's
        // work is done
        const bool lpop = work && lempty && d > dbase;
        const bool lfin = work && lempty && d <= dbase;
        {
            uint32_t mr[Stk::M];
#pragma unroll
            for (int j = 0; j < Stk::M; ++j) mr[j] = 0u;
            if (lpop) {
                --d;
                stk.get(d, P, X, mr);
            }
            if (__ballot_sync(FULL, lpop) != 0u) {
                unsigned pe2, rs2;
                uint64_t S2;
                meta_unpack<G, K>(g, mr, pe2, rs2, S2);
                if (lpop) {
                    pe = pe2;
                    rs = rs2;
                    S = S2;
                    lempty = false;
                    uint32_t rp[K];
                    load_row<K, SMEM>(rp, rowp((int)(pe & 0xffffu)));
#pragma unroll
                    for (int k = 0; k < K; ++k) L[k] = P[k] & ~rp[k] & g.below(k, pe >> 16);
                }
            }
        }
        if (lfin) {
            work = false;
            lempty = false;
            if (g.leader()) {
                cn.note(kDiagBusyNs, global_ns() - t_busy);
                atomicAdd(&lq.h->idle, 1u);
                // the last work of the block gives back its unit
                if (atomicSub(&lq.h->bwork, 1u) == 1u) atomicSub(&ctl->pending, 1u);
            }
        }

        // ---- B1: the block ring (idle groups take, busy groups refill)
        const unsigned busy_b = __ballot_sync(FULL, work);
        if (busy_b != FULL || (it & (prm.tune.local_check - 1u)) == 0u) {
            unsigned lh = 0, lt = 0, li = 0, ld = 0;
            if (g.lane == 0) {
                lh = vld(&lq.h->head);
                lt = vld(&lq.h->tail);
                li = vld(&lq.h->idle);
                ld = vld(&lq.h->done);
            }
            lh = __shfl_sync(FULL, lh, 0);
            lt = __shfl_sync(FULL, lt, 0);
            li = __shfl_sync(FULL, li, 0);
            ld = __shfl_sync(FULL, ld, 0);
            if (busy_b == 0u && ld && !t2any) break;
            const unsigned lqueued = lt - lh;
            unsigned ticket = 0, got = 0;
            if (!work && !held && lqueued != 0u && g.leader()) got = lq_reserve_pop(lq.h, lq.seq, lq.mask, ticket) ? 1u : 0u;
            got = g.from_leader(got);
            ticket = g.from_leader(ticket);
            if (got) {
                __threadfence_block();
                const volatile uint32_t *fr = lq.frames + (size_t)(ticket & lq.mask) * lfs;
                pe = fr[0];
                rs = fr[1];
                S = (uint64_t)fr[2] | ((uint64_t)fr[3] << 32);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    P[k] = fr[kFrameHdr + g.gl * K + k];
                    X[k] = fr[kFrameHdr + WP + g.gl * K + k];
                }
                if (list) {
                    uint32_t *b = prm.lst.base + (size_t)gidx * WP + g.gl * K;
#pragma unroll
                    for (int k = 0; k < K; ++k) b[k] = fr[kFrameHdr + 2 * WP + g.gl * K + k];
                }
            }
            __syncwarp();
            if (got) {
                if (g.leader()) {
                    __threadfence_block();
                    vst(&lq.seq[ticket & lq.mask], ticket + lq.mask + 1u);
                    atomicSub(&lq.h->idle, 1u);
                    cn.note(kDiagSteals);
                }
                start_frame();
            }
            const bool hungry = work && !got && li > lqueued;
            // with half the block's groups idle, smaller frames are worth moving
            const unsigned bgroups = (blockDim.x >> 5) * (32u / G);
            const int lmin = 2u * li > bgroups ? (int)min(th.share_local, prm.tune.share_tail) : (int)th.share_local;
            if (__ballot_sync(FULL, hungry) != 0u) share(hungry, true, lmin);
        }

        // ---- B2: the global ring and the end of the search.  Global state is
        // read by the block's polling warp (an all-idle warp) or, at most
        // every tune.refresh_ns, by one busy warp, and cached in shared memory.
        const unsigned busy2 = __ballot_sync(FULL, work);
        const bool anyheld = __ballot_sync(FULL, held) != 0u;
        const bool periodic = busy2 == 0u || (it & (prm.tune.global_check - 1u)) == 0u;
        // a held ticket is looked at every eighth iteration of a warp whose
        // other groups are busy (each look is a round trip to L2)
        if (periodic || (anyheld && (it & 7u) == 0u)) {
            unsigned head = 0, tail = 0, pend = 1, starving = 0, ab = 0, lh = 0, lt = 0, done = 0;
            bool pol = poller;
            if (g.lane == 0) {
                lh = vld(&lq.h->head);
                lt = vld(&lq.h->tail);
                // the polling warp is one with nothing at all to do (no frame and no
                // lane-tier subproblem): it polls every iteration
                if (busy2 == 0u && !pol && !t2any) pol = atomicCAS(&lq.h->poller, 0u, 1u) == 0u;
                const uint64_t now = global_ns();
                bool refresh = pol;
                if (!refresh && now - *reinterpret_cast<volatile unsigned long long *>(&lq.h->stamp) > prm.tune.refresh_ns)
                    refresh = atomicCAS(&lq.h->refreshing, 0u, 1u) == 0u;
                if (refresh) {
                    ab = ld_relaxed(&ctl->abort);
                    pend = ld_relaxed(&ctl->pending);
                    head = ld_relaxed(&ctl->head);
                    tail = ld_relaxed(&ctl->tail);
                    starving = ld_relaxed(&ctl->starving);
                    // this block is starving while it has idle groups and an empty ring
                    const bool st = vld(&lq.h->idle) != 0u && lt == lh;
                    if (st != (vld(&lq.h->starving) != 0u)) {
                        if (st) {
                            if (atomicExch(&lq.h->starving, 1u) == 0u) atomicAdd(&ctl->starving, 1u);
                        } else {
                            if (atomicExch(&lq.h->starving, 0u) == 1u) atomicSub(&ctl->starving, 1u);
                        }
                    }
                    vst(&lq.h->g_head, head);
                    vst(&lq.h->g_tail, tail);
                    vst(&lq.h->g_starving, starving);
                    if (ab || pend == 0u) vst(&lq.h->done, ab ? 2u : 1u);
                    *reinterpret_cast<volatile unsigned long long *>(&lq.h->stamp) = now;
                    if (prm.trace) {
                        const unsigned ti = atomicAdd(&lq.h->trace_n, 1u);
                        if (ti < prm.trace_per_block) {
                            const unsigned groups = prm.total_groups / gridDim.x;
                            const unsigned busy = groups - min(groups, vld(&lq.h->idle));
                            const unsigned qg = (int)(tail - head) > 0 ? min(tail - head, 65535u) : 0u;
                            const unsigned sv = min(starving, 65535u);
                            unsigned long long *rec = prm.trace + 2ull * ((size_t)blockIdx.x * prm.trace_per_block + ti);
                            rec[0] = now;
                            rec[1] = (unsigned long long)busy | ((unsigned long long)min(vld(&lq.h->t2_busy), 65535u) << 16) |
                                     ((unsigned long long)qg << 32) | ((unsigned long long)sv << 48);
                        }
                    }
                    if (now - t_start > 10ull * prm.timeout_ns) set_status(prm.out, ctl, MCE_ETIMEOUT);
                    if (!pol) atomicExch(&lq.h->refreshing, 0u);
                } else {
                    head = vld(&lq.h->g_head);
                    tail = vld(&lq.h->g_tail);
                    starving = vld(&lq.h->g_starving);
                    ab = vld(&lq.h->done) == 2u ? 1u : 0u;
                }
                done = vld(&lq.h->done);
            }
            pol = __shfl_sync(FULL, pol ? 1u : 0u, 0) != 0u;
            poller = pol;
            ab = __shfl_sync(FULL, ab, 0);
            pend = __shfl_sync(FULL, pend, 0);
            head = __shfl_sync(FULL, head, 0);
            tail = __shfl_sync(FULL, tail, 0);
            starving = __shfl_sync(FULL, starving, 0);
            lh = __shfl_sync(FULL, lh, 0);
            lt = __shfl_sync(FULL, lt, 0);
            done = __shfl_sync(FULL, done, 0);
            if (ab) break;
            if (busy2 == 0u && done && !t2any) break;
            // (claimed tickets can run ahead of the producers': nothing queued)
            const unsigned queued = (int)(tail - head) > 0 ? tail - head : 0u;
            gq = queued;

            // An idle group takes a global frame when its block's ring is
            // empty; only the block's polling warp asks, one group per try, so
            // the ring's head sees one contender per block instead of one per
            // idle group (the block's other groups get work from the taker
            // through the block ring).
            // (A block-private ring, as in the batched form, has no other
            // contenders: there every idle group asks.)
            // The polling warp's first asking group takes frames for up to four
            // of the warp's asking groups with one ticket advance.
            unsigned ticket = 0, got = 0;
            const bool ring_shared = prm.total_groups > (blockDim.x >> 5) * (32u / G);
            const bool ask = !work && !held && queued != 0u && lt == lh && (poller || !ring_shared) && g.leader();
            const unsigned askers = __ballot_sync(FULL, ask);
            if (!ring_shared) {
                if (ask) {
                    cn.note(kDiagGtry);
                    got = q_reserve_pop(ctl, prm.seq, qmask, ticket, cn.diag + kDiagCasFail, prm.tune.pop_tries) ? 1u : 0u;
                }
            } else if (askers != 0u) {
                const unsigned lead = (unsigned)(__ffs(askers) - 1);
                unsigned first = 0u, k = 0u;
                if (g.lane == lead) {
                    cn.note(kDiagGtry);
                    k = q_claim(ctl, min(4u, (unsigned)__popc(askers)), first);
                }
                k = __shfl_sync(FULL, k, (int)lead);
                first = __shfl_sync(FULL, first, (int)lead);
                const unsigned rank = (unsigned)__popc(askers & ((1u << g.lane) - 1u));
                if (ask && rank < k) {
                    held = true;
                    hticket = first + rank;
                }
            }
            got = g.from_leader(got);
            ticket = g.from_leader(ticket);
            held = g.from_leader(held ? 1u : 0u) != 0u;
            hticket = g.from_leader(hticket);
            if (ring_shared && __ballot_sync(FULL, held) != 0u) {
                // a held ticket's frame, once its producer has published it
                unsigned rdy = 0u;
                if (held && g.leader()) rdy = ld_acquire(&prm.seq[hticket & qmask]) == hticket + 1u ? 1u : 0u;
                rdy = g.from_leader(rdy);
                if (rdy) {
                    got = 1u;
                    ticket = hticket;
                    held = false;
                }
            }
            if (got) {
                __threadfence();
                const uint32_t *fr = prm.frames + (size_t)(ticket & qmask) * prm.fs;
                pe = __ldcg(fr + 0);
                rs = __ldcg(fr + 1);
                S = (uint64_t)__ldcg(fr + 2) | ((uint64_t)__ldcg(fr + 3) << 32);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    P[k] = __ldcg(fr + kFrameHdr + g.gl * K + k);
                    X[k] = __ldcg(fr + kFrameHdr + WP + g.gl * K + k);
                }
                if (list) {
                    uint32_t *b = prm.lst.base + (size_t)gidx * WP + g.gl * K;
#pragma unroll
                    for (int k = 0; k < K; ++k) b[k] = __ldcg(fr + kFrameHdr + 2 * WP + g.gl * K + k);
                }
            }
            __syncwarp();
            if (got) {
                if (g.leader()) {
                    st_release(&prm.seq[ticket & qmask], ticket + prm.qcap);
                    atomicSub(&lq.h->idle, 1u);
                    // an already active block absorbs the frame's unit
                    if (atomicAdd(&lq.h->bwork, 1u) != 0u) atomicSub(&ctl->pending, 1u);
                    cn.note(kDiagSteals);
                    cn.note(kDiagGlobal);
                }
                start_frame();
            }
            if (poller && __ballot_sync(FULL, work) != 0u) {
                // busy now: hand the polling role to another idle warp
                if (g.lane == 0) atomicExch(&lq.h->poller, 0u);
                poller = false;
            }

            // busy groups feed starving blocks
            const bool hungry = periodic && work && !got && starving > queued;
            // with half the blocks starving (the search is draining), so are
            // smaller frames
            const int gmin = 2u * starving > gridDim.x ? (int)min(th.share_global, prm.tune.share_tail)
                                                       : (int)th.share_global;
            if (__ballot_sync(FULL, hungry) != 0u) share(hungry, false, gmin);

            if (__ballot_sync(FULL, work) == 0u) {
                if (T2 && t2any) continue;  // no frame, but subproblems: back to the lane tier
                // nobody here has work: back off; the poller watches for a
                // stalled search
                if (g.lane == 0 && poller) {
                    const uint64_t now = global_ns();
                    if (pend != last_pend || head != last_head || quiet_since == 0) {
                        quiet_since = now;
                        last_pend = pend;
                        last_head = head;
                    } else if (now - quiet_since > prm.timeout_ns) {
                        set_status(prm.out, ctl, MCE_ETIMEOUT);
                    }
                }
                // the poller backs off to 1 us; other idle warps only wait for
                // the block ring and may sleep longer (fewer issue slots taken
                // from the busy warps of the SM)
                __nanosleep(backoff);
                const unsigned cap = (poller || anyheld) ? 1024u : prm.tune.idle_sleep_ns;
                backoff = backoff < cap ? backoff * 2u : cap;
                continue;
            }
            backoff = 32;
        }

        // ---- C: expand one child v = first(L) of every active frame.  After
        // A and B every busy group has a non-empty branching set: pops and
        // queued frames always carry children, and giving work away always
        // leaves the giver at least one.
        // (a frame without children would give v < 0; the group then just
        // returns from it, reading no row)
        const int v = g.first(L);
        const bool act = work && v >= 0;
        uint32_t Pc[K], Xc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) Pc[k] = Xc[k] = 0u;
        if (act) {
            g.clear(L, v);
            uint32_t r[K];
            load_row<K, SMEM>(r, rowp(v));
#pragma unroll
            for (int k = 0; k < K; ++k) {
                Pc[k] = P[k] & r[k];  // P n N(v)
                Xc[k] = X[k] & r[k];  // X n N(v)
            }
            g.clear(P, v);  // P <- P \ {v}
            g.set(X, v);    // X <- X u {v}
        }
        // first vertices of X' and P' (ChoosePivotOrdered's candidates) also
        // answer the emptiness tests of the leaf test
        bool bx, bp;
        int fp = -1, pg = -1;
        if (PIVOT == MCE_PIVOT_GREEDY) {
            pg = g.first_either(Xc, Pc, bx, bp);
        } else {
            const int fx = g.first(Xc);
            fp = g.first(Pc);
            bx = fx >= 0;
            bp = fp >= 0;
        }
        uint64_t Sc = 0;
        if (act) Sc = S + hv[v];  // every lane keeps |R| and S
        // every node is internal, a leaf or a dead end (nodes = their sum,
        // formed when the counters are flushed)
        const bool lead = act && g.leader();
        cn.intl += (lead && bp) ? 1u : 0u;
        cn.dead += (lead && !bp && bx) ? 1u : 0u;
        if (lead && !bp && !bx) {  // P u X empty: R u {v} is a maximal clique
            const unsigned k = rs + 1u;
            ++cn.cnt;
            cn.hash += mix64(Sc ^ mix64((uint64_t)k));
            cn.max = k > cn.max ? k : cn.max;
            const unsigned old = atomicAdd(&hist[k], 1u);
            if (old == 0xffffffffu)
                atomicAdd(reinterpret_cast<unsigned long long *>(prm.out + MCE_OUT_HIST + k), 1ull << 32);
        }
        if (list) {
            const bool emit = act && !bp && !bx;
            if (__ballot_sync(FULL, emit) != 0u) emit_clique(emit, v);
        }
        const bool inter = act && bp;

        // ChoosePivotOrdered on the child (P', X')
        int pc;
        if (PIVOT == MCE_PIVOT_GREEDY) {
            pc = pg;
        } else if (T2 && prm.t2_max_p != 0u) {
            // argmax |P' n N(u)| over X' (TX, NX) or P' u X' (TomitaBB), all
            // candidates at once: the lanes' words of P' go to the warp's
            // scratch, every lane scores the candidates in its own words
            // against the whole of P' (16-byte loads starting at a chunk
            // rotated by lane, so a phase of eight lanes hits distinct
            // banks), and one packed max (score + 1, 0xffff - position) over
            // the group keeps the highest score, earliest on ties.  NX has
            // TX's pivot (its early exit only saves work).
            Stk::st_vec(t2m.piv + g.lane * K, Pc);
            __syncwarp();
            const uint32_t *pw = t2m.piv + g.gbase * K;  // this group's P' (WP words)
            unsigned best = 0u;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                uint32_t w = 0u;
                if (inter) w = (PIVOT == MCE_PIVOT_GREEDY_TX) ? (bx ? Xc[k] : 0u) : (Pc[k] | Xc[k]);
                while (w) {
                    const unsigned b = (unsigned)(__ffs(w) - 1);
                    w &= w - 1u;
                    const unsigned u = (g.gl * K + k) * 32u + b;
                    const uint32_t *ru = rows + (size_t)u * WP;
                    int c = 0;
                    if (WP >= 4) {
                        constexpr int NC = WP >= 4 ? WP / 4 : 1;
#pragma unroll 4
                        for (int j = 0; j < NC; ++j) {
                            const int jj = ((j + (int)g.lane) & (NC - 1)) * 4;
                            const uint4 a = *reinterpret_cast<const uint4 *>(pw + jj);
                            const uint4 r = SMEM ? *reinterpret_cast<const uint4 *>(ru + jj)
                                                 : __ldg(reinterpret_cast<const uint4 *>(ru + jj));
                            c += __popc(a.x & r.x) + __popc(a.y & r.y) + __popc(a.z & r.z) + __popc(a.w & r.w);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < WP; ++j) c += __popc(pw[j] & (SMEM ? ru[j] : __ldg(ru + j)));
                    }
                    const unsigned key = ((unsigned)(c + 1) << 16) | (0xffffu - u);
                    best = key > best ? key : best;
                }
            }
            if (G > 1) {
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) {
                    const unsigned y = __shfl_xor_sync(FULL, best, o);
                    best = y > best ? y : best;
                }
            }
            __syncwarp();
            pc = best ? (int)(0xffffu - (best & 0xffffu)) : ((PIVOT == MCE_PIVOT_GREEDY_TX) ? fp : -1);
        } else {
            // argmax |P' n N(u)| over X' (TX) or P' u X' (TomitaBB); scanning
            // candidates in increasing position with '>' keeps the earliest
            uint32_t cand[K];
#pragma unroll
            for (int k = 0; k < K; ++k) cand[k] = (PIVOT == MCE_PIVOT_GREEDY_TX) ? (bx ? Xc[k] : 0u) : (Pc[k] | Xc[k]);
            if (!inter) {
#pragma unroll
                for (int k = 0; k < K; ++k) cand[k] = 0u;
            }
            int best = -1;
            pc = (PIVOT == MCE_PIVOT_GREEDY_TX) ? fp : -1;  // X' empty: first of P'
            // GreedyBBNX (the TX kernel with pivot_mode NX): Naude's early exit.
            // A candidate's count is one group-wide popcount here, so the
            // exit is at candidate level: once a candidate covers all of P'
            // (|P' n K(u)| = 0), no later one can beat it and the scan stops.
            const bool nx = PIVOT == MCE_PIVOT_GREEDY_TX && prm.pivot_mode == MCE_PIVOT_GREEDY_NX;
            int npc = 0;
            if (nx) {
#pragma unroll
                for (int k = 0; k < K; ++k) npc += __popc(Pc[k]);
                npc = g.sum(npc);
            }
            for (;;) {
                uint32_t o = 0;
#pragma unroll
                for (int k = 0; k < K; ++k) o |= cand[k];
                if (__ballot_sync(FULL, o != 0u) == 0u) break;
                const int u = g.first(cand);
                uint32_t r[K];
#pragma unroll
                for (int k = 0; k < K; ++k) r[k] = 0u;
                if (u >= 0) load_row<K, SMEM>(r, rowp(u));
                int cnt = 0;
#pragma unroll
                for (int k = 0; k < K; ++k) cnt += __popc(Pc[k] & r[k]);
                cnt = g.sum(cnt);
                if (u >= 0) {
                    if (cnt > best) {
                        best = cnt;
                        pc = u;
                    }
                    g.clear(cand, u);
                    if (nx && best == npc) {
#pragma unroll
                        for (int k = 0; k < K; ++k) cand[k] = 0u;
                    }
                }
            }
        }

        uint32_t Lc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) Lc[k] = 0u;
        if (inter) {
            uint32_t r[K];
            load_row<K, SMEM>(r, rowp(pc));
#pragma unroll
            for (int k = 0; k < K; ++k) Lc[k] = Pc[k] & ~r[k];  // L' = P' \ N(p)
        }
        bool hasLc, more;
        g.any2(Lc, L, hasLc, more);
        bool desc = inter && hasLc;
        if (T2 && t2p != 0u) {
            // a child whose P' u X' has at most 32 vertices and whose P' is
            // small enough goes to a free lane of the warp instead
            int cu = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) cu += (__popc(Pc[k] | Xc[k]) << 16) | __popc(Pc[k]);
            cu = g.sum(cu);
            const bool comp = desc && (cu >> 16) <= 32 && (unsigned)(cu & 0xffff) <= t2p;
            if (__ballot_sync(FULL, comp) != 0u) {
                if (t2_take(comp, Pc, Xc, Lc, rs + 1u, Sc)) desc = false;
            }
        }
        // Breadth-first split of the top of the tree: a new subtree with a
        // large candidate set goes to the global ring (while the ring is short
        // of frames; gq is the same in every lane) instead of being descended
        // into here.
        const bool split_open = gq < prm.split_target;  // warp-uniform
        const bool try_split = desc && split_open;
        bool any_split = false;
        if (split_open) any_split = __ballot_sync(FULL, try_split) != 0u;
        if (any_split) {
            int cp = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) cp += __popc(Pc[k]);
            const int np = g.sum(cp);
            const bool sp = try_split && (unsigned)np >= th.split;
            uint32_t sR[K];
#pragma unroll
            for (int k = 0; k < K; ++k) sR[k] = 0u;
            if (list && sp) r_bits(rs, v, sR);
            const bool pushed = push_global<G, K>(g, prm, sp, Pc, Xc, (unsigned)pc | (n << 16), rs + 1u, Sc, list, sR, cn);
            if (pushed) {
                desc = false;
                if (g.leader()) cn.note(kDiagDonations);
            }
        }
        bool spill = false;
        if (desc && more) {
            if (d < (int)prm.stack_levels) {
                stk.put(d, g.gl, P, X, pe, rs, S);
                ++d;
            } else {
                spill = true;
            }
        }
        if (__ballot_sync(FULL, spill) != 0u) {
            // stack full: the rest of this frame (L is non-empty) goes to the
            // global ring as it stands, and the group descends without it
            uint32_t sR[K];
#pragma unroll
            for (int k = 0; k < K; ++k) sR[k] = 0u;
            if (list && spill) r_bits(rs, -1, sR);
            const bool pushed = push_global<G, K>(g, prm, spill, P, X, pe, rs, S, list, sR, cn);
            if (pushed && g.leader()) cn.note(kDiagDonations);
            if (spill && !pushed && g.leader()) set_status(prm.out, ctl, MCE_EOVERFLOW);
        }
        lempty = (act && !desc && !more) || (work && v < 0);
        if (desc) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                P[k] = Pc[k];
                X[k] = Xc[k];
                L[k] = Lc[k];
            }
            if (list) prm.lst.path[(size_t)gidx * n + rs] = (uint16_t)v;  // R grows by v at |R| = rs
            pe = (unsigned)pc | (n << 16);
            rs = rs + 1u;
            S = Sc;
        }
    }
    if (list && g.leader() && cend)  // retire the last chunk
        prm.lst.fill[cend / prm.lst.chunk_words - 1u] = cpos - (cend - prm.lst.chunk_words);
}

template <int G, int K, bool SMEM, int PIVOT, bool LIST>
__global__ void __launch_bounds__(512) search_kernel(const SearchParams prm)
{
    constexpr int WP = G * K;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;

    const uint32_t n = prm.n;
    const size_t rbytes = smem_rows_bytes(n, WP, SMEM);
    uint32_t *srows = reinterpret_cast<uint32_t *>(smem_raw);
    uint64_t *hv = reinterpret_cast<uint64_t *>(smem_raw + rbytes);
    uint32_t *hist = reinterpret_cast<uint32_t *>(hv + n);
    const LocalQ lq = local_queue_at(smem_raw + smem_local_offset(n, WP, SMEM), WP, prm.local_slots);
    local_queue_reset(lq, (blockDim.x / 32u) * (32u / G));

    // ---- prologue: stage the rows (bulk copy), hash terms, histogram
    if (SMEM) {
        if (threadIdx.x == 0) mbar_init(&mbar);
        __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) hv[i] = mix64((uint64_t)prm.order[i] + 1u);
    for (uint32_t i = threadIdx.x; i <= n; i += blockDim.x) hist[i] = 0u;
    bool staged = true;
    if (SMEM) staged = stage_rows(srows, prm.rows, (uint32_t)rbytes, (uint32_t)__cvta_generic_to_shared(&mbar), 0u);
    if (!staged && threadIdx.x == 0) set_status(prm.out, prm.ctl, MCE_ETIMEOUT);
    const bool ok = __syncthreads_and(staged) != 0;

    __shared__ unsigned deg_sum;
    const Thresholds th = density_thresholds(SMEM ? srows : prm.rows, n, WP, prm.tune.share_local,
                                             prm.tune.share_global, prm.split_min_p, &deg_sum,
                                             prm.tune.small_split != 0u);
    uint32_t *stack_smem = reinterpret_cast<uint32_t *>(smem_raw + prm.stack_offset);
    Counters cn;
    cn.diag = lq.h->diag;
    if (ok)
        search_loop<G, K, SMEM, PIVOT, LIST>(prm, SMEM ? srows : prm.rows, hv, hist, lq, th, stack_smem,
                                       (int)prm.stack_smem_levels, smem_raw + prm.t2_offset, cn);
    flush_counters(cn, prm.out);
    __syncthreads();
    if (threadIdx.x == 0) flush_diag(lq.h->diag, prm.out);
    for (uint32_t i = threadIdx.x; i <= n; i += blockDim.x)
        if (hist[i]) atomicAdd(reinterpret_cast<unsigned long long *>(prm.out + MCE_OUT_HIST + i), (unsigned long long)hist[i]);
}

// Batched form: each block takes graphs of its bucket one at a time, most
// expensive first, and searches each with its own block-local queue region
// (the same frame ring as the single-graph kernel, private to the block).
// Per graph: output initialised with the root counted (status kept), rows
// bulk-copied to shared memory, root frame queued, search, reduction into the
// graph's own result array.
template <int G, int K, bool SMEM, int PIVOT>
__global__ void __launch_bounds__(512) batch_kernel(const BatchParams bp)
{
    constexpr int WP = G * K;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ unsigned cur, root_key;

    unsigned char *region = bp.qbase + (size_t)blockIdx.x * bp.qstride;
    Ctl *ctl = reinterpret_cast<Ctl *>(region);
    unsigned *seq = reinterpret_cast<unsigned *>(region + batch_seq_offset());
    uint32_t *frames = reinterpret_cast<uint32_t *>(region + batch_frames_offset(bp.qcap));
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (SMEM) {
        if (threadIdx.x == 0) mbar_init(&mbar);
        __syncthreads();
    }
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(bp.next, 1u);
        __syncthreads();
        const unsigned idx = cur;
        if (idx >= bp.count) break;
        // a work item: graph index | part << 16 | parts << 24; a graph split
        // into parts (parts >= 2) spreads over several blocks, each searching
        // the root's children t = part, part + parts, ... (independent
        // subtrees; the root node is counted by part 0)
        const unsigned item = bp.list[idx];
        const unsigned part = (item >> 16) & 0xffu, parts = item >> 24;
        const BatchGraph gd = bp.graphs[item & 0xffffu];
        const uint32_t n = gd.n;
        const size_t rbytes = smem_rows_bytes(n, WP, SMEM);
        uint32_t *srows = reinterpret_cast<uint32_t *>(smem_raw);
        uint64_t *hv = reinterpret_cast<uint64_t *>(smem_raw + rbytes);
        uint32_t *hist = reinterpret_cast<uint32_t *>(hv + n);
        const LocalQ lq = local_queue_at(smem_raw + smem_local_offset(n, WP, SMEM), WP);
        local_queue_reset(lq, bp.groups_per_block);
        const bool valid = gd.out[MCE_OUT_STATUS] == 0ull;
        // The root's P and X over positions: all of V and nothing, or, for a
        // subproblem of the outer loop (Alg. 3), the given sets carried
        // through the order, with R = {rv} already chosen.
        const bool sub = gd.root != nullptr;
        bool pne = false, xne = false;
        for (uint32_t w = threadIdx.x; w < (uint32_t)WP; w += blockDim.x) {
            uint32_t pw = 0u, xw = 0u;
            if (!sub) {
                const uint32_t base = w * 32u;
                if (n >= base + 32u) pw = FULL;
                else if (n > base) pw = (1u << (n - base)) - 1u;
            } else {
                for (uint32_t b = 0; b < 32u && w * 32u + b < n; ++b) {
                    const uint32_t loc = gd.order[w * 32u + b];
                    pw |= ((gd.root[loc >> 5] >> (loc & 31u)) & 1u) << b;
                    xw |= ((gd.root[gd.w + (loc >> 5)] >> (loc & 31u)) & 1u) << b;
                }
            }
            frames[kFrameHdr + w] = pw;
            frames[kFrameHdr + WP + w] = xw;
            pne = pne || pw != 0u;
            xne = xne || xw != 0u;
        }
        pne = __syncthreads_or(pne) != 0;
        xne = __syncthreads_or(xne) != 0;
        const unsigned r0 = sub ? 1u : 0u;
        const uint64_t s0 = sub ? mix64((uint64_t)gd.label[gd.rv] + 1u) : 0ull;

        // the root is one node: internal, a leaf (R is maximal) or a dead end;
        // the graph's result array starts zeroed (cleared with the batch) and
        // every part adds to it
        const bool split = parts >= 2u && !sub;
        if (threadIdx.x == 0 && (!split || part == 0u)) {
            unsigned long long *o = reinterpret_cast<unsigned long long *>(gd.out);
            atomicAdd(o + MCE_OUT_NODES, 1ull);
            if (pne) atomicAdd(o + MCE_OUT_INTERNAL, 1ull);
            if (!pne && xne) atomicAdd(o + MCE_OUT_DEAD_ENDS, 1ull);
            if (!pne && !xne) {
                atomicAdd(o + MCE_OUT_COUNT, 1ull);
                atomicAdd(o + MCE_OUT_HIST + r0, 1ull);
                atomicAdd(o + MCE_OUT_HASH, (unsigned long long)mix64(s0 ^ mix64((uint64_t)r0)));
                atomicMax(o + MCE_OUT_MAX_SIZE, (unsigned long long)r0);
            }
        }
        for (uint32_t j = threadIdx.x; j < n; j += blockDim.x)
            hv[j] = mix64((uint64_t)(sub ? gd.label[gd.order[j]] : gd.order[j]) + 1u);
        for (uint32_t j = threadIdx.x; j <= n; j += blockDim.x) hist[j] = 0u;

        // ChoosePivotOrdered at the root: the key (score + 1) << 12 | (4095 -
        // position) is largest for the best score, earliest on ties; GreedyBB
        // scores nothing (first of X, else of P), GreedyBBTX/NX score
        // |P n N(u)| over X (else first of P), TomitaBB over P u X.
        if (threadIdx.x == 0) root_key = 0u;
        __syncthreads();
        {
            unsigned mine = 0u;
            for (uint32_t u = threadIdx.x; u < n; u += blockDim.x) {
                const bool inp = (frames[kFrameHdr + (u >> 5)] >> (u & 31u)) & 1u;
                const bool inx = (frames[kFrameHdr + WP + (u >> 5)] >> (u & 31u)) & 1u;
                const bool cand = (PIVOT == MCE_PIVOT_TOMITA) ? (inp || inx) : (xne ? inx : inp);
                if (!cand) continue;
                unsigned score = 0;
                if (PIVOT == MCE_PIVOT_TOMITA || (PIVOT == MCE_PIVOT_GREEDY_TX && xne))
                    for (uint32_t w = 0; w < (uint32_t)WP; ++w)
                        score += __popc(frames[kFrameHdr + w] & gd.ren[(size_t)u * WP + w]);
                const unsigned key = ((score + 1u) << 12) | (4095u - u);
                mine = key > mine ? key : mine;
            }
            atomicMax(&root_key, mine);
        }
        __syncthreads();
        // the root frame is queued only with children to expand: with X
        // non-empty the pivot may cover all of P (an internal node without
        // children), and a queued frame must always carry a branching vertex
        const unsigned p0 = root_key ? (4095u - (root_key & 4095u)) : 0u;
        bool lne = false;
        if (pne)
            for (uint32_t w = threadIdx.x; w < (uint32_t)WP; w += blockDim.x)
                lne = lne || (frames[kFrameHdr + w] & ~gd.ren[(size_t)p0 * WP + w]) != 0u;
        lne = __syncthreads_or(lne) != 0;
        const bool root = valid && pne && lne;
        // a part queues one frame per root child of the part instead of the
        // root frame: child t branches on the t-th vertex v_t of L = P \ N(p0)
        // with v_1..v_{t-1} already in X, i.e. the frame (P minus those, X =
        // those, p0, end = v_t + 1); frames go to slots 1.. (slot 0 keeps the
        // root frame's layout)
        unsigned queued = root ? 1u : 0u;
        if (split) {
            __shared__ unsigned lpre[kBatchPartWords + 1];
            const uint32_t *rp0 = gd.ren + (size_t)p0 * WP;
            if (threadIdx.x == 0) {
                unsigned acc = 0;
                for (uint32_t w = 0; w < (uint32_t)WP; ++w) {
                    lpre[w] = acc;
                    acc += (unsigned)__popc(frames[kFrameHdr + w] & ~rp0[w]);
                }
                lpre[WP] = acc;
            }
            __syncthreads();
            const unsigned nl = lpre[WP];
            const unsigned mine = nl > part ? (nl - part + parts - 1u) / parts : 0u;
            for (unsigned j = threadIdx.x; j < mine && j + 1u < bp.qcap; j += blockDim.x) {
                const unsigned t = part + j * parts;
                unsigned w = 0;
                while (w + 1u < (unsigned)WP && lpre[w + 1] <= t) ++w;
                uint32_t lw = frames[kFrameHdr + w] & ~rp0[w];
                for (unsigned r = t - lpre[w]; r > 0u; --r) lw &= lw - 1u;
                const unsigned v = w * 32u + (unsigned)(__ffs(lw) - 1);
                uint32_t *fr = frames + (size_t)(j + 1u) * bp.fs;
                for (uint32_t q = 0; q < (uint32_t)WP; ++q) {
                    const uint32_t pw = frames[kFrameHdr + q];
                    uint32_t below = 0u;
                    if (v >= q * 32u + 32u) below = FULL;
                    else if (v > q * 32u) below = (1u << (v - q * 32u)) - 1u;
                    const uint32_t x = pw & ~rp0[q] & below;
                    fr[kFrameHdr + q] = pw & ~x;
                    fr[kFrameHdr + WP + q] = x;
                }
                fr[0] = (p0 & 0xffffu) | ((v + 1u) << 16);
                fr[1] = 0u;
                fr[2] = 0u;
                fr[3] = 0u;
                fr[4] = 0u;
            }
            queued = valid && pne ? min(mine, bp.qcap - 1u) : 0u;
            if (threadIdx.x == 0 && valid && mine + 1u > bp.qcap)  // the host sizes the ring for this
                atomicCAS(reinterpret_cast<unsigned long long *>(gd.out + MCE_OUT_STATUS), 0ull,
                          static_cast<unsigned long long>(static_cast<long long>(MCE_EOVERFLOW)));
        }
        // ring state: the root frame is consumer ticket 0 in slot 0; a part's
        // frames are consumer tickets 1..queued in slots 1..queued (slot 0 is
        // then free for producer ticket qcap)
        for (uint32_t j = threadIdx.x; j < bp.qcap; j += blockDim.x) {
            unsigned sv = j;
            if (!split && j == 0u && root) sv = 1u;
            if (split && j == 0u) sv = bp.qcap;
            if (split && j >= 1u && j <= queued) sv = j + 1u;
            seq[j] = sv;
        }
        bool staged = true;
        if (SMEM) staged = stage_rows(srows, gd.ren, (uint32_t)rbytes, mb, phase & 1u);
        ++phase;
        __syncthreads();
        if (threadIdx.x == 0) {
            frames[0] = (p0 & 0xffffu) | (n << 16);
            frames[1] = r0;
            frames[2] = (uint32_t)s0;
            frames[3] = (uint32_t)(s0 >> 32);
            ctl->head = split ? 1u : 0u;
            ctl->abort = 0u;
            ctl->tail = split ? queued + 1u : (root ? 1u : 0u);
            ctl->pending = split ? queued : (root ? 1u : 0u);
            ctl->starving = 0u;
            if (!staged) {
                atomicCAS(reinterpret_cast<unsigned long long *>(gd.out + MCE_OUT_STATUS), 0ull,
                          static_cast<unsigned long long>(static_cast<long long>(MCE_ETIMEOUT)));
            }
        }
        __threadfence();
        const bool ok = __syncthreads_and(staged) != 0;

        SearchParams prm;
        prm.n = n;
        prm.wp = WP;
        prm.rows = gd.ren;
        prm.order = gd.order;
        prm.ctl = ctl;
        prm.seq = seq;
        prm.frames = frames;
        prm.qcap = bp.qcap;
        prm.fs = bp.fs;
        prm.out = gd.out;
        prm.timeout_ns = bp.timeout_ns;
        prm.total_groups = bp.groups_per_block;
        prm.pivot_mode = bp.pivot_mode;
        prm.stack_levels = bp.stack_levels;
        prm.split_min_p = bp.split_min_p;
        prm.split_target = bp.split_target;
        prm.stack_smem_levels = bp.stack_smem_levels;
        prm.stack_offset = bp.stack_offset;
        prm.trace = nullptr;
        prm.trace_per_block = 0;
        prm.tune = bp.tune;
        prm.lst = ListParams{};
        prm.part = nullptr;
        prm.part_k = 0;
        prm.count_root = 1;
        prm.seed_children = 0;
        prm.local_slots = kLocalSlots;
        prm.t2_offset = bp.t2_offset;
        prm.t2_levels = bp.t2_levels;
        prm.t2_max_p = bp.t2_max_p;
        const Thresholds th = density_thresholds(SMEM ? srows : gd.ren, n, WP, bp.tune.share_local,
                                                 bp.tune.share_global, bp.split_min_p, &root_key,
                                                 bp.tune.small_split != 0u);
        Counters cn;
        cn.diag = lq.h->diag;
        if (ok)
            search_loop<G, K, SMEM, PIVOT, false>(prm, SMEM ? srows : gd.ren, hv, hist, lq, th,
                                           reinterpret_cast<uint32_t *>(smem_raw + bp.stack_offset),
                                           (int)bp.stack_smem_levels, smem_raw + bp.t2_offset, cn);
        flush_counters(cn, gd.out);
        __syncthreads();
        if (threadIdx.x == 0) flush_diag(lq.h->diag, gd.out);
        for (uint32_t j = threadIdx.x; j <= n; j += blockDim.x)
            if (hist[j]) atomicAdd(reinterpret_cast<unsigned long long *>(gd.out + MCE_OUT_HIST + j), (unsigned long long)hist[j]);
        __syncthreads();
    }
}

// Root of Alg. 4 (P = V, X = R = {}) as the first queued frame, empty queue
// otherwise, and the result array with the root already counted: one node,
// internal when n > 0; for n = 0 the root is a leaf and the empty set is the
// one maximal clique.  A non-zero status left by an earlier step (invalid
// input) suppresses the root frame, so the search returns at once.
// root_pivot (device, nullable = position 0) is the
// root's pivot: with X empty every rule but TomitaBB takes the first vertex.
template <int G, int K>
__global__ void search_init_kernel(const SearchParams prm, const unsigned *root_pivot)
{
    constexpr int WP = G * K;
    const uint32_t n = prm.n;
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned nth = gridDim.x * blockDim.x;
    // a part of the root's branching queues part_k child frames (written by
    // the part-frames kernel that follows) and counts the root only when
    // asked to
    const bool part = prm.part != nullptr;
    // seeded: the root's children are queued by the seeding kernel that
    // follows, so the queue starts empty here
    const bool seeded = part || prm.seed_children;
    const unsigned queued = part ? prm.part_k : (prm.seed_children ? 0u : (n > 0u ? 1u : 0u));
    const bool root = !part || prm.count_root;
    for (unsigned i = tid; i < prm.qcap; i += nth) prm.seq[i] = i < queued ? i + 1u : i;
    for (unsigned i = tid; i < MCE_OUT_WORDS(n); i += nth) {
        if (i == MCE_OUT_STATUS) continue;  // sticky: an earlier step's error stays
        uint64_t v = 0ull;
        if (root && i == MCE_OUT_NODES) v = 1ull;
        if (root && n > 0u && i == MCE_OUT_INTERNAL) v = 1ull;
        if (root && n == 0u && (i == MCE_OUT_COUNT || i == MCE_OUT_HIST)) v = 1ull;
        if (root && n == 0u && i == MCE_OUT_HASH) v = mix64(0ull ^ mix64(0ull));
        if (i == MCE_OUT_GROUPS) v = prm.total_groups;
        prm.out[i] = v;
    }
    if (seeded) {
        if (tid == 0) {
            Ctl *c = prm.ctl;
            c->head = 0u;
            c->abort = 0u;
            const bool go = queued > 0u && prm.out[MCE_OUT_STATUS] == 0ull;
            c->tail = go ? queued : 0u;
            c->pending = go ? queued : 0u;
            c->starving = 0u;
        }
        return;
    }
    if (n > 0u) {
        for (unsigned w = tid; w < (unsigned)WP; w += nth) {
            const unsigned base = w * 32u;
            uint32_t pw = 0u;
            if (n >= base + 32u) pw = FULL;
            else if (n > base) pw = (1u << (n - base)) - 1u;
            prm.frames[kFrameHdr + w] = pw;       // P = V
            prm.frames[kFrameHdr + WP + w] = 0u;  // X = {}
            if (prm.lst.rec) prm.frames[kFrameHdr + 2 * WP + w] = 0u;  // R = {}
        }
    }
    if (tid == 0) {
        Ctl *c = prm.ctl;
        c->head = 0u;
        c->abort = 0u;
        if (n > 0u && prm.out[MCE_OUT_STATUS] == 0ull) {
            const unsigned p0 = root_pivot ? *root_pivot : 0u;
            prm.frames[0] = (p0 & 0xffffu) | (n << 16);
            prm.frames[1] = 0u;
            prm.frames[2] = 0u;
            prm.frames[3] = 0u;
            c->tail = 1u;
            c->pending = 1u;
        } else {
            c->tail = 0u;
            c->pending = 0u;
        }
        c->starving = 0u;
    }
}

// Root pivot for TomitaBB: the vertex of maximum degree, earliest on ties.
template <int D = 0>
__global__ void root_tomita_pivot_kernel(const uint32_t *rows, uint32_t n, uint32_t wp, unsigned *dst)
{
    __shared__ unsigned best;
    if (threadIdx.x == 0) best = 0u;
    __syncthreads();
    unsigned mine = 0u;
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
        unsigned deg = 0;
        for (uint32_t w = 0; w < wp; ++w) deg += __popc(rows[(size_t)v * wp + w]);
        const unsigned key = ((deg + 1u) << 12) | (4095u - v);
        mine = key > mine ? key : mine;
    }
    atomicMax(&best, mine);
    __syncthreads();
    if (threadIdx.x == 0) *dst = n ? (4095u - (best & 4095u)) : 0u;
}

}  // namespace mce
