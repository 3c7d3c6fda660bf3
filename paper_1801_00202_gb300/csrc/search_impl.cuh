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
//  * Idle groups take frames from a global bounded MPMC queue; busy groups
//    give away the upper half of their shallowest frame's branching set when
//    idle groups outnumber queued frames.  Splitting a branching set L into
//    a lower part L1 (kept) and upper part L2 (given away) as
//    (P, X, end = min L2) and (P \ L1, X u L1, end) reproduces exactly the
//    sequential P/X updates of Alg. 4, so node counts do not depend on how
//    the work was split.
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
constexpr unsigned kCheckEvery = 8;      // iterations between queue polls
constexpr unsigned kCasTries = 1u << 14; // bound of one queue ticket loop

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

__device__ __forceinline__ bool q_reserve_push(Ctl *ctl, unsigned *seq, unsigned mask, unsigned &ticket)
{
    unsigned pos = ld_relaxed(&ctl->tail);
    for (unsigned t = 0; t < kCasTries; ++t) {
        unsigned s = ld_acquire(&seq[pos & mask]);
        int dif = (int)(s - pos);
        if (dif == 0) {
            unsigned prev = atomicCAS(&ctl->tail, pos, pos + 1);
            if (prev == pos) { ticket = pos; return true; }
            pos = prev;
        } else if (dif < 0) {
            return false;  // full
        } else {
            pos = ld_relaxed(&ctl->tail);
        }
    }
    return false;
}

__device__ __forceinline__ bool q_reserve_pop(Ctl *ctl, unsigned *seq, unsigned mask, unsigned &ticket)
{
    unsigned pos = ld_relaxed(&ctl->head);
    for (unsigned t = 0; t < kCasTries; ++t) {
        unsigned s = ld_acquire(&seq[pos & mask]);
        int dif = (int)(s - (pos + 1));
        if (dif == 0) {
            unsigned prev = atomicCAS(&ctl->head, pos, pos + 1);
            if (prev == pos) { ticket = pos; return true; }
            pos = prev;
        } else if (dif < 0) {
            return false;  // empty
        } else {
            pos = ld_relaxed(&ctl->head);
        }
    }
    return false;
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
    // in the order), or -1 if the set is empty.
    __device__ __forceinline__ int first(const uint32_t (&s)[K]) const
    {
        int loc = -1;
#pragma unroll
        for (int k = K - 1; k >= 0; --k)
            if (s[k]) loc = (int)((gl * K + k) * 32u) + __ffs(s[k]) - 1;
        if (G == 1) return loc;
        unsigned b = __ballot_sync(FULL, loc >= 0) & gmask;
        int src = b ? (__ffs(b) - 1) : (int)lane;
        int r = __shfl_sync(FULL, loc, src);
        return b ? r : -1;
    }
    __device__ __forceinline__ int sum(int x) const
    {
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
// Give away the upper part of a frame's branching set L (c elements).  The
// owner keeps the lowest `keep` of them:
//   kKeepHalf       keep = ceil(c/2); a single element is not given away;
//   kKeepHalfOrNone keep = ceil(c/2) for c >= 2, else 0 (the whole frame);
//   kKeepNone       keep = 0.
// The given-away frame is (P \ L1, X u L1, pivot, end) with L1 the kept part;
// the owner continues with end = the first given-away position, which the
// call returns (or -1 when nothing was given).  `whole` tells the owner that
// it kept nothing.
enum KeepPolicy { kKeepHalf = 0, kKeepHalfOrNone = 1, kKeepNone = 2 };

template <int G, int K>
__device__ __forceinline__ int donate(const Grp<G, K> &g, const SearchParams &prm, bool pred, int policy,
                                      const uint32_t (&P)[K], const uint32_t (&X)[K], const uint32_t (&L)[K],
                                      unsigned pe, unsigned rs, uint64_t S, bool &whole, uint64_t &c_don)
{
    constexpr int WP = G * K;
    int cl = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) cl += __popc(L[k]);
    const int c = g.sum(cl);
    int keep = 0;
    if (policy != kKeepNone) keep = (c >= 2) ? (c + 1) / 2 : (policy == kKeepHalf ? c : 0);
    const bool ok = pred && c > keep;
    const int pre = g.excl_scan(cl);
    int pos = -1;
    if (ok && pre <= keep && keep < pre + cl) {
        int r = keep - pre;
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
        unsigned b = __ballot_sync(FULL, pos >= 0) & g.gmask;
        split = __shfl_sync(FULL, pos, b ? (__ffs(b) - 1) : (int)g.lane);
    }

    unsigned ticket = 0, got = 0;
    if (ok && g.leader()) {
        atomicAdd(&prm.ctl->pending, 1u);
        got = q_reserve_push(prm.ctl, prm.seq, prm.qcap - 1u, ticket) ? 1u : 0u;
        if (!got) atomicSub(&prm.ctl->pending, 1u);
    }
    got = g.from_leader(got);
    ticket = g.from_leader(ticket);
    if (got) {
        uint32_t *fr = prm.frames + (size_t)(ticket & (prm.qcap - 1u)) * prm.fs;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t l1 = L[k] & g.below(k, (unsigned)split);
            __stcg(fr + kFrameHdr + g.gl * K + k, P[k] & ~l1);
            __stcg(fr + kFrameHdr + WP + g.gl * K + k, X[k] | l1);
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
    if (got && g.leader()) {
        st_release(&prm.seq[ticket & (prm.qcap - 1u)], ticket + 1u);
        ++c_don;
    }
    whole = (keep == 0);
    return got ? split : -1;
}

// ---------------------------------------------------------------------------

template <int G, int K, bool SMEM, int PIVOT>
__global__ void __launch_bounds__(K >= 4 ? 512 : 1024) search_kernel(const SearchParams prm)
{
    using Gp = Grp<G, K>;
    constexpr int WP = G * K;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int stage_failed;

    const uint32_t n = prm.n;
    const size_t rbytes = smem_rows_bytes(n, WP, SMEM);
    uint32_t *srows = reinterpret_cast<uint32_t *>(smem_raw);
    uint64_t *hv = reinterpret_cast<uint64_t *>(smem_raw + rbytes);
    uint32_t *hist = reinterpret_cast<uint32_t *>(hv + n);
    Ctl *ctl = prm.ctl;

    // ---- prologue: stage the rows (bulk copy), hash table, histogram
    if (threadIdx.x == 0) stage_failed = 0;
    if (SMEM) {
        const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"((uint32_t)rbytes)
                         : "memory");
            const uint32_t dst0 = (uint32_t)__cvta_generic_to_shared(srows);
            for (size_t off = 0; off < rbytes; off += 65536) {
                const uint32_t len = (uint32_t)((rbytes - off) < 65536 ? (rbytes - off) : 65536);
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        dst0 + (uint32_t)off),
                    "l"(reinterpret_cast<const unsigned char *>(prm.rows) + off), "r"(len), "r"(mb)
                    : "memory");
            }
        }
    }
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) hv[i] = mix64((uint64_t)prm.order[i] + 1u);
    for (uint32_t i = threadIdx.x; i <= n; i += blockDim.x) hist[i] = 0u;
    if (SMEM) {
        // bounded wait for the bulk copy (phase 0)
        const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
        bool done = false;
        const uint64_t t0 = global_ns();
        for (unsigned t = 0; !done; ++t) {
            uint32_t ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(ok)
                : "r"(mb)
                : "memory");
            done = ok != 0;
            if (!done && (t & 63u) == 63u && global_ns() - t0 > 2000000000ull) break;
        }
        if (!done) {
            stage_failed = 1;
            if (threadIdx.x == 0) set_status(prm.out, ctl, MCE_ETIMEOUT);
            // give copies still in flight a second bounded chance to land
            // before the block retires its shared memory
            const uint64_t t1 = global_ns();
            for (unsigned t = 0; !done; ++t) {
                uint32_t ok;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                    : "=r"(ok)
                    : "r"(mb)
                    : "memory");
                done = ok != 0;
                if (!done && (t & 63u) == 63u && global_ns() - t1 > 2000000000ull) break;
            }
        }
    }
    __syncthreads();
    const uint32_t *rows = SMEM ? srows : prm.rows;

    Gp g;
    g.init();
    uint32_t P[K], X[K], L[K];
#pragma unroll
    for (int k = 0; k < K; ++k) P[k] = X[k] = L[k] = 0u;
    unsigned pe = 0, rs = 0;
    uint64_t S = 0;
    int d = 0, dbase = 0;
    bool work = false;
    uint64_t c_cnt = 0, c_nodes = 0, c_int = 0, c_dead = 0, c_hash = 0, c_don = 0;
    unsigned c_max = 0;

    uint32_t stP[kStackDepth][K], stX[kStackDepth][K];
    unsigned stPE[kStackDepth], stRS[kStackDepth];
    uint64_t stS[kStackDepth];

    uint64_t quiet_since = 0;
    const uint64_t t_start = global_ns();
    unsigned last_pend = 0xffffffffu, last_head = 0xffffffffu;
    unsigned backoff = 64;
    const unsigned qmask = prm.qcap - 1u;
    bool stop = stage_failed != 0;

    auto rowp = [&](int v) -> const uint32_t * { return rows + (size_t)v * WP + g.gl * K; };

    for (unsigned it = 0; !stop; ++it) {
        // ---- A: a frame whose branching set is exhausted returns to its parent
        const bool hasL = g.any(L);
        if (work && !hasL) {
            if (d > dbase) {
                --d;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    P[k] = stP[d][k];
                    X[k] = stX[d][k];
                }
                pe = stPE[d];
                if (g.leader()) {
                    rs = stRS[d];
                    S = stS[d];
                }
                uint32_t rp[K];
                load_row<K, SMEM>(rp, rowp((int)(pe & 0xffffu)));
#pragma unroll
                for (int k = 0; k < K; ++k) L[k] = P[k] & ~rp[k] & g.below(k, pe >> 16);
            } else {
                work = false;
                if (g.leader()) {
                    atomicSub(&ctl->pending, 1u);
                    atomicAdd(&ctl->idle, 1u);
                }
            }
        }

        // ---- B: queue traffic (every kCheckEvery iterations, or when idle)
        const bool all_idle = __ballot_sync(FULL, work) == 0u;
        if (all_idle || (it % kCheckEvery) == 0u) {
            unsigned head = 0, tail = 0, idl = 0, pend = 0, ab = 0;
            if (g.lane == 0) {
                ab = ld_relaxed(&ctl->abort);
                pend = ld_relaxed(&ctl->pending);
                head = ld_relaxed(&ctl->head);
                tail = ld_relaxed(&ctl->tail);
                idl = ld_relaxed(&ctl->idle);
            }
            ab = __shfl_sync(FULL, ab, 0);
            pend = __shfl_sync(FULL, pend, 0);
            head = __shfl_sync(FULL, head, 0);
            tail = __shfl_sync(FULL, tail, 0);
            idl = __shfl_sync(FULL, idl, 0);
            if (ab) break;
            if (all_idle && pend == 0u) break;
            // hard cap on the whole search: ten idle budgets
            if (g.lane == 0 && global_ns() - t_start > 10ull * prm.timeout_ns) set_status(prm.out, ctl, MCE_ETIMEOUT);
            const unsigned queued = tail - head;

            // idle groups take a frame
            unsigned ticket = 0, got = 0;
            if (!work && queued != 0u && g.leader()) got = q_reserve_pop(ctl, prm.seq, qmask, ticket) ? 1u : 0u;
            got = g.from_leader(got);
            ticket = g.from_leader(ticket);
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
            }
            __syncwarp();
            if (got) {
                if (g.leader()) {
                    st_release(&prm.seq[ticket & qmask], ticket + prm.qcap);
                    atomicSub(&ctl->idle, 1u);
                }
                work = true;
                d = dbase = 0;
                uint32_t rp[K];
                load_row<K, SMEM>(rp, rowp((int)(pe & 0xffffu)));
#pragma unroll
                for (int k = 0; k < K; ++k) L[k] = P[k] & ~rp[k] & g.below(k, pe >> 16);
            }

            // busy groups feed idle ones: split the shallowest frame
            const bool hungry = work && !got && idl > queued;
            if (__ballot_sync(FULL, hungry) != 0u) {
                const bool from_stack = hungry && d > dbase;
                uint32_t sP[K], sX[K], sL[K];
                unsigned spe = pe, srs = rs;
                uint64_t sS = S;
                if (from_stack) {
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        sP[k] = stP[dbase][k];
                        sX[k] = stX[dbase][k];
                    }
                    spe = stPE[dbase];
                    if (g.leader()) {
                        srs = stRS[dbase];
                        sS = stS[dbase];
                    }
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
                bool whole = false;
                const int ne = donate<G, K>(g, prm, hungry, from_stack ? kKeepHalfOrNone : kKeepHalf, sP, sX, sL, spe,
                                            srs, sS, whole, c_don);
                if (ne >= 0) {
                    const unsigned npe = (spe & 0xffffu) | ((unsigned)ne << 16);
                    if (from_stack) {
                        if (whole) ++dbase;
                        else stPE[dbase] = npe;
                    } else {
                        pe = npe;
#pragma unroll
                        for (int k = 0; k < K; ++k) L[k] &= g.below(k, (unsigned)ne);
                    }
                }
            }

            if (__ballot_sync(FULL, work) == 0u) {
                // nobody here has work: back off, watch for a stalled search
                if (g.lane == 0) {
                    const uint64_t now = global_ns();
                    if (pend != last_pend || head != last_head || quiet_since == 0) {
                        quiet_since = now;
                        last_pend = pend;
                        last_head = head;
                    } else if (now - quiet_since > prm.timeout_ns) {
                        set_status(prm.out, ctl, MCE_ETIMEOUT);
                    }
                }
                __nanosleep(backoff);
                backoff = backoff < 2048u ? backoff * 2u : 2048u;
                continue;
            }
            backoff = 64;
        }

        // ---- C: expand one child v = first(L) of every active frame
        const bool anyL = g.any(L);  // collective: never inside && or ?:
        const bool act = work && anyL;
        const int v = g.first(L);
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
        const bool bp = g.any(Pc);
        const bool bx = g.any(Xc);
        uint64_t Sc = 0;
        if (act && g.leader()) {
            ++c_nodes;
            Sc = S + hv[v];
            if (!bp) {
                if (!bx) {  // P u X empty: R u {v} is a maximal clique
                    const unsigned k = rs + 1u;
                    ++c_cnt;
                    c_hash += mix64(Sc ^ mix64((uint64_t)k));
                    c_max = k > c_max ? k : c_max;
                    const unsigned old = atomicAdd(&hist[k], 1u);
                    if (old == 0xffffffffu)
                        atomicAdd(reinterpret_cast<unsigned long long *>(prm.out + MCE_OUT_HIST + k), 1ull << 32);
                } else {
                    ++c_dead;
                }
            } else {
                ++c_int;
            }
        }
        const bool inter = act && bp;

        // ChoosePivotOrdered on the child (P', X')
        int pc;
        if (PIVOT == MCE_PIVOT_GREEDY) {
            uint32_t sel[K];
#pragma unroll
            for (int k = 0; k < K; ++k) sel[k] = bx ? Xc[k] : Pc[k];
            pc = g.first(sel);
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
            const int firstP = g.first(Pc);
            pc = (PIVOT == MCE_PIVOT_GREEDY_TX) ? firstP : -1;  // X' empty: first of P'
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
        const bool hasLc = g.any(Lc);
        const bool more = g.any(L);
        const bool desc = inter && hasLc;
        bool spill = false;
        if (desc && more) {
            if (d < (int)prm.stack_levels) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    stP[d][k] = P[k];
                    stX[d][k] = X[k];
                }
                stPE[d] = pe;
                if (g.leader()) {
                    stRS[d] = rs;
                    stS[d] = S;
                }
                ++d;
            } else {
                spill = true;
            }
        }
        if (__ballot_sync(FULL, spill) != 0u) {
            // stack full: the rest of this frame goes to the queue whole
            bool whole = false;
            const int ne = donate<G, K>(g, prm, spill, kKeepNone, P, X, L, pe, rs, S, whole, c_don);
            if (spill && ne < 0 && g.leader()) set_status(prm.out, ctl, MCE_EOVERFLOW);
        }
        if (desc) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                P[k] = Pc[k];
                X[k] = Xc[k];
                L[k] = Lc[k];
            }
            pe = (unsigned)pc | (n << 16);
            rs = rs + 1u;
            S = Sc;
        }
    }

    // ---- reduction: warp, then one atomic per counter per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c_cnt += __shfl_xor_sync(FULL, c_cnt, o);
        c_nodes += __shfl_xor_sync(FULL, c_nodes, o);
        c_int += __shfl_xor_sync(FULL, c_int, o);
        c_dead += __shfl_xor_sync(FULL, c_dead, o);
        c_hash += __shfl_xor_sync(FULL, c_hash, o);
        c_don += __shfl_xor_sync(FULL, c_don, o);
        c_max = max(c_max, __shfl_xor_sync(FULL, c_max, o));
    }
    if (g.lane == 0) {
        unsigned long long *o = reinterpret_cast<unsigned long long *>(prm.out);
        if (c_cnt) atomicAdd(o + MCE_OUT_COUNT, c_cnt);
        if (c_nodes) atomicAdd(o + MCE_OUT_NODES, c_nodes);
        if (c_int) atomicAdd(o + MCE_OUT_INTERNAL, c_int);
        if (c_dead) atomicAdd(o + MCE_OUT_DEAD_ENDS, c_dead);
        if (c_hash) atomicAdd(o + MCE_OUT_HASH, c_hash);
        if (c_don) atomicAdd(o + MCE_OUT_DONATIONS, c_don);
        if (c_max) atomicMax(o + MCE_OUT_MAX_SIZE, (unsigned long long)c_max);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i <= n; i += blockDim.x)
        if (hist[i]) atomicAdd(reinterpret_cast<unsigned long long *>(prm.out + MCE_OUT_HIST + i), (unsigned long long)hist[i]);
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
    for (unsigned i = tid; i < prm.qcap; i += nth) prm.seq[i] = (i == 0u && n > 0u) ? 1u : i;
    for (unsigned i = tid; i < MCE_OUT_WORDS(n); i += nth) {
        if (i == MCE_OUT_STATUS) continue;  // sticky: an earlier step's error stays
        uint64_t v = 0ull;
        if (i == MCE_OUT_NODES) v = 1ull;
        if (n > 0u && i == MCE_OUT_INTERNAL) v = 1ull;
        if (n == 0u && (i == MCE_OUT_COUNT || i == MCE_OUT_HIST)) v = 1ull;
        if (n == 0u && i == MCE_OUT_HASH) v = mix64(0ull ^ mix64(0ull));
        prm.out[i] = v;
    }
    if (n > 0u) {
        for (unsigned w = tid; w < (unsigned)WP; w += nth) {
            const unsigned base = w * 32u;
            uint32_t pw = 0u;
            if (n >= base + 32u) pw = FULL;
            else if (n > base) pw = (1u << (n - base)) - 1u;
            prm.frames[kFrameHdr + w] = pw;       // P = V
            prm.frames[kFrameHdr + WP + w] = 0u;  // X = {}
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
        c->idle = prm.total_groups;
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
