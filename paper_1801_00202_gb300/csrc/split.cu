// The root's children of Alg. 4 as independent subtrees: the unit a search
// is split into across GPUs.
//
// Alg. 3 (Section 3.3) decomposes the enumeration into independent
// subproblems because each branch of the sequential loop receives sets that
// the branches before it fixed: branch v gets P n N(v) and X n N(v) where P
// has lost, and X gained, every earlier branch vertex.  The root of Alg. 4
// decomposes the same way.  With the root's branching set L = V \ N(p0)
// walked in order v_1 < v_2 < ..., child t is the search from R = {v_t},
// P = P_t n N(v_t), X = {v_1..v_{t-1}} n N(v_t), P_t = V minus v_1..v_{t-1}.
// In the frame encoding of the search kernel (P, X, pivot, end: "expand the
// vertices of P \ N(pivot) below end") child t alone is the frame
// (P_t, {v_1..v_{t-1}}, p0, v_t + 1), since every vertex of L below v_t has
// already moved to X.  Any set of children can therefore be searched on its
// own, and the counters of a partition of the children add up modulo 2^64 to
// the whole search once one part counts the root node.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "mce_internal.h"

namespace mce {
namespace {

__device__ __forceinline__ uint32_t valid_bits(uint32_t w, uint32_t n)
{
    const uint32_t base = w * 32u;
    if (n >= base + 32u) return 0xffffffffu;
    if (n <= base) return 0u;
    return (1u << (n - base)) - 1u;
}

__device__ __forceinline__ uint32_t below_bits(uint32_t w, uint32_t v)
{
    const uint32_t base = w * 32u;
    if (v >= base + 32u) return 0xffffffffu;
    if (v <= base) return 0u;
    return (1u << (v - base)) - 1u;
}

// Position of the t-th vertex (0-based) of L = V \ N(p0), or -1.
__device__ int select_child(const uint32_t *rows, uint32_t n, uint32_t wp, uint32_t p0, uint32_t t)
{
    const uint32_t *rp = rows + (size_t)p0 * wp;
    for (uint32_t w = 0; w * 32u < n; ++w) {
        uint32_t L = valid_bits(w, n) & ~rp[w];
        const uint32_t c = (uint32_t)__popc(L);
        if (t < c) {
            for (uint32_t j = 0; j < t; ++j) L &= L - 1u;
            return (int)(w * 32u + (uint32_t)(__ffs(L) - 1));
        }
        t -= c;
    }
    return -1;
}

__global__ void root_children_kernel(const uint32_t *rows, uint32_t n, uint32_t wp, const unsigned *root_pivot,
                                     uint32_t *sizes, uint32_t cap, uint32_t *count)
{
    const uint32_t p0 = root_pivot ? *root_pivot : 0u;
    const uint32_t *rp = rows + (size_t)p0 * wp;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        uint32_t c = 0;
        for (uint32_t w = 0; w * 32u < n; ++w) c += (uint32_t)__popc(valid_bits(w, n) & ~rp[w]);
        *count = c;
    }
    if (t >= n || t >= cap) return;
    const int v = select_child(rows, n, wp, p0, t);
    if (v < 0) return;
    const uint32_t *rv = rows + (size_t)v * wp;
    uint32_t size = 0;
    for (uint32_t w = 0; w * 32u < n; ++w) {
        const uint32_t L = valid_bits(w, n) & ~rp[w];
        const uint32_t P = valid_bits(w, n) & ~(L & below_bits(w, (uint32_t)v));
        size += (uint32_t)__popc(P & rv[w]);
    }
    sizes[t] = size;
}

// One block per queued child frame.
__global__ void part_frames_kernel(const SearchParams prm, const unsigned *root_pivot)
{
    __shared__ int v;
    const uint32_t j = blockIdx.x;
    const uint32_t n = prm.n, wp = prm.wp;
    const uint32_t p0 = root_pivot ? *root_pivot : 0u;
    if (threadIdx.x == 0) {
        const uint32_t t = prm.part[j];
        v = (j > 0 && prm.part[j - 1] >= t) ? -1 : select_child(prm.rows, n, wp, p0, t);
        if (v < 0) {
            atomicCAS(reinterpret_cast<unsigned long long *>(prm.out + MCE_OUT_STATUS), 0ull,
                      static_cast<unsigned long long>(static_cast<long long>(MCE_EINVAL)));
            atomicExch(&prm.ctl->abort, 1u);
        }
    }
    __syncthreads();
    if (v < 0) return;
    uint32_t *fr = prm.frames + (size_t)j * prm.fs;
    const uint32_t *rp = prm.rows + (size_t)p0 * wp;
    for (uint32_t w = threadIdx.x; w < wp; w += blockDim.x) {
        const uint32_t valid = valid_bits(w, n);
        const uint32_t X = valid & ~rp[w] & below_bits(w, (uint32_t)v);  // v_1..v_{t-1}
        fr[kFrameHdr + w] = valid & ~X;                                   // P_t
        fr[kFrameHdr + wp + w] = X;
        if (prm.lst.rec) fr[kFrameHdr + 2 * wp + w] = 0u;
    }
    if (threadIdx.x == 0) {
        fr[0] = (p0 & 0xffffu) | (((uint32_t)v + 1u) << 16);
        fr[1] = 0u;
        fr[2] = 0u;
        fr[3] = 0u;
        fr[4] = 0u;
    }
}

// Every root child as its own frame, one block per candidate child t < n.
__global__ void seed_children_kernel(const SearchParams prm, const unsigned *root_pivot)
{
    __shared__ int v;
    __shared__ uint32_t c;
    const uint32_t t = blockIdx.x;
    const uint32_t n = prm.n, wp = prm.wp;
    const uint32_t p0 = root_pivot ? *root_pivot : 0u;
    const uint32_t *rp = prm.rows + (size_t)p0 * wp;
    if (threadIdx.x == 0) {
        uint32_t cnt = 0;
        for (uint32_t w = 0; w * 32u < n; ++w) cnt += (uint32_t)__popc(valid_bits(w, n) & ~rp[w]);
        c = cnt;
        v = t < cnt ? select_child(prm.rows, n, wp, p0, t) : -1;
    }
    __syncthreads();
    const bool go = prm.out[MCE_OUT_STATUS] == 0ull;  // an invalid input queues nothing
    if (t == 0 && threadIdx.x == 0 && go) {
        prm.ctl->tail = c;
        prm.ctl->pending = c;
    }
    if (v < 0 || !go) return;
    uint32_t *fr = prm.frames + (size_t)t * prm.fs;
    for (uint32_t w = threadIdx.x; w < wp; w += blockDim.x) {
        const uint32_t valid = valid_bits(w, n);
        const uint32_t X = valid & ~rp[w] & below_bits(w, (uint32_t)v);
        fr[kFrameHdr + w] = valid & ~X;
        fr[kFrameHdr + wp + w] = X;
        if (prm.lst.rec) fr[kFrameHdr + 2 * wp + w] = 0u;
    }
    if (threadIdx.x == 0) {
        fr[0] = (p0 & 0xffffu) | (((uint32_t)v + 1u) << 16);
        fr[1] = 0u;
        fr[2] = 0u;
        fr[3] = 0u;
        fr[4] = 0u;
        prm.seq[t] = t + 1u;  // the frame is ready for consumer ticket t
    }
}

// TomitaBB's root pivot: with X empty, the vertex of P = V with the most
// neighbours in P (its degree), earliest in the order on ties.
__global__ void root_degree_pivot_kernel(const uint32_t *rows, uint32_t n, uint32_t wp, unsigned *dst)
{
    __shared__ unsigned best;
    if (threadIdx.x == 0) best = 0u;
    __syncthreads();
    unsigned mine = 0u;
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
        unsigned deg = 0;
        for (uint32_t w = 0; w < wp; ++w) deg += (unsigned)__popc(rows[(size_t)v * wp + w]);
        const unsigned key = ((deg + 1u) << 12) | (4095u - v);
        mine = key > mine ? key : mine;
    }
    atomicMax(&best, mine);
    __syncthreads();
    if (threadIdx.x == 0) *dst = n ? (4095u - (best & 4095u)) : 0u;
}

}  // namespace

cudaError_t launch_root_degree_pivot(const uint32_t *rows, uint32_t n, uint32_t wp, unsigned *dst, cudaStream_t s)
{
    root_degree_pivot_kernel<<<1, 1024, 0, s>>>(rows, n, wp, dst);
    return cudaGetLastError();
}

cudaError_t launch_root_children(const uint32_t *rows, uint32_t n, uint32_t wp, const unsigned *root_pivot,
                                 uint32_t *sizes, uint32_t cap, uint32_t *count, cudaStream_t s)
{
    const unsigned threads = 128;
    const unsigned blocks = (std::max<uint32_t>(n, 1u) + threads - 1) / threads;
    root_children_kernel<<<blocks, threads, 0, s>>>(rows, n, wp, root_pivot, sizes, cap, count);
    return cudaGetLastError();
}

cudaError_t launch_seed_children(const SearchParams &prm, const unsigned *root_pivot, cudaStream_t s)
{
    if (prm.n == 0) return cudaSuccess;
    seed_children_kernel<<<prm.n, 64, 0, s>>>(prm, root_pivot);
    return cudaGetLastError();
}

cudaError_t launch_part_frames(const SearchParams &prm, const unsigned *root_pivot, cudaStream_t s)
{
    if (prm.part_k == 0) return cudaSuccess;
    part_frames_kernel<<<prm.part_k, 128, 0, s>>>(prm, root_pivot);
    return cudaGetLastError();
}

}  // namespace mce
