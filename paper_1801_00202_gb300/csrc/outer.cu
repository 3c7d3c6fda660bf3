// Alg. 3's outer loop for graphs beyond the bitset path: device CSR,
// degeneracy ordering, and one subproblem per vertex for the batched search.
//
// For every vertex v, in degeneracy order (Section 3.3), the subproblem is
// the graph H_v = G[{v} u N(v)] with its vertices in increasing label; the
// batched search kernel orders it maximum-degree-first, renumbers it
// (Section 4.2) and runs Alg. 4 from R = {v}, P = the neighbours after v in
// the degeneracy order, X = those before.  Each maximal clique is reported
// once, in the subproblem of its vertex earliest in that order; counts,
// histograms and hashes of the subproblems add up to the graph's.
#include <cstdint>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_select.cuh>

#include "mce_internal.h"

namespace mce {
namespace {

constexpr unsigned FULLM = 0xffffffffu;

unsigned blocks_for(uint64_t items, unsigned threads)
{
    uint64_t g = (items + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535u * 16u) g = 65535u * 16u;
    return (unsigned)g;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// ---------------------------------------------------------------------------
// CSR from an edge list: both orientations as 64-bit keys (src << 32 | dst),
// sorted and deduplicated; invalid edges become the largest key, which no
// vertex's range reaches.

__global__ void edge_keys_kernel(uint32_t n, uint64_t m, const uint32_t *__restrict__ uv, uint64_t *keys,
                                 uint64_t *out)
{
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = uv[2 * e], v = uv[2 * e + 1];
        if (u == v || u >= n || v >= n) {
            atomicCAS(reinterpret_cast<unsigned long long *>(out + MCE_OUT_STATUS), 0ull,
                      static_cast<unsigned long long>(static_cast<long long>(MCE_EINVAL)));
            keys[2 * e] = keys[2 * e + 1] = ~0ull;
        } else {
            keys[2 * e] = ((uint64_t)u << 32) | v;
            keys[2 * e + 1] = ((uint64_t)v << 32) | u;
        }
    }
}

// off[v] = first key with source >= v (v = 0..n), by binary search.
__global__ void csr_offsets_kernel(uint32_t n, const uint64_t *__restrict__ keys, const uint32_t *count,
                                   uint32_t *off)
{
    const uint32_t num = *count;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
        const uint64_t want = (uint64_t)v << 32;
        uint32_t lo = 0, hi = num;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) / 2;
            if (keys[mid] < want) lo = mid + 1;
            else hi = mid;
        }
        off[v] = lo;
    }
}

__global__ void csr_targets_kernel(const uint64_t *__restrict__ keys, const uint32_t *off, uint32_t n, uint32_t *adj)
{
    const uint32_t total = off[n];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        adj[i] = (uint32_t)keys[i];
}

struct EdgeTemp {
    size_t keys0, keys1, count, sort, unique, total, sort_bytes, unique_bytes;
};

EdgeTemp edge_temp(uint64_t m)
{
    EdgeTemp t{};
    const uint64_t k = 2 * (m ? m : 1);
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t at = off;
        off += align256(b);
        return at;
    };
    t.keys0 = take(k * 8);
    t.keys1 = take(k * 8);
    t.count = take(8);
    cub::DeviceRadixSort::SortKeys(nullptr, t.sort_bytes, (const uint64_t *)nullptr, (uint64_t *)nullptr, (int64_t)k);
    cub::DeviceSelect::Unique(nullptr, t.unique_bytes, (const uint64_t *)nullptr, (uint64_t *)nullptr,
                              (uint32_t *)nullptr, (int64_t)k);
    t.sort = take(t.sort_bytes);
    t.unique = take(t.unique_bytes);
    t.total = off;
    return t;
}

// ---------------------------------------------------------------------------
// CSR from a bitset: per-row counts, a scan, then each row's set bits.

__global__ void row_count_kernel(uint32_t n, uint32_t w, const uint32_t *__restrict__ rows, uint32_t *cnt)
{
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
        uint32_t c = 0;
        if (v < n)
            for (uint32_t i = 0; i < w; ++i) c += __popc(rows[(size_t)v * w + i]);
        cnt[v] = c;
    }
}

__global__ void row_fill_kernel(uint32_t n, uint32_t w, const uint32_t *__restrict__ rows, const uint32_t *off,
                                uint32_t *adj)
{
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t k = off[v];
        for (uint32_t i = 0; i < w; ++i) {
            uint32_t word = rows[(size_t)v * w + i];
            while (word) {
                adj[k++] = i * 32u + (uint32_t)(__ffs(word) - 1);
                word &= word - 1u;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Degeneracy order, one block: every round takes the remaining vertex of
// smallest key (degree << 16 | label) and lowers its remaining neighbours'
// degrees.  Degrees live in shared memory as 16-bit values (0xffff marks a
// removed vertex); the smallest key of every chunk of 32 vertices and of
// every super-chunk of 32 chunks is kept beside them.  A lowered degree only
// lowers keys, so it updates both minima with atomicMin; the removed
// vertex's chunk and super-chunk are recomputed.  Warp 0 picks the vertex
// (from the at most 64 super-chunk minima) and recomputes the minima; the
// whole block lowers the neighbours' degrees; two barriers per round.  With
// SOFF the offsets are staged in shared memory too (one global round trip
// fewer per round).

constexpr unsigned kDegeneracyThreads = 256;

__device__ __forceinline__ unsigned degeneracy_key(const uint16_t *sdeg, uint32_t n, uint32_t v)
{
    if (v >= n) return FULLM;
    const unsigned d = sdeg[v];
    return d == 0xffffu ? FULLM : ((d << 16) | v);
}

template <bool SOFF>
__global__ void __launch_bounds__(kDegeneracyThreads) degeneracy_kernel(uint32_t n, const uint32_t *__restrict__ goff,
                                                                        const uint32_t *__restrict__ adj,
                                                                        uint32_t *order, uint32_t *pos)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ unsigned chosen;
    const uint32_t C = (n + 31u) / 32u, C2 = (C + 31u) / 32u;
    unsigned *cmin = reinterpret_cast<unsigned *>(dsm);  // C chunk minima
    unsigned *cmin2 = cmin + C;                          // C2 super-chunk minima
    uint32_t *soff = cmin2 + C2;                         // n + 1 offsets (SOFF)
    uint16_t *sdeg = reinterpret_cast<uint16_t *>(SOFF ? soff + n + 1 : soff);
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (SOFF)
        for (uint32_t v = threadIdx.x; v <= n; v += blockDim.x) soff[v] = __ldg(goff + v);
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) sdeg[v] = (uint16_t)(__ldg(goff + v + 1) - __ldg(goff + v));
    __syncthreads();
    const uint32_t *off = SOFF ? soff : goff;
    for (uint32_t c = warp; c < C; c += nw) {
        const unsigned k = __reduce_min_sync(FULLM, degeneracy_key(sdeg, n, c * 32u + lane));
        if (lane == 0) cmin[c] = k;
    }
    __syncthreads();
    if (warp == 0) {
        for (uint32_t c2 = 0; c2 < C2; ++c2) {
            const uint32_t c = c2 * 32u + lane;
            const unsigned k = __reduce_min_sync(FULLM, c < C ? cmin[c] : FULLM);
            if (lane == 0) cmin2[c2] = k;
        }
    }
    for (uint32_t i = 0; i < n; ++i) {
        if (warp == 0) {
            unsigned best = FULLM;
            for (uint32_t j = lane; j < C2; j += 32u) best = min(best, cmin2[j]);
            best = __reduce_min_sync(FULLM, best);
            if (lane == 0) {
                chosen = best;
                if (best != FULLM) {
                    order[i] = best & 0xffffu;
                    pos[best & 0xffffu] = i;
                }
            }
        }
        __syncthreads();
        const unsigned best = chosen;
        if (best == FULLM) break;  // nothing left (only on an asymmetric adjacency)
        const uint32_t v = best & 0xffffu;
        const uint32_t e = off[v + 1];
        for (uint32_t k = off[v] + threadIdx.x; k < e; k += blockDim.x) {
            const uint32_t u = __ldg(adj + k);  // a list holds u once: no two threads write sdeg[u]
            const unsigned d = sdeg[u];
            if (d == 0xffffu) continue;
            sdeg[u] = (uint16_t)(d - 1u);
            // minima only fall until warp 0 recomputes them after the
            // barrier, so a stored minimum at or below the key needs no atomic
            const unsigned key = ((d - 1u) << 16) | u;
            if (key < cmin[u >> 5]) atomicMin(cmin + (u >> 5), key);
            if (key < cmin2[u >> 10]) atomicMin(cmin2 + (u >> 10), key);
        }
        if (threadIdx.x == 0) sdeg[v] = 0xffffu;
        __syncthreads();
        if (warp == 0) {  // v's chunk and super-chunk, read before the next pick
            const unsigned kc = __reduce_min_sync(FULLM, degeneracy_key(sdeg, n, (v & ~31u) + lane));
            if (lane == 0) cmin[v >> 5] = kc;
            __syncwarp();
            const uint32_t c = (v >> 10) * 32u + lane;
            const unsigned k2 = __reduce_min_sync(FULLM, c < C ? cmin[c] : FULLM);
            if (lane == 0) cmin2[v >> 10] = k2;
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Subproblem extraction, one block per vertex of the degeneracy order.
// Shared memory: U (h labels, sorted), one row buffer of max_w words per warp.

__device__ __forceinline__ int find_sorted(const uint32_t *U, uint32_t h, uint32_t x)
{
    uint32_t lo = 0, hi = h;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (U[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return (lo < h && U[lo] == x) ? (int)lo : -1;
}

__global__ void __launch_bounds__(256) extract_kernel(const BatchGraph *__restrict__ table, uint32_t max_w,
                                                      const uint32_t *__restrict__ order,
                                                      const uint32_t *__restrict__ pos,
                                                      const uint32_t *__restrict__ off,
                                                      const uint32_t *__restrict__ adj)
{
    extern __shared__ uint32_t sx[];
    __shared__ unsigned rank;
    const BatchGraph gd = table[blockIdx.x];
    const uint32_t i = blockIdx.x, v = order[i], h = gd.n, wl = gd.w;
    const uint32_t d = off[v + 1] - off[v];
    uint32_t *U = sx;
    uint32_t *rb = sx + ((max_w * 32u + 3u) & ~3u) + (threadIdx.x >> 5) * max_w;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) rank = 0;
    __syncthreads();
    unsigned below = 0;
    for (uint32_t j = threadIdx.x; j < d; j += blockDim.x) below += adj[off[v] + j] < v ? 1u : 0u;
    atomicAdd(&rank, below);
    __syncthreads();
    const uint32_t rv = rank;
    for (uint32_t j = threadIdx.x; j < d; j += blockDim.x) {
        const uint32_t a = adj[off[v] + j];
        U[j + (j >= rv ? 1u : 0u)] = a;
    }
    if (threadIdx.x == 0) {
        U[rv] = v;
        const_cast<BatchGraph *>(table)[blockIdx.x].rv = rv;  // read by the search after this kernel
    }
    __syncthreads();
    uint32_t *label = const_cast<uint32_t *>(gd.label);
    uint32_t *root = const_cast<uint32_t *>(gd.root);
    uint32_t *rows = const_cast<uint32_t *>(gd.rows);
    for (uint32_t j = threadIdx.x; j < h; j += blockDim.x) label[j] = U[j];
    // root sets over local vertices: P = later neighbours, X = earlier ones
    for (uint32_t w = threadIdx.x; w < wl; w += blockDim.x) {
        uint32_t pw = 0u, xw = 0u;
        for (uint32_t b = 0; b < 32u; ++b) {
            const uint32_t j = w * 32u + b;
            if (j >= h || j == rv) continue;
            if (pos[U[j]] > i) pw |= 1u << b;
            else xw |= 1u << b;
        }
        root[w] = pw;
        root[wl + w] = xw;
    }
    // adjacency of H_v over local vertices, one warp per row
    for (uint32_t a = warp; a < h; a += nwarps) {
        for (uint32_t w = lane; w < wl; w += 32u) rb[w] = 0u;
        __syncwarp();
        const uint32_t ua = U[a];
        for (uint32_t e = off[ua] + lane; e < off[ua + 1]; e += 32u) {
            const int b = find_sorted(U, h, adj[e]);
            if (b >= 0) atomicOr(&rb[b >> 5], 1u << (b & 31));
        }
        __syncwarp();
        for (uint32_t w = lane; w < wl; w += 32u) rows[(size_t)a * wl + w] = rb[w];
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// The subproblems' result arrays summed into the graph's (one block each).

__global__ void outer_reduce_kernel(const BatchGraph *__restrict__ table, uint32_t n, uint64_t *out)
{
    const BatchGraph gd = table[blockIdx.x];
    unsigned long long *o = reinterpret_cast<unsigned long long *>(out);
    const uint64_t *s = gd.out;
    const uint32_t words = (uint32_t)MCE_OUT_WORDS(gd.n);
    for (uint32_t j = threadIdx.x; j < words; j += blockDim.x) {
        const uint64_t x = s[j];
        if (j == MCE_OUT_STATUS) {
            if (x) atomicCAS(o + MCE_OUT_STATUS, 0ull, (unsigned long long)x);
        } else if (j == MCE_OUT_MAX_SIZE || j == MCE_OUT_GROUPS) {
            if (x) atomicMax(o + j, (unsigned long long)x);
        } else if (j >= MCE_OUT_HIST) {
            if (x && j - MCE_OUT_HIST <= n) atomicAdd(o + j, (unsigned long long)x);
        } else if (x) {
            atomicAdd(o + j, (unsigned long long)x);
        }
    }
}

}  // namespace

cudaError_t outer_csr_from_edges_bytes(uint32_t n, uint64_t m, size_t *temp_bytes)
{
    (void)n;
    *temp_bytes = edge_temp(m).total;
    return cudaSuccess;
}

cudaError_t outer_csr_from_edges(uint32_t n, uint64_t m, const uint32_t *d_uv, void *temp, size_t temp_bytes,
                                 uint32_t *off, uint32_t *adj, uint64_t *out, cudaStream_t s)
{
    const EdgeTemp t = edge_temp(m);
    if (temp_bytes < t.total) return cudaErrorInvalidValue;
    unsigned char *b = static_cast<unsigned char *>(temp);
    uint64_t *k0 = reinterpret_cast<uint64_t *>(b + t.keys0), *k1 = reinterpret_cast<uint64_t *>(b + t.keys1);
    uint32_t *count = reinterpret_cast<uint32_t *>(b + t.count);
    const uint64_t k = 2 * m;
    cudaError_t e = cudaMemsetAsync(count, 0, 4, s);
    if (e == cudaSuccess && m) {
        edge_keys_kernel<<<blocks_for(m, 256), 256, 0, s>>>(n, m, d_uv, k0, out);
        e = cudaGetLastError();
        size_t sb = t.sort_bytes, ub = t.unique_bytes;
        if (e == cudaSuccess) e = cub::DeviceRadixSort::SortKeys(b + t.sort, sb, k0, k1, (int64_t)k, 0, 64, s);
        if (e == cudaSuccess) e = cub::DeviceSelect::Unique(b + t.unique, ub, k1, k0, count, (int64_t)k, s);
    }
    if (e == cudaSuccess) {
        csr_offsets_kernel<<<blocks_for((uint64_t)n + 1, 256), 256, 0, s>>>(n, k0, count, off);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && m) {
        csr_targets_kernel<<<blocks_for(k, 256), 256, 0, s>>>(k0, off, n, adj);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t outer_csr_from_rows(uint32_t n, uint32_t w, const uint32_t *rows, uint32_t *off, uint32_t *adj,
                                void *temp, size_t temp_bytes, size_t *need, cudaStream_t s)
{
    size_t scan = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, scan, (uint32_t *)nullptr, (uint32_t *)nullptr, (int64_t)n + 1);
    const size_t total = align256(((size_t)n + 1) * 4) + align256(scan);
    if (need) *need = total;
    if (!temp) return cudaSuccess;
    if (temp_bytes < total) return cudaErrorInvalidValue;
    uint32_t *cnt = static_cast<uint32_t *>(temp);
    void *st = static_cast<unsigned char *>(temp) + align256(((size_t)n + 1) * 4);
    row_count_kernel<<<blocks_for((uint64_t)n + 1, 256), 256, 0, s>>>(n, w, rows, cnt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(st, scan, cnt, off, (int64_t)n + 1, s);
    if (e == cudaSuccess && adj) {
        row_fill_kernel<<<blocks_for(n, 128), 128, 0, s>>>(n, w, rows, off, adj);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t outer_degeneracy(uint32_t n, const uint32_t *off, const uint32_t *adj, uint32_t *order, uint32_t *pos,
                             cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const size_t C = (n + 31u) / 32u, C2 = (C + 31u) / 32u;
    const size_t plain = ((C + C2) * 4 + (size_t)n * 2 + 15) / 16 * 16;
    const size_t staged = plain + ((size_t)n + 1) * 4;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (staged + 1024 <= (size_t)optin) {
        e = kernel_smem_setup((const void *)degeneracy_kernel<true>);
        if (e != cudaSuccess) return e;
        degeneracy_kernel<true><<<1, kDegeneracyThreads, staged, s>>>(n, off, adj, order, pos);
    } else {
        e = kernel_smem_setup((const void *)degeneracy_kernel<false>);
        if (e != cudaSuccess) return e;
        degeneracy_kernel<false><<<1, kDegeneracyThreads, plain, s>>>(n, off, adj, order, pos);
    }
    return cudaGetLastError();
}

cudaError_t outer_extract(const BatchGraph *table, uint32_t count, uint32_t max_w, const uint32_t *order,
                          const uint32_t *pos, const uint32_t *off, const uint32_t *adj, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const size_t smem = ((size_t)((max_w * 32u + 3u) & ~3u) + 8u * max_w) * 4;
    cudaError_t e = kernel_smem_setup((const void *)extract_kernel);
    if (e != cudaSuccess) return e;
    extract_kernel<<<count, 256, smem, s>>>(table, max_w, order, pos, off, adj);
    return cudaGetLastError();
}

cudaError_t outer_reduce(const BatchGraph *table, uint32_t count, uint32_t n, uint64_t *out, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    outer_reduce_kernel<<<count, 128, 0, s>>>(table, n, out);
    return cudaGetLastError();
}

}  // namespace mce
