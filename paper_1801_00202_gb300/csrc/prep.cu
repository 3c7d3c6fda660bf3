// Preprocessing steps of the search path on the device:
//  * input canonicalisation (Section 2: simple undirected graph) from an edge
//    list or a bitset,
//  * the maximum-degree-first ordering (Section 4.2),
//  * renumbering by position (Section 4.2, "How we use the vertex ordering").
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "mce_internal.h"

namespace mce {
namespace {

constexpr unsigned FULLM = 0xffffffffu;

__device__ __forceinline__ void flag_invalid(uint64_t *out)
{
    atomicCAS(reinterpret_cast<unsigned long long *>(out + MCE_OUT_STATUS), 0ull,
              static_cast<unsigned long long>(static_cast<long long>(MCE_EINVAL)));
}

// Edge list -> symmetric bitset (rows cleared beforehand).
__global__ void edges_kernel(uint32_t n, uint64_t m, const uint32_t *__restrict__ uv, uint32_t w,
                             uint32_t *__restrict__ rows, uint64_t *out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint32_t a = uv[2 * e], b = uv[2 * e + 1];
        if (a >= n || b >= n || a == b) {
            flag_invalid(out);
            continue;
        }
        atomicOr(rows + (size_t)a * w + (b >> 5), 1u << (b & 31));
        atomicOr(rows + (size_t)b * w + (a >> 5), 1u << (a & 31));
    }
}

// Bitset checks: zero diagonal, zero bits at positions >= n, symmetry.
__global__ void validate_kernel(uint32_t n, uint32_t w, const uint32_t *__restrict__ rows, uint64_t *out)
{
    const uint64_t total = (uint64_t)n * w;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        const uint32_t i = (uint32_t)(idx / w), j = (uint32_t)(idx % w);
        uint32_t word = rows[idx];
        if (word == 0u) continue;
        const uint32_t base = j * 32u;
        uint32_t valid = FULLM;
        if (base >= n) valid = 0u;
        else if (n - base < 32u) valid = (1u << (n - base)) - 1u;
        if (word & ~valid) { flag_invalid(out); continue; }
        if (i >= base && i < base + 32u && ((word >> (i - base)) & 1u)) { flag_invalid(out); continue; }
        while (word) {
            const uint32_t b = (uint32_t)__ffs(word) - 1u;
            word &= word - 1u;
            const uint32_t u = base + b;
            if (!((rows[(size_t)u * w + (i >> 5)] >> (i & 31)) & 1u)) { flag_invalid(out); break; }
        }
    }
}

// Maximum-degree-first order.  The block stages the rows in shared memory
// (when they fit) and computes all degrees; then warp 0 runs the n rounds
// with the keys in registers: lane l owns the vertices of words
// [l*JW, l*JW + JW), key = (degree + 1) << 12 | (4095 - u) while u is not
// placed (0 once placed), so the maximum key is the highest remaining degree
// with the smallest label.  A round takes the warp's two largest keys,
// places the first vertex and, when the second is not adjacent to it, the
// second too (its key is then unchanged while every other key can only
// fall, so it is the next pick), and decrements the keys of the placed
// vertices' remaining neighbours.
template <int JW>
__device__ __forceinline__ void order_body(uint32_t n, uint32_t w, const uint32_t *__restrict__ rows,
                                           uint32_t *__restrict__ order, int rows_in_smem, uint32_t *sm)
{
    uint32_t *sdeg = sm;                                  // n keys
    uint32_t *srows = sm + ((n + 3u) & ~3u);              // n * w words (optional)
    const uint32_t *R = rows;
    if (rows_in_smem) {
        for (uint32_t i = threadIdx.x; i < n * w; i += blockDim.x) srows[i] = rows[i];
        R = srows;
    }
    __syncthreads();
    for (uint32_t u = threadIdx.x; u < n; u += blockDim.x) {
        uint32_t deg = 0;
        for (uint32_t j = 0; j < w; ++j) deg += __popc(R[(size_t)u * w + j]);
        sdeg[u] = ((deg + 1u) << 12) | (4095u - u);
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;

    const uint32_t lane = threadIdx.x;
    uint32_t key[32 * JW];
#pragma unroll
    for (int q = 0; q < JW; ++q)
#pragma unroll
        for (int b = 0; b < 32; ++b) {
            const uint32_t u = (lane * JW + q) * 32u + b;
            key[q * 32 + b] = u < n ? sdeg[u] : 0u;
        }

    for (uint32_t i = 0; i < n;) {
        uint32_t a1 = 0u, a2 = 0u;
#pragma unroll
        for (int t = 0; t < 32 * JW; ++t) {
            const uint32_t k = key[t];
            if (k > a1) {
                a2 = a1;
                a1 = k;
            } else if (k > a2) {
                a2 = k;
            }
        }
        const uint32_t b1 = __reduce_max_sync(FULLM, a1);
        const uint32_t b2 = __reduce_max_sync(FULLM, a1 == b1 ? a2 : a1);
        const uint32_t v = 4095u - (b1 & 4095u);
        const uint32_t v2 = 4095u - (b2 & 4095u);
        const uint32_t *rv = R + (size_t)v * w;
        const bool two = b2 != 0u && !((rv[v2 >> 5] >> (v2 & 31u)) & 1u);
        const uint32_t *rv2 = R + (size_t)v2 * w;
        if (lane == 0) {
            order[i] = v;
            if (two) order[i + 1] = v2;
        }
#pragma unroll
        for (int q = 0; q < JW; ++q) {
            const uint32_t wi = lane * JW + q;
            const uint32_t word = wi < w ? rv[wi] : 0u;
            const uint32_t word2 = (two && wi < w) ? rv2[wi] : 0u;
#pragma unroll
            for (int b = 0; b < 32; ++b) {
                uint32_t k = key[q * 32 + b];
                const uint32_t u = wi * 32u + b;
                if (u == v || (two && u == v2)) k = 0u;
                else if (k) k -= (((word >> b) & 1u) + ((word2 >> b) & 1u)) << 12;
                key[q * 32 + b] = k;
            }
        }
        i += two ? 2u : 1u;
    }
}

// The same order for one graph with the whole block (eight warps): thread t
// owns the keys of vertices t, t + 256, ... (KP of them).  A round finds the
// two largest keys of the block (each warp's two largest by two
// __reduce_max_sync, the block's through a double-buffered pair of slots
// per warp in shared memory: one barrier per round -- a warp cannot reach
// round r + 2's write before every warp has passed round r + 1's barrier,
// after its reads of round r), places the first vertex v1, and places the
// second one v2 in the same round when v2 is not adjacent to v1: then v2's
// key is unchanged by placing v1 while every other key can only fall, so v2
// is exactly the next maximum-degree vertex (labels make keys distinct).  On
// G(n, 0.3) about two vertices in three rounds go in pairs.  Finally the keys
// of the placed vertices' remaining neighbours are decremented.
template <int KP>
__global__ void __launch_bounds__(256) order_kernel(uint32_t n, uint32_t w, const uint32_t *__restrict__ rows,
                                                   uint32_t *__restrict__ order, int rows_in_smem)
{
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *mx = sm;              // [2 rounds][8 warps][2 keys]
    uint32_t *srows = sm + 32;      // n * w words (optional)
    const uint32_t *R = rows;
    if (rows_in_smem) {
        for (uint32_t i = threadIdx.x; i < n * w; i += blockDim.x) srows[i] = rows[i];
        R = srows;
    }
    __syncthreads();
    const uint32_t t = threadIdx.x;
    uint32_t key[KP];
#pragma unroll
    for (int q = 0; q < KP; ++q) {
        const uint32_t u = t + 256u * q;
        uint32_t k = 0u;
        if (u < n) {
            uint32_t deg = 0;
            for (uint32_t j = 0; j < w; ++j) deg += __popc(R[(size_t)u * w + j]);
            k = ((deg + 1u) << 12) | (4095u - u);
        }
        key[q] = k;
    }
    uint32_t i = 0, rd = 0;
    while (i < n) {
        uint32_t a1 = 0u, a2 = 0u;  // this thread's two largest keys
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            const uint32_t k = key[q];
            if (k > a1) {
                a2 = a1;
                a1 = k;
            } else if (k > a2) {
                a2 = k;
            }
        }
        const uint32_t w1 = __reduce_max_sync(FULLM, a1);
        const uint32_t w2 = __reduce_max_sync(FULLM, a1 == w1 ? a2 : a1);
        volatile uint32_t *slot = mx + (rd & 1u) * 16u;
        if ((t & 31u) == 0u) {
            slot[2u * (t >> 5)] = w1;
            slot[2u * (t >> 5) + 1u] = w2;
        }
        __syncthreads();
        uint32_t b1 = 0u, b2 = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t x1 = slot[2 * j], x2 = slot[2 * j + 1];
            if (x1 > b1) {
                b2 = x2 > b1 ? x2 : b1;
                b1 = x1;
            } else if (x1 > b2) {
                b2 = x1;
            }
        }
        const uint32_t v1 = 4095u - (b1 & 4095u);
        const uint32_t v2 = 4095u - (b2 & 4095u);
        const uint32_t *r1 = R + (size_t)v1 * w;
        const bool two = b2 != 0u && !((r1[v2 >> 5] >> (v2 & 31u)) & 1u);
        const uint32_t *r2 = R + (size_t)v2 * w;
        if (t == 0) {
            order[i] = v1;
            if (two) order[i + 1] = v2;
        }
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            const uint32_t u = t + 256u * q;
            if (u < n) {
                uint32_t k = key[q];
                if (u == v1 || (two && u == v2)) {
                    k = 0u;
                } else if (k) {
                    uint32_t dec = (r1[u >> 5] >> (u & 31u)) & 1u;
                    if (two) dec += (r2[u >> 5] >> (u & 31u)) & 1u;
                    k -= dec << 12;
                }
                key[q] = k;
            }
        }
        i += two ? 2u : 1u;
        ++rd;
    }
}

// One block per graph of a batch; the rows go to shared memory when they fit
// in the launch's dynamic shared memory.
template <int JW>
__global__ void __launch_bounds__(256) order_batch_kernel(const BatchGraph *__restrict__ graphs, size_t smem_bytes)
{
    extern __shared__ __align__(16) uint32_t sm[];
    const BatchGraph gd = graphs[blockIdx.x];
    const size_t need = (size_t)((gd.n + 3u) & ~3u) * 4 + (size_t)gd.n * gd.w * 4;
    order_body<JW>(gd.n, gd.w, gd.rows, gd.order, need <= smem_bytes, sm);
}

__global__ void identity_kernel(uint32_t n, uint32_t *order)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) order[i] = i;
}

// A'[i][j] = A[order[i]][order[j]]: one warp per output word, each lane
// fetching one bit and a ballot assembling the word.
__global__ void renumber_kernel(uint32_t n, uint32_t w, const uint32_t *__restrict__ rows,
                                const uint32_t *__restrict__ order, uint32_t wout, uint32_t *__restrict__ out)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t total = (uint64_t)n * wout;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < total; t += nwarps) {
        const uint32_t i = (uint32_t)(t / wout), jw = (uint32_t)(t % wout);
        const uint32_t j = jw * 32u + lane;
        bool bit = false;
        if (j < n) {
            const uint32_t src = __ldg(order + i), col = __ldg(order + j);
            bit = (__ldg(rows + (size_t)src * w + (col >> 5)) >> (col & 31)) & 1u;
        }
        const uint32_t word = __ballot_sync(FULLM, bit);
        if (lane == 0) out[t] = word;
    }
}

// Renumbering for a batch: blockIdx.y selects the graph, the block's warps
// stride over its output words.
__global__ void renumber_batch_kernel(const BatchGraph *__restrict__ graphs)
{
    const BatchGraph gd = graphs[blockIdx.y];
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t total = (uint64_t)gd.n * gd.wp;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < total; t += nwarps) {
        const uint32_t i = (uint32_t)(t / gd.wp), jw = (uint32_t)(t % gd.wp);
        const uint32_t j = jw * 32u + lane;
        bool bit = false;
        if (j < gd.n) {
            const uint32_t src = gd.order[i], col = gd.order[j];
            bit = (__ldg(gd.rows + (size_t)src * gd.w + (col >> 5)) >> (col & 31)) & 1u;
        }
        const uint32_t word = __ballot_sync(FULLM, bit);
        if (lane == 0) gd.ren[t] = word;
    }
}

unsigned grid_for(uint64_t work, unsigned threads)
{
    uint64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535u) g = 65535u;
    return (unsigned)g;
}

}  // namespace

cudaError_t launch_edges_to_rows(uint32_t n, uint64_t m, const uint32_t *uv, uint32_t w, uint32_t *rows,
                                 uint64_t *out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(rows, 0, (size_t)n * w * 4, s);
    if (e != cudaSuccess || m == 0) return e;
    edges_kernel<<<grid_for(m, 256), 256, 0, s>>>(n, m, uv, w, rows, out);
    return cudaGetLastError();
}

cudaError_t launch_validate_rows(uint32_t n, uint32_t w, const uint32_t *rows, uint64_t *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    validate_kernel<<<grid_for((uint64_t)n * w, 256), 256, 0, s>>>(n, w, rows, out);
    return cudaGetLastError();
}

cudaError_t launch_order(uint32_t n, uint32_t w, const uint32_t *rows, uint32_t *order, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const size_t rbytes = (size_t)n * w * 4;
    const int in_smem = (128 + rbytes) <= 200u * 1024u;
    const size_t smem = 128 + (in_smem ? rbytes : 0);
    const void *k = nullptr;
    void (*f)(uint32_t, uint32_t, const uint32_t *, uint32_t *, int) = nullptr;
    if (n <= 256) f = order_kernel<1>;
    else if (n <= 512) f = order_kernel<2>;
    else if (n <= 1024) f = order_kernel<4>;
    else if (n <= 2048) f = order_kernel<8>;
    else f = order_kernel<16>;
    k = (const void *)f;
    cudaError_t e = kernel_smem_setup(k);
    if (e != cudaSuccess) return e;
    f<<<1, 256, smem, s>>>(n, w, rows, order, in_smem);
    return cudaGetLastError();
}

cudaError_t launch_identity(uint32_t n, uint32_t *order, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    identity_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, order);
    return cudaGetLastError();
}

cudaError_t launch_renumber(uint32_t n, uint32_t w, const uint32_t *rows, const uint32_t *order, uint32_t wout,
                            uint32_t *rows_out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t warps = (uint64_t)n * wout;
    renumber_kernel<<<grid_for(warps * 32, 256), 256, 0, s>>>(n, w, rows, order, wout, rows_out);
    return cudaGetLastError();
}


cudaError_t kernel_smem_setup(const void *func)
{
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    for (const auto &d : done)
        if (d.first == func && d.second == dev) return cudaSuccess;
    int optin = 0;
    cudaFuncAttributes fa{};
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
    if (e == cudaSuccess)  // static shared memory counts against the same limit
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess && (int)done.size() < kMaxDev * 256) done.emplace_back(func, dev);
    return e;
}

cudaError_t prepare_order_batch(uint32_t max_n, uint32_t max_w, size_t *smem)
{
    const size_t keys = ((max_n + 3u) & ~3u) * sizeof(uint32_t);
    const size_t rbytes = (size_t)max_n * max_w * 4;
    *smem = keys + ((keys + rbytes) <= 200u * 1024u ? rbytes : 0);
    const uint32_t words = (max_n + 31) / 32;
    cudaError_t e;
    if (words <= 32) e = cudaFuncSetAttribute(order_batch_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    else if (words <= 64) e = cudaFuncSetAttribute(order_batch_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    else e = cudaFuncSetAttribute(order_batch_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    return e;
}

cudaError_t launch_order_batch(const BatchGraph *graphs, uint32_t count, uint32_t max_n, size_t smem, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const uint32_t words = (max_n + 31) / 32;
    if (words <= 32) order_batch_kernel<1><<<count, 256, smem, s>>>(graphs, smem);
    else if (words <= 64) order_batch_kernel<2><<<count, 256, smem, s>>>(graphs, smem);
    else order_batch_kernel<4><<<count, 256, smem, s>>>(graphs, smem);
    return cudaGetLastError();
}

cudaError_t launch_renumber_batch(const BatchGraph *graphs, uint32_t count, uint32_t max_n, uint32_t max_wp,
                                  cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const uint64_t warps = (uint64_t)max_n * max_wp;
    unsigned gx = (unsigned)std::min<uint64_t>((warps + 7) / 8, 1024);
    if (gx == 0) gx = 1;
    renumber_batch_kernel<<<dim3(gx, count), 256, 0, s>>>(graphs);
    return cudaGetLastError();
}

}  // namespace mce
