// Clique listing (MCE_LIST / MCE_LIST_SORTED): turning the search's record
// chunks into the CSR listing of the result contract.
//
// During the search every group appends, at each maximal clique it reports,
// a record [0x80000000 | k, pos_1 .. pos_k] (positions in the search order,
// all < 4096 so the top bit marks headers) to a chunk of the record buffer
// it claimed (ListParams in mce_internal.h).  Chunks are filled in claim order
// per group, so records never straddle chunks; `fill[c]` is the number of
// words used in chunk c.  This file builds, on the device:
//   1. per chunk, its number of cliques (header words) and member ids;
//   2. exclusive scans of both over the chunks (clique index and id offset
//      of each chunk's first record);
//   3. the CSR listing: off[i] = offset of clique i's members in ids[],
//      off[count] = total; every clique's members as original labels in
//      ascending order (a per-warp bitset of the labels, read out in order);
//   4. for MCE_LIST_SORTED, the cliques in lexicographic order: a stable
//      least-significant-digit radix sort of the clique indices whose digits
//      are groups of four members (label + 1 in 13 bits each, 0 past the
//      clique's end), then a gather into the final CSR.
// The sorts and scans are CUB primitives; the record walk, the per-clique
// ordering and the gathers are kernels of this file.
#include <cstdint>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "mce_internal.h"

namespace mce {
namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int kListWarps = 8;  // warps per block of the listing kernels

// 1. cliques per used chunk (ids = fill - cliques)
__global__ void list_count_kernel(const uint32_t *rec, const uint32_t *fill, uint32_t chunks, uint32_t cw,
                                  uint64_t *cliques, uint64_t *ids)
{
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t c = warp; c < chunks; c += nwarps) {
        const uint32_t f = fill[c];
        const uint32_t *r = rec + c * (uint64_t)cw;
        unsigned h = 0;
        for (uint32_t i = lane; i < f; i += 32u) h += r[i] >> 31;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(FULLM, h, o);
        if (lane == 0) {
            cliques[c] = h;
            ids[c] = f - h;
        }
    }
}

// 3. one warp per chunk: walk its records, write off[] and each clique's
// members as labels in ascending order.  bits: per-warp scratch of
// ceil(n/32) words in shared memory.
__global__ void list_emit_kernel(const uint32_t *rec, const uint32_t *fill, uint32_t chunks, uint32_t cw,
                                 const uint64_t *clique_base, const uint64_t *id_base, const uint32_t *order,
                                 uint32_t n, uint64_t count, uint64_t ids_total, uint32_t *ids_out, uint64_t *off_out)
{
    extern __shared__ uint32_t lbits[];
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t wl = (n + 31u) / 32u;
    uint32_t *bits = lbits + (size_t)(threadIdx.x >> 5) * wl;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t c = warp; c < chunks; c += nwarps) {
        const uint32_t f = fill[c];
        const uint32_t *r = rec + c * (uint64_t)cw;
        uint64_t cl = clique_base[c], id = id_base[c];
        for (uint32_t pos = 0; pos < f;) {
            const uint32_t k = r[pos] & 0x7fffffffu;
            for (uint32_t w = lane; w < wl; w += 32u) bits[w] = 0u;
            __syncwarp();
            for (uint32_t t = lane; t < k && pos + 1u + t < f; t += 32u) {
                const uint32_t p = r[pos + 1u + t];
                const uint32_t lab = p < n ? order[p] : 0u;
                atomicOr(&bits[lab >> 5], 1u << (lab & 31u));
            }
            __syncwarp();
            uint64_t run = id;
            for (uint32_t w0 = 0; w0 < wl; w0 += 32u) {
                const uint32_t w = w0 + lane;
                uint32_t b = w < wl ? bits[w] : 0u;
                const unsigned cnt = (unsigned)__popc(b);
                unsigned incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(FULLM, incl, o);
                    if ((int)lane >= o) incl += y;
                }
                uint64_t at = run + (incl - cnt);
                while (b) {
                    if (at < ids_total) ids_out[at] = w * 32u + (unsigned)(__ffs(b) - 1);
                    ++at;
                    b &= b - 1u;
                }
                run += __shfl_sync(FULLM, incl, 31);
            }
            if (lane == 0 && cl < count) off_out[cl] = id;
            __syncwarp();
            ++cl;
            id += k;
            pos += k + 1u;
        }
    }
}

// 4a. digit group t of clique perm[j]: members 4t .. 4t+3 as (label + 1) in
// 13-bit fields, most significant first; 0 past the end of the clique.
__global__ void list_key_kernel(const uint32_t *perm, uint64_t count, const uint64_t *off, const uint32_t *ids,
                                uint32_t t, uint64_t *keys)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = perm[j];
        const uint64_t a = off[c], e = off[c + 1];
        uint64_t key = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t at = a + 4ull * t + (uint64_t)i;
            const uint64_t d = at < e ? (uint64_t)ids[at] + 1ull : 0ull;
            key |= d << (13 * (3 - i));
        }
        keys[j] = key;
    }
}

__global__ void list_iota_kernel(uint32_t *perm, uint64_t count)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += (uint64_t)gridDim.x * blockDim.x)
        perm[j] = (uint32_t)j;
}

// 4b. sizes in the new order
__global__ void list_size_kernel(const uint32_t *perm, uint64_t count, const uint64_t *off, uint64_t *sizes)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = perm[j];
        sizes[j] = off[c + 1] - off[c];
    }
}

// 4c. one warp per clique of the new order: copy its members
__global__ void list_gather_kernel(const uint32_t *perm, uint64_t count, const uint64_t *off_in, const uint32_t *ids_in,
                                   const uint64_t *off_out, uint32_t *ids_out)
{
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t j = warp; j < count; j += nwarps) {
        const uint32_t c = perm[j];
        const uint64_t a = off_in[c], k = off_in[c + 1] - a, b = off_out[j];
        for (uint64_t t = lane; t < k; t += 32u) ids_out[b + t] = ids_in[a + t];
    }
}

__global__ void list_set_kernel(uint64_t *p, uint64_t v) { *p = v; }

unsigned grid_for_items(uint64_t items, unsigned per_block)
{
    const uint64_t g = (items + per_block - 1) / per_block;
    return (unsigned)(g < 1 ? 1 : (g > 65535ull * 32ull ? 65535ull * 32ull : g));
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct TempLayout {
    size_t cl, idn, clb, idb, cub_scan, t_ids, t_off, keys0, keys1, perm0, perm1, sizes, cub_sort, total;
    size_t scan_bytes, sort_bytes;  // CUB scratch sizes at cub_scan / cub_sort
};

TempLayout temp_layout(uint64_t count, uint64_t ids, uint32_t chunks, bool sorted)
{
    TempLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += align256(bytes);
        return at;
    };
    const uint64_t nc = chunks ? chunks : 1;
    L.cl = take(nc * 8);
    L.idn = take(nc * 8);
    L.clb = take(nc * 8);
    L.idb = take(nc * 8);
    size_t scan_bytes = 0, scan2 = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, (uint64_t *)nullptr, (uint64_t *)nullptr, (int64_t)nc);
    if (sorted) {
        const uint64_t m = count ? count : 1;
        cub::DeviceScan::ExclusiveSum(nullptr, scan2, (uint64_t *)nullptr, (uint64_t *)nullptr, (int64_t)m);
    }
    L.scan_bytes = scan_bytes > scan2 ? scan_bytes : scan2;
    L.cub_scan = take(L.scan_bytes);
    if (sorted) {
        const uint64_t m = count ? count : 1;
        L.t_ids = take((ids ? ids : 1) * 4);
        L.t_off = take((m + 1) * 8);
        L.keys0 = take(m * 8);
        L.keys1 = take(m * 8);
        L.perm0 = take(m * 4);
        L.perm1 = take(m * 4);
        L.sizes = take(m * 8);
        size_t sort_bytes = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, (const uint64_t *)nullptr, (uint64_t *)nullptr,
                                        (const uint32_t *)nullptr, (uint32_t *)nullptr, (int64_t)m, 0, 52);
        L.sort_bytes = sort_bytes;
        L.cub_sort = take(sort_bytes);
    }
    L.total = off;
    return L;
}

}  // namespace

size_t list_temp_bytes(uint64_t count, uint64_t ids, uint32_t chunks, bool sorted)
{
    return temp_layout(count, ids, chunks, sorted).total;
}

cudaError_t list_build(const ListJob &j, cudaStream_t s)
{
    const TempLayout L = temp_layout(j.count, j.ids, j.chunks, j.sorted);
    if (j.temp_bytes < L.total) return cudaErrorInvalidValue;
    unsigned char *t = static_cast<unsigned char *>(j.temp);
    uint64_t *cl = reinterpret_cast<uint64_t *>(t + L.cl), *idn = reinterpret_cast<uint64_t *>(t + L.idn);
    uint64_t *clb = reinterpret_cast<uint64_t *>(t + L.clb), *idb = reinterpret_cast<uint64_t *>(t + L.idb);
    const int threads = 32 * kListWarps;
    cudaError_t e = cudaSuccess;
    if (j.chunks) {
        list_count_kernel<<<grid_for_items(j.chunks, kListWarps), threads, 0, s>>>(j.rec, j.fill, j.chunks, j.chunk_words,
                                                                                  cl, idn);
        e = cudaGetLastError();
        size_t sb = L.scan_bytes;
        if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(t + L.cub_scan, sb, cl, clb, (int64_t)j.chunks, s);
        sb = L.scan_bytes;
        if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(t + L.cub_scan, sb, idn, idb, (int64_t)j.chunks, s);
    }
    uint32_t *ids_e = j.sorted ? reinterpret_cast<uint32_t *>(t + L.t_ids) : j.ids_out;
    uint64_t *off_e = j.sorted ? reinterpret_cast<uint64_t *>(t + L.t_off) : j.off_out;
    if (e == cudaSuccess && j.chunks) {
        const size_t smem = (size_t)kListWarps * ((j.n + 31) / 32) * 4;
        list_emit_kernel<<<grid_for_items(j.chunks, kListWarps), threads, smem, s>>>(
            j.rec, j.fill, j.chunks, j.chunk_words, clb, idb, j.order, j.n, j.count, j.ids, ids_e, off_e);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        list_set_kernel<<<1, 1, 0, s>>>(off_e + j.count, j.ids);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess || !j.sorted || j.count == 0) return e;

    // lexicographic order: LSD passes over groups of four members
    uint64_t *k0 = reinterpret_cast<uint64_t *>(t + L.keys0), *k1 = reinterpret_cast<uint64_t *>(t + L.keys1);
    uint32_t *p0 = reinterpret_cast<uint32_t *>(t + L.perm0), *p1 = reinterpret_cast<uint32_t *>(t + L.perm1);
    list_iota_kernel<<<grid_for_items(j.count, 256), 256, 0, s>>>(p0, j.count);
    e = cudaGetLastError();
    const uint32_t groups = (j.max_size + 3) / 4;
    for (uint32_t g = groups; e == cudaSuccess && g-- > 0;) {
        list_key_kernel<<<grid_for_items(j.count, 256), 256, 0, s>>>(p0, j.count, off_e, ids_e, g, k0);
        e = cudaGetLastError();
        size_t sb = L.sort_bytes;
        if (e == cudaSuccess)
            e = cub::DeviceRadixSort::SortPairs(t + L.cub_sort, sb, k0, k1, p0, p1, (int64_t)j.count, 0, 52, s);
        uint32_t *tmp = p0;
        p0 = p1;
        p1 = tmp;
    }
    uint64_t *sizes = reinterpret_cast<uint64_t *>(t + L.sizes);
    if (e == cudaSuccess) {
        list_size_kernel<<<grid_for_items(j.count, 256), 256, 0, s>>>(p0, j.count, off_e, sizes);
        e = cudaGetLastError();
    }
    size_t sb = L.scan_bytes;
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(t + L.cub_scan, sb, sizes, j.off_out, (int64_t)j.count, s);
    if (e == cudaSuccess) {
        list_set_kernel<<<1, 1, 0, s>>>(j.off_out + j.count, j.ids);
        list_gather_kernel<<<grid_for_items(j.count, kListWarps), threads, 0, s>>>(p0, j.count, off_e, ids_e, j.off_out,
                                                                                  j.ids_out);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace mce
