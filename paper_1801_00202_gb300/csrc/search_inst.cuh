// Launch wrappers for one (lanes per group, words per lane) instantiation of
// the search kernel; each search_gN.cu instantiates a few of them so the
// library compiles in parallel.
#pragma once

#include "search_impl.cuh"

namespace mce {

template <int G, int K, bool SMEM, int PIVOT, bool LIST>
cudaError_t run_search_t(const SearchParams &prm, const LaunchShape &sh, cudaStream_t s)
{
    const unsigned *rp = nullptr;
    if (PIVOT == MCE_PIVOT_TOMITA && prm.n > 0) {
        unsigned *dst = &prm.ctl->pad4[0];
        root_tomita_pivot_kernel<0><<<1, 1024, 0, s>>>(prm.rows, prm.n, prm.wp, dst);
        rp = dst;
    }
    search_init_kernel<G, K><<<64, 256, 0, s>>>(prm, rp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (prm.part) {
        e = launch_part_frames(prm, rp, s);
        if (e != cudaSuccess) return e;
    } else if (prm.seed_children) {
        e = launch_seed_children(prm, rp, s);
        if (e != cudaSuccess) return e;
    }
    e = kernel_smem_setup((const void *)search_kernel<G, K, SMEM, PIVOT, LIST>);
    if (e != cudaSuccess) return e;
    search_kernel<G, K, SMEM, PIVOT, LIST><<<sh.blocks, sh.threads, sh.smem, s>>>(prm);
    return cudaGetLastError();
}

template <int G, int K, bool SMEM, int PIVOT, bool LIST>
cudaError_t occupancy_t(int threads, size_t smem, int *blocks_per_sm)
{
    cudaError_t e = kernel_smem_setup((const void *)search_kernel<G, K, SMEM, PIVOT, LIST>);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel<G, K, SMEM, PIVOT, LIST>,
                                                         threads, smem);
}

template <int G, int K, bool SMEM, int PIVOT>
cudaError_t run_batch_t(const BatchParams &bp, const LaunchShape &sh, cudaStream_t s)
{
    batch_kernel<G, K, SMEM, PIVOT><<<sh.blocks, sh.threads, sh.smem, s>>>(bp);
    return cudaGetLastError();
}

template <int G, int K, bool SMEM, int PIVOT>
cudaError_t batch_occupancy_t(int threads, size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<G, K, SMEM, PIVOT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<G, K, SMEM, PIVOT>, threads,
                                                         smem);
}

// The listing variant (LIST) has no batched form.
template <int G, int K, bool SMEM, int PIVOT, bool LIST>
SearchImpl impl_t()
{
    if constexpr (LIST)
        return {run_search_t<G, K, SMEM, PIVOT, true>, occupancy_t<G, K, SMEM, PIVOT, true>, nullptr, nullptr};
    else
        return {run_search_t<G, K, SMEM, PIVOT, false>, occupancy_t<G, K, SMEM, PIVOT, false>,
                run_batch_t<G, K, SMEM, PIVOT>, batch_occupancy_t<G, K, SMEM, PIVOT>};
}

template <int G, int K, bool SMEM, bool LIST>
SearchImpl pick_pivot(int pivot)
{
    switch (pivot) {
    case MCE_PIVOT_GREEDY: return impl_t<G, K, SMEM, MCE_PIVOT_GREEDY, LIST>();
    case MCE_PIVOT_GREEDY_TX: return impl_t<G, K, SMEM, MCE_PIVOT_GREEDY_TX, LIST>();
    case MCE_PIVOT_TOMITA: return impl_t<G, K, SMEM, MCE_PIVOT_TOMITA, LIST>();
    default: return {nullptr, nullptr, nullptr, nullptr};
    }
}

// Rows live in shared memory only for sets of at most 32 words.
template <int G, int K, bool LIST>
SearchImpl pick(bool smem, int pivot)
{
    if constexpr (G * K <= 32) {
        if (smem) return pick_pivot<G, K, true, LIST>(pivot);
    }
    if (smem) return {nullptr, nullptr, nullptr, nullptr};
    return pick_pivot<G, K, false, LIST>(pivot);
}

}  // namespace mce

#define MCE_DEFINE_SEARCH(G, K) \
    namespace mce { SearchImpl search_impl_##G##_##K(bool smem, int pivot) { return pick<G, K, false>(smem, pivot); } }
#define MCE_DEFINE_SEARCH_LIST(G, K)                                        \
    namespace mce {                                                         \
    SearchImpl search_list_impl_##G##_##K(bool smem, int pivot) { return pick<G, K, true>(smem, pivot); } \
    }
