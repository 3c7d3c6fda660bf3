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
constexpr int kFrameHdr = 8;

// Levels of the per-group explicit stack (local memory).  Deeper paths spill
// their frames to the global work queue, so this bounds nothing but
// register/local footprint.
constexpr int kStackDepth = 64;

// Global control block of one search, each counter on its own 128-byte line.
struct Ctl {
    unsigned head;    unsigned pad0[31];   // queue consumer ticket
    unsigned tail;    unsigned pad1[31];   // queue producer ticket
    unsigned pending; unsigned pad2[31];   // frames queued or being expanded
    unsigned idle;    unsigned pad3[31];   // groups without a frame
    unsigned abort;   unsigned pad4[31];   // set on error: every warp stops
};

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
};

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
};
SearchImpl search_impl_1_1(bool smem, int pivot);
SearchImpl search_impl_1_2(bool smem, int pivot);
SearchImpl search_impl_2_1(bool smem, int pivot);
SearchImpl search_impl_2_2(bool smem, int pivot);
SearchImpl search_impl_4_1(bool smem, int pivot);
SearchImpl search_impl_4_2(bool smem, int pivot);
SearchImpl search_impl_8_1(bool smem, int pivot);
SearchImpl search_impl_8_2(bool smem, int pivot);
SearchImpl search_impl_16_1(bool smem, int pivot);
SearchImpl search_impl_16_2(bool smem, int pivot);
SearchImpl search_impl_32_1(bool smem, int pivot);
SearchImpl search_impl_32_2(bool smem, int pivot);
SearchImpl search_impl_32_4(bool smem, int pivot);


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

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Shared-memory layout of the search kernel:
//   [rows (when staged), padded to 16 B][hv: n x u64][hist: (n + 1) x u32]
__host__ __device__ inline size_t smem_rows_bytes(uint32_t n, uint32_t wp, bool rows_in_smem)
{
    return rows_in_smem ? ((size_t)n * wp * 4 + 15) / 16 * 16 : 0;
}


}  // namespace mce
