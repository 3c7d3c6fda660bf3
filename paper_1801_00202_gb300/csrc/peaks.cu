// Throughput microbenchmarks for the roofline of the search kernels: the
// search does no dense contraction and, once the rows are staged, no HBM
// traffic, so what bounds it is the integer/logic pipe (AND, ANDNOT, OR of
// set words: LOP3; popcounts: POPC) and shared-memory bandwidth (row reads).
// Each kernel keeps eight independent dependency chains per thread so that
// issue, not latency, is the limit, and writes its chains' final values so
// that nothing can be removed.  Timed with CUDA events on a private stream
// after one warm-up launch; nothing here changes a clock or any other
// setting of the GPU.
#include <cstdint>

#include <cuda_runtime.h>

#include "mce.h"

namespace {

constexpr int kIters = 4096;
constexpr int kThreads = 1024;

// 8 chains x 16 LOP3 per loop trip: a_i <- a_i ^ a_{i+1} ^ c (lop3 0x96);
// each step reads a neighbouring chain, so no two steps fold into one.
__global__ void __launch_bounds__(kThreads) lop3_kernel(uint32_t seed, uint32_t *sink)
{
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed * (threadIdx.x + 1u) + (uint32_t)i * 0x9e3779b9u + blockIdx.x;
    for (int it = 0; it < kIters; ++it) {
        const uint32_t c = (uint32_t)it;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[i]) : "r"(a[(i + 1) & 7]), "r"(c));
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x ^= a[i];
    if (x == 0x12345678u) sink[blockIdx.x] = x;  // practically never: keeps the chains live
}

// 8 chains x 16 POPC per loop trip: a_i <- popc(a_i ^ c) (one LOP3 every
// other step keeps the operand changing; counted as POPC only).
__global__ void __launch_bounds__(kThreads) popc_kernel(uint32_t seed, uint32_t *sink)
{
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed ^ (threadIdx.x * 0x01000193u + (uint32_t)i);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) asm volatile("popc.b32 %0, %0;" : "+r"(a[i]));
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] ^= (uint32_t)it << i;
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x += a[i];
    if (x == 0xffffffffu) sink[blockIdx.x] = x;
}

// 128-bit shared-memory loads, consecutive lanes on consecutive 16-byte
// words (conflict-free), folded into two accumulators per load.
constexpr int kLdsWords = 8192;  // 32 KB per block
__global__ void __launch_bounds__(kThreads) lds_kernel(uint32_t seed, uint32_t *sink)
{
    __shared__ __align__(16) uint32_t buf[kLdsWords];
    for (int i = threadIdx.x; i < kLdsWords; i += blockDim.x) buf[i] = seed + (uint32_t)i * 2654435761u;
    __syncthreads();
    uint32_t x0 = 0, x1 = 0;
    const uint4 *v = reinterpret_cast<const uint4 *>(buf);
    constexpr int nv = kLdsWords / 4;
    unsigned idx = threadIdx.x % nv;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            uint4 t;
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(t.x), "=r"(t.y), "=r"(t.z), "=r"(t.w)
                         : "r"((uint32_t)__cvta_generic_to_shared(v + idx)));
            x0 ^= t.x ^ t.y;
            x1 ^= t.z ^ t.w;
            idx = (idx + 32u) & (unsigned)(nv - 1);
        }
    }
    if ((x0 ^ x1) == 0x12345678u) sink[blockIdx.x] = x0;
}

// Warp collectives the search issues per node (first vertex of a set: a
// ballot; group sums and broadcasts: shuffles; the pivot argmax: a packed
// max reduction).  8 chains x 8 collectives per loop trip, each chain's
// operand changed by one LOP3 between collectives; counted as collectives.
constexpr int kCollIters = 1024;
__global__ void __launch_bounds__(kThreads) ballot_kernel(uint32_t seed, uint32_t *sink)
{
    uint32_t a[8];
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed * (threadIdx.x + 1u) + (uint32_t)i * 0x9e3779b9u;
    for (int it = 0; it < kCollIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = __ballot_sync(0xffffffffu, (a[i] >> lane) & 1u) ^ (uint32_t)(it + i);
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x ^= a[i];
    if (x == 0x12345678u) sink[blockIdx.x] = x;
}

__global__ void __launch_bounds__(kThreads) shfl_kernel(uint32_t seed, uint32_t *sink)
{
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed * (threadIdx.x + 1u) + (uint32_t)i * 0x9e3779b9u;
    for (int it = 0; it < kCollIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = __shfl_xor_sync(0xffffffffu, a[i], (it + i) & 31) ^ (uint32_t)it;
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x ^= a[i];
    if (x == 0x12345678u) sink[blockIdx.x] = x;
}

__global__ void __launch_bounds__(kThreads) redux_kernel(uint32_t seed, uint32_t *sink)
{
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed * (threadIdx.x + 1u) + (uint32_t)i * 0x9e3779b9u;
    for (int it = 0; it < kCollIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = __reduce_max_sync(0xffffffffu, a[i] ^ (threadIdx.x * (uint32_t)(it + 1)));
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x ^= a[i];
    if (x == 0x12345678u) sink[blockIdx.x] = x;
}

template <typename F>
int time_kernel(F launch, cudaStream_t s, double *ms)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MCE_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MCE_ECUDA;
    }
    launch();  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) launch();
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / 3.0;
    return e == cudaSuccess ? MCE_OK : MCE_ECUDA;
}

}  // namespace

extern "C" int mce_measure_peaks(int device, mce_peaks *out)
{
    if (!out) return MCE_EINVAL;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return MCE_ECUDA;
    int sms = 0, khz = 0;
    int rc = MCE_OK;
    cudaStream_t s = nullptr;
    uint32_t *sink = nullptr;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        rc = MCE_ECUDA;
    const unsigned blocks = (unsigned)sms * 2u;  // 64 warps per SM
    if (rc == MCE_OK && cudaMalloc(&sink, blocks * sizeof(uint32_t)) != cudaSuccess) rc = MCE_ENOMEM;
    double ms_lop = 0, ms_popc = 0, ms_lds = 0;
    if (rc == MCE_OK)
        rc = time_kernel([&] { lop3_kernel<<<blocks, kThreads, 0, s>>>(0x2545f491u, sink); }, s, &ms_lop);
    if (rc == MCE_OK)
        rc = time_kernel([&] { popc_kernel<<<blocks, kThreads, 0, s>>>(0x2545f491u, sink); }, s, &ms_popc);
    if (rc == MCE_OK)
        rc = time_kernel([&] { lds_kernel<<<blocks, kThreads, 0, s>>>(0x2545f491u, sink); }, s, &ms_lds);
    double ms_ballot = 0, ms_shfl = 0, ms_redux = 0;
    if (rc == MCE_OK)
        rc = time_kernel([&] { ballot_kernel<<<blocks, kThreads, 0, s>>>(0x2545f491u, sink); }, s, &ms_ballot);
    if (rc == MCE_OK)
        rc = time_kernel([&] { shfl_kernel<<<blocks, kThreads, 0, s>>>(0x2545f491u, sink); }, s, &ms_shfl);
    if (rc == MCE_OK)
        rc = time_kernel([&] { redux_kernel<<<blocks, kThreads, 0, s>>>(0x2545f491u, sink); }, s, &ms_redux);
    if (rc == MCE_OK) {
        const double lanes = (double)blocks * kThreads;
        out->lop3_lane_ops_per_s = lanes * kIters * 16.0 / (ms_lop * 1e-3);
        out->popc_lane_ops_per_s = lanes * kIters * 16.0 / (ms_popc * 1e-3);
        out->lds_bytes_per_s = lanes * kIters * 8.0 * 16.0 / (ms_lds * 1e-3);
        out->sm_count = (uint32_t)sms;
        out->sm_clock_max_khz = (uint32_t)khz;
        out->ms_lop3 = ms_lop;
        out->ms_popc = ms_popc;
        out->ms_lds = ms_lds;
        const double warps = (double)blocks * (kThreads / 32);
        out->ballot_warp_ops_per_s = warps * kCollIters * 8.0 / (ms_ballot * 1e-3);
        out->shfl_warp_ops_per_s = warps * kCollIters * 8.0 / (ms_shfl * 1e-3);
        out->redux_warp_ops_per_s = warps * kCollIters * 8.0 / (ms_redux * 1e-3);
    }
    if (sink) cudaFree(sink);
    if (s) cudaStreamDestroy(s);
    cudaSetDevice(prev);
    return rc;
}
