// mce_enumerate_device_static: the whole search path on a device bitset,
// with its scratch memory in a fixed area of device memory that the library
// owns, so that the call itself allocates nothing.
//
// Who needs this: callers that are handed input and output buffers but may
// not allocate device memory themselves -- a plug-in or custom operator whose
// host framework owns every device allocation (a serving runtime or a tensor
// framework's caching allocator), and latency-critical request paths that
// must not pay for, or fragment memory with, an allocation per call.
//
// The area is MCE_STATIC_SCRATCH_BYTES of __device__ memory per GPU that
// loads the library, held until the process exits.  In host code the symbol
// is only a stand-in, so its device address is looked up with
// cudaGetSymbolAddress, with the device current, on every call: a device
// reset, or a primary context released and created again, reloads the module
// and may move the area, so no address is kept between calls.  The first
// call on a device loads the module there.  Every call uses the same area
// and the search re-initialises all
// of it that must start from zero or a known state (queue tickets, control
// counters, root frame; the caller's d_out is zeroed by the search too), but
// two calls whose work overlaps on the GPU -- on different streams, or on one
// device from two host threads -- race on the area and must not be issued.
#include <cstdint>

#include <cuda_runtime.h>

#include "mce.h"

static __device__ __align__(256) unsigned char g_static_scratch[MCE_STATIC_SCRATCH_BYTES];

namespace {

// Device address of the area on the current device, looked up afresh.
int static_area(void **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return MCE_ECUDA;
    }
    *out = p;
    return MCE_OK;
}

}  // namespace

extern "C" int mce_enumerate_device_static(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows,
                                           const mce_options *opts, uint64_t *d_out, void *stream)
{
    if (n > MCE_NMAX || !d_out || (n && !d_rows) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    uint64_t need = 0;
    int rc = mce_scratch_bytes(n, opts, &need);
    if (rc != MCE_OK) return rc;
    if (need > MCE_STATIC_SCRATCH_BYTES) return MCE_ENOMEM;  // options need more than the fixed area
    void *area = nullptr;
    rc = static_area(&area);
    if (rc != MCE_OK) return rc;
    return mce_enumerate_device(n, words_per_row, d_rows, opts, area, MCE_STATIC_SCRATCH_BYTES, d_out, stream);
}
