// C ABI of libmce (include/mce.h): launch configuration, scratch layout,
// device-level step calls and the host-level handle API.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mce_internal.h"

using namespace mce;

namespace {

// ---------------------------------------------------------------------------
// Launch configuration

struct Config {
    int G = 32, K = 1;
    bool smem = false;
    unsigned threads = 0, blocks = 0;
    uint32_t wp = 32;
    uint32_t qcap = 1024, fs = 0;
    uint32_t total_groups = 0;
    int pivot = 0;
    SearchImpl impl{nullptr, nullptr};
};

struct Layout {
    size_t ctl = 0, order = 0, rows = 0, seq = 0, frames = 0, total = 0;
};

mce_options defaults(const mce_options *o)
{
    mce_options d{};
    if (o) d = *o;
    return d;
}

SearchImpl impl_for(int G, int K, bool smem, int pivot)
{
    switch (G * 8 + K) {
    case 1 * 8 + 1: return search_impl_1_1(smem, pivot);
    case 1 * 8 + 2: return search_impl_1_2(smem, pivot);
    case 2 * 8 + 1: return search_impl_2_1(smem, pivot);
    case 2 * 8 + 2: return search_impl_2_2(smem, pivot);
    case 4 * 8 + 1: return search_impl_4_1(smem, pivot);
    case 4 * 8 + 2: return search_impl_4_2(smem, pivot);
    case 8 * 8 + 1: return search_impl_8_1(smem, pivot);
    case 8 * 8 + 2: return search_impl_8_2(smem, pivot);
    case 16 * 8 + 1: return search_impl_16_1(smem, pivot);
    case 16 * 8 + 2: return search_impl_16_2(smem, pivot);
    case 32 * 8 + 1: return search_impl_32_1(smem, pivot);
    case 32 * 8 + 2: return search_impl_32_2(smem, pivot);
    case 32 * 8 + 4: return search_impl_32_4(smem, pivot);
    default: return {nullptr, nullptr};
    }
}

uint32_t next_pow2(uint64_t x)
{
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return (uint32_t)p;
}

size_t search_smem(uint32_t n, uint32_t wp, bool rows_in_smem)
{
    return smem_rows_bytes(n, wp, rows_in_smem) + (size_t)n * 8 + ((size_t)n + 1) * 4;
}

// Default subtree width: the narrowest group whose sets still fit one word
// per lane, one thread per subtree below 65 vertices.
void default_shape(uint32_t n, int &G, int &K)
{
    const uint32_t W = std::max<uint32_t>(1, (n + 31) / 32);
    if (W <= 1) { G = 1; K = 1; }
    else if (W <= 2) { G = 1; K = 2; }
    else if (W <= 4) { G = 4; K = 1; }
    else if (W <= 8) { G = 8; K = 1; }
    else if (W <= 16) { G = 16; K = 1; }
    else if (W <= 32) { G = 32; K = 1; }
    else if (W <= 64) { G = 32; K = 2; }
    else { G = 32; K = 4; }
}

int choose(uint32_t n, const mce_options &o, Config &c)
{
    if (o.pivot_mode > MCE_PIVOT_TOMITA || o.stack_levels > (uint32_t)kStackDepth || o.queue_log2 > 24)
        return MCE_EINVAL;
    const uint32_t W = std::max<uint32_t>(1, (n + 31) / 32);
    int G, K;
    default_shape(n, G, K);
    if (o.lanes_per_subtree || o.words_per_lane) {
        if (o.lanes_per_subtree) G = (int)o.lanes_per_subtree;
        if (o.words_per_lane) K = (int)o.words_per_lane;
        else K = (int)std::max<uint32_t>(1, (W + G - 1) / G);
        if (K == 3) K = 4;
    }
    if ((uint32_t)(G * K) < W) return MCE_EINVAL;
    c.impl = impl_for(G, K, false, (int)o.pivot_mode);
    if (!c.impl.run) return MCE_EINVAL;
    c.G = G;
    c.K = K;
    c.wp = (uint32_t)(G * K);
    c.pivot = (int)o.pivot_mode;

    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MCE_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MCE_ECUDA;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return MCE_ECUDA;
    const size_t limit = (size_t)optin - 1024;  // static shared memory + slack

    c.smem = c.wp <= 32 && search_smem(n, c.wp, true) <= limit;
    if (c.smem) c.impl = impl_for(G, K, true, (int)o.pivot_mode);
    if (search_smem(n, c.wp, c.smem) > limit) return MCE_EINVAL;

    c.threads = o.threads_per_block ? o.threads_per_block : (K >= 4 ? 512u : 1024u);
    if (c.threads % 32 || c.threads > (K >= 4 ? 512u : 1024u)) return MCE_EINVAL;
    if (o.blocks) {
        c.blocks = o.blocks;
    } else {
        int per_sm = 0;
        if (c.impl.occupancy((int)c.threads, search_smem(n, c.wp, c.smem), &per_sm) != cudaSuccess) return MCE_ECUDA;
        if (per_sm < 1) return MCE_ENOMEM;
        c.blocks = (unsigned)(per_sm * sms);
    }
    c.total_groups = c.blocks * (c.threads / 32) * (32 / G);
    c.qcap = next_pow2(std::max<uint64_t>(1024, 2ull * c.total_groups + 256));
    if (o.queue_log2) c.qcap = std::max<uint32_t>(c.qcap, 1u << o.queue_log2);
    c.fs = (uint32_t)round_up(kFrameHdr + 2 * c.wp, 4);
    return MCE_OK;
}

Layout layout(uint32_t n, const Config &c)
{
    Layout L;
    size_t off = 0;
    L.ctl = off;
    off += round_up(sizeof(Ctl), 256);
    L.order = off;
    off += round_up((size_t)std::max<uint32_t>(n, 1) * 4, 256);
    L.rows = off;
    off += round_up((size_t)n * c.wp * 4 + 16, 256);
    L.seq = off;
    off += round_up((size_t)c.qcap * 4, 256);
    L.frames = off;
    off += round_up((size_t)c.qcap * c.fs * 4, 256);
    L.total = off;
    return L;
}

int cuda_code(cudaError_t e) { return e == cudaSuccess ? MCE_OK : (e == cudaErrorMemoryAllocation ? MCE_ENOMEM : MCE_ECUDA); }

SearchParams params(uint32_t n, const Config &c, const Layout &L, unsigned char *scratch, const uint32_t *rows,
                    const uint32_t *order, uint64_t *out, const mce_options &o)
{
    SearchParams p{};
    p.n = n;
    p.wp = c.wp;
    p.rows = rows;
    p.order = order;
    p.ctl = reinterpret_cast<Ctl *>(scratch + L.ctl);
    p.seq = reinterpret_cast<unsigned *>(scratch + L.seq);
    p.frames = reinterpret_cast<uint32_t *>(scratch + L.frames);
    p.qcap = c.qcap;
    p.fs = c.fs;
    p.out = out;
    p.timeout_ns = o.timeout_ns ? o.timeout_ns : 60ull * 1000000000ull;
    p.total_groups = c.total_groups;
    p.pivot_mode = (uint32_t)c.pivot;
    p.stack_levels = o.stack_levels ? std::min<uint32_t>(o.stack_levels, kStackDepth) : kStackDepth;
    return p;
}

int run_search(uint32_t n, const Config &c, const Layout &L, unsigned char *scratch, const uint32_t *rows,
               const uint32_t *order, uint64_t *out, const mce_options &o, cudaStream_t s)
{
    SearchParams p = params(n, c, L, scratch, rows, order, out, o);
    LaunchShape sh{c.blocks, c.threads, search_smem(n, c.wp, c.smem), c.smem};
    return cuda_code(c.impl.run(p, sh, s));
}

}  // namespace

// ---------------------------------------------------------------------------
// Device-level calls

extern "C" int mce_edges_to_rows(uint32_t n, uint64_t m, const uint32_t *d_uv, uint32_t words_per_row,
                                 uint32_t *d_rows, uint64_t *d_out, void *stream)
{
    if (n > MCE_NMAX || !d_out || (m && !d_uv) || (n && !d_rows) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    return cuda_code(launch_edges_to_rows(n, m, d_uv, words_per_row, d_rows, d_out, (cudaStream_t)stream));
}

extern "C" int mce_validate_rows(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows, uint64_t *d_out,
                                 void *stream)
{
    if (n > MCE_NMAX || !d_out || (n && !d_rows) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    return cuda_code(launch_validate_rows(n, words_per_row, d_rows, d_out, (cudaStream_t)stream));
}

extern "C" int mce_order(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows, uint32_t *d_order, void *stream)
{
    if (n > MCE_NMAX || (n && (!d_rows || !d_order)) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    return cuda_code(launch_order(n, words_per_row, d_rows, d_order, (cudaStream_t)stream));
}

extern "C" int mce_renumber(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows, const uint32_t *d_order,
                            uint32_t out_words_per_row, uint32_t *d_rows_out, void *stream)
{
    if (n > MCE_NMAX || (n && (!d_rows || !d_order || !d_rows_out)) || words_per_row < (n + 31) / 32 ||
        out_words_per_row < (n + 31) / 32)
        return MCE_EINVAL;
    return cuda_code(launch_renumber(n, words_per_row, d_rows, d_order, out_words_per_row, d_rows_out,
                                     (cudaStream_t)stream));
}

extern "C" uint32_t mce_search_words(uint32_t n, const mce_options *opts)
{
    Config c;
    if (n > MCE_NMAX || choose(n, defaults(opts), c) != MCE_OK) return 0;
    return c.wp;
}

extern "C" int mce_scratch_bytes(uint32_t n, const mce_options *opts, uint64_t *bytes)
{
    if (!bytes || n > MCE_NMAX) return MCE_EINVAL;
    Config c;
    int rc = choose(n, defaults(opts), c);
    if (rc) return rc;
    *bytes = layout(n, c).total;
    return MCE_OK;
}

extern "C" int mce_search(uint32_t n, const uint32_t *d_rows_renum, const uint32_t *d_order, const mce_options *opts,
                          void *d_scratch, uint64_t scratch_bytes, uint64_t *d_out, void *stream)
{
    if (n > MCE_NMAX || !d_out || !d_scratch || (n && (!d_rows_renum || !d_order))) return MCE_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_scratch) % 256 || reinterpret_cast<uintptr_t>(d_rows_renum) % 16)
        return MCE_EINVAL;
    const mce_options o = defaults(opts);
    Config c;
    int rc = choose(n, o, c);
    if (rc) return rc;
    const Layout L = layout(n, c);
    if (scratch_bytes < L.total) return MCE_ENOMEM;
    return run_search(n, c, L, static_cast<unsigned char *>(d_scratch), d_rows_renum, d_order, d_out, o,
                      (cudaStream_t)stream);
}

extern "C" int mce_enumerate_device(uint32_t n, uint32_t words_per_row, const uint32_t *d_rows,
                                    const mce_options *opts, void *d_scratch, uint64_t scratch_bytes,
                                    uint64_t *d_out, void *stream)
{
    if (n > MCE_NMAX || !d_out || !d_scratch || (n && !d_rows) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_scratch) % 256) return MCE_EINVAL;
    const mce_options o = defaults(opts);
    Config c;
    int rc = choose(n, o, c);
    if (rc) return rc;
    const Layout L = layout(n, c);
    if (scratch_bytes < L.total) return MCE_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *scr = static_cast<unsigned char *>(d_scratch);
    uint32_t *order = reinterpret_cast<uint32_t *>(scr + L.order);
    uint32_t *rows = reinterpret_cast<uint32_t *>(scr + L.rows);
    cudaError_t e = cudaMemsetAsync(d_out + MCE_OUT_STATUS, 0, sizeof(uint64_t), s);
    if (e == cudaSuccess) e = launch_validate_rows(n, words_per_row, d_rows, d_out, s);
    if (e == cudaSuccess)
        e = (o.flags & MCE_ORDER_IDENTITY) ? launch_identity(n, order, s) : launch_order(n, words_per_row, d_rows, order, s);
    if (e == cudaSuccess) e = launch_renumber(n, words_per_row, d_rows, order, c.wp, rows, s);
    if (e != cudaSuccess) return cuda_code(e);
    return run_search(n, c, L, scr, rows, order, d_out, o, s);
}

// ---------------------------------------------------------------------------
// Host-level API

struct mce_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;
    uint64_t budget = 0;
    uint64_t used = 0;
};

struct mce_graph {
    mce_ctx *ctx = nullptr;
    uint32_t n = 0, w = 0;
    uint32_t *d_rows = nullptr;
    uint64_t bytes = 0;
};

namespace {

struct DevicePick {
    int prev = -1;
    explicit DevicePick(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevicePick()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int dalloc(mce_ctx *ctx, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (ctx->budget && ctx->used + bytes > ctx->budget) return MCE_ENOMEM;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MCE_ENOMEM;
    }
    ctx->used += bytes;
    return MCE_OK;
}

void dfree(mce_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    cudaFreeAsync(p, ctx->stream);
    if (bytes == 0) bytes = 256;
    ctx->used -= std::min<uint64_t>(ctx->used, bytes);
}

double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" int mce_ctx_create(int device, uint64_t mem_budget_bytes, void *stream, mce_ctx **out)
{
    if (!out) return MCE_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return device < 0 ? MCE_EINVAL : MCE_ECUDA;
    }
    mce_ctx *c = new (std::nothrow) mce_ctx;
    if (!c) return MCE_ENOMEM;
    DevicePick pick(device);
    c->device = device;
    cudaError_t e = cudaSuccess;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = true;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&c->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = ~0ull;  // keep freed blocks for reuse
        e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    size_t fr = 0, tot = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
        if (c->pool) cudaMemPoolDestroy(c->pool);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return MCE_ECUDA;
    }
    c->budget = mem_budget_bytes ? mem_budget_bytes : (uint64_t)(fr * 0.9);
    *out = c;
    return MCE_OK;
}

extern "C" void mce_ctx_destroy(mce_ctx *ctx)
{
    if (!ctx) return;
    {
        DevicePick pick(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
}

namespace {

int finish_load(mce_ctx *ctx, mce_graph *g, uint64_t *d_status, mce_graph **out)
{
    uint64_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, d_status + MCE_OUT_STATUS, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, d_status, 64);
    if (e != cudaSuccess || st != 0) {
        dfree(ctx, g->d_rows, g->bytes);
        cudaStreamSynchronize(ctx->stream);
        delete g;
        return e != cudaSuccess ? MCE_ECUDA : (int)(int64_t)st;
    }
    *out = g;
    return MCE_OK;
}

}  // namespace

extern "C" int mce_load_edges(mce_ctx *ctx, uint32_t n, const uint32_t *uv, uint64_t m, mce_graph **out)
{
    if (!ctx || !out || n > MCE_NMAX || (m && !uv)) return MCE_EINVAL;
    *out = nullptr;
    DevicePick pick(ctx->device);
    mce_graph *g = new (std::nothrow) mce_graph;
    if (!g) return MCE_ENOMEM;
    g->ctx = ctx;
    g->n = n;
    g->w = std::max<uint32_t>(1, (n + 31) / 32);
    g->bytes = (uint64_t)std::max<uint32_t>(n, 1) * g->w * 4;
    uint32_t *d_uv = nullptr;
    uint64_t *d_status = nullptr;
    int rc = dalloc(ctx, (void **)&g->d_rows, g->bytes);
    if (rc == MCE_OK) rc = dalloc(ctx, (void **)&d_status, 64);
    if (rc == MCE_OK && m) rc = dalloc(ctx, (void **)&d_uv, m * 8);
    cudaError_t e = cudaSuccess;
    if (rc == MCE_OK) {
        e = cudaMemsetAsync(d_status, 0, 64, ctx->stream);
        if (e == cudaSuccess && m) e = cudaMemcpyAsync(d_uv, uv, m * 8, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = launch_edges_to_rows(n, m, d_uv, g->w, g->d_rows, d_status, ctx->stream);
        if (e != cudaSuccess) rc = MCE_ECUDA;
    }
    dfree(ctx, d_uv, m * 8);
    if (rc != MCE_OK) {
        dfree(ctx, d_status, 64);
        dfree(ctx, g->d_rows, g->bytes);
        cudaStreamSynchronize(ctx->stream);
        delete g;
        return rc;
    }
    return finish_load(ctx, g, d_status, out);
}

extern "C" int mce_load_bitset(mce_ctx *ctx, uint32_t n, const uint32_t *rows, uint32_t words_per_row,
                               mce_graph **out)
{
    if (!ctx || !out || n > MCE_NMAX || (n && !rows) || words_per_row < (n + 31) / 32) return MCE_EINVAL;
    *out = nullptr;
    DevicePick pick(ctx->device);
    mce_graph *g = new (std::nothrow) mce_graph;
    if (!g) return MCE_ENOMEM;
    g->ctx = ctx;
    g->n = n;
    g->w = std::max<uint32_t>(1, words_per_row);
    g->bytes = (uint64_t)std::max<uint32_t>(n, 1) * g->w * 4;
    uint64_t *d_status = nullptr;
    int rc = dalloc(ctx, (void **)&g->d_rows, g->bytes);
    if (rc == MCE_OK) rc = dalloc(ctx, (void **)&d_status, 64);
    cudaError_t e = cudaSuccess;
    if (rc == MCE_OK) {
        e = cudaMemsetAsync(d_status, 0, 64, ctx->stream);
        if (e == cudaSuccess && n)
            e = cudaMemcpyAsync(g->d_rows, rows, (size_t)n * words_per_row * 4, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = launch_validate_rows(n, g->w, g->d_rows, d_status, ctx->stream);
        if (e != cudaSuccess) rc = MCE_ECUDA;
    }
    if (rc != MCE_OK) {
        dfree(ctx, d_status, 64);
        dfree(ctx, g->d_rows, g->bytes);
        cudaStreamSynchronize(ctx->stream);
        delete g;
        return rc;
    }
    return finish_load(ctx, g, d_status, out);
}

extern "C" void mce_graph_free(mce_graph *g)
{
    if (!g) return;
    DevicePick pick(g->ctx->device);
    dfree(g->ctx, g->d_rows, g->bytes);
    cudaStreamSynchronize(g->ctx->stream);
    delete g;
}

namespace {

int fill_result(const std::vector<uint64_t> &h, uint32_t n, mce_result *res)
{
    res->count = h[MCE_OUT_COUNT];
    res->nodes = h[MCE_OUT_NODES];
    res->internal_nodes = h[MCE_OUT_INTERNAL];
    res->dead_ends = h[MCE_OUT_DEAD_ENDS];
    res->hash = h[MCE_OUT_HASH];
    res->max_size = (uint32_t)h[MCE_OUT_MAX_SIZE];
    const int st = (int)(int64_t)h[MCE_OUT_STATUS];
    res->status = (uint32_t)st;
    if (st) return st;
    if (res->hist) {
        const uint32_t k = std::min<uint32_t>(res->hist_cap, n + 1);
        for (uint32_t i = 0; i < k; ++i) res->hist[i] = h[MCE_OUT_HIST + i];
        for (uint32_t i = k; i < res->hist_cap; ++i) res->hist[i] = 0;
        if (res->hist_cap <= res->max_size && res->count) return MCE_ETRUNC;
    }
    return MCE_OK;
}

}  // namespace

namespace {
int enumerate_once(mce_graph *g, const mce_options &o, mce_result *res, std::chrono::steady_clock::time_point t0);
}

extern "C" int mce_enumerate(mce_graph *g, const mce_options *opts, mce_result *res)
{
    if (!g || !res) return MCE_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    DevicePick pick(g->ctx->device);
    mce_options o = defaults(opts);
    int rc = enumerate_once(g, o, res, t0);
    // a queue overflow leaves no partial state behind: retry with 16x the slots
    for (int tries = 0; rc == MCE_EOVERFLOW && tries < 2; ++tries) {
        Config c;
        if (choose(g->n, o, c) != MCE_OK) break;
        uint32_t lg = 0;
        while ((1u << lg) < c.qcap) ++lg;
        if (lg + 4 > 24) break;
        o.queue_log2 = lg + 4;
        rc = enumerate_once(g, o, res, t0);
    }
    return rc;
}

namespace {
int enumerate_once(mce_graph *g, const mce_options &o, mce_result *res, std::chrono::steady_clock::time_point t0)
{
    mce_ctx *ctx = g->ctx;
    if (o.flags & (MCE_LIST | MCE_LIST_SORTED)) return MCE_ENOTIMPL;
    uint64_t sbytes = 0;
    int rc = mce_scratch_bytes(g->n, &o, &sbytes);
    if (rc) return rc;
    const size_t obytes = MCE_OUT_WORDS(g->n) * 8;
    void *scr = nullptr;
    uint64_t *d_out = nullptr;
    rc = dalloc(ctx, &scr, sbytes);
    if (rc == MCE_OK) rc = dalloc(ctx, (void **)&d_out, obytes);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<uint64_t> h(MCE_OUT_WORDS(g->n), 0);
    if (rc == MCE_OK) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, ctx->stream);
        rc = mce_enumerate_device(g->n, g->w, g->d_rows, &o, scr, sbytes, d_out, ctx->stream);
        cudaEventRecord(e1, ctx->stream);
        if (rc == MCE_OK) {
            cudaError_t e = cudaMemcpyAsync(h.data(), d_out, obytes, cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) rc = MCE_ECUDA;
        }
    }
    float kms = 0.f;
    if (rc == MCE_OK && e0 && e1) cudaEventElapsedTime(&kms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(ctx, d_out, obytes);
    dfree(ctx, scr, sbytes);
    if (rc != MCE_OK) {
        cudaStreamSynchronize(ctx->stream);
        return rc;
    }
    rc = fill_result(h, g->n, res);
    res->kernel_ms = kms;
    res->total_ms = ms_since(t0);
    return rc;
}
}  // namespace

extern "C" int mce_enumerate_batch(mce_ctx *ctx, mce_graph *const *graphs, uint32_t count, const mce_options *opts,
                                   mce_result *res)
{
    (void)ctx; (void)graphs; (void)count; (void)opts; (void)res;
    return MCE_ENOTIMPL;
}

extern "C" int mce_submit(mce_ctx *ctx, mce_graph *g, const mce_options *opts, mce_ticket *out)
{
    (void)ctx; (void)g; (void)opts; (void)out;
    return MCE_ENOTIMPL;
}

extern "C" int mce_poll(mce_ctx *ctx, mce_ticket t, mce_result *res)
{
    (void)ctx; (void)t; (void)res;
    return MCE_ENOTIMPL;
}

extern "C" int mce_wait(mce_ctx *ctx, mce_ticket t, uint64_t timeout_ns, mce_result *res)
{
    (void)ctx; (void)t; (void)timeout_ns; (void)res;
    return MCE_ENOTIMPL;
}

extern "C" const char *mce_strerror(int code)
{
    switch (code) {
    case MCE_OK: return "ok";
    case MCE_PENDING: return "pending";
    case MCE_EINVAL: return "invalid argument or graph";
    case MCE_ENOMEM: return "out of memory";
    case MCE_ECUDA: return "CUDA error";
    case MCE_ETRUNC: return "output buffer too small";
    case MCE_ETIMEOUT: return "timed out";
    case MCE_EOVERFLOW: return "work queue overflow";
    case MCE_ENOTIMPL: return "not implemented";
    default: return "unknown error";
    }
}
