"""Python binding of libmce (include/mce.h).

Argument marshalling only: every step of the search path runs in the CUDA
kernels of ``libmce.so``.  There is no CPU fallback -- if the library is
missing, ``lib()`` raises.  PyTorch is used by callers only for device memory
and streams (tensors are passed by ``data_ptr()``).

The functions keep the C names: ``mce_enumerate_device``, ``mce_search``,
``mce_load_edges`` and so on.  ``Context`` / ``Graph`` wrap the handle API.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

# The served form runs every admitted request on its own stream; CUDA maps
# streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 unless set), and
# streams sharing a queue run one after another.  Ask for the most queues
# unless the caller chose; it takes effect only if no CUDA context exists yet.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from .build import LIB as _LIB_PATH, build  # noqa: F401

MCE_OK, MCE_PENDING = 0, 1
MCE_EINVAL, MCE_ENOMEM, MCE_ECUDA, MCE_ETRUNC = -1, -2, -3, -4
MCE_ETIMEOUT, MCE_EOVERFLOW, MCE_ENOTIMPL = -5, -6, -7
MCE_ECANCELED, MCE_EBUSY = -8, -9
MCE_FAULT_ALLOC, MCE_FAULT_COPY, MCE_FAULT_ADMIT = 1, 2, 3
MCE_NMAX, MCE_NMAX_SPARSE = 4096, 65535

MCE_PIVOT_GREEDY, MCE_PIVOT_GREEDY_TX, MCE_PIVOT_TOMITA, MCE_PIVOT_GREEDY_NX = 0, 1, 2, 3
PIVOTS = {"greedy": 0, "tx": 1, "tomita": 2, "nx": 3}
MCE_ORDER_IDENTITY, MCE_LIST, MCE_LIST_SORTED, MCE_AUTOTUNE, MCE_OUTER = 0x1, 0x2, 0x4, 0x8, 0x10

MCE_OUT_COUNT, MCE_OUT_NODES, MCE_OUT_INTERNAL, MCE_OUT_DEAD_ENDS = 0, 1, 2, 3
MCE_OUT_HASH, MCE_OUT_STATUS, MCE_OUT_MAX_SIZE, MCE_OUT_DONATIONS = 4, 5, 6, 7
MCE_OUT_STEALS, MCE_OUT_GLOBAL, MCE_OUT_BUSY_NS, MCE_OUT_GROUPS = 8, 9, 10, 11
MCE_OUT_GPUSH, MCE_OUT_GTRY, MCE_OUT_CAS_FAIL, MCE_OUT_LANE_TASKS = 12, 13, 14, 15
MCE_OUT_HIST = 16


def MCE_OUT_WORDS(n: int) -> int:
    return MCE_OUT_HIST + n + 1


class MceError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {mce_strerror(code)} ({code})" if what else f"{mce_strerror(code)} ({code})")


class Options(C.Structure):
    _fields_ = [("pivot_mode", C.c_uint32), ("flags", C.c_uint32), ("lanes_per_subtree", C.c_uint32),
                ("words_per_lane", C.c_uint32), ("blocks", C.c_uint32), ("threads_per_block", C.c_uint32),
                ("timeout_ns", C.c_uint64), ("stack_levels", C.c_uint32), ("queue_log2", C.c_uint32),
                ("split_min_p", C.c_uint32), ("_reserved", C.c_uint32)]


class BatchBucket(C.Structure):
    _fields_ = [("words_class", C.c_uint32), ("graphs", C.c_uint32), ("lanes_per_subtree", C.c_uint32),
                ("words_per_lane", C.c_uint32), ("threads_per_block", C.c_uint32), ("blocks", C.c_uint32),
                ("split_min_p", C.c_uint32), ("tuned", C.c_uint32), ("tuned_ms_per_graph", C.c_double),
                ("work_items", C.c_uint32), ("split_graphs", C.c_uint32)]


class Peaks(C.Structure):
    _fields_ = [("lop3_lane_ops_per_s", C.c_double), ("popc_lane_ops_per_s", C.c_double),
                ("lds_bytes_per_s", C.c_double), ("ms_lop3", C.c_double), ("ms_popc", C.c_double),
                ("ms_lds", C.c_double), ("sm_count", C.c_uint32), ("sm_clock_max_khz", C.c_uint32),
                ("ballot_warp_ops_per_s", C.c_double), ("shfl_warp_ops_per_s", C.c_double),
                ("redux_warp_ops_per_s", C.c_double)]


class Result(C.Structure):
    _fields_ = [("count", C.c_uint64), ("nodes", C.c_uint64), ("internal_nodes", C.c_uint64),
                ("dead_ends", C.c_uint64), ("hash", C.c_uint64), ("max_size", C.c_uint32),
                ("status", C.c_uint32), ("hist", C.POINTER(C.c_uint64)), ("hist_cap", C.c_uint32),
                ("_pad", C.c_uint32), ("list_ids", C.POINTER(C.c_uint32)), ("list_cap", C.c_uint64),
                ("list_off", C.POINTER(C.c_uint64)), ("list_off_cap", C.c_uint64),
                ("list_ids_needed", C.c_uint64), ("kernel_ms", C.c_double), ("total_ms", C.c_double)]


def options(pivot: str | int = "greedy", identity_order: bool = False, lanes: int = 0, words: int = 0,
            blocks: int = 0, threads: int = 0, timeout_ns: int = 0, stack_levels: int = 0,
            queue_log2: int = 0, split_min_p: int = 0, flags: int = 0, autotune: bool = False,
            outer: bool = False) -> Options:
    o = Options()
    o.pivot_mode = PIVOTS[pivot] if isinstance(pivot, str) else int(pivot)
    o.flags = flags | (MCE_ORDER_IDENTITY if identity_order else 0) | (MCE_AUTOTUNE if autotune else 0) | \
        (MCE_OUTER if outer else 0)
    o.lanes_per_subtree, o.words_per_lane = lanes, words
    o.blocks, o.threads_per_block = blocks, threads
    o.timeout_ns, o.stack_levels, o.queue_log2 = timeout_ns, stack_levels, queue_log2
    o.split_min_p = split_min_p
    return o


_lib = None
_VP, _U32, _U64 = C.c_void_p, C.c_uint32, C.c_uint64

_SIGS = {
    "mce_edges_to_rows": (C.c_int, [_U32, _U64, _VP, _U32, _VP, _VP, _VP]),
    "mce_validate_rows": (C.c_int, [_U32, _U32, _VP, _VP, _VP]),
    "mce_order": (C.c_int, [_U32, _U32, _VP, _VP, _VP]),
    "mce_renumber": (C.c_int, [_U32, _U32, _VP, _VP, _U32, _VP, _VP]),
    "mce_scratch_bytes": (C.c_int, [_U32, C.POINTER(Options), C.POINTER(_U64)]),
    "mce_search": (C.c_int, [_U32, _VP, _VP, C.POINTER(Options), _VP, _U64, _VP, _VP]),
    "mce_search_words": (_U32, [_U32, C.POINTER(Options)]),
    "mce_enumerate_device": (C.c_int, [_U32, _U32, _VP, C.POINTER(Options), _VP, _U64, _VP, _VP]),
    "mce_enumerate_device_static": (C.c_int, [_U32, _U32, _VP, C.POINTER(Options), _VP, _VP]),
    "mce_ctx_create": (C.c_int, [C.c_int, _U64, _VP, C.POINTER(_VP)]),
    "mce_ctx_destroy": (None, [_VP]),
    "mce_load_edges": (C.c_int, [_VP, _U32, _VP, _U64, C.POINTER(_VP)]),
    "mce_load_bitset": (C.c_int, [_VP, _U32, _VP, _U32, C.POINTER(_VP)]),
    "mce_graph_free": (None, [_VP]),
    "mce_enumerate": (C.c_int, [_VP, C.POINTER(Options), C.POINTER(Result)]),
    "mce_enumerate_batch": (C.c_int, [_VP, C.POINTER(_VP), _U32, C.POINTER(Options), C.POINTER(Result)]),
    "mce_batch_create": (C.c_int, [_VP, C.POINTER(_VP), _U32, C.POINTER(Options), C.POINTER(_VP)]),
    "mce_batch_launch": (C.c_int, [_VP]),
    "mce_batch_results": (C.c_int, [_VP, C.POINTER(Result)]),
    "mce_batch_run": (C.c_int, [_VP, C.POINTER(Result)]),
    "mce_batch_destroy": (None, [_VP]),
    "mce_batch_buckets": (C.c_int, [_VP, C.POINTER(BatchBucket), _U32, C.POINTER(_U32)]),
    "mce_submit": (C.c_int, [_VP, _VP, C.POINTER(Options), C.POINTER(_U64)]),
    "mce_poll": (C.c_int, [_VP, _U64, C.POINTER(Result)]),
    "mce_wait": (C.c_int, [_VP, _U64, _U64, C.POINTER(Result)]),
    "mce_cancel": (C.c_int, [_VP, _U64]),
    "mce_fault_inject": (C.c_int, [C.c_int, _U32, _U32]),
    "mce_ctx_mem_used": (_U64, [_VP]),
    "mce_strerror": (C.c_char_p, [C.c_int]),
    "mce_trace_enable": (C.c_int, [_VP, _U64]),
    "mce_measure_peaks": (C.c_int, [C.c_int, C.POINTER(Peaks)]),
    "mce_root_children": (C.c_int, [_VP, C.POINTER(Options), _VP, _U32, C.POINTER(_U32)]),
    "mce_enumerate_part": (C.c_int, [_VP, C.POINTER(Options), _VP, _U32, C.c_int, C.POINTER(Result)]),
    "mce_enumerate_stream": (C.c_int, [_VP, C.POINTER(Options), _VP, _VP, C.POINTER(Result)]),
}

# mce_clique_sink: int (*)(const uint32_t *ids, const uint64_t *off, uint64_t count, void *user)
CliqueSink = C.CFUNCTYPE(C.c_int, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64), C.c_uint64, C.c_void_p)


def lib():
    """The loaded libmce.so; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libmce.so is not built ({_LIB_PATH}); run paper_1801_00202_gb300.build.build()")
        L = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def _opt(o):
    return C.byref(o if o is not None else Options())


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise MceError(rc, what)
    return rc


# --- C names, one to one ---------------------------------------------------

def mce_strerror(code: int) -> str:
    return lib().mce_strerror(code).decode()


def mce_fault_inject(site: int, skip: int = 0, count: int = 1) -> int:
    """Arm a host-side fault site (MCE_FAULT_ALLOC / COPY / ADMIT): after
    `skip` passes, the next `count` fail; count 0 disarms."""
    return int(lib().mce_fault_inject(site, skip, count))


def mce_measure_peaks(device: int = 0) -> dict:
    """LOP3 / POPC lane-ops per second and 128-bit shared-memory load bytes
    per second measured on ``device`` (the search's roofline denominators)."""
    pk = Peaks()
    _check(lib().mce_measure_peaks(device, C.byref(pk)), "mce_measure_peaks")
    return {f: getattr(pk, f) for f, _ in Peaks._fields_}


def mce_edges_to_rows(n, m, d_uv, words_per_row, d_rows, d_out, stream=None) -> int:
    return lib().mce_edges_to_rows(n, m, _ptr(d_uv), words_per_row, _ptr(d_rows), _ptr(d_out), _stream(stream))


def mce_validate_rows(n, words_per_row, d_rows, d_out, stream=None) -> int:
    return lib().mce_validate_rows(n, words_per_row, _ptr(d_rows), _ptr(d_out), _stream(stream))


def mce_order(n, words_per_row, d_rows, d_order, stream=None) -> int:
    return lib().mce_order(n, words_per_row, _ptr(d_rows), _ptr(d_order), _stream(stream))


def mce_renumber(n, words_per_row, d_rows, d_order, out_words_per_row, d_rows_out, stream=None) -> int:
    return lib().mce_renumber(n, words_per_row, _ptr(d_rows), _ptr(d_order), out_words_per_row,
                              _ptr(d_rows_out), _stream(stream))


def mce_scratch_bytes(n, opts=None) -> int:
    b = C.c_uint64(0)
    _check(lib().mce_scratch_bytes(n, _opt(opts), C.byref(b)), "mce_scratch_bytes")
    return int(b.value)


def mce_search_words(n, opts=None) -> int:
    return int(lib().mce_search_words(n, _opt(opts)))


def mce_search(n, d_rows_renum, d_order, opts, d_scratch, scratch_bytes, d_out, stream=None) -> int:
    return lib().mce_search(n, _ptr(d_rows_renum), _ptr(d_order), _opt(opts), _ptr(d_scratch), scratch_bytes,
                            _ptr(d_out), _stream(stream))


def mce_enumerate_device(n, words_per_row, d_rows, opts, d_scratch, scratch_bytes, d_out, stream=None) -> int:
    return lib().mce_enumerate_device(n, words_per_row, _ptr(d_rows), _opt(opts), _ptr(d_scratch), scratch_bytes,
                                      _ptr(d_out), _stream(stream))


def mce_trace_enable(d_buf, nbytes: int) -> int:
    return lib().mce_trace_enable(_ptr(d_buf), nbytes)


MCE_STATIC_SCRATCH_BYTES = 32 << 20


def mce_enumerate_device_static(n, words_per_row, d_rows, opts, d_out, stream=None) -> int:
    """The whole path with the library's fixed scratch area: nothing is
    allocated, for callers that may not allocate device memory."""
    return lib().mce_enumerate_device_static(n, words_per_row, _ptr(d_rows), _opt(opts), _ptr(d_out),
                                             _stream(stream))


def decode_out(out, n: int) -> dict:
    """Result dict from a device/host d_out array of MCE_OUT_WORDS(n) uint64."""
    a = np.asarray(out.cpu().numpy() if hasattr(out, "cpu") else out).view(np.uint64)
    return {"count": int(a[MCE_OUT_COUNT]), "nodes": int(a[MCE_OUT_NODES]),
            "internal": int(a[MCE_OUT_INTERNAL]), "dead_ends": int(a[MCE_OUT_DEAD_ENDS]),
            "hash": int(a[MCE_OUT_HASH]), "status": int(a[MCE_OUT_STATUS].astype(np.int64)),
            "max_size": int(a[MCE_OUT_MAX_SIZE]), "donations": int(a[MCE_OUT_DONATIONS]),
            "steals": int(a[MCE_OUT_STEALS]), "global_steals": int(a[MCE_OUT_GLOBAL]),
            "busy_ns": int(a[MCE_OUT_BUSY_NS]), "groups": int(a[MCE_OUT_GROUPS]),
            "global_pushes": int(a[MCE_OUT_GPUSH]), "global_tries": int(a[MCE_OUT_GTRY]),
            "cas_fails": int(a[MCE_OUT_CAS_FAIL]), "lane_tasks": int(a[MCE_OUT_LANE_TASKS]),
            "hist": a[MCE_OUT_HIST:MCE_OUT_HIST + n + 1].copy()}


# --- handle API -------------------------------------------------------------

class Context:
    """mce_ctx: a device, a stream and a device-memory budget.  Graphs and
    batches made from a context are released before it is destroyed."""

    def __init__(self, device: int = 0, mem_budget: int = 0, stream=None):
        import weakref
        h = C.c_void_p()
        _check(lib().mce_ctx_create(device, mem_budget, _stream(stream), C.byref(h)), "mce_ctx_create")
        self.handle = h
        self._owned = weakref.WeakSet()

    def close(self):
        if self.handle:
            for obj in list(self._owned):
                obj.close()
            lib().mce_ctx_destroy(self.handle)
            self.handle = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def load_edges(self, n: int, uv) -> "Graph":
        uv = np.ascontiguousarray(np.asarray(uv, dtype=np.uint32).reshape(-1, 2))
        h = C.c_void_p()
        _check(lib().mce_load_edges(self.handle, n, uv.ctypes.data if uv.size else None, uv.shape[0], C.byref(h)),
               "mce_load_edges")
        g = Graph(self, h, n)
        self._owned.add(g)
        return g

    # --- served form ------------------------------------------------------
    def submit(self, graph: "Graph", opts: Options | None = None) -> int:
        t = C.c_uint64(0)
        _check(lib().mce_submit(self.handle, graph.handle, _opt(opts), C.byref(t)), "mce_submit")
        if not hasattr(self, "_tickets"):
            self._tickets = {}
        self._tickets[int(t.value)] = graph.n
        return int(t.value)

    def _collect(self, ticket: int, call, *extra):
        n = self._tickets[ticket]
        hist = np.zeros(n + 1, dtype=np.uint64)
        r = Result()
        r.hist = hist.ctypes.data_as(C.POINTER(C.c_uint64))
        r.hist_cap = hist.size
        rc = call(self.handle, ticket, *extra, C.byref(r))
        if rc == MCE_PENDING or rc == MCE_ETIMEOUT:
            return rc, None
        del self._tickets[ticket]
        return rc, {"rc": rc, "count": r.count, "nodes": r.nodes, "internal": r.internal_nodes,
                    "dead_ends": r.dead_ends, "hash": r.hash, "max_size": r.max_size, "hist": hist,
                    "kernel_ms": r.kernel_ms, "total_ms": r.total_ms}

    def poll(self, ticket: int):
        """mce_poll: None while pending, else the result dict (rc inside)."""
        rc, res = self._collect(ticket, lib().mce_poll)
        return res

    def wait(self, ticket: int, timeout_ns: int = 0):
        rc, res = self._collect(ticket, lib().mce_wait, timeout_ns)
        if res is None:
            raise MceError(rc, "mce_wait")
        return res

    def cancel(self, ticket: int) -> int:
        """mce_cancel: MCE_OK when the queued request will not run (its
        result then carries MCE_ECANCELED), MCE_EBUSY when it already runs."""
        return int(lib().mce_cancel(self.handle, ticket))

    def mem_used(self) -> int:
        """mce_ctx_mem_used: device bytes the context's allocations hold."""
        return int(lib().mce_ctx_mem_used(self.handle))

    def load_bitset(self, n: int, rows) -> "Graph":
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.uint32))
        w = rows.shape[1] if rows.ndim == 2 else max(1, (n + 31) // 32)
        h = C.c_void_p()
        _check(lib().mce_load_bitset(self.handle, n, rows.ctypes.data if rows.size else None, w, C.byref(h)),
               "mce_load_bitset")
        g = Graph(self, h, n)
        self._owned.add(g)
        return g


class Graph:
    """mce_graph: a validated graph resident on the device."""

    def __init__(self, ctx: Context, handle, n: int):
        self.ctx, self.handle, self.n = ctx, handle, n

    def free(self):
        if self.handle:
            if self.ctx.handle:
                lib().mce_graph_free(self.handle)
            self.handle = None

    close = free
    __del__ = free

    def enumerate(self, opts: Options | None = None, raise_on_error: bool = True,
                  list_cap: int | None = None, off_cap: int | None = None) -> dict:
        """mce_enumerate.  With MCE_LIST / MCE_LIST_SORTED in opts.flags the
        result also holds the listing ("list_ids", "list_off": CSR, original
        labels, each clique ascending; MCE_LIST_SORTED also orders the
        cliques lexicographically).  Without capacities, a first call learns
        the sizes (MCE_ETRUNC) and a second one lists."""
        listing = opts is not None and (opts.flags & (MCE_LIST | MCE_LIST_SORTED)) != 0
        hist = np.zeros(self.n + 1, dtype=np.uint64)
        r = Result()
        r.hist = hist.ctypes.data_as(C.POINTER(C.c_uint64))
        r.hist_cap = hist.size
        ids = off = None
        if listing:
            if list_cap is None or off_cap is None:
                probe = self.enumerate(opts, raise_on_error=False, list_cap=0, off_cap=0)
                if probe["rc"] not in (0, MCE_ETRUNC):
                    if raise_on_error:
                        _check(probe["rc"], "mce_enumerate")
                    return probe
                list_cap, off_cap = int(probe["list_ids_needed"]), int(probe["count"]) + 1
            ids = np.zeros(max(list_cap, 1), dtype=np.uint32)
            off = np.zeros(max(off_cap, 1), dtype=np.uint64)
            r.list_ids = ids.ctypes.data_as(C.POINTER(C.c_uint32))
            r.list_cap = list_cap
            r.list_off = off.ctypes.data_as(C.POINTER(C.c_uint64))
            r.list_off_cap = off_cap
        rc = lib().mce_enumerate(self.handle, _opt(opts), C.byref(r))
        if raise_on_error:
            _check(rc, "mce_enumerate")
        out = {"rc": rc, "count": r.count, "nodes": r.nodes, "internal": r.internal_nodes,
               "dead_ends": r.dead_ends, "hash": r.hash, "max_size": r.max_size, "hist": hist,
               "kernel_ms": r.kernel_ms, "total_ms": r.total_ms, "list_ids_needed": r.list_ids_needed}
        if listing and rc == 0:
            # exact capacities (the usual case) hand back the buffers as they
            # are; larger ones are trimmed by a copy
            no, ni = r.count + 1, r.list_ids_needed
            out["list_off"] = off if off.size == no else off[:no].copy()
            out["list_ids"] = ids if ids.size == ni else ids[:ni].copy()
        return out


    def root_children(self, opts: Options | None = None) -> np.ndarray:
        """mce_root_children: candidate-set sizes of the root's children
        (independent subtrees, in order)."""
        cnt = C.c_uint32(0)
        rc = lib().mce_root_children(self.handle, _opt(opts), None, 0, C.byref(cnt))
        if rc not in (MCE_OK, MCE_ETRUNC):
            _check(rc, "mce_root_children")
        sizes = np.zeros(max(cnt.value, 1), dtype=np.uint32)
        _check(lib().mce_root_children(self.handle, _opt(opts), sizes.ctypes.data, sizes.size, C.byref(cnt)),
               "mce_root_children")
        return sizes[:cnt.value].copy()

    def enumerate_part(self, children, count_root: bool, opts: Options | None = None,
                       raise_on_error: bool = True) -> dict:
        """mce_enumerate_part: the search restricted to the listed root
        children (strictly increasing indices); the root node is counted
        only with count_root."""
        ch = np.ascontiguousarray(np.asarray(children, dtype=np.uint32).reshape(-1))
        hist = np.zeros(self.n + 1, dtype=np.uint64)
        r = Result()
        r.hist = hist.ctypes.data_as(C.POINTER(C.c_uint64))
        r.hist_cap = hist.size
        rc = lib().mce_enumerate_part(self.handle, _opt(opts), ch.ctypes.data if ch.size else None, ch.size,
                                      1 if count_root else 0, C.byref(r))
        if raise_on_error:
            _check(rc, "mce_enumerate_part")
        return {"rc": rc, "count": r.count, "nodes": r.nodes, "internal": r.internal_nodes,
                "dead_ends": r.dead_ends, "hash": r.hash, "max_size": r.max_size, "hist": hist,
                "kernel_ms": r.kernel_ms, "total_ms": r.total_ms}


    def enumerate_stream(self, sink, opts: Options | None = None, raise_on_error: bool = True) -> dict:
        """mce_enumerate_stream: every maximal clique handed to sink(ids,
        off, count) in chunks (numpy copies: clique i is ids[off[i]:off[i+1]],
        original labels); a truthy return from sink stops the stream."""
        def _cb(ids_p, off_p, count, _user):
            off = np.ctypeslib.as_array(off_p, shape=(count + 1,)).copy()
            nid = int(off[-1])
            ids = np.ctypeslib.as_array(ids_p, shape=(nid,)).copy() if nid else np.zeros(0, dtype=np.uint32)
            return 1 if sink(ids, off, int(count)) else 0
        cb = CliqueSink(_cb)
        hist = np.zeros(self.n + 1, dtype=np.uint64)
        r = Result()
        r.hist = hist.ctypes.data_as(C.POINTER(C.c_uint64))
        r.hist_cap = hist.size
        rc = lib().mce_enumerate_stream(self.handle, _opt(opts), C.cast(cb, C.c_void_p), None, C.byref(r))
        if raise_on_error:
            _check(rc, "mce_enumerate_stream")
        return {"rc": rc, "count": r.count, "nodes": r.nodes, "internal": r.internal_nodes,
                "dead_ends": r.dead_ends, "hash": r.hash, "max_size": r.max_size, "hist": hist,
                "kernel_ms": r.kernel_ms, "total_ms": r.total_ms}


def cliques(res: dict) -> list:
    """The listing of an enumerate() result as a list of label arrays."""
    off, ids = res["list_off"], res["list_ids"]
    return [ids[int(off[i]):int(off[i + 1])] for i in range(len(off) - 1)]


def _results_array(ns):
    res = (Result * max(len(ns), 1))()
    hists = []
    for i, n in enumerate(ns):
        h = np.zeros(n + 1, dtype=np.uint64)
        hists.append(h)
        res[i].hist = h.ctypes.data_as(C.POINTER(C.c_uint64))
        res[i].hist_cap = h.size
    return res, hists


def _result_dicts(res, hists):
    out = []
    for i, h in enumerate(hists):
        r = res[i]
        out.append({"status": int(C.c_int32(r.status).value), "count": r.count, "nodes": r.nodes,
                    "internal": r.internal_nodes, "dead_ends": r.dead_ends, "hash": r.hash,
                    "max_size": r.max_size, "hist": h, "kernel_ms": r.kernel_ms})
    return out


class Batch:
    """mce_batch: graphs planned once and captured into one CUDA graph."""

    def __init__(self, ctx: Context, graphs, opts: Options | None = None):
        self.handle = None
        self.ctx, self.graphs = ctx, list(graphs)
        arr = (C.c_void_p * max(len(self.graphs), 1))(*[g.handle for g in self.graphs])
        h = C.c_void_p()
        _check(lib().mce_batch_create(ctx.handle, arr, len(self.graphs), _opt(opts), C.byref(h)), "mce_batch_create")
        self.handle = h
        ctx._owned.add(self)
        self._res, self._hists = _results_array([g.n for g in self.graphs])

    def launch(self):
        _check(lib().mce_batch_launch(self.handle), "mce_batch_launch")

    def buckets(self) -> list:
        """mce_batch_buckets: the launch choice of every bucket."""
        n = C.c_uint32(0)
        _check(lib().mce_batch_buckets(self.handle, None, 0, C.byref(n)), "mce_batch_buckets")
        arr = (BatchBucket * max(n.value, 1))()
        _check(lib().mce_batch_buckets(self.handle, arr, n.value, C.byref(n)), "mce_batch_buckets")
        return [{f: getattr(arr[i], f) for f, _ in BatchBucket._fields_} for i in range(n.value)]

    def results(self, raise_on_error: bool = True):
        rc = lib().mce_batch_results(self.handle, self._res)
        if raise_on_error:
            _check(rc, "mce_batch_results")
        return _result_dicts(self._res, [h.copy() for h in self._hists])

    def run(self, raise_on_error: bool = True):
        self.launch()
        return self.results(raise_on_error)

    def close(self):
        if self.handle:
            if self.ctx.handle:
                lib().mce_batch_destroy(self.handle)
            self.handle = None

    __del__ = close


def enumerate_batch(ctx: Context, graphs, opts: Options | None = None):
    """mce_enumerate_batch: create, run and destroy a batch in one call."""
    graphs = list(graphs)
    arr = (C.c_void_p * max(len(graphs), 1))(*[g.handle for g in graphs])
    res, hists = _results_array([g.n for g in graphs])
    rc = lib().mce_enumerate_batch(ctx.handle, arr, len(graphs), _opt(opts), res)
    _check(rc, "mce_enumerate_batch")
    return _result_dicts(res, hists)
