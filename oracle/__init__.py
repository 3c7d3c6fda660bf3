"""CPU oracle for maximal clique enumeration -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, built
with gcc into ``liboracle.so`` next to it) and shares nothing with the CUDA
library: no code, headers, tables or helpers.

What each function follows in the paper:

* ``tomita``   -- Bron-Kerbosch with pivoting, Alg. 2 (Section 3.2), Tomita
  pivot argmax_{u in P u X} |P n N(u)|; defines the set of maximal cliques.
* ``ordered``  -- the paper's search tree: maximum-degree-first ordering and
  renumbering (Section 4.2), BKPivotOrdered / ChoosePivotOrdered (Alg. 4)
  with the GreedyBB, GreedyBBTX or TomitaBB pivot (Section 4.3).
* ``mdf_order`` -- the maximum-degree-first ordering alone (Section 4.2).
* ``root_children`` / ``ordered_part`` -- the root's children of Alg. 4 as
  independent subtrees (the decomposition Alg. 3 makes over vertices,
  Section 3.3): the candidate-set size of every child, and the search of a
  chosen set of children.
* ``clique_hash`` / ``mix64`` -- the order-independent clique hash of the
  library's output contract (not in the paper; SplitMix64 finaliser).

Every function is pinned by tests against brute force, closed forms and the
Section 5 example, never against the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MODES = {"greedy": 0, "tx": 1, "tomita": 2, "nx": 3}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        u32p = C.POINTER(C.c_uint32)
        u64p = C.POINTER(C.c_uint64)
        i32p = C.POINTER(C.c_int32)
        lib.oracle_mix64.restype = C.c_uint64
        lib.oracle_mix64.argtypes = [C.c_uint64]
        lib.oracle_clique_hash.restype = C.c_uint64
        lib.oracle_clique_hash.argtypes = [u32p, C.c_uint32]
        lib.oracle_mdf_order.restype = None
        lib.oracle_mdf_order.argtypes = [C.c_uint32, u32p, u32p, u32p]
        lib.oracle_tomita.restype = C.c_int
        lib.oracle_tomita.argtypes = [C.c_uint32, u32p, u32p, u64p, u64p, u32p, C.c_uint64, u64p, C.c_uint64]
        lib.oracle_ordered.restype = C.c_int
        lib.oracle_ordered.argtypes = [C.c_uint32, u32p, u32p, C.c_int, u32p, u32p, u64p, u64p,
                                       u32p, C.c_uint64, u64p, i32p, C.c_uint64, u64p]
        lib.oracle_root_children.restype = C.c_int
        lib.oracle_root_children.argtypes = [C.c_uint32, u32p, u32p, C.c_int, u32p, u32p, C.c_uint32, u32p]
        lib.oracle_ordered_part.restype = C.c_int
        lib.oracle_ordered_part.argtypes = [C.c_uint32, u32p, u32p, C.c_int, u32p, C.POINTER(C.c_ubyte),
                                            C.c_uint32, C.c_int, u64p, u64p]
        lib.oracle_degeneracy_order.restype = None
        lib.oracle_degeneracy_order.argtypes = [C.c_uint32, u32p, u32p, u32p]
        lib.oracle_outer.restype = C.c_int
        lib.oracle_outer.argtypes = [C.c_uint32, u32p, u32p, C.c_int, u32p, u64p, u64p, u32p, C.c_uint64, u64p]
        _lib = lib
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(C.POINTER(t))


def csr(n: int, uv: np.ndarray):
    """Sorted symmetric CSR (off, adj) from an edge array (duplicates and
    both orientations allowed, self-loops rejected)."""
    uv = np.asarray(uv, dtype=np.int64).reshape(-1, 2)
    if uv.size and (uv.min() < 0 or uv.max() >= n):
        raise ValueError("vertex id out of range")
    if np.any(uv[:, 0] == uv[:, 1]):
        raise ValueError("self-loop")
    a = np.concatenate([uv[:, 0], uv[:, 1]])
    b = np.concatenate([uv[:, 1], uv[:, 0]])
    key = np.unique(a * max(n, 1) + b)
    src = key // max(n, 1)
    dst = (key % max(n, 1)).astype(np.uint32)
    off = np.zeros(n + 1, dtype=np.uint32)
    if n:
        np.add.at(off, src + 1, 1)
        off = np.cumsum(off, dtype=np.uint64).astype(np.uint32)
    return np.ascontiguousarray(off), np.ascontiguousarray(dst)


def _unpack_listing(buf: np.ndarray, used: int):
    out, i = [], 0
    while i < used:
        k = int(buf[i])
        out.append(tuple(int(x) for x in buf[i + 1:i + 1 + k]))
        i += k + 1
    out.sort()
    return out


def _result(stats, hist, n):
    return {"count": int(stats[0]), "nodes": int(stats[1]), "internal": int(stats[2]),
            "dead_ends": int(stats[3]), "hash": int(stats[4]), "hist": hist.copy()}


def tomita(n: int, uv, listing: bool = False, list_cap: int = 1 << 22, max_nodes: int = 0):
    """Maximal cliques by Alg. 2 with the Tomita pivot.  ``max_nodes`` > 0
    stops after that many search nodes (result flagged ``partial``)."""
    lib = _load()
    off, adj = csr(n, uv)
    stats = np.zeros(5, dtype=np.uint64)
    hist = np.zeros(n + 1, dtype=np.uint64)
    lst = np.zeros(list_cap if listing else 1, dtype=np.uint32)
    used = np.zeros(1, dtype=np.uint64)
    rc = lib.oracle_tomita(n, _p(off, C.c_uint32), _p(adj if adj.size else np.zeros(1, np.uint32), C.c_uint32),
                           _p(stats, C.c_uint64), _p(hist, C.c_uint64),
                           _p(lst, C.c_uint32) if listing else None, lst.size, _p(used, C.c_uint64), max_nodes)
    if rc < 0:
        raise MemoryError("oracle ran out of memory")
    res = _result(stats, hist, n)
    res["partial"] = rc == 1
    if listing:
        if int(used[0]) > lst.size:
            return tomita(n, uv, True, int(used[0]) + 16, max_nodes)
        res["listing"] = _unpack_listing(lst, int(used[0]))
    return res


def ordered(n: int, uv, mode: str = "greedy", order=None, listing: bool = False,
            list_cap: int = 1 << 22, trace_cap: int = 0):
    """The paper's ordered search (Alg. 4) with the given pivot rule.

    ``order`` fixes the vertex order (order[i] = vertex at position i);
    None computes the maximum-degree-first order of Section 4.2.
    Returns the result dict plus ``order`` and, when ``trace_cap`` > 0, the
    first internal nodes as (depth, pivot, L) tuples in original labels.
    """
    lib = _load()
    off, adj = csr(n, uv)
    stats = np.zeros(5, dtype=np.uint64)
    hist = np.zeros(n + 1, dtype=np.uint64)
    lst = np.zeros(list_cap if listing else 1, dtype=np.uint32)
    used = np.zeros(1, dtype=np.uint64)
    ordv = None if order is None else np.ascontiguousarray(order, dtype=np.uint32)
    oout = np.zeros(max(n, 1), dtype=np.uint32)
    trace = np.zeros(max(trace_cap, 1), dtype=np.int32)
    tused = np.zeros(1, dtype=np.uint64)
    rc = lib.oracle_ordered(n, _p(off, C.c_uint32), _p(adj if adj.size else np.zeros(1, np.uint32), C.c_uint32),
                            MODES[mode], _p(ordv, C.c_uint32), _p(oout, C.c_uint32),
                            _p(stats, C.c_uint64), _p(hist, C.c_uint64),
                            _p(lst, C.c_uint32) if listing else None, lst.size, _p(used, C.c_uint64),
                            _p(trace, C.c_int32) if trace_cap else None, trace_cap, _p(tused, C.c_uint64))
    if rc:
        raise MemoryError("oracle ran out of memory")
    res = _result(stats, hist, n)
    res["order"] = oout[:n].copy()
    if listing:
        if int(used[0]) > lst.size:
            return ordered(n, uv, mode, order, True, int(used[0]) + 16, trace_cap)
        res["listing"] = _unpack_listing(lst, int(used[0]))
    if trace_cap:
        recs, i, u = [], 0, int(tused[0])
        while i < u:
            d, p, k = int(trace[i]), int(trace[i + 1]), int(trace[i + 2])
            recs.append((d, p, tuple(int(x) for x in trace[i + 3:i + 3 + k])))
            i += 3 + k
        res["trace"] = recs
    return res


def root_children(n: int, uv, mode: str = "greedy", order=None) -> np.ndarray:
    """Candidate-set sizes |P_t| of the root's children t = 0, 1, ... of
    Alg. 4 (the root's branching set in order)."""
    lib = _load()
    off, adj = csr(n, uv)
    sizes = np.zeros(max(n, 1), dtype=np.uint32)
    cnt = np.zeros(1, dtype=np.uint32)
    ordv = None if order is None else np.ascontiguousarray(order, dtype=np.uint32)
    rc = lib.oracle_root_children(n, _p(off, C.c_uint32), _p(adj if adj.size else np.zeros(1, np.uint32), C.c_uint32),
                                  MODES[mode], _p(ordv, C.c_uint32), _p(sizes, C.c_uint32), sizes.size,
                                  _p(cnt, C.c_uint32))
    if rc:
        raise MemoryError("oracle ran out of memory")
    return sizes[:int(cnt[0])].copy()


def ordered_part(n: int, uv, mode: str, children, count_root: bool, order=None):
    """Alg. 4 searching only the root children listed in ``children``
    (indices into the root's branching set); the root node is counted only
    when ``count_root``."""
    lib = _load()
    off, adj = csr(n, uv)
    sel = np.zeros(max(n, 1), dtype=np.uint8)
    for t in children:
        sel[int(t)] = 1
    stats = np.zeros(5, dtype=np.uint64)
    hist = np.zeros(n + 1, dtype=np.uint64)
    ordv = None if order is None else np.ascontiguousarray(order, dtype=np.uint32)
    rc = lib.oracle_ordered_part(n, _p(off, C.c_uint32), _p(adj if adj.size else np.zeros(1, np.uint32), C.c_uint32),
                                 MODES[mode], _p(ordv, C.c_uint32), _p(sel, C.c_ubyte), sel.size,
                                 1 if count_root else 0, _p(stats, C.c_uint64), _p(hist, C.c_uint64))
    if rc:
        raise MemoryError("oracle ran out of memory")
    return _result(stats, hist, n)


def mdf_order(n: int, uv) -> np.ndarray:
    """Maximum-degree-first order (Section 4.2), ties to the smallest label."""
    lib = _load()
    off, adj = csr(n, uv)
    out = np.zeros(max(n, 1), dtype=np.uint32)
    lib.oracle_mdf_order(n, _p(off, C.c_uint32), _p(adj if adj.size else np.zeros(1, np.uint32), C.c_uint32),
                         _p(out, C.c_uint32))
    return out[:n].copy()


def mix64(z: int) -> int:
    return int(_load().oracle_mix64(z & 0xFFFFFFFFFFFFFFFF))


def clique_hash(labels) -> int:
    a = np.ascontiguousarray(np.asarray(labels, dtype=np.uint32).reshape(-1))
    return int(_load().oracle_clique_hash(_p(a if a.size else np.zeros(1, np.uint32), C.c_uint32), a.size))


def degeneracy_order(n: int, uv) -> np.ndarray:
    """Alg. 3's outer order: minimum remaining degree first, smallest label
    on ties."""
    off, adj = csr(n, uv)
    out = np.zeros(max(n, 1), dtype=np.uint32)
    _load().oracle_degeneracy_order(n, _p(off, C.c_uint32), _p(adj if adj.size else np.zeros(1, np.uint32), C.c_uint32),
                                    _p(out, C.c_uint32))
    return out[:n]


def outer(n: int, uv, mode: str = "greedy", listing: bool = False, list_cap: int = 1 << 22):
    """Alg. 3: for every vertex v in degeneracy order, the ordered search
    (Alg. 4, pivot rule ``mode``) on G[{v} u N(v)] from R = {v}, P = later
    neighbours, X = earlier neighbours.  Returns the result dict plus the
    outer ``order``."""
    lib = _load()
    off, adj = csr(n, uv)
    stats = np.zeros(5, dtype=np.uint64)
    hist = np.zeros(n + 1, dtype=np.uint64)
    lst = np.zeros(list_cap if listing else 1, dtype=np.uint32)
    used = np.zeros(1, dtype=np.uint64)
    oout = np.zeros(max(n, 1), dtype=np.uint32)
    rc = lib.oracle_outer(n, _p(off, C.c_uint32), _p(adj if adj.size else np.zeros(1, np.uint32), C.c_uint32),
                          MODES[mode], _p(oout, C.c_uint32), _p(stats, C.c_uint64), _p(hist, C.c_uint64),
                          _p(lst, C.c_uint32) if listing else None, lst.size, _p(used, C.c_uint64))
    if rc < 0:
        raise MemoryError("oracle ran out of memory")
    if listing and int(used[0]) > lst.size:
        return outer(n, uv, mode, True, int(used[0]) + 16)
    res = _result(stats, hist, n)
    res["order"] = oout[:n].copy()
    if listing:
        res["listing"] = _unpack_listing(lst, int(used[0]))
    return res

