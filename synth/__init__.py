"""Seeded synthetic inputs for maximal clique enumeration.

This module only *builds graphs*.  It holds none of the enumeration
arithmetic: no ordering, no pivoting, no clique hash.  Both the CPU oracle
(tests) and the CUDA path (library, bench) take their inputs from here, so the
two never share code beyond these generators.

Graphs are simple and undirected on V = {0, ..., n-1} (the paper numbers
vertices from 1, Section 2; the library is 0-based).  A graph is returned as
an edge array ``uv`` of shape (m, 2), dtype uint32, each unordered pair once
with u < v, sorted row-major.

Random stream
-------------
Every random draw comes from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): the state advances
by the golden-ratio increment 0x9E3779B97F4A7C15 and each output is the
state passed through the 64-bit finaliser.  The k-th output (k = 0, 1, ...)
of a stream seeded with s is therefore finalise(s + (k + 1) * increment),
which lets numpy draw a whole block at once.

Workload families (the paper's Table 1 uses uniform random graphs G(n, p);
its instances are not available, so seeded G(n, p) stands in for them):

* ``gnp(n, p, seed)``: pair (i, j), i < j, visited in row-major upper
  triangle order, is an edge iff (next() >> 11) * 2**-53 < p.
* ``moon_moser(k)``: complement of k disjoint triangles (n = 3k), the graph
  that attains the 3^(n/3) bound cited in the paper's introduction.
* ``moon_moser_deleted(k, frac, seed)``: the same with round(frac * m) edges
  removed, chosen uniformly without replacement by a partial Fisher-Yates
  shuffle driven by the seed's stream.
* ``batch_graph(s)`` / ``served_graph`` / ``served_requests``: the multi-graph
  workloads (one stream per graph, so any graph can be built alone), with
  (n, p) redrawn while the expected number of maximal cliques exceeds a cap.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import gammaln

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO53 = float(2 ** 53)


def _finalise(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


class SplitMix64:
    """Sequential SplitMix64 stream; ``block(k)`` draws k outputs at once."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def block(self, k: int) -> np.ndarray:
        steps = np.arange(1, k + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            states = self.state + steps * GOLDEN
            self.state = self.state + np.uint64(k) * GOLDEN
        return _finalise(states)

    def next(self) -> int:
        return int(self.block(1)[0])

    def uniform(self) -> float:
        """(next() >> 11) * 2**-53, a double in [0, 1)."""
        return float(self.next() >> 11) / _TWO53

    def uniform_block(self, k: int) -> np.ndarray:
        return (self.block(k) >> np.uint64(11)).astype(np.float64) / _TWO53


def _upper_pairs(n: int) -> tuple[np.ndarray, np.ndarray]:
    iu, ju = np.triu_indices(n, k=1)
    return iu.astype(np.uint32), ju.astype(np.uint32)


def gnp_from_stream(n: int, p: float, rng: SplitMix64) -> np.ndarray:
    """G(n, p) edges drawn from an existing stream (row-major upper triangle)."""
    if n < 2:
        return np.zeros((0, 2), dtype=np.uint32)
    iu, ju = _upper_pairs(n)
    keep = rng.uniform_block(iu.size) < p
    return np.stack([iu[keep], ju[keep]], axis=1)


def gnp(n: int, p: float, seed: int) -> np.ndarray:
    """Erdos-Renyi G(n, p) with the SplitMix64 stream seeded by ``seed``."""
    return gnp_from_stream(n, p, SplitMix64(seed))


def moon_moser(k: int) -> np.ndarray:
    """Complement of k disjoint triangles on n = 3k vertices."""
    n = 3 * k
    iu, ju = _upper_pairs(n)
    keep = (iu // 3) != (ju // 3)
    return np.stack([iu[keep], ju[keep]], axis=1)


def moon_moser_deleted(k: int, frac: float, seed: int) -> np.ndarray:
    """``moon_moser(k)`` with round(frac * m) edges removed uniformly.

    Partial Fisher-Yates over the row-major edge list: for t = 0, 1, ...,
    d - 1 swap slot t with slot t + (next() mod (m - t)); the first d slots
    are deleted.
    """
    uv = moon_moser(k)
    m = uv.shape[0]
    d = int(round(frac * m))
    rng = SplitMix64(seed)
    idx = np.arange(m)
    for t in range(d):
        j = t + int(rng.next() % (m - t))
        idx[t], idx[j] = idx[j], idx[t]
    keep = np.ones(m, dtype=bool)
    keep[idx[:d]] = False
    return uv[keep]


# ----------------------------------------------------------------------------
# Deterministic structured families (closed forms are pinned in tests).

def complete(n: int) -> np.ndarray:
    iu, ju = _upper_pairs(n)
    return np.stack([iu, ju], axis=1)


def empty(n: int) -> np.ndarray:
    return np.zeros((0, 2), dtype=np.uint32)


def cycle(n: int) -> np.ndarray:
    u = np.arange(n, dtype=np.uint32)
    v = (u + 1) % n
    uv = np.stack([np.minimum(u, v), np.maximum(u, v)], axis=1)
    return canonical(uv)


def complete_multipartite(sizes) -> np.ndarray:
    part = np.repeat(np.arange(len(sizes)), sizes)
    n = int(part.size)
    iu, ju = _upper_pairs(n)
    keep = part[iu] != part[ju]
    return np.stack([iu[keep], ju[keep]], axis=1)


def disjoint_union(uv1: np.ndarray, n1: int, uv2: np.ndarray) -> np.ndarray:
    """G + H with H's vertices shifted by n1."""
    return canonical(np.concatenate([uv1, uv2 + np.uint32(n1)], axis=0))


def join(uv1: np.ndarray, n1: int, uv2: np.ndarray, n2: int) -> np.ndarray:
    """G v H: disjoint union plus every edge between the two vertex sets."""
    a = np.repeat(np.arange(n1, dtype=np.uint32), n2)
    b = np.tile(np.arange(n1, n1 + n2, dtype=np.uint32), n1)
    cross = np.stack([a, b], axis=1)
    return canonical(np.concatenate([uv1, uv2 + np.uint32(n1), cross], axis=0))


def relabel(uv: np.ndarray, perm: np.ndarray) -> np.ndarray:
    """Vertex v becomes perm[v]."""
    p = np.asarray(perm, dtype=np.uint32)
    return canonical(p[uv])


def canonical(uv: np.ndarray) -> np.ndarray:
    """Each pair once as (min, max), sorted row-major, self-loops dropped."""
    uv = np.asarray(uv, dtype=np.uint32).reshape(-1, 2)
    a = np.minimum(uv[:, 0], uv[:, 1])
    b = np.maximum(uv[:, 0], uv[:, 1])
    keep = a != b
    key = np.unique(a[keep].astype(np.uint64) << np.uint64(32) | b[keep].astype(np.uint64))
    return np.stack([(key >> np.uint64(32)).astype(np.uint32),
                     (key & np.uint64(0xFFFFFFFF)).astype(np.uint32)], axis=1)


def random_order(n: int, seed: int) -> np.ndarray:
    """A seeded permutation of 0..n-1 (Fisher-Yates on the seed's stream)."""
    rng = SplitMix64(seed)
    perm = np.arange(n, dtype=np.uint32)
    for i in range(n - 1, 0, -1):
        j = int(rng.next() % (i + 1))
        perm[i], perm[j] = perm[j], perm[i]
    return perm


# ----------------------------------------------------------------------------
# Bitset layout used at the library boundary.

def words_per_row(n: int) -> int:
    return (n + 31) // 32


def to_bitset(n: int, uv: np.ndarray, words: int | None = None) -> np.ndarray:
    """Symmetric bitset adjacency, shape (n, words) uint32, bit j of row i =
    word j // 32, bit j % 32; diagonal and padding bits zero."""
    w = words_per_row(n) if words is None else words
    rows = np.zeros((n, w), dtype=np.uint32)
    if uv.size:
        u = uv[:, 0].astype(np.int64)
        v = uv[:, 1].astype(np.int64)
        for a, b in ((u, v), (v, u)):
            np.bitwise_or.at(rows, (a, b // 32), (np.uint32(1) << (b % 32).astype(np.uint32)))
    return rows


# ----------------------------------------------------------------------------
# Multi-graph workloads.

def expected_maximal_cliques(n: int, p: float) -> float:
    """E[mu(G(n, p))] = sum_k C(n, k) p^C(k, 2) (1 - p^k)^(n - k).

    Used only to cap the size of generated workloads (a cliquer's textbook
    expectation, not part of the enumeration method).
    """
    if n == 0:
        return 1.0
    if p <= 0.0:
        return float(n)
    k = np.arange(1, n + 1, dtype=np.float64)
    lc = gammaln(n + 1.0) - gammaln(k + 1.0) - gammaln(n - k + 1.0)
    with np.errstate(divide="ignore"):
        lp = (k * (k - 1) / 2.0) * math.log(p) if p < 1.0 else np.zeros_like(k)
        pk = np.power(p, k)
        lq = (n - k) * np.log1p(-pk) if p < 1.0 else np.where(k == n, 0.0, -np.inf)
    terms = lc + lp + lq
    mx = np.max(terms)
    return float(math.exp(mx) * np.sum(np.exp(terms - mx)))


@dataclass
class GraphSpec:
    index: int
    seed: int
    n: int
    p: float
    draws: int          # how many (n, p) draws it took (1 = accepted first time)
    uv: np.ndarray


def _capped_params(rng: SplitMix64, draw, cap: float):
    draws = 0
    while True:
        draws += 1
        n, p = draw(rng)
        if expected_maximal_cliques(n, p) <= cap:
            return n, p, draws


def batch_graph(i: int, cap: float = 1e6, first_seed: int = 0,
                n_lo: int = 32, n_hi: int = 512, p_lo: float = 0.2, p_hi: float = 0.8) -> GraphSpec:
    """Graph i of the batched workload, from its own stream seeded first_seed + i:
    n = n_lo + (next() mod (n_hi - n_lo + 1)), p = p_lo + (p_hi - p_lo) * u,
    redrawn from the same stream while E[mu](n, p) > cap; the edges follow on
    the same stream."""
    def draw(rng):
        n = n_lo + int(rng.next() % (n_hi - n_lo + 1))
        p = p_lo + (p_hi - p_lo) * rng.uniform()
        return n, p

    seed = first_seed + i
    rng = SplitMix64(seed)
    n, p, draws = _capped_params(rng, draw, cap)
    return GraphSpec(i, seed, n, p, draws, gnp_from_stream(n, p, rng))


def batch_graphs(count: int = 4096, cap: float = 1e6, first_seed: int = 0, **kw):
    """The batched workload: graphs 0 .. count-1 of ``batch_graph``."""
    return [batch_graph(i, cap, first_seed, **kw) for i in range(count)]


@dataclass
class Request:
    index: int
    arrival_s: float
    spec: GraphSpec


def served_arrivals(count: int, rate_per_s: float, seed: int = 5) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps of
    mean 1 / rate_per_s drawn from the stream seeded ``seed``."""
    arrivals = SplitMix64(seed)
    gaps = -np.log1p(-arrivals.uniform_block(count)) / rate_per_s
    return np.cumsum(gaps)


def served_graph(r: int, cap: float = 1e6, seed: int = 5,
                 n_lo: int = 64, n_hi: int = 2048, p_lo: float = 0.1, p_hi: float = 0.9) -> GraphSpec:
    """Request r's graph, from the stream seeded (seed << 32) + r:
    n = round(exp(U[ln n_lo, ln n_hi])), p ~ U[p_lo, p_hi], capped like
    ``batch_graph``."""
    lo, hi = math.log(n_lo), math.log(n_hi)

    def draw(rng):
        n = int(round(math.exp(lo + (hi - lo) * rng.uniform())))
        p = p_lo + (p_hi - p_lo) * rng.uniform()
        return n, p

    s = (seed << 32) + r
    rng = SplitMix64(s)
    n, p, draws = _capped_params(rng, draw, cap)
    return GraphSpec(r, s, n, p, draws, gnp_from_stream(n, p, rng))


def served_requests(count: int, rate_per_s: float, cap: float = 1e6, seed: int = 5, **kw):
    """Served workload: Poisson arrivals (``served_arrivals``) of the
    requests ``served_graph`` draws."""
    t = served_arrivals(count, rate_per_s, seed)
    return [Request(r, float(t[r]), served_graph(r, cap, seed, **kw)) for r in range(count)]
