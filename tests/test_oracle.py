"""Pins for the CPU oracle (``-m "not gpu"``).

The oracle is checked against things fixed by the paper or by mathematics,
never against itself or the CUDA path:

* brute-force subset enumeration (every graph on n <= 5, random graphs up to
  n = 20): count, histogram, listing and hash;
* closed forms: Moon-Moser 3^k, complete multipartite prod s_i, C_n -> n,
  K_n -> 1, empty -> n, n = 0 -> {{}}, disjoint union and join;
* per-clique checks (clique, maximal, unique) and invariants (relabelling);
* the Section 5 example (pivot and branching set at the node under 9);
* the paper's Table 1 mu values as a statistical check;
* exact search-tree sizes of Alg. 4 on graphs where the tree can be worked
  out by hand (K_n, empty graph, Moon-Moser).
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MASK = (1 << 64) - 1


# --- an independent statement of the output contract, for the tests only --

def _mix64(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def _h(clique) -> int:
    s = sum(_mix64(c + 1) for c in clique) & MASK
    return _mix64(s ^ _mix64(len(clique)))


def brute_force(n: int, uv: np.ndarray):
    """All maximal cliques by checking every vertex subset (n <= 20)."""
    assert n <= 20
    nb = [0] * n
    for a, b in np.asarray(uv, dtype=np.int64).reshape(-1, 2):
        nb[a] |= 1 << int(b)
        nb[b] |= 1 << int(a)
    S = np.arange(1 << n, dtype=np.int64)
    clique = np.ones(S.size, dtype=bool)
    for v in range(n):
        inS = ((S >> v) & 1).astype(bool)
        clique &= ~(inS & ((S & ~(nb[v] | (1 << v))) != 0))
    maximal = clique.copy()
    for u in range(n):
        outside = ((S >> u) & 1) == 0
        maximal &= ~(outside & ((S & ~nb[u]) == 0))
    out = []
    for s in S[maximal]:
        out.append(tuple(v for v in range(n) if (int(s) >> v) & 1))
    return sorted(out)


def summary(cliques, n):
    hist = np.zeros(n + 1, dtype=np.uint64)
    h = 0
    for c in cliques:
        hist[len(c)] += 1
        h = (h + _h(c)) & MASK
    return len(cliques), hist, h


def check_all_against(n, uv, cliques):
    cnt, hist, h = summary(cliques, n)
    for res in (oracle.tomita(n, uv, listing=True),
                oracle.ordered(n, uv, "greedy", listing=True),
                oracle.ordered(n, uv, "tx", listing=True),
                oracle.ordered(n, uv, "tomita", listing=True),
                oracle.ordered(n, uv, "nx", listing=True)):
        assert res["count"] == cnt
        assert np.array_equal(res["hist"], hist)
        assert res["hash"] == h
        assert res["listing"] == cliques
        assert res["nodes"] == res["count"] + res["internal"] + res["dead_ends"]


# --- hash primitive ---------------------------------------------------------

def test_mix64_published_vectors():
    """The finaliser reproduces SplitMix64's published reference outputs."""
    with open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) as f:
        rows = [list(map(int, l.split())) for l in f if l.strip() and not l.startswith("#")]
    for seed, *outs in rows:
        state = seed
        for o in outs:
            state = (state + 0x9E3779B97F4A7C15) & MASK
            assert oracle.mix64(state) == o
            assert _mix64(state) == o


def test_clique_hash_is_a_set_function():
    rng = np.random.default_rng(0)
    for k in range(0, 12):
        c = rng.choice(1000, size=k, replace=False)
        assert oracle.clique_hash(c) == oracle.clique_hash(np.sort(c)) == _h(sorted(c.tolist()))


# --- brute force ------------------------------------------------------------

def test_every_graph_up_to_five_vertices():
    for n in range(0, 6):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            uv = np.array([pairs[i] for i in range(len(pairs)) if (mask >> i) & 1],
                          dtype=np.uint32).reshape(-1, 2)
            check_all_against(n, uv, brute_force(n, uv) if n else [()])


@pytest.mark.parametrize("n,p,seed", [(8, 0.5, 1), (12, 0.3, 2), (12, 0.7, 3), (16, 0.5, 4),
                                      (18, 0.8, 5), (20, 0.5, 6), (20, 0.25, 7), (20, 0.9, 8)])
def test_random_against_brute_force(n, p, seed):
    uv = synth.gnp(n, p, seed)
    check_all_against(n, uv, brute_force(n, uv))


# --- closed forms -----------------------------------------------------------

@pytest.mark.parametrize("k", range(1, 9))
def test_moon_moser(k):
    n = 3 * k
    for mode in ("greedy", "tx", "tomita", "nx"):
        r = oracle.ordered(n, synth.moon_moser(k), mode)
        assert r["count"] == 3 ** k
        assert r["hist"][k] == 3 ** k and r["hist"].sum() == 3 ** k
    r = oracle.tomita(n, synth.moon_moser(k))
    assert r["count"] == 3 ** k


@pytest.mark.parametrize("sizes", [(1,), (2, 3), (2, 3, 4), (3, 3, 3), (1, 5, 2, 4), (6, 1, 1, 2, 3)])
def test_complete_multipartite(sizes):
    n = sum(sizes)
    uv = synth.complete_multipartite(sizes)
    want = math.prod(sizes)
    for r in (oracle.tomita(n, uv), oracle.ordered(n, uv)):
        assert r["count"] == want
        assert r["hist"][len(sizes)] == want


@pytest.mark.parametrize("n", [4, 5, 7, 30, 101])
def test_cycle(n):
    r = oracle.tomita(n, synth.cycle(n))
    assert r["count"] == n and r["hist"][2] == n
    assert oracle.ordered(n, synth.cycle(n))["count"] == n


@pytest.mark.parametrize("n", [1, 2, 3, 10, 64, 200])
def test_complete_and_empty(n):
    rk = oracle.ordered(n, synth.complete(n))
    assert rk["count"] == 1 and rk["hist"][n] == 1
    assert rk["hash"] == _h(list(range(n)))
    re_ = oracle.ordered(n, synth.empty(n))
    assert re_["count"] == n and re_["hist"][1] == n
    assert re_["hash"] == sum(_h([v]) for v in range(n)) & MASK
    assert oracle.tomita(n, synth.complete(n))["count"] == 1
    assert oracle.tomita(n, synth.empty(n))["count"] == n


def test_zero_vertices():
    for r in (oracle.tomita(0, synth.empty(0)), oracle.ordered(0, synth.empty(0))):
        assert r["count"] == 1 and r["hist"][0] == 1 and r["hash"] == _h([])
        assert r["nodes"] == 1


def test_disjoint_union_adds():
    n1, n2 = 40, 35
    g, h = synth.gnp(n1, 0.4, 11), synth.gnp(n2, 0.5, 12)
    rg, rh = oracle.tomita(n1, g, listing=True), oracle.tomita(n2, h, listing=True)
    ru = oracle.tomita(n1 + n2, synth.disjoint_union(g, n1, h))
    assert ru["count"] == rg["count"] + rh["count"]
    hh = np.zeros(n1 + n2 + 1, dtype=np.uint64)
    hh[:n1 + 1] += rg["hist"]
    hh[:n2 + 1] += rh["hist"]
    assert np.array_equal(ru["hist"], hh)
    shifted = sum(_h([c + n1 for c in k]) for k in rh["listing"]) & MASK
    assert ru["hash"] == (rg["hash"] + shifted) & MASK


def test_join_multiplies():
    n1, n2 = 25, 20
    g, h = synth.gnp(n1, 0.5, 13), synth.gnp(n2, 0.3, 14)
    rg, rh = oracle.tomita(n1, g), oracle.tomita(n2, h)
    rj = oracle.ordered(n1 + n2, synth.join(g, n1, h, n2))
    assert rj["count"] == rg["count"] * rh["count"]
    conv = np.convolve(rg["hist"].astype(np.int64), rh["hist"].astype(np.int64))
    assert np.array_equal(rj["hist"][:conv.size].astype(np.int64), conv)


# --- per-clique checks and invariants --------------------------------------

@pytest.mark.parametrize("n,p,seed", [(60, 0.5, 21), (90, 0.3, 22), (45, 0.8, 23)])
def test_listing_is_maximal_unique(n, p, seed):
    uv = synth.gnp(n, p, seed)
    off, adj = oracle.csr(n, uv)
    nbrs = [set(adj[off[v]:off[v + 1]].tolist()) for v in range(n)]
    r = oracle.ordered(n, uv, listing=True)
    L = r["listing"]
    assert len(L) == r["count"] == len(set(L)) == int(r["hist"].sum())
    for K in L:
        for a, b in itertools.combinations(K, 2):
            assert b in nbrs[a]
        common = set(range(n)).difference(K)
        for c in K:
            common &= nbrs[c]
        assert not common, "clique is not maximal"
    assert r["hash"] == sum(_h(K) for K in L) & MASK


def test_relabelling_invariance():
    n = 70
    uv = synth.gnp(n, 0.45, 31)
    perm = synth.random_order(n, 32)
    a = oracle.tomita(n, uv, listing=True)
    b = oracle.ordered(n, synth.relabel(uv, perm), listing=True)
    assert a["count"] == b["count"] and np.array_equal(a["hist"], b["hist"])
    mapped = sorted(tuple(sorted(int(perm[c]) for c in K)) for K in a["listing"])
    assert mapped == b["listing"]


def test_moon_moser_bound_on_random_graphs():
    for seed in range(12):
        n = 18
        uv = synth.gnp(n, 0.3 + 0.05 * seed, 40 + seed)
        assert oracle.ordered(n, uv)["count"] <= 3 ** (n // 3)


def test_moon_moser_deleted_below_bound():
    uv = synth.moon_moser_deleted(6, 0.05, 3)
    r = oracle.ordered(18, uv, listing=True)
    assert r["count"] < 3 ** 6
    assert r["listing"] == brute_force(18, uv)


# --- ordering (Section 4.2) -------------------------------------------------

def test_mdf_order_hand_worked_path():
    # path 0-1-2-3-4: degrees 1,2,2,2,1 -> 1 (smallest label among degree 2);
    # then 3 has degree 2 in {0,2,3,4}; then all remaining have degree 0.
    uv = np.array([[0, 1], [1, 2], [2, 3], [3, 4]], dtype=np.uint32)
    assert oracle.mdf_order(5, uv).tolist() == [1, 3, 0, 2, 4]


@pytest.mark.parametrize("n,p,seed", [(50, 0.3, 51), (120, 0.5, 52), (200, 0.1, 53)])
def test_mdf_order_property(n, p, seed):
    """Each v_i has maximum degree in the graph induced by v_i..v_n, and the
    smallest label among the vertices that share that degree."""
    uv = synth.gnp(n, p, seed)
    order = oracle.mdf_order(n, uv).tolist()
    assert sorted(order) == list(range(n))
    A = synth.to_bitset(n, uv)
    dense = np.unpackbits(A.view(np.uint8), bitorder="little").reshape(n, -1)[:, :n].astype(bool)
    remaining = np.ones(n, dtype=bool)
    for v in order:
        deg = (dense & remaining[None, :]).sum(axis=1)
        deg[~remaining] = -1
        best = deg.max()
        assert deg[v] == best and v == int(np.flatnonzero(deg == best)[0])
        remaining[v] = False


# --- the Section 5 example --------------------------------------------------

def _example():
    order, edges, cliques, expect = None, [], [], {}
    with open(os.path.join(GOLDEN, "section5_example.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "order":
                order = [int(x) for x in t[1:]]
            elif t[0] == "edge":
                edges.append((int(t[1]), int(t[2])))
            elif t[0] == "clique":
                cliques.append(tuple(int(x) for x in t[1:]))
            else:
                i = t.index(":")
                expect[t[0]] = (int(t[1]), tuple(int(x) for x in t[i + 1:]))
    return order, edges, cliques, expect


def test_section5_example():
    order, edges, cliques, expect = _example()
    labels = sorted(order)                       # paper labels -> 0..6
    idx = {v: i for i, v in enumerate(labels)}
    uv = np.array([[idx[a], idx[b]] for a, b in edges], dtype=np.uint32)
    n = len(labels)
    ordv = np.array([idx[v] for v in order], dtype=np.uint32)
    want = sorted(tuple(sorted(idx[c] for c in K)) for K in cliques)
    assert brute_force(n, uv) == want
    for mode in ("greedy", "tomita"):
        r = oracle.ordered(n, uv, mode, order=ordv, listing=True, trace_cap=256)
        assert r["listing"] == want
        # trace[0] is the root (R = {}); trace[1] is the node R = {9}
        depth, pivot, L = r["trace"][1]
        p_want, L_want = expect[mode]
        assert depth == 1
        assert labels[pivot] == p_want
        assert tuple(labels[v] for v in L) == L_want


def _tie_example():
    order, edges, cliques, expect = None, [], [], {}
    for line in open(os.path.join(GOLDEN, "tx_tie_example.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "order":
            order = [int(x) for x in t[1:]]
        elif t[0] == "edge":
            edges.append((int(t[1]), int(t[2])))
        elif t[0] == "clique":
            cliques.append(tuple(int(x) for x in t[1:]))
        else:
            i = t.index(":")
            expect[t[0]] = (int(t[1]), tuple(int(x) for x in t[i + 1:]))
    return order, edges, cliques, expect


def test_tx_tie_goes_to_the_earliest_vertex_of_x():
    # Section 4.3: two vertices of X tie on |P n N(u)| at the node R = {5} of
    # the hand-worked graph in tests/golden/tx_tie_example.txt; GreedyBBTX
    # and GreedyBBNX must both pivot on the earlier one (3, not 4).
    order, edges, cliques, expect = _tie_example()
    n = len(order)
    uv = np.array(edges, dtype=np.uint32)
    assert brute_force(n, uv) == sorted(cliques)
    for mode in ("tx", "nx", "greedy"):
        r = oracle.ordered(n, uv, mode, order=np.array(order, dtype=np.uint32), listing=True, trace_cap=256)
        assert r["listing"] == sorted(cliques)
        node = [(p, L) for d, p, L in r["trace"] if d == 1 and 5 not in L and p in (2, 3, 4)]
        assert node == [expect[mode]], (mode, r["trace"])


# --- exact search-tree sizes of Alg. 4 --------------------------------------

@pytest.mark.parametrize("n", [1, 2, 9, 100])
def test_tree_size_complete_graph(n):
    # pivot = first of P, L = {pivot}: a chain of n internal nodes, one leaf
    r = oracle.ordered(n, synth.complete(n))
    assert (r["nodes"], r["internal"], r["dead_ends"]) == (n + 1, n, 0)


@pytest.mark.parametrize("n", [1, 2, 9, 100])
def test_tree_size_empty_graph(n):
    # root pivots on vertex 0, L = V: n leaves with P = X = {}
    r = oracle.ordered(n, synth.empty(n))
    assert (r["nodes"], r["internal"], r["dead_ends"]) == (n + 1, 1, 0)


@pytest.mark.parametrize("k", range(1, 9))
def test_tree_size_moon_moser(k):
    # the first vertex's triangle forms L; each child is Moon-Moser on k-1
    # triangles with X empty: T(k) = 1 + 3 T(k-1), T(0) = 1
    r = oracle.ordered(3 * k, synth.moon_moser(k))
    assert r["nodes"] == (3 ** (k + 1) - 1) // 2
    assert r["internal"] == (3 ** k - 1) // 2 and r["dead_ends"] == 0


# --- statistical check against Table 1 --------------------------------------

def _table1_mu():
    rows = []
    with open(os.path.join(GOLDEN, "table1_random_mu.txt")) as f:
        for line in f:
            t = line.split()
            if t and not t[0].startswith("#"):
                rows.append((int(t[0]), float(t[1]), int(t[2])))
    return rows


@pytest.mark.parametrize("n,p,mu", _table1_mu())
def test_table1_mean_mu(n, p, mu):
    """Mean mu over 10 seeded G(n, p) vs the paper's 10-graph mean and the
    textbook expectation (sanity only: different instances)."""
    counts = [oracle.ordered(n, synth.gnp(n, p, 1000 + s))["count"] for s in range(10)]
    mean = float(np.mean(counts))
    assert abs(mean / mu - 1.0) < 0.12
    assert abs(mean / synth.expected_maximal_cliques(n, p) - 1.0) < 0.12


# --- GreedyBBNX picks GreedyBBTX's pivot ------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_nx_pivot_is_tx_pivot(seed):
    # For u in X (disjoint from P), |P n K(u)| = |P| - |P n N(u)|, so the
    # argmin of NX is TX's argmax with the same earliest-on-ties rule, and
    # the early exit only drops candidates that cannot win: every traced
    # node must pick the same pivot and branching set, and the trees agree.
    n, p = 16 + 9 * seed, 0.25 + 0.07 * seed
    uv = synth.gnp(n, p, 700 + seed)
    a = oracle.ordered(n, uv, "nx", trace_cap=4096)
    b = oracle.ordered(n, uv, "tx", trace_cap=4096)
    assert a["trace"] == b["trace"]
    assert (a["nodes"], a["internal"], a["dead_ends"]) == (b["nodes"], b["internal"], b["dead_ends"])
    ref = oracle.tomita(n, uv)
    assert (a["count"], a["hash"]) == (ref["count"], ref["hash"])



# --- the paper's step counts (Table 1) ----------------------------------------

def _table1():
    rows = {}
    for line in open(os.path.join(GOLDEN, "table1_random.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        rows[(int(t[0]), float(t[1]))] = {"mu": int(t[2]), "tomita": int(t[3]), "nx": int(t[5]), "greedy": int(t[7])}
    return rows


@pytest.mark.parametrize("n,p", [(100, 0.6), (300, 0.1), (300, 0.2), (300, 0.3), (500, 0.1), (500, 0.2),
                                 (700, 0.1), (1000, 0.1)])
def test_steps_per_clique_match_table1(n, p):
    # Table 1 reports, per shape G(n, p), the mean maximal cliques mu and the
    # mean search steps of GreedyBB, GreedyBBNX and TomitaBB over 10
    # unpublished instances.  A step is a call with P non-empty (our
    # "internal" node): the steps-per-clique ratio of the oracle's Alg. 4
    # tree on 3 seeded instances must match the paper's within 6 %, and the
    # three pivot rules must keep the paper's order (TomitaBB < NX < GreedyBB).
    paper = _table1()[(n, p)]
    got = {m: [0, 0] for m in ("greedy", "nx", "tomita")}
    for seed in range(3):
        uv = synth.gnp(n, p, seed)
        for m in got:
            r = oracle.ordered(n, uv, m)
            got[m][0] += r["internal"]
            got[m][1] += r["count"]
    for m, (steps, mu) in got.items():
        ours, theirs = steps / mu, paper[m] / paper["mu"]
        assert abs(ours / theirs - 1.0) < 0.06, (m, ours, theirs)
    assert got["tomita"][0] <= got["nx"][0] <= got["greedy"][0]


# --- the root's children as independent subtrees (multi-GPU split) -----------

@pytest.mark.parametrize("mode", ["greedy", "tx", "tomita", "nx"])
@pytest.mark.parametrize("n,p,seed", [(12, 0.5, 900), (16, 0.4, 901), (18, 0.6, 902)])
def test_root_child_reports_the_cliques_it_owns(mode, n, p, seed):
    # Child t of the root branches on v_t with v_1..v_{t-1} already moved to
    # X, so it reports exactly the maximal cliques that contain v_t and none
    # of v_1..v_{t-1} (brute force); the parts of any partition add up.
    uv = synth.gnp(n, p, seed)
    cliques = brute_force(n, uv)
    whole = oracle.ordered(n, uv, mode, trace_cap=1 << 16)
    depth, pivot, L = whole["trace"][0]
    assert depth == 0
    sizes = oracle.root_children(n, uv, mode)
    assert len(sizes) == len(L)
    tot = {"count": 0, "nodes": 0, "internal": 0, "dead_ends": 0, "hash": 0}
    for t, v in enumerate(L):
        own = [K for K in cliques if v in K and not set(L[:t]) & set(K)]
        r = oracle.ordered_part(n, uv, mode, [t], count_root=(t == 0))
        cnt, hist, h = summary(own, n)
        assert (r["count"], r["hash"]) == (cnt, h) and np.array_equal(r["hist"], hist), (t, v)
        for k in tot:
            tot[k] = (tot[k] + r[k]) & MASK
    for k in tot:
        assert tot[k] == whole[k], k


@pytest.mark.parametrize("mode", ["greedy", "tomita"])
def test_root_children_sizes_and_partition_sums(mode):
    # sizes on graphs worked by hand: the empty graph branches on every
    # vertex with nothing left (sizes 0); K_n on one child with n - 1 others;
    # Moon-Moser on k triangles branches on one triangle, each child keeping
    # the other 3(k-1) vertices
    assert oracle.root_children(7, synth.empty(7), mode).tolist() == [0] * 7
    assert oracle.root_children(9, synth.complete(9), mode).tolist() == [8]
    assert oracle.root_children(15, synth.moon_moser(5), mode).tolist() == [12, 12, 12]
    # a two-way split of a larger graph adds up to the whole search
    n, uv = 60, synth.gnp(60, 0.5, 903)
    whole = oracle.ordered(n, uv, mode)
    k = len(oracle.root_children(n, uv, mode))
    a = oracle.ordered_part(n, uv, mode, range(0, k, 2), count_root=True)
    b = oracle.ordered_part(n, uv, mode, range(1, k, 2), count_root=False)
    for key in ("count", "nodes", "internal", "dead_ends"):
        assert a[key] + b[key] == whole[key], key
    assert (a["hash"] + b["hash"]) & MASK == whole["hash"]
    assert np.array_equal(a["hist"] + b["hist"], whole["hist"])


# --- Alg. 3: degeneracy-ordered outer loop ----------------------------------

def _remaining_degree_check(n, uv, order):
    adj = [set() for _ in range(n)]
    for a, b in uv:
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    left = set(range(n))
    for v in order:
        v = int(v)
        deg = {u: len(adj[u] & left) for u in left}
        dmin = min(deg.values())
        assert deg[v] == dmin and v == min(u for u in left if deg[u] == dmin)
        left.remove(v)


@pytest.mark.parametrize("n,p,seed", [(20, 0.3, 1), (40, 0.15, 2), (60, 0.5, 3)])
def test_degeneracy_order_definition(n, p, seed):
    uv = synth.gnp(n, p, seed)
    _remaining_degree_check(n, uv, oracle.degeneracy_order(n, uv))


def test_degeneracy_order_bounds_later_neighbours_by_the_core_number():
    nx = pytest.importorskip("networkx")
    n, uv = 300, synth.gnp(300, 0.05, 9)
    order = oracle.degeneracy_order(n, uv)
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    later = np.zeros(n, dtype=np.int64)
    for a, b in uv:
        later[a if pos[a] < pos[b] else b] += 1
    g = nx.Graph()
    g.add_nodes_from(range(n))
    g.add_edges_from(uv.tolist())
    assert later.max() == max(nx.core_number(g).values())


@pytest.mark.parametrize("mode", ["greedy", "tx", "tomita", "nx"])
@pytest.mark.parametrize("n,p,seed", [(16, 0.5, 1), (80, 0.1, 2), (300, 0.03, 3), (120, 0.3, 4)])
def test_outer_loop_lists_the_maximal_cliques(mode, n, p, seed):
    uv = synth.gnp(n, p, seed)
    a = oracle.outer(n, uv, mode, listing=True)
    ref = oracle.tomita(n, uv, listing=True)
    assert (a["count"], a["hash"]) == (ref["count"], ref["hash"])
    assert np.array_equal(a["hist"], ref["hist"])
    assert a["listing"] == ref["listing"]
    assert a["nodes"] == a["count"] + a["internal"] + a["dead_ends"]


@pytest.mark.parametrize("n", [2, 5, 9, 30])
def test_outer_loop_tree_on_complete_and_empty_graphs(n):
    # K_n: v_0's subproblem is a chain of n calls; every later v_i has its
    # earlier neighbour v_0 in X, which pivots away all of P (one internal
    # call) except the last, whose P is empty (one dead end).
    a = oracle.outer(n, synth.complete(n))
    assert (a["count"], a["nodes"], a["internal"], a["dead_ends"]) == (1, 2 * n - 1, 2 * n - 3, 1)
    e = oracle.outer(n, synth.empty(n))
    assert (e["count"], e["nodes"], e["internal"], e["dead_ends"]) == (n, n, 0, 0)


@pytest.mark.parametrize("k", [3, 5, 7])
def test_outer_loop_moon_moser(k):
    a = oracle.outer(3 * k, synth.moon_moser(k))
    assert a["count"] == 3 ** k and int(a["hist"][k]) == 3 ** k
