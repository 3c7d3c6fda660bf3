#!/usr/bin/env python
"""Benchmark of the maximal clique enumeration path on GB300.

One *step* is one pass of the whole search path over one synthetic graph
already resident in HBM: input validation, maximum-degree-first ordering,
renumbering, the search itself and the reduction (every kernel of
mce_enumerate_device, called step by step so the search launch can be timed
on its own).  The workload is G(n = 1000, p = 0.3) with seed 1, the shape of
the paper's Table 1 row n = 1000, p = 0.3.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  ``value`` is maximal cliques per second over
all ranks (each rank runs its own replica: the plain form does not shard).
``e2e`` is the same metric through the handle API from pinned host memory
(mce_load_edges + mce_enumerate + mce_graph_free).  ``forms`` holds the
batched form (4096 graphs of uneven size in one captured launch,
mce_batch_launch) and the served form (a Poisson request stream through
mce_submit / mce_poll: graphs/s and p50/p99 latency), each beside the plain
form (one mce_enumerate call per graph) on the same graphs.  ``--impl
reference`` times the CPU oracle (Bron-Kerbosch with the Tomita pivot) on
bounded samples of the same graph on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# more hardware queues for the served form's per-request streams (read when
# the CUDA context is created)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import synth  # noqa: E402

METRIC = "maximal cliques/s & BK nodes/s, plain vs batched/served; p50/p99 latency"
UNIT = "maximal cliques/s"
# name -> (n, p, seed); the default is the measured workload, the others are
# smaller cases of the same kernels for profiling.
WORKLOADS = {
    "gnp_1000_0.3_s1": (1000, 0.3, 1),
    "gnp_700_0.3_s2": (700, 0.3, 2),
    "gnp_100_0.5_s0": (100, 0.5, 0),
}
DEFAULT_WORKLOAD = "gnp_1000_0.3_s1"
N, P, SEED = WORKLOADS[DEFAULT_WORKLOAD]
WORKLOAD = ""
GOLDEN_KEY = DEFAULT_WORKLOAD


def select_workload(name: str):
    global N, P, SEED, WORKLOAD, GOLDEN_KEY
    N, P, SEED = WORKLOADS[name]
    GOLDEN_KEY = name
    WORKLOAD = (f"G(n={N}, p={P}) seed {SEED}, one graph, plain form "
                f"(whole path: validate, order, renumber, search, reduce)")
# Table 1, n = 1000, p = 0.3: GreedyBB found 15.487755M cliques in 4.964 s on one
# Xeon E5-2690 v2 core (10-graph mean; other instances of the same shape).
PAPER_CLIQUES_PER_S = 15487755 / 4.964
L2_FLUSH_BYTES = 256 << 20          # > 129 MB of L2
# Roofline denominators: measured at the start of every run by
# mce_measure_peaks (LOP3 lane-operations and 128-bit shared-memory load
# bandwidth on every SM, CUDA events) -- see measure_peaks().  Until then,
# and as context in the JSON line, the figures derived from the GB300 unit
# counts and maximum clock: 152 SMs x 4 schedulers x 32 lanes x 2.07 GHz
# lane-operations per second and 152 SMs x 128 B/clk x 2.07 GHz.
SMS, SM_MHZ = 152, 2070.0
DERIVED_ALU_OPS = SMS * 4 * 32 * SM_MHZ * 1e6
DERIVED_SMEM_BPS = SMS * 128 * SM_MHZ * 1e6
ALU_PEAK_OPS = DERIVED_ALU_OPS
SMEM_PEAK_BPS = DERIVED_SMEM_BPS
PEAKS = {"source": "derived"}


def measure_peaks(mce, device: int) -> dict:
    """Measure the integer-pipe and shared-memory peaks on this GPU and make
    them the roofline denominators of this run."""
    global ALU_PEAK_OPS, SMEM_PEAK_BPS, PEAKS
    pk = mce.mce_measure_peaks(device)
    ALU_PEAK_OPS = pk["lop3_lane_ops_per_s"]
    SMEM_PEAK_BPS = pk["lds_bytes_per_s"]
    PEAKS = {"source": "measured: mce_measure_peaks (LOP3 / POPC lane-op, LDS.128 and warp-collective "
                       "microbenchmarks, CUDA events, all SMs)",
             "lop3_tops": pk["lop3_lane_ops_per_s"] / 1e12, "popc_tops": pk["popc_lane_ops_per_s"] / 1e12,
             "lds_gbs": pk["lds_bytes_per_s"] / 1e9,
             "ballot_g_warp_ops": pk["ballot_warp_ops_per_s"] / 1e9,
             "shfl_g_warp_ops": pk["shfl_warp_ops_per_s"] / 1e9,
             "redux_g_warp_ops": pk["redux_warp_ops_per_s"] / 1e9, "sm_count": pk["sm_count"],
             "sm_clock_max_mhz": pk["sm_clock_max_khz"] / 1e3,
             "derived_alu_tops": DERIVED_ALU_OPS / 1e12, "derived_lds_gbs": DERIVED_SMEM_BPS / 1e9}
    return PEAKS
ORACLE_SAMPLE_NODES = 1_500_000     # per reference step
BASELINE_SAMPLE_NODES = 5_000_000   # cpu_baseline leg (about 10-30 s)
# Batched form: 4096 G(n, p), n uniform in [32, 512], p uniform in [0.2, 0.8],
# seeds 0..4095, (n, p) redrawn while E[maximal cliques] > 1e6.  Served form:
# Poisson stream of G(n, p), n log-uniform in [64, 2048], p uniform in
# [0.1, 0.9], same cap, arrivals at SERVE_LOAD x the capacity measured on the
# warm-up requests (saturating), then a second pass at LATENCY_LOAD x capacity.
BATCH_GRAPHS = 4096
# The literal (uncapped) batched distribution, attempted on a few graphs with a
# short budget and reported as did-not-finish.
LITERAL_SAMPLE, LITERAL_TIMEOUT_NS = 32, 20_000_000
SERVE_LOAD, LATENCY_LOAD = 1.2, 0.7
# DRAM bytes (read + write) of one search-kernel launch, from a one-pass ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel built
# from device sources with this fingerprint (sha256 of the files below, first
# 16 hex digits); reported only while they match, else null.
KERNEL_SOURCES = ("search_impl.cuh", "search_inst.cuh", "mce_internal.h")
TRAFFIC = {"fingerprint": "88558c41864e7c4c", "workload": "gnp_1000_0.3_s1", "bytes": 3_768_832 + 798_720}


def words(n: int) -> int:
    return max(1, (n + 31) // 32)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"mce_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            t = [x.strip() for x in line.split(",")]
            if len(t) >= 7:
                rows.append(t)
        os.unlink(self.path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def kernel_fingerprint() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1801_00202_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic():
    if TRAFFIC["bytes"] and TRAFFIC["workload"] == GOLDEN_KEY and TRAFFIC["fingerprint"] == kernel_fingerprint():
        return TRAFFIC["bytes"]
    return None


def max_over_ranks(values, dist=None, device=None):
    """Element-wise maximum of per-rank timings over all ranks (the job's
    time is its slowest rank's); identity without a process group."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_rate(world: int, steps: int, units_per_step: float, max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (weak scaling: each rank runs its own replica)."""
    return world * steps * units_per_step / (max_ms / 1e3)


def golden_for(key):
    p = os.path.join(ROOT, "tests", "golden", "config_results.json")
    if os.path.exists(p):
        return json.load(open(p)).get(key)
    return None


def golden():
    p = os.path.join(ROOT, "tests", "golden", "config_results.json")
    if os.path.exists(p):
        return json.load(open(p)).get(GOLDEN_KEY)
    return None


def base_line(args, world):
    return {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "p": P, "seed": SEED, "words_per_row": words(N),
                       "l2": "flushed between timed steps (256 MiB write)", "replicas": world}}


def cpu_baseline(uv, max_nodes: int) -> dict:
    import oracle
    t = time.perf_counter()
    r = oracle.tomita(N, uv, max_nodes=max_nodes)
    dt = time.perf_counter() - t
    return {"value": r["count"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"Bron-Kerbosch with the Tomita pivot on the same graph, first {r['nodes']} search nodes "
                      f"({r['count']} maximal cliques, {dt:.1f} s on one host core)",
            "nodes_per_s": r["nodes"] / dt}


def _oracle_part(job):
    import oracle
    n, uv, mode, children, count_root = job
    t = time.perf_counter()
    r = oracle.ordered_part(n, uv, mode, children, count_root)
    return r["count"], r["nodes"], r["hash"], time.perf_counter() - t


def cpu_split_baseline(n, uv, cores: int, mode: str = "greedy") -> dict:
    """The oracle's Alg. 4 tree (the paper's GreedyBB) on all host cores: the
    root's children partitioned by candidate-set size over `cores` spawned
    processes (each an independent subtree), wall time of the whole search."""
    import multiprocessing as mp

    import oracle
    from paper_1801_00202_gb300 import split
    oracle.build()
    sizes = oracle.root_children(n, uv, mode)
    parts = [x for x in split.partition(sizes, cores)]
    jobs = [(n, uv, mode, ch, i == 0) for i, ch in enumerate(parts) if ch or i == 0]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        pool.map(abs, range(len(jobs)))          # start the workers outside the timed region
        t = time.perf_counter()
        res = pool.map(_oracle_part, jobs, chunksize=1)
        wall = time.perf_counter() - t
    count = sum(c for c, _, _, _ in res)
    nodes = sum(x for _, x, _, _ in res)
    h = sum(x for _, _, x, _ in res) % (1 << 64)
    return {"value": count / wall, "unit": UNIT, "cores": len(jobs), "kind": "oracle", "nodes_per_s": nodes / wall,
            "seconds": wall, "count": count, "hash": h, "root_children": int(len(sizes)),
            "busiest_part_s": max(x for _, _, _, x in res),
            "sample": f"whole graph: the oracle's GreedyBB tree (Alg. 4), the root's {len(sizes)} children split "
                      f"over {len(jobs)} host processes by candidate-set size"}


def root_child_work(mce, ctx, n, uv) -> dict:
    """Search nodes of every root child (mce_enumerate_part, one child per
    call): the tree's imbalance as max / mean work per root child."""
    g = ctx.load_edges(n, uv)
    try:
        sizes = g.root_children()
        work = [g.enumerate_part([t], False)["nodes"] for t in range(len(sizes))]
    finally:
        g.free()
    mean = sum(work) / max(1, len(work))
    return {"children": len(work), "nodes_per_child": work, "max_over_mean": max(work) / mean if mean else None}


# ---------------------------------------------------------------------------
# Batched and served forms

def _gen_batch(i: int):
    g = synth.batch_graph(i)
    return g.n, g.p, g.draws, synth.to_bitset(g.n, g.uv)


def _gen_literal(i: int):
    g = synth.batch_graph(i, cap=math.inf)   # the literal distribution: first draw kept
    return g.n, g.p, g.draws, synth.to_bitset(g.n, g.uv)


def _gen_served(r: int):
    g = synth.served_graph(r)
    return g.n, g.p, g.draws, synth.to_bitset(g.n, g.uv)


def _oracle_batch_graph(i: int):
    import oracle
    g = synth.batch_graph(i)
    t = time.perf_counter()
    r = oracle.tomita(g.n, g.uv)
    return r["count"], time.perf_counter() - t


def generate_forms(args):
    """Build the batched and served graphs on all host cores (spawned pool,
    before any CUDA call); bitset rows come back.  The same pool then times
    the CPU oracle, one graph per core, on an evenly spaced sample of the
    batched workload (its all-cores baseline)."""
    import multiprocessing as mp
    total = args.served_warmup + args.served_requests
    cores = max(1, min(os.cpu_count() or 1, 32))
    t = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        batch = pool.map(_gen_batch, range(args.batch_graphs), chunksize=32)
        served = pool.map(_gen_served, range(total), chunksize=64)
        literal = pool.map(_gen_literal, range(LITERAL_SAMPLE), chunksize=4)
        gen_s = time.perf_counter() - t
        base = None
        if args.oracle_sample and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            step = max(1, args.batch_graphs // args.oracle_sample)
            sample = list(range(0, args.batch_graphs, step))[:args.oracle_sample]
            t = time.perf_counter()
            res = pool.map(_oracle_batch_graph, sample, chunksize=1)
            wall = time.perf_counter() - t
            cliques = sum(c for c, _ in res)
            base = {"value": len(sample) / wall, "unit": "graphs/s", "cores": cores, "kind": "oracle",
                    "cliques_per_s": cliques / wall,
                    "sample": f"Bron-Kerbosch with the Tomita pivot, one graph per host core, on every "
                              f"{step}th graph of the batched workload ({len(sample)} graphs, "
                              f"{cliques} maximal cliques, {wall:.1f} s)"}
    return batch, served, {"cores": cores, "seconds": gen_s}, base, literal


def _work(results, ns):
    """Algorithmic lane-ops and row bytes (6W and 8W per search node)."""
    ops = sum(6 * words(n) * r["nodes"] for r, n in zip(results, ns))
    return ops, 8 * ops // 6


def _rates(graphs, cliques, nodes, ops, row_bytes, seconds):
    return {"graphs_per_s": graphs / seconds, "cliques_per_s": cliques / seconds, "nodes_per_s": nodes / seconds,
            "alu_frac": ops / seconds / ALU_PEAK_OPS, "smem_frac": row_bytes / seconds / SMEM_PEAK_BPS}


def _same(a, b) -> bool:
    return (a["count"] == b["count"] and a["hash"] == b["hash"] and a["nodes"] == b["nodes"]
            and np.array_equal(a["hist"], b["hist"]))


def plain_pass(mce, torch, graphs, opts):
    """Plain form: one mce_enumerate call (whole path, result to host) per
    graph, back to back."""
    torch.cuda.synchronize()
    t = time.perf_counter()
    res = [g.enumerate(opts) for g in graphs]
    return res, time.perf_counter() - t


def batched_form(mce, torch, ctx, s, specs, opts, args, flush_l2):
    graphs = [ctx.load_bitset(n, rows) for n, _, _, rows in specs]
    ns = [n for n, _, _, _ in specs]
    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(b):
        for _ in range(max(1, args.warmup // 3)):
            b.run()
        evs = [(mk(), mk()) for _ in range(args.batch_steps)]
        torch.cuda.synchronize()
        for e0, e1 in evs:
            flush_l2()
            e0.record(s)
            b.launch()
            e1.record(s)
        res = b.results()
        return res, [e0.elapsed_time(e1) for e0, e1 in evs]

    # the launch choices come from the autotuner (timed on these graphs at
    # plan time, outside the timed region); the defaults are measured beside
    t = time.perf_counter()
    b = mce.Batch(ctx, graphs, mce.options(autotune=True))
    plan_s = time.perf_counter() - t
    res, ms = timed(b)
    buckets = b.buckets()
    b.close()
    b = mce.Batch(ctx, graphs, opts)
    res_d, ms_d = timed(b)
    b.close()
    plain, plain_s = plain_pass(mce, torch, graphs, opts)
    for g in graphs:
        g.free()
    sec = statistics.mean(ms) / 1e3
    cliques, nodes = sum(r["count"] for r in res), sum(r["nodes"] for r in res)
    ops, rb = _work(res, ns)
    out = {"workload": f"{len(ns)} G(n,p), n uniform [32,512], p uniform [0.2,0.8], seeds 0..{len(ns) - 1}, "
                       f"(n,p) redrawn while E[maximal cliques] > 1e6",
           "graphs": len(ns), "acceptance": len(ns) / sum(d for _, _, d, _ in specs),
           "mean_n": float(np.mean(ns)), "cliques": cliques, "nodes": nodes,
           "steps": args.batch_steps, "ms_per_step": statistics.mean(ms), "autotune_plan_and_capture_s": plan_s,
           "batched": _rates(len(ns), cliques, nodes, ops, rb, sec),
           "batched_default_choices": _rates(len(ns), cliques, nodes, ops, rb, statistics.mean(ms_d) / 1e3),
           "autotuned_buckets": [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in x.items()}
                                 for x in buckets],
           "plain": _rates(len(ns), cliques, nodes, ops, rb, plain_s),
           "plain_note": "one mce_enumerate per graph, back to back (wall clock, results read per graph)",
           "status_ok": all(r["status"] == 0 for r in res),
           "batched_equals_plain": all(_same(a, c) for a, c in zip(res, plain)) and
                                   all(_same(a, c) for a, c in zip(res_d, plain)),
           "launches_per_step": "one CUDA graph: a batched ordering kernel, a batched renumbering "
                                "kernel and one persistent search kernel per subtree shape"}
    out["speedup_graphs_per_s"] = out["batched"]["graphs_per_s"] / out["plain"]["graphs_per_s"]
    return out


def _open_loop(ctx, graphs, arrivals, opts):
    """Submit graph i at arrivals[i] (s from the start), poll the oldest
    requests; latency = submit delay + the library's submit-to-done time."""
    R = len(graphs)
    lat = [0.0] * R
    res = [None] * R
    pend = []           # (index, ticket, submit time)
    nxt = done = 0
    t0 = time.perf_counter()
    while done < R:
        now = time.perf_counter() - t0
        while nxt < R and arrivals[nxt] <= now:
            ts = time.perf_counter() - t0
            pend.append((nxt, ctx.submit(graphs[nxt], opts), ts))
            nxt += 1
        keep = []
        for k, (i, tk, ts) in enumerate(pend):
            if k >= 64:
                keep.extend(pend[k:])
                break
            r = ctx.poll(tk)
            if r is None:
                keep.append((i, tk, ts))
                continue
            res[i] = r
            lat[i] = (ts - arrivals[i]) + r["total_ms"] / 1e3
            done += 1
        pend = keep
    finish = max(a + l for a, l in zip(arrivals, lat))
    return res, lat, finish - arrivals[0]


def literal_form(mce, ctx, specs, cliques_per_s):
    """The first LITERAL_SAMPLE graphs of the batched workload as written, with
    no cap on E[maximal cliques]: one batch with a short per-graph budget
    (MCE_ETIMEOUT after 10 x LITERAL_TIMEOUT_NS of search), reported as did
    not finish where the budget ran out, with the time the expected clique
    counts project at the capped workload's measured rate."""
    graphs = [ctx.load_bitset(n, rows) for n, _, _, rows in specs]
    t = time.perf_counter()
    b = mce.Batch(ctx, graphs, mce.options(timeout_ns=LITERAL_TIMEOUT_NS))
    res = b.run(raise_on_error=False)
    wall = time.perf_counter() - t
    b.close()
    for g in graphs:
        g.free()
    emu = [synth.expected_maximal_cliques(n, p) for n, p, _, _ in specs]
    done = [r["status"] == 0 for r in res]
    dnf = [r["status"] == mce.MCE_ETIMEOUT for r in res]
    left = sum(e for e, d in zip(emu, done) if not d)
    return {"graphs": len(specs), "finished": sum(done), "did_not_finish": sum(dnf),
            "other_status": len(specs) - sum(done) - sum(dnf), "budget_s_per_graph": 10 * LITERAL_TIMEOUT_NS / 1e9,
            "wall_s": wall, "cliques_finished": sum(r["count"] for r, d in zip(res, done) if d),
            "expected_cliques_unfinished": left, "largest_expected": max(emu),
            "projected_hours_at_capped_rate": left / cliques_per_s / 3600.0,
            "note": "n uniform [32,512], p uniform [0.2,0.8] with no cap on E[maximal cliques] "
                    "(the capped workload redraws (n,p) while E > 1e6); first draws of graphs 0.."
                    f"{len(specs) - 1}"}


def served_form(mce, torch, ctx, specs, opts, args):
    graphs = [ctx.load_bitset(n, rows) for n, _, _, rows in specs]
    ns = [n for n, _, _, _ in specs]
    W = args.served_warmup
    warm, timed = graphs[:W], graphs[W:]
    # warm-up, closed loop: everything submitted at once -> capacity
    t = time.perf_counter()
    tickets = [ctx.submit(g, opts) for g in warm]
    for tk in tickets:
        ctx.wait(tk)
    capacity = len(warm) / (time.perf_counter() - t)
    out = {"workload": f"Poisson stream of G(n,p), n log-uniform [64,2048], p uniform [0.1,0.9], "
                       f"(n,p) redrawn while E[maximal cliques] > 1e6; {W} warm-up + {len(timed)} timed requests",
           "requests": len(timed), "warmup_requests": W,
           "acceptance": len(specs) / sum(d for _, _, d, _ in specs), "mean_n": float(np.mean(ns[W:])),
           "capacity_closed_loop_graphs_per_s": capacity}
    for name, load in (("saturating", SERVE_LOAD), ("latency", LATENCY_LOAD)):
        arr = synth.served_arrivals(len(timed), load * capacity)
        arr = arr - arr[0]
        res, lat, span = _open_loop(ctx, timed, arr, opts)
        cliques, nodes = sum(r["count"] for r in res), sum(r["nodes"] for r in res)
        ops, rb = _work(res, ns[W:])
        lat_ms = np.array(lat) * 1e3
        out[name] = {"offered_graphs_per_s": load * capacity, "load": load,
                     **_rates(len(timed), cliques, nodes, ops, rb, span),
                     "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                     "mean_ms": float(lat_ms.mean()), "status_ok": all(r["rc"] == 0 for r in res)}
        if name == "saturating":
            first = res
    k = min(args.plain_sample, len(timed))
    plain, plain_s = plain_pass(mce, torch, timed[:k], opts)
    ops, rb = _work(plain, ns[W:W + k])
    out["plain"] = _rates(k, sum(r["count"] for r in plain), sum(r["nodes"] for r in plain), ops, rb, plain_s)
    out["plain_note"] = f"one mce_enumerate per request, back to back, first {k} timed requests"
    out["served_equals_plain"] = all(_same(a, c) for a, c in zip(first[:k], plain))
    out["speedup_graphs_per_s"] = out["saturating"]["graphs_per_s"] / out["plain"]["graphs_per_s"]
    for g in graphs:
        g.free()
    return out


# ---------------------------------------------------------------------------

def other_configs():
    """The other single-graph configurations: G(100, 0.5) seed 0, Moon-Moser
    on 45 vertices, and the same with 5% of its edges deleted (seed 3)."""
    return [("gnp_100_0.5_s0", 100, synth.gnp(100, 0.5, 0)),
            ("moon_moser_45", 45, synth.moon_moser(15)),
            ("moon_moser_45_del5", 45, synth.moon_moser_deleted(15, 0.05, 3))]


def plain_config(mce, torch, s, dev, name, n, uv, reps, flush_l2):
    """One graph through mce_enumerate_device on resident device input, the
    whole path timed with events (median of `reps` after one warm-up)."""
    opts = mce.options()
    W = words(n)
    rows = torch.from_numpy(synth.to_bitset(n, uv).view(np.int32).reshape(-1)).to(dev)
    nb = mce.mce_scratch_bytes(n, opts)
    scr = torch.empty(nb, dtype=torch.uint8, device=dev)
    out = torch.zeros(mce.MCE_OUT_WORDS(n), dtype=torch.int64, device=dev)
    ms = []
    for i in range(reps + 1):
        flush_l2()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            e0.record(s)
            rc = mce.mce_enumerate_device(n, W, rows, opts, scr, nb, out, s)
            e1.record(s)
        if rc:
            raise mce.MceError(rc, name)
        torch.cuda.synchronize()
        if i:
            ms.append(e0.elapsed_time(e1))
    r = mce.decode_out(out, n)
    t = statistics.median(ms) / 1e3
    gold = golden_for(name)
    ops = 6 * W * r["nodes"]
    return {"n": n, "count": r["count"], "nodes": r["nodes"], "ms": 1e3 * t,
            "cliques_per_s": r["count"] / t, "nodes_per_s": r["nodes"] / t,
            "alu_frac": ops / t / ALU_PEAK_OPS, "smem_frac": 8 * W * r["nodes"] / t / SMEM_PEAK_BPS,
            "utilisation": r["busy_ns"] / max(1, r["groups"]) / (t * 1e9),
            "donations": r["donations"], "steals": r["steals"], "global_steals": r["global_steals"],
            "matches_oracle": bool(gold) and r["count"] == gold["count"] and r["hash"] == gold["hash"]
                              and r["nodes"] == gold["greedy"]["nodes"] and r["status"] == 0}


def listing_runs(mce, torch, device, stream, uv):
    """The listing through mce_enumerate on the measured graph: every maximal
    clique returned to host buffers (CSR), unsorted and in lexicographic
    order; wall time of the call (search, record chunks -> CSR on the
    device, copy to the host)."""
    gold = golden() or {}
    need_ids = sum(int(k) * c for k, c in gold.get("hist", {}).items())
    if not need_ids:
        return None
    ctx = mce.Context(device, stream=stream)
    g = ctx.load_edges(N, uv)
    out = {}
    for name, flags in (("unsorted", mce.MCE_LIST), ("sorted", mce.MCE_LIST_SORTED)):
        o = mce.options(flags=flags)
        g.enumerate(o, list_cap=need_ids, off_cap=gold["count"] + 1)   # warm
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = g.enumerate(o, list_cap=need_ids, off_cap=gold["count"] + 1)
        sec = time.perf_counter() - t
        out[name] = {"ms": 1e3 * sec, "cliques_per_s": r["count"] / sec, "ids": int(r["list_off"][-1]),
                     "host_bytes": int(r["list_off"][-1]) * 4 + (r["count"] + 1) * 8,
                     "matches_oracle": r["count"] == gold["count"] and r["hash"] == gold["hash"]}
    g.free()
    ctx.close()
    return out


def table1_rows():
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "table1_random.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        rows.append({"n": int(t[0]), "p": float(t[1]), "mu": int(t[2]),
                     "tomita": (int(t[3]), t[4]), "nx": (int(t[5]), t[6]), "greedy": (int(t[7]), t[8])})
    return rows


def run_sweep(args):
    """The paper's Table 1 grid (every shape with n <= 4096) on seeded
    G(n, p): maximal cliques, search nodes and time per pivot rule through
    mce_enumerate, beside the paper's steps and seconds (one CPU core, 10
    other instances of each shape)."""
    import torch

    import paper_1801_00202_gb300 as mce
    mce.build()
    mce.lib()
    ctx = mce.Context(0)
    clocks = ClockSampler(0)
    clocks.start()
    out = []
    for row in table1_rows():
        if row["n"] > mce.MCE_NMAX_SPARSE or row["n"] < args.sweep_min_n:
            continue
        cell = {"n": row["n"], "p": row["p"], "paper_mu": row["mu"], "seeds": args.sweep_seeds}
        mus = []
        seen = {}           # seed -> (count, hash) of the first pivot rule
        consistent = True
        for pivot in ("greedy", "nx", "tomita"):
            nodes, internal, ms, total = [], [], [], []
            for seed in range(args.sweep_seeds):
                g = ctx.load_edges(row["n"], synth.gnp(row["n"], row["p"], seed))
                torch.cuda.synchronize()
                r = g.enumerate(mce.options(pivot=pivot))
                g.free()
                key = (r["count"], r["hash"], tuple(int(x) for x in r["hist"]))
                consistent = consistent and seen.setdefault(seed, key) == key
                if pivot == "greedy":
                    mus.append(r["count"])
                nodes.append(r["nodes"])
                internal.append(r["internal"])
                ms.append(r["kernel_ms"])
                total.append(r["total_ms"])
            steps, secs = row[pivot]
            cell[pivot] = {"nodes": statistics.mean(nodes), "internal_nodes": statistics.mean(internal),
                           "ms": statistics.mean(ms), "call_ms": statistics.mean(total),
                           "paper_steps": steps, "paper_s": secs}
            if row["n"] > mce.MCE_NMAX:
                cell[pivot]["path"] = "outer loop of Alg. 3 (nodes: sum of the subproblem trees)"
            if not secs.startswith("<"):
                cell[pivot]["speedup_vs_paper_core"] = float(secs) * 1e3 / statistics.mean(ms)
        cell["mu"] = statistics.mean(mus)
        # the results do not depend on the pivot rule: the three rules must
        # agree on every seed; where the oracle finishes in seconds
        # (expected maximal cliques <= 3e5), seed 0 is checked against it
        cell["pivot_rules_agree"] = consistent
        if synth.expected_maximal_cliques(row["n"], row["p"]) <= 3e5:
            import oracle
            ref = oracle.tomita(row["n"], synth.gnp(row["n"], row["p"], 0))
            cell["matches_oracle"] = seen[0] == (ref["count"], ref["hash"], tuple(int(x) for x in ref["hist"]))
        out.append(cell)
        print(json.dumps(cell), file=sys.stderr, flush=True)
    ctx.close()
    print(json.dumps({"sweep": "Table 1 shapes", "unit": "ms per graph (whole path, device time); call_ms: "
                                                        "the mce_enumerate call",
                      "clocks": clocks.stop(), "rows": out}), flush=True)
    return 0


def run_batch_probe(args):
    """The first --batch-probe graphs of the batched workload as one batch
    with the default launch choices: three warm-up launches, then one timed
    launch (the case the ncu captures of batch_kernel profile)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(os.cpu_count() or 1, 32))) as pool:
        specs = pool.map(_gen_batch, range(args.batch_probe), chunksize=16)
    import torch

    import paper_1801_00202_gb300 as mce
    mce.build()
    mce.lib()
    ctx = mce.Context(0)
    graphs = [ctx.load_bitset(n, rows) for n, _, _, rows in specs]
    b = mce.Batch(ctx, graphs)
    for _ in range(3):
        b.run()
    torch.cuda.synchronize()
    t = time.perf_counter()
    b.launch()
    res = b.results()
    dt = time.perf_counter() - t
    print(json.dumps({"batch_probe": len(graphs), "ms": 1e3 * dt, "graphs_per_s": len(graphs) / dt,
                      "cliques": sum(r["count"] for r in res), "status_ok": all(r["status"] == 0 for r in res),
                      "buckets": [{k: x[k] for k in ("words_class", "graphs", "lanes_per_subtree", "words_per_lane",
                                                     "threads_per_block", "blocks")} for x in b.buckets()]}),
          flush=True)
    b.close()
    for g in graphs:
        g.free()
    ctx.close()
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    uv = synth.gnp(N, P, SEED)
    rates, times = [], []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        r = oracle.tomita(N, uv, max_nodes=ORACLE_SAMPLE_NODES)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            rates.append(r["count"] / dt)
            times.append(dt)
    value = statistics.mean(rates)
    line = base_line(args, world)
    line.update({"impl": "reference", "value": value, "ms_per_step": 1e3 * statistics.mean(times),
                 "vs_baseline": value / PAPER_CLIQUES_PER_S,
                 "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                  "sample": f"each step: Bron-Kerbosch with the Tomita pivot on the same graph, "
                                            f"first {ORACLE_SAMPLE_NODES} search nodes, one host core"},
                 "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    print(json.dumps(line), flush=True)
    return 0


def run_sharded(args, mce, torch, dist, rank, world, local, dev):
    """N > 1: one graph split over the ranks (the root's children are
    independent subtrees; paper_1801_00202_gb300/split.py), strong scaling.
    A step is this rank's share of the search (mce_enumerate_part: validate,
    order, renumber, search its children; device time from the library's CUDA
    events) and one all-reduce of the result vector."""
    from paper_1801_00202_gb300 import split
    uv = synth.gnp(N, P, SEED)
    ctx = mce.Context(local)
    g = ctx.load_edges(N, uv)
    sizes = g.root_children()
    mine = split.part_of(sizes, rank, world)
    for _ in range(args.warmup):
        split.all_reduce_result(g.enumerate_part(mine, rank == 0), N, dist, dev)
    dist.barrier()
    torch.cuda.synchronize()
    dev_ms = []
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.steps):
        r = g.enumerate_part(mine, rank == 0)
        dev_ms.append(r["kernel_ms"])
        whole = split.all_reduce_result(r, N, dist, dev)
    torch.cuda.synchronize()
    clk = clocks.stop()
    g.free()
    # end to end: the edge list from pinned host memory every step
    pinned = torch.from_numpy(uv.astype(np.int32)).pin_memory()
    host_uv = pinned.numpy().view(np.uint32)
    dist.barrier()
    wall = time.perf_counter()
    for _ in range(args.steps):
        g2 = ctx.load_edges(N, host_uv)
        split.all_reduce_result(g2.enumerate_part(mine, rank == 0), N, dist, dev)
        g2.free()
    wall = time.perf_counter() - wall
    total_ms, wall_ms = max_over_ranks([sum(dev_ms), 1e3 * wall], dist, dev)
    ctx.close()
    if rank != 0:
        return 0
    gold = golden()
    line = base_line(args, world)
    line["scaling"] = "strong"
    line["config"].update({"parallelism": f"root children split over {world} GPUs", "replicas": 1})
    line.update({"impl": "ours", "value": args.steps * whole["count"] / (total_ms / 1e3),
                 "ms_per_step": total_ms / args.steps, "vs_baseline": None,
                 "nodes_per_s": args.steps * whole["nodes"] / (total_ms / 1e3),
                 "check": {"count": whole["count"], "hash": whole["hash"], "nodes": whole["nodes"],
                           "matches_oracle": bool(gold) and whole["count"] == gold["count"]
                           and whole["hash"] == gold["hash"] and whole["nodes"] == gold["greedy"]["nodes"]},
                 "e2e": {"value": args.steps * whole["count"] / (wall_ms / 1e3), "unit": UNIT,
                         "h2d_bytes_per_step": int(uv.shape[0]) * 8, "d2h_bytes_per_step": 8 * (N + 22),
                         "api": "per rank and step: mce_load_edges (pinned host edge list) + mce_enumerate_part + "
                                "all-reduce of the result vector + mce_graph_free"},
                 "gpu_launches": 7 * args.steps, "clocks": clk,
                 "root_children": int(len(sizes))})
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    forms_in = None
    if not args.no_forms and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        forms_in = generate_forms(args)     # host cores, before any CUDA call
    import torch

    import paper_1801_00202_gb300 as mce

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mce.build()
    mce.lib()
    if world > 1:
        try:
            return run_sharded(args, mce, torch, dist, rank, world, local, dev)
        finally:
            dist.destroy_process_group()

    uv = synth.gnp(N, P, SEED)
    W = words(N)
    opts = mce.options(lanes=args.lanes, words=args.words, threads=args.threads, blocks=args.blocks,
                       split_min_p=args.split)
    wp = mce.mce_search_words(N, opts)
    s = torch.cuda.Stream(device=dev)
    rows = torch.from_numpy(synth.to_bitset(N, uv).view(np.int32).reshape(-1)).to(dev)
    order = torch.zeros(N, dtype=torch.int32, device=dev)
    ren = torch.zeros(N * wp + 4, dtype=torch.int32, device=dev)
    nbytes = mce.mce_scratch_bytes(N, opts)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = torch.zeros(mce.MCE_OUT_WORDS(N), dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def step(ev0, ev1, ev2):
        with torch.cuda.stream(s):
            ev0.record(s)
            out.zero_()
            rc = mce.mce_validate_rows(N, W, rows, out, s)
            rc = rc or mce.mce_order(N, W, rows, order, s)
            rc = rc or mce.mce_renumber(N, W, rows, order, wp, ren, s)
            ev1.record(s)
            rc = rc or mce.mce_search(N, ren, order, opts, scratch, nbytes, out, s)
            ev2.record(s)
        if rc:
            raise mce.MceError(rc, "step")

    def flush_l2():
        with torch.cuda.stream(s):
            flush.zero_()

    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    for _ in range(args.warmup):
        flush_l2()
        step(mk(), mk(), mk())
    torch.cuda.synchronize()
    res = mce.decode_out(out, N)
    if res["status"] != 0:
        raise mce.MceError(res["status"], "warm-up")
    peaks = measure_peaks(mce, local)

    clocks = ClockSampler(local)
    evs = [(mk(), mk(), mk()) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for e in evs:
        flush_l2()
        step(*e)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(c) for a, b, c in evs]
    search_ms = [b.elapsed_time(c) for a, b, c in evs]
    prep_ms = [a.elapsed_time(b) for a, b, c in evs]
    res = mce.decode_out(out, N)
    if res["status"] != 0:
        raise mce.MceError(res["status"], "timed steps")

    # --- end to end through the handle API, host buffers in pinned memory
    e2e_s, r2 = [], {"count": res["count"]}
    if not args.no_e2e:
        ctx = mce.Context(local, stream=s)
        pinned = torch.from_numpy(uv.astype(np.int32)).pin_memory()
        host_uv = pinned.numpy().view(np.uint32)
        for _ in range(args.warmup):
            g = ctx.load_edges(N, host_uv)
            g.enumerate(opts)
            g.free()
        for _ in range(args.steps):
            flush_l2()
            torch.cuda.synchronize()
            t = time.perf_counter()
            g = ctx.load_edges(N, host_uv)
            r2 = g.enumerate(opts)
            g.free()
            e2e_s.append(time.perf_counter() - t)
        ctx.close()
    clk = clocks.stop()

    total_ms = float(sum(step_ms))
    e2e_total = float(sum(e2e_s)) if e2e_s else 0.0
    total_ms, e2e_total = max_over_ranks([total_ms, e2e_total], dist, dev)
    if rank != 0:
        dist.destroy_process_group()
        return 0
    configs = {name: plain_config(mce, torch, s, dev, name, n, cuv, 5, flush_l2)
               for name, n, cuv in other_configs()}
    ictx = mce.Context(local, stream=s)
    for name, n, cuv in other_configs():
        if name.startswith("moon_moser"):
            configs[name]["root_child_work"] = root_child_work(mce, ictx, n, cuv)
    ictx.close()
    listing = listing_runs(mce, torch, local, s, uv)

    forms = None
    if forms_in is not None:
        batch_specs, served_specs, gen, batch_base, literal_specs = forms_in
        fctx = mce.Context(local, stream=s)
        fclk = ClockSampler(local)
        fclk.start()
        forms = {"batched": batched_form(mce, torch, fctx, s, batch_specs, mce.options(), args, flush_l2)}
        forms["batched"]["cpu_oracle_all_cores"] = batch_base
        forms["served"] = served_form(mce, torch, fctx, served_specs, mce.options(), args)
        forms["literal_batched_sample"] = literal_form(mce, fctx, literal_specs,
                                                       forms["batched"]["batched"]["cliques_per_s"])
        forms["clocks"] = fclk.stop()
        forms["generation"] = gen
        fctx.close()

    count, nodes = res["count"], res["nodes"]
    value = job_rate(world, args.steps, count, total_ms)
    gold = golden()
    check = {"status": res["status"], "count": count, "nodes": nodes, "hash": res["hash"],
             "lane_tasks": res["lane_tasks"], "steals": res["steals"], "donations": res["donations"]}
    if gold:
        check["matches_oracle"] = (count == gold["count"] and res["hash"] == gold["hash"]
                                   and nodes == gold["greedy"]["nodes"] and r2["count"] == gold["count"])
    search_avg = statistics.mean(search_ms)
    ops = 6 * W * nodes                 # algorithmic 32-bit lane-ops per search launch
    smem_bytes = 8 * W * nodes          # two adjacency rows per node
    line = base_line(args, world)
    line.update({
        "impl": "ours",
        "value": value,
        "ms_per_step": total_ms / args.steps,
        "vs_baseline": value / PAPER_CLIQUES_PER_S,
        "vs_baseline_note": "paper's GreedyBB, Table 1 n=1000 p=0.3 (10-graph mean, one Xeon E5-2690 v2 core)",
        "nodes_per_s": job_rate(world, args.steps, nodes, total_ms),
        "breakdown_ms": {"prep (validate+order+renumber)": statistics.mean(prep_ms),
                         "search (init+persistent kernel)": search_avg,
                         "wall_per_step_incl_l2_flush": 1e3 * t_wall / args.steps},
        "check": check,
        "roofline": {"bound": "alu", "kernel": "search_kernel",
                     "achieved": ops / (search_avg / 1e3) / 1e12, "peak": ALU_PEAK_OPS / 1e12,
                     "unit": "T lane-ops/s (32-bit LOP3)", "frac": ops / (search_avg / 1e3) / ALU_PEAK_OPS,
                     "traffic": measured_traffic(), "traffic_fingerprint": kernel_fingerprint(),
                     "peak_source": peaks["source"],
                     "ops_per_node": 6 * W, "nodes_per_launch": nodes},
        "roofline_smem": {"achieved": smem_bytes / (search_avg / 1e3) / 1e9, "peak": SMEM_PEAK_BPS / 1e9,
                          "unit": "GB/s", "frac": smem_bytes / (search_avg / 1e3) / SMEM_PEAK_BPS,
                          "bytes_per_node": 8 * W, "peak_source": peaks["source"]},
        "peaks": peaks,
        "e2e": None if args.no_e2e else {
            "value": job_rate(world, args.steps, r2["count"], 1e3 * e2e_total), "unit": UNIT,
            "h2d_bytes_per_step": int(uv.shape[0]) * 8,
            "d2h_bytes_per_step": mce.MCE_OUT_WORDS(N) * 8 + 8,
            "ms_per_step": 1e3 * e2e_total / args.steps,
            "api": "mce_load_edges (pinned host edge list) + mce_enumerate + mce_graph_free"},
        "gpu_launches": 5 * args.steps + (0 if args.no_e2e else 6 * args.steps),
        "clocks": clk,
        "other_configs": configs,
        "listing": listing,
        "forms": forms,
    })
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(uv, BASELINE_SAMPLE_NODES)
        cores = max(1, min(os.cpu_count() or 1, 32))
        allc = {DEFAULT_WORKLOAD: cpu_split_baseline(N, uv, cores)}
        for name, n, cuv in other_configs():
            allc[name] = cpu_split_baseline(n, cuv, cores)
        line["cpu_baseline"]["all_cores"] = allc
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and served forms")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the benchmark: the paper's Table 1 grid, per pivot rule")
    ap.add_argument("--sweep-seeds", type=int, default=3)
    ap.add_argument("--sweep-min-n", type=int, default=0)
    ap.add_argument("--batch-graphs", type=int, default=BATCH_GRAPHS)
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--batch-probe", type=int, default=0,
                    help="instead of the benchmark: time one launch of a batch of the first N batched graphs")
    ap.add_argument("--served-requests", type=int, default=20000)
    ap.add_argument("--served-warmup", type=int, default=2000)
    ap.add_argument("--oracle-sample", type=int, default=256,
                    help="batched graphs the CPU oracle runs on all host cores (0: skip)")
    ap.add_argument("--plain-sample", type=int, default=4000,
                    help="served requests also run through the plain form for the comparison")
    # launch-shape overrides (0 = the library's choice)
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--words", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--blocks", type=int, default=0)
    ap.add_argument("--split", type=int, default=0)
    args = ap.parse_args()
    select_workload(args.workload)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.sweep:
        return run_sweep(args)
    if args.batch_probe:
        return run_batch_probe(args)
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
