"""Write the expected per-graph results of the multi-graph workloads, computed
by the CPU oracle only, one graph per host core:

  batch4096_results.txt   every graph of the batched workload
                          (synth.batch_graphs(4096): capped G(n, p), n in
                          [32, 512], p in [0.2, 0.8], seeds 0..4095)
  served2000_results.txt  the first 2,000 requests of the served workload
                          (synth.served_graph(r), r = 0..1999: capped G(n, p),
                          n log-uniform in [64, 2048], p in [0.1, 0.9])

Per graph:  index n m count hash nodes internal dead_ends hist
  count / hist / hash           oracle.tomita  (Alg. 2 with the Tomita pivot)
  nodes / internal / dead_ends  oracle.ordered (Alg. 4 with the GreedyBB
                                pivot and the order of Section 4.2)
  hist                          k:v pairs of the non-zero buckets

Usage: python tests/golden/make_workload_golden.py [batch|served ...]
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

FILES = {"batch": ("batch4096_results.txt", 4096), "served": ("served2000_results.txt", 2000)}


def _one(job):
    kind, i = job
    import oracle
    import synth
    s = synth.batch_graph(i) if kind == "batch" else synth.served_graph(i)
    ref = oracle.tomita(s.n, s.uv)
    tree = oracle.ordered(s.n, s.uv, "greedy")
    assert (tree["count"], tree["hash"]) == (ref["count"], ref["hash"])
    hist = ",".join(f"{k}:{int(v)}" for k, v in enumerate(ref["hist"]) if v)
    return (f"{i} {s.n} {s.uv.shape[0]} {ref['count']} {ref['hash']} {tree['nodes']} {tree['internal']} "
            f"{tree['dead_ends']} {hist}")


def main(kinds):
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count() or 4) as pool:
        for kind in kinds:
            name, count = FILES[kind]
            t = time.time()
            lines = pool.map(_one, [(kind, i) for i in range(count)], chunksize=4)
            with open(os.path.join(HERE, name), "w") as f:
                f.write(f"# {name}: written by make_workload_golden.py from the CPU oracle only\n")
                f.write("# index n m count hash nodes internal dead_ends hist(k:v,...)\n")
                f.write("\n".join(lines) + "\n")
            print(kind, count, f"{time.time() - t:.1f}s", flush=True)


def load(kind):
    """Parsed rows of a stored file: dicts with the fields above (hist as a
    {size: count} dict)."""
    name, _ = FILES[kind]
    rows = []
    for line in open(os.path.join(HERE, name)):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        rows.append({"index": int(t[0]), "n": int(t[1]), "m": int(t[2]), "count": int(t[3]), "hash": int(t[4]),
                     "nodes": int(t[5]), "internal": int(t[6]), "dead_ends": int(t[7]),
                     "hist": {int(a): int(b) for a, b in (x.split(":") for x in t[8].split(","))}})
    return rows


if __name__ == "__main__":
    main(sys.argv[1:] or list(FILES))
