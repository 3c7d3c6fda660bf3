"""Write tests/golden/config_results.json: expected results of the full-size
workloads, computed by the CPU oracle only.

  count / hist / hash      oracle.tomita  (Alg. 2 with the Tomita pivot)
  nodes / internal / dead  oracle.ordered (Alg. 4, each pivot rule, with the
                           maximum-degree-first order of Section 4.2)

Workloads (seeded, from synth):
  gnp_100_0.5_s0    G(100, 0.5), seed 0
  gnp_1000_0.3_s1   G(1000, 0.3), seed 1   (Table 1's n = 1000, p = 0.3 shape)
  moon_moser_45     complement of 15 disjoint triangles (closed form 3^15)
  moon_moser_45_del5  the same with round(0.05 * 945) = 47 edges removed, seed 3

Usage: python tests/golden/make_config_golden.py [name ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

WORKLOADS = {
    "gnp_100_0.5_s0": lambda: (100, synth.gnp(100, 0.5, 0)),
    "gnp_1000_0.3_s1": lambda: (1000, synth.gnp(1000, 0.3, 1)),
    "moon_moser_45": lambda: (45, synth.moon_moser(15)),
    "moon_moser_45_del5": lambda: (45, synth.moon_moser_deleted(15, 0.05, 3)),
}

OUT = os.path.join(HERE, "config_results.json")


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        n, uv = WORKLOADS[name]()
        t = time.time()
        ref = oracle.tomita(n, uv)
        t_tomita = time.time() - t
        entry = {"n": n, "m": int(uv.shape[0]), "count": ref["count"], "hash": ref["hash"],
                 "hist": {str(k): int(v) for k, v in enumerate(ref["hist"]) if v},
                 "tomita_nodes": ref["nodes"], "oracle_seconds": {"bk_tomita": round(t_tomita, 2)}}
        for mode in ("greedy", "tx", "tomita"):
            t = time.time()
            r = oracle.ordered(n, uv, mode)
            assert (r["count"], r["hash"]) == (ref["count"], ref["hash"])
            entry[mode] = {"nodes": r["nodes"], "internal": r["internal"], "dead_ends": r["dead_ends"]}
            entry["oracle_seconds"][mode] = round(time.time() - t, 2)
        data[name] = entry
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(name, entry["count"], entry["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
