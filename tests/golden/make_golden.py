"""Write the full-size expected counts of the benchmark workloads.

Calls only the oracle (and the shared seeded generators).  Run from the
repository root:

    python tests/golden/make_golden.py [workload ...]

and commit the resulting workload_counts.json.  Workloads:
  motif3   ER G(2000, 0.005): induced triangles and wedges
  cliques  Chung-Lu 1M / 10M, gamma 2.1: 3-, 4- and 5-cliques
  motif4   R-MAT scale 20, edge factor 16: the six induced 4-vertex motifs
  fsm      Chung-Lu 500K / 5M, gamma 2.3, Zipf(1.2) labels over 20: frequent
           labeled patterns with 1..3 edges, MNI support >= 1000
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synthgraph as sg  # noqa: E402

OUT = os.path.join(HERE, "workload_counts.json")


def run(name):
    t = time.time()
    if name == "motif3":
        g = sg.workload_graph(1)
        res = {"induced_triangle": oracle.triangles(g), "induced_wedge": oracle.wedges_induced(g)}
    elif name == "cliques":
        g = sg.workload_graph(2)
        res = {f"{k}-clique": oracle.kcliques(g, k) for k in (3, 4, 5)}
    elif name == "motif4":
        g = sg.workload_graph(3)
        res = {f"induced_{k}": v for k, v in oracle.motif4_induced(g).items()}
    elif name == "fsm":
        g = sg.workload_graph(4)
        freq = oracle.fsm(g, 20, 1000)
        res = {f"{shape}:{','.join(map(str, labels))}": v for (shape, labels), v in sorted(freq.items())}
    else:
        raise SystemExit(f"unknown workload {name}")
    return {"graph": {k: v for k, v in g.meta.items() if k != "abcd"},
            "counts": {k: str(v) for k, v in res.items()},
            "oracle_seconds": round(time.time() - t, 1)}


if __name__ == "__main__":
    names = sys.argv[1:] or ["motif3", "cliques", "motif4", "fsm"]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data["_about"] = ("Expected counts written by tests/golden/make_golden.py from the oracle "
                      "only; counts are decimal strings (exact).")
    for n in names:
        data[n] = run(n)
        print(n, data[n], flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
