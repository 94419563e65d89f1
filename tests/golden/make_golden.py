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
  fsm_domains  the same graph: MNI supports recomputed by the per-vertex
           domain search (oracle.domain_sizes) for a seeded sample of the
           frequent set (every edge and triangle, 600 wedges, 1000 paths, 1000
           stars) and of the infrequent candidates one edge away from it
           (anti-monotone extensions of frequent patterns that are not
           frequent): a second, independent oracle for the FSM workload
"""
import json
import os
import sys
import time

import numpy as np

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
    elif name == "fsm_domains":
        g = sg.workload_graph(4)
        res = fsm_domain_sample(g)
    else:
        raise SystemExit(f"unknown workload {name}")
    return {"graph": {k: v for k, v in g.meta.items() if k != "abcd"},
            "counts": {k: str(v) for k, v in res.items()},
            "oracle_seconds": round(time.time() - t, 1)}


def _key(shape, labels):
    """Canonical label tuple of a shape (the FSM output's key)."""
    if shape == "edge":
        return tuple(sorted(labels))
    if shape == "wedge":
        return (labels[0],) + tuple(sorted(labels[1:]))
    if shape == "triangle":
        return tuple(sorted(labels))
    if shape == "path":
        return min(tuple(labels), tuple(reversed(labels)))
    return (labels[0],) + tuple(sorted(labels[1:]))


def fsm_domain_sample(g, threshold=1000, seed=0x5EED0404):
    """Supports by oracle.domain_sizes for a seeded sample of frequent
    patterns and of infrequent one-edge extensions of frequent ones."""
    data = json.load(open(OUT))
    freq = {}
    for key in data["fsm"]["counts"]:
        shape, labels = key.split(":")
        freq[(shape, tuple(int(x) for x in labels.split(",")))] = True
    L = 20
    edges = [k for k in freq if k[0] == "edge"]
    wedges = [k for k in freq if k[0] == "wedge"]
    cand = set()
    for (_, (x, y)) in edges:  # wedges from two frequent edges sharing the centre
        for c, a in ((x, y), (y, x)):
            for b in range(L):
                if ("edge", _key("edge", (c, b))) in freq:
                    cand.add(("wedge", _key("wedge", (c, a, b))))
    for (_, (c, x, y)) in wedges:  # 3-edge extensions of a frequent wedge
        for z in range(L):
            cand.add(("star", _key("star", (c, x, y, z))))
            cand.add(("path", _key("path", (z, x, c, y))))
            cand.add(("path", _key("path", (x, c, y, z))))
        cand.add(("triangle", _key("triangle", (c, x, y))))
    infrequent = sorted(k for k in cand if k not in freq)
    rng = np.random.default_rng(seed)

    def pick(pool, n):
        pool = sorted(pool)
        if len(pool) <= n:
            return pool
        return [pool[i] for i in sorted(rng.choice(len(pool), n, replace=False))]

    sample = (pick([k for k in freq if k[0] in ("edge", "triangle")], 10 ** 9)
              + pick([k for k in freq if k[0] == "wedge"], 600)
              + pick([k for k in freq if k[0] == "path"], 1000)
              + pick([k for k in freq if k[0] == "star"], 1000))
    sample += (pick([k for k in infrequent if k[0] in ("wedge", "triangle")], 400)
               + pick([k for k in infrequent if k[0] == "path"], 500)
               + pick([k for k in infrequent if k[0] == "star"], 500))
    out = {}
    for i, (shape, labels) in enumerate(sample):
        s = oracle.mni_support(g, oracle.fsm_pattern(shape, labels))
        out[f"{shape}:{','.join(map(str, labels))}"] = s
        if i % 500 == 0:
            print(f"  fsm_domains {i}/{len(sample)}", flush=True)
    return out


if __name__ == "__main__":
    names = sys.argv[1:] or ["motif3", "cliques", "motif4", "fsm", "fsm_domains"]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data["_about"] = ("Expected counts written by tests/golden/make_golden.py from the oracle "
                      "only; counts are decimal strings (exact).")
    for n in names:
        data[n] = run(n)
        print(n, data[n], flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
