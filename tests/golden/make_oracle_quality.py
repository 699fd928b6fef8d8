"""Write the oracle's mean final best objective per instance of a workload.

Runs only the FP64 oracle (oracle/) on the seeded inputs of qqa_inputs; the
output file is the target of bench.py's time-to-oracle-quality figure (the
time until an instance's best feasible objective reaches 99% of this mean).

    python tests/golden/make_oracle_quality.py mis_er700_800 4
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from qqa_inputs import workloads as W  # noqa: E402


def workload(name):
    if name == "mis_er700_800":
        return W.er_mis_paper(num_graphs=16, S=128, steps=3000, base_seed=1000)
    if name == "mis_er100":
        return W.er_mis_small()
    raise SystemExit(f"unknown workload {name}")


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else "mis_er700_800"
    seeds = int(sys.argv[2]) if len(sys.argv) > 2 else 4
    wl = workload(name)
    out = {"workload": wl.name, "seeds": seeds, "threads": oracle.num_threads(), "instances": []}
    for inst in wl.instances:
        t0 = time.time()
        bests = []
        for seed in range(seeds):
            r = oracle.anneal(inst.kind, inst.graph, inst.params.with_(seed=1000 + seed))
            bests.append(int(r.eval.obj[r.eval.best]) if r.eval.best >= 0 else None)
        ok = [b for b in bests if b is not None]
        out["instances"].append({"name": inst.name, "n": inst.graph.n, "nnz": inst.graph.nnz,
                                 "oracle_best": bests, "oracle_mean_best": float(np.mean(ok)) if ok else None})
        print(inst.name, bests, f"{time.time() - t0:.1f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_quality_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
