"""Write the FP64 oracle's final best objective per seed for a quality set.

Runs only the FP64 oracle (oracle/) on the seeded inputs of qqa_inputs. The
files it writes are the targets of the GPU quality tests (best feasible
objective per instance, mean over seeds, within 1% of the oracle's) and of
bench.py's time-to-oracle-quality figure.

    python tests/golden/make_oracle_quality.py mis_er700_800 4
    python tests/golden/make_oracle_quality.py mis_er700_800_s16
    python tests/golden/make_oracle_quality.py maxcut_regular3_n10000

Each set names a workload recipe, the instances it takes and the number of
oracle seeds (run seed 1000 + k for seed k). The output is rewritten after
every seed, so an interrupted run keeps what it finished and a rerun resumes.

Long sets can run their seeds in parallel processes: `--seed k` computes run
k of a single-instance set alone into oracle_quality_<set>.seed<k>.json, and
the main mode takes such a file in place of computing that run (and removes
it once the run is in the set's file).

    python tests/golden/make_oracle_quality.py maxcut_regular3_n100000 --seed 3
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


def _er_paper():
    return W.er_mis_paper(num_graphs=16, S=128, steps=3000, base_seed=1000)


def _ablation(**kw):
    """The first ER-[700-800]-shaped graph with one ablation setting changed
    (Sec. 6: schedule length, initial gamma, communication strength)."""
    inst = _er_paper().instances[0]
    p = inst.params.with_(**kw)
    tag = "_".join(f"{k}{v}" for k, v in kw.items())
    return W.Workload(f"ablation_{tag}_{inst.name}_S{p.S}", [W.Instance(inst.kind, inst.graph, p, inst.name)])


# name -> (workload factory, default seeds, instances taken (None = all))
SETS = {
    "mis_er100": (W.er_mis_small, 4, None),
    "mis_er700_800": (_er_paper, 4, None),
    "mis_er700_800_s16": (_er_paper, 16, 6),
    "maxcut_regular3_n10000": (lambda: W.maxcut_large(n=10_000, family="regular3"), 16, None),
    "maxcut_ba4_n10000": (lambda: W.maxcut_large(n=10_000, family="ba4"), 16, None),
    "maxcut_regular3_n100000": (lambda: W.maxcut_large(n=100_000, family="regular3"), 4, None),
    "maxcut_ba4_n100000": (lambda: W.maxcut_large(n=100_000, family="ba4"), 4, None),
    "ablation_K100": (lambda: _ablation(steps=100), 16, None),
    "ablation_gamma0_0": (lambda: _ablation(gamma_min=0.0), 16, None),
    "ablation_alpha1": (lambda: _ablation(alpha_comm=1.0), 16, None),
}


def _one_run(inst, seed):
    """Run `seed` of an instance: best feasible objective, feasible count, lowest energy."""
    r = oracle.anneal(inst.kind, inst.graph, inst.params.with_(seed=1000 + seed))
    e = r.eval
    return (int(e.obj[e.best]) if e.best >= 0 else None, int(np.count_nonzero(e.feasible)),
            float(np.min(e.energy)))


def main():
    args = [a for a in sys.argv[1:]]
    only = None
    if "--seed" in args:
        k = args.index("--seed")
        only = int(args[k + 1])
        del args[k:k + 2]
    name = args[0] if args else "mis_er700_800"
    factory, seeds, take = SETS[name]
    if len(args) > 1:
        seeds = int(args[1])
    wl = factory()
    insts = wl.instances if take is None else wl.instances[:take]
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, f"oracle_quality_{name}.json")
    part = lambda k: os.path.join(here, f"oracle_quality_{name}.seed{k}.json")  # noqa: E731
    if only is not None:   # one run of a single-instance set, for a parallel process
        assert len(insts) == 1, "--seed is for single-instance sets"
        best, feas, emin = _one_run(insts[0], only)
        with open(part(only) + ".tmp", "w") as f:
            json.dump({"set": name, "name": insts[0].name, "seed": only, "oracle_best": best,
                       "oracle_feasible": feas, "oracle_min_energy": emin}, f, indent=1)
        os.replace(part(only) + ".tmp", part(only))
        print(name, insts[0].name, only, best, "(part file)", flush=True)
        return
    done = {}
    if os.path.exists(path):
        for rec in json.load(open(path)).get("instances", []):
            done[rec["name"]] = rec
    out = {"workload": wl.name, "set": name, "seeds": seeds, "threads": oracle.num_threads(),
           "oracle_seed": "1000 + k", "instances": []}

    def write():
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(out, f, indent=1)
        os.replace(tmp, path)

    for inst in insts:
        p0 = inst.params
        rec = done.get(inst.name)
        if rec is None or "oracle_min_energy" not in rec:
            rec = {"name": inst.name, "n": inst.graph.n, "nnz": inst.graph.nnz, "kind": inst.kind, "S": p0.S,
                   "steps": p0.steps, "gamma_min": p0.gamma_min, "alpha_comm": p0.alpha_comm,
                   "precision_of_recipe": "fp32" if p0.precision == W.FP32 else "bf16",
                   "oracle_best": [], "oracle_feasible": [], "oracle_min_energy": []}
        out["instances"].append(rec)
        for seed in range(len(rec["oracle_best"]), seeds):
            t0 = time.time()
            pf = part(seed)
            if len(insts) == 1 and os.path.exists(pf):   # computed by a parallel process
                with open(pf) as f:
                    got = json.load(f)
                assert got["set"] == name and got["seed"] == seed
                best, feas, emin = got["oracle_best"], got["oracle_feasible"], got["oracle_min_energy"]
            else:
                best, feas, emin = _one_run(inst, seed)
                pf = None
            rec["oracle_best"].append(best)
            rec["oracle_feasible"].append(feas)
            rec["oracle_min_energy"].append(emin)
            ok = [b for b in rec["oracle_best"] if b is not None]
            rec["oracle_mean_best"] = float(np.mean(ok)) if ok else None
            rec["oracle_mean_min_energy"] = float(np.mean(rec["oracle_min_energy"]))
            write()
            if pf:
                os.remove(pf)
            print(name, inst.name, seed, rec["oracle_best"][-1], f"{time.time() - t0:.1f}s", flush=True)
        ok = [b for b in rec["oracle_best"] if b is not None]
        rec["oracle_mean_best"] = float(np.mean(ok)) if ok else None
        rec["oracle_mean_min_energy"] = float(np.mean(rec["oracle_min_energy"])) if rec["oracle_min_energy"] else None
    write()
    print("wrote", path)


if __name__ == "__main__":
    main()
