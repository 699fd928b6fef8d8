"""Workload recipes: seeded graphs plus hyper-parameters for each configuration.

Hyper-parameters follow the paper where it states them (Sec. 5 "Implementation",
App. C.2, App. C.3): alpha-entropy exponent 4, gamma from -2 to 0.1 (max-cut:
-20 on large graphs, -5 otherwise), weight decay 0.01, temperature 1e-3,
penalty 2 (App. D.1). The learning rate is one of {1, 0.1, 0.01} in the paper,
chosen per problem; an oracle sweep on ER(n~U[700,800], 0.15) MIS (4 graphs x
2 seeds, S = 128, 3000 steps) gave mean best sizes 44.25 / 43.25 / 41.25 for
1 / 0.1 / 0.01, and on max-cut (random 3-regular n = 2000 and BA(1100, 4),
S = 64, 2000 steps) lr 1 beat 0.1 and 0.01 as well, so every recipe uses 1
(RECIPE_LR). AdamW's beta1, beta2 and eps are not
stated; PyTorch's defaults are used. The communication strength alpha is not
printed (Fig. 4 has no values); see DEFAULT_ALPHA_COMM.

No number here is computed by the method: these are inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from . import graphs as G

MIS, MAXCUT, MAXCLIQUE = 0, 1, 2
FP32, BF16 = 0, 1

# Communication strength alpha (Eq. 10). The paper gives no value; an oracle
# sweep over {0, 0.1, 0.3, 1} on the ER MIS shape above gave 43.1 / 43.3 / 43.0
# at lr 0.1 (alpha = 1 left most rounded replicas infeasible) and 44.0 / 44.25
# for alpha 0 / 0.1 at lr 1.
DEFAULT_ALPHA_COMM = 0.1
RECIPE_LR = 1.0


@dataclass
class Params:
    S: int = 128
    steps: int = 3000
    round_every: int = 50
    a_ent: int = 4
    lr: float = 0.1
    weight_decay: float = 0.01
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-8
    gamma_min: float = -2.0
    gamma_max: float = 0.1
    alpha_comm: float = DEFAULT_ALPHA_COMM
    comm_eps: float = 1e-8
    temperature: float = 1e-3
    lam: float = 2.0
    seed: int = 0
    precision: int = FP32

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


@dataclass
class Instance:
    kind: int
    graph: G.CSRGraph
    params: Params
    name: str = ""


@dataclass
class Workload:
    name: str
    instances: list = field(default_factory=list)
    description: str = ""

    @property
    def replica_steps(self) -> int:
        return sum(inst.params.S * inst.params.steps for inst in self.instances)

    @property
    def element_steps(self) -> int:
        return sum(inst.graph.n * inst.params.S * inst.params.steps for inst in self.instances)


def er_mis_small(seed: int = 0) -> Workload:
    """MIS on one G(n=100, p=0.05) graph, S=8, 1000 steps, FP32."""
    g = G.erdos_renyi(100, 0.05, seed)
    p = Params(S=8, steps=1000, seed=0, lr=RECIPE_LR)
    return Workload("mis_er100_S8_K1000", [Instance(MIS, g, p, "er100")],
                    "MIS, ER G(100,0.05) seed 0, lambda 2, S=8, 1000 steps, FP32")


def er_mis_paper(num_graphs: int = 16, S: int = 128, steps: int = 3000, base_seed: int = 1000,
                 run_seed: int = 0, precision: int = FP32) -> Workload:
    """MIS on ER graphs shaped like ER-[700-800] (Sec. 5.1; Table 7: n in [700, 800],
    edge density implied by 47,885 edges at 800 nodes, p = 0.15)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x57524B31, base_seed]))
    ns = rng.integers(700, 801, size=num_graphs)
    insts = []
    for k in range(num_graphs):
        g = G.erdos_renyi(int(ns[k]), 0.15, base_seed + k)
        insts.append(Instance(MIS, g, Params(S=S, steps=steps, seed=run_seed, precision=precision, lr=RECIPE_LR),
                              f"er{int(ns[k])}_{k}"))
    return Workload(f"mis_er700-800_x{num_graphs}_S{S}_K{steps}", insts,
                    f"MIS, {num_graphs} ER graphs n~U[700,800], p=0.15, S={S}, {steps} steps")


def rrg_mis(n: int = 100_000, d: int = 20, steps: int = 3000, num_graphs: int = 5, base_seed: int = 3000,
            run_seed: int = 0, precision: int = FP32) -> Workload:
    """MIS on random d-regular graphs with a single replica (S = 1), the setting of
    the paper's RRG study (Sec. 5.1, regular random graphs: d = 20 and 100, n from
    1e4 to 1e6, five graphs, 3000 or 30000 steps). The quality measure is the
    independence density |IS| / n."""
    insts = []
    for k in range(num_graphs):
        g = G.random_regular(n, d, base_seed + k)
        insts.append(Instance(MIS, g, Params(S=1, steps=steps, seed=run_seed + k, precision=precision, lr=RECIPE_LR),
                              f"rrg{d}_{n}_{k}"))
    return Workload(f"mis_rrg_d{d}_n{n}_x{num_graphs}_S1_K{steps}", insts,
                    f"{num_graphs} MIS random {d}-regular graphs, n={n}, S=1, {steps} steps")


def maxcut_large(n: int = 100_000, S: int = 256, steps: int = 5000, family: str = "regular3",
                 seed: int = 7, run_seed: int = 0, precision: int = BF16) -> Workload:
    """Max-cut on a random 3-regular or Barabasi-Albert (m=4) graph with unit
    weights (Sec. 5.3; BA m=4 from Table 7: 4,384 edges at 1,100 nodes);
    gamma_min = -20 for large graphs (App. C.2)."""
    if family == "regular3":
        g = G.random_regular(n, 3, seed)
    elif family == "ba4":
        g = G.barabasi_albert(n, 4, seed)
    else:
        raise ValueError(family)
    gmin = -20.0 if n >= 10_000 else -5.0
    p = Params(S=S, steps=steps, gamma_min=gmin, seed=run_seed, precision=precision, lr=RECIPE_LR)
    return Workload(f"maxcut_{family}_n{n}_S{S}_K{steps}", [Instance(MAXCUT, g, p, family)],
                    f"max-cut, {family}, n={n}, unit weights, S={S}, {steps} steps")


def batched_mis(num: int = 512, S: int = 64, steps: int = 2000, base_seed: int = 5000,
                run_seed: int = 0, precision: int = BF16) -> Workload:
    """Many uneven MIS instances from the clique-block generator (n in [200, 1200],
    cliques of 5-25 nodes, inter-clique edge probability 0.02)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x42415443, base_seed]))
    ns = rng.integers(200, 1201, size=num)
    insts = []
    for k in range(num):
        g = G.clique_blocks(int(ns[k]), base_seed + k)
        insts.append(Instance(MIS, g, Params(S=S, steps=steps, seed=run_seed + k, precision=precision, lr=RECIPE_LR),
                              f"cb{int(ns[k])}_{k}"))
    return Workload(f"mis_cliqueblocks_x{num}_S{S}_K{steps}", insts,
                    f"{num} MIS clique-block instances, n~U[200,1200], S={S}, {steps} steps")


@dataclass
class Request:
    arrival_s: float
    instance: Instance


def serving_trace(num: int = 2000, rate_per_s: float = 200.0, seed: int = 9, n_lo: float = 1e3,
                  n_hi: float = 1e6, avg_degree: float = 10.0, precision: int = BF16,
                  lazy_graphs: bool = True):
    """Poisson arrivals of mixed MIS / max-cut requests on ER graphs with average
    degree 10, n log-uniform in [n_lo, n_hi], S in {32, 64, 128, 256},
    steps uniform in [1000, 5000]. Graphs are generated on demand when
    lazy_graphs is set (returned as (kind, n, graph_seed) specs)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x53525645, seed]))
    gaps = rng.exponential(1.0 / rate_per_s, size=num)
    arrivals = np.cumsum(gaps)
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=num)).astype(np.int64)
    kinds = rng.integers(0, 2, size=num)  # 0 = MIS, 1 = max-cut
    Ss = rng.choice(np.array([32, 64, 128, 256]), size=num)
    Ks = rng.integers(1000, 5001, size=num)
    gseeds = rng.integers(0, 2**31, size=num)
    out = []
    for k in range(num):
        kind = MIS if kinds[k] == 0 else MAXCUT
        gmin = -2.0 if kind == MIS else (-20.0 if ns[k] >= 10_000 else -5.0)
        p = Params(S=int(Ss[k]), steps=int(Ks[k]), gamma_min=gmin, seed=int(k), precision=precision,
                   lr=RECIPE_LR)
        spec = (kind, int(ns[k]), float(avg_degree), int(gseeds[k]))
        out.append((float(arrivals[k]), spec, p))
    return out


def graph_from_spec(spec) -> G.CSRGraph:
    kind, n, avg_degree, gseed = spec
    return G.erdos_renyi_avg_degree(n, avg_degree, gseed)


# Graph colouring instances of the paper's Table 9 that have a definition
# (Mycielski and queens graphs; the book graphs are dataset files): name,
# generator and the number of colours K the paper runs them with.
COLOR_GRAPHS = [
    ("myciel5", lambda: G.mycielski(5), 6),
    ("myciel6", lambda: G.mycielski(6), 7),
    ("queen5-5", lambda: G.queens(5, 5), 5),
    ("queen6-6", lambda: G.queens(6, 6), 7),
    ("queen7-7", lambda: G.queens(7, 7), 7),
    ("queen8-8", lambda: G.queens(8, 8), 9),
    ("queen9-9", lambda: G.queens(9, 9), 10),
    ("queen8-12", lambda: G.queens(8, 12), 12),
    ("queen11-11", lambda: G.queens(11, 11), 11),
    ("queen13-13", lambda: G.queens(13, 13), 13),
]
