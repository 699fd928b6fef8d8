"""GPU parity of categorical PQQA for graph colouring (App. B, App. C.4): the
CUDA path through the C ABI (qqa_color_*) against the FP64 oracle on the same
seeded inputs. The initial draw and the rounding (argmax, conflict counts,
best replica) must be bit-exact; a single step is compared element by element
within the propagated FP32 bound of tests/parity.py; whole anneals reach the
conflict counts of Table 6 like the oracle does."""
import os

import numpy as np
import pytest

import oracle
import paper_2409_02135_gb300 as qqa
from parity import as_f32, assert_within, step_tolerance
from qqa_inputs import graphs as G
from qqa_inputs.workloads import FP32, Params

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_02135_gb300 import _build
    _build.build()
    import torch
    assert torch.cuda.is_available()


def _table6():
    rows = {}
    with open(os.path.join(GOLDEN, "paper_color_graphs.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, gen, nodes, edges, colours, conflicts = line.split()
                rows[name] = (gen, int(colours), int(conflicts))
    return rows


def _graph(gen):
    parts = gen.split(":")
    return G.mycielski(int(parts[1])) if parts[0] == "mycielski" else G.queens(int(parts[1]), int(parts[2]))


def _check_step(g, K, p, c):
    W0, m0, v0, t = c.get_state()
    grad = c.step_debug()
    W1, m1, v1, t1 = c.get_state()
    assert t1 == t + 1
    po = as_f32(p)
    out = oracle.color_step(g, K, po, t, W0.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64))
    tg, tm, tv, tp = step_tolerance(po, FP32, t, W0.astype(np.float64), m0.astype(np.float64),
                                    v0.astype(np.float64), out)
    assert_within("gradient", grad, out.grad, tg)
    assert_within("m", m1, out.m, tm)
    assert_within("v", v1, out.v, tv)
    assert_within("W", W1, out.X, tp)


@pytest.mark.parametrize("K,S", [(3, 1), (5, 37), (13, 64), (32, 300)])
def test_color_init_is_the_oracle_draw(K, S):
    g = G.erdos_renyi(41, 0.2, 5)
    p = Params(S=S, steps=10, seed=0xC0FFEE123456789, precision=FP32)
    c = qqa.Coloring(g, K, qqa.make_params(p))
    W, m, v, t = c.get_state()
    assert t == 0 and not m.any() and not v.any()
    np.testing.assert_array_equal(W.astype(np.float64), oracle.color_init(g.n, K, S, p.seed))


@pytest.mark.parametrize("gen,K", [("queens:5:5", 5), ("mycielski:4", 5), ("queens:6:6", 7), ("queens:8:12", 12),
                                   ("queens:13:13", 13), ("er", 20), ("er_large", 6)])
@pytest.mark.parametrize("S", [8, 37, 300])
def test_color_single_step_matches_oracle(gen, K, S):
    """Cold moments at t = 0, warm moments at t = 60, with the communication term on.
    The dense graph of 112 nodes or more (queen13-13) takes the tensor-core
    neighbour sums, the other small graphs the shared-memory ones, the sparse
    2000-node graph the direct gather."""
    if gen == "er_large":
        g = G.erdos_renyi(2000, 0.005, 9)
    else:
        g = G.erdos_renyi(60, 0.15, 8) if gen == "er" else _graph(gen)
    p = Params(S=S, steps=400, lr=0.1, alpha_comm=0.3, seed=11, precision=FP32)
    c = qqa.Coloring(g, K, qqa.make_params(p))
    _check_step(g, K, p, c)
    c.steps(59)
    _check_step(g, K, p, c)


@pytest.mark.parametrize("gen,K", [("queens:13:13", 13), ("queens:8:12", 12), ("er_large", 6)])
def test_color_single_step_at_the_bench_replica_count(gen, K):
    """S = 1024, the replica count the colouring benchmark runs: all eight
    128-replica chunks of the carried partial sums of sigma, for the
    tensor-core, shared-memory and direct neighbour sums."""
    g = G.erdos_renyi(2000, 0.005, 9) if gen == "er_large" else _graph(gen)
    p = Params(S=1024, steps=3000, lr=0.1, alpha_comm=0.3, seed=12, precision=FP32)
    c = qqa.Coloring(g, K, qqa.make_params(p))
    _check_step(g, K, p, c)
    c.steps(30)
    _check_step(g, K, p, c)


def test_color_graph_replay_equals_single_launches():
    """Chunks of steps replayed from a captured CUDA graph (the step index read
    from the device counter) give the same state, bit for bit, as the same
    steps launched one at a time, for the shared-memory, tensor-core and
    direct neighbour sums."""
    for g, K in ((G.queens(6, 6), 7), (G.queens(11, 11), 11), (G.erdos_renyi(1700, 0.004, 2), 5)):
        p = Params(S=96, steps=200, lr=0.1, alpha_comm=0.2, seed=4, precision=FP32)
        a = qqa.Coloring(g, K, qqa.make_params(p))
        b = qqa.Coloring(g, K, qqa.make_params(p))
        assert a.steps(70) == 70
        for _ in range(70):
            b.steps(1)
        for x, y in zip(a.get_state(), b.get_state()):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("a_ent,alpha,T", [(2, 0.0, 1e-3), (4, 1.0, 0.0), (6, 0.5, 1e-3), (8, 0.0, 1e-3)])
def test_color_single_step_entropy_exponents_alpha_and_temperature(a_ent, alpha, T):
    g = G.queens(7, 7)
    p = Params(S=64, steps=100, lr=0.1, a_ent=a_ent, alpha_comm=alpha, temperature=T, seed=21, precision=FP32)
    c = qqa.Coloring(g, 7, qqa.make_params(p))
    _check_step(g, 7, p, c)
    c.steps(30)
    _check_step(g, 7, p, c)


def test_color_step_from_planted_state_with_zero_and_saturated_rows():
    """A state with rows of zeros (sigma = 1/K, gradient 0), rows at the upper
    bound and converged replicas (STD close to sqrt(eps)) steps like the oracle."""
    g = G.queens(5, 5)
    K, S = 5, 40
    rng = np.random.default_rng(4)
    W = rng.random((g.n, K, S)).astype(np.float32)
    W[0] = 0.0
    W[1] = 1.0
    W[2, :, :] = W[2, :, :1]                    # all replicas equal at node 2
    W[3, :, 5] = 0.0
    m = (rng.standard_normal((g.n, K, S)) * 0.01).astype(np.float32)
    v = (rng.random((g.n, K, S)) * 1e-3).astype(np.float32)
    p = Params(S=S, steps=100, lr=0.1, alpha_comm=0.5, seed=5, precision=FP32)
    c = qqa.Coloring(g, K, qqa.make_params(p))
    c.set_state(W, m, v, 17)
    _check_step(g, K, p, c)


@pytest.mark.parametrize("K,S", [(4, 33), (9, 128), (32, 7)])
def test_color_rounding_is_exact(K, S):
    """argmax with ties to the lowest colour, conflicts per replica and the best
    replica are identical to the oracle's, on states with planted ties."""
    g = G.erdos_renyi(150, 0.05, 13)
    rng = np.random.default_rng(K * 100 + S)
    W = (rng.integers(0, 4, size=(g.n, K, S)) / 4.0).astype(np.float32)   # many exact ties
    W[::7] = 0.0                                                            # zero rows -> colour 0
    p = Params(S=S, steps=10, seed=3, precision=FP32)
    c = qqa.Coloring(g, K, qqa.make_params(p))
    c.set_state(W, np.zeros_like(W), np.zeros_like(W), 0)
    r = c.round()
    x, conf, best = oracle.color_round(g, K, W.astype(np.float64))
    np.testing.assert_array_equal(r["x"].astype(np.int32), x)
    np.testing.assert_array_equal(r["conflicts"], conf)
    assert r["best_s"] == best


def test_color_anneal_rounding_matches_oracle_rounding_of_the_same_state():
    g = G.queens(8, 8)
    p = Params(S=96, steps=300, lr=0.1, seed=2, precision=FP32)
    c, r = qqa.color_anneal(g, 9, qqa.make_params(p))
    W, _, _, t = c.get_state()
    assert t == 300
    x, conf, best = oracle.color_round(g, 9, W.astype(np.float64))
    np.testing.assert_array_equal(r["x"].astype(np.int32), x)
    np.testing.assert_array_equal(r["conflicts"], conf)
    assert r["best_s"] == best


@pytest.mark.parametrize("name", ["queen5-5", "queen6-6", "myciel5"])
def test_color_anneal_reaches_the_papers_conflicts(name):
    """At the oracle pin's settings (S = 32, 2000 steps) the GPU anneal reaches
    the conflicts PQQA reports in Table 6."""
    gen, K, want = _table6()[name]
    g = _graph(gen)
    _, r = qqa.color_anneal(g, K, qqa.make_params(Params(S=32, steps=2000, seed=1, lr=0.1, precision=FP32)))
    assert r["conflicts"][r["best_s"]] <= want


def test_color_quality_matches_oracle_over_seeds():
    """Best conflicts on queen7-7 with 7 colours (S = 32, 2000 steps) over 8 seeds:
    the GPU's mean is within one conflict of the oracle's."""
    g = G.queens(7, 7)
    gpu, ora = [], []
    for seed in range(8):
        p = Params(S=32, steps=2000, seed=seed, lr=0.1, precision=FP32)
        _, r = qqa.color_anneal(g, 7, qqa.make_params(p))
        gpu.append(int(r["conflicts"][r["best_s"]]))
        conf, best, _, _ = oracle.color_anneal(g, 7, as_f32(p))
        ora.append(int(conf[best]))
    assert np.mean(gpu) <= np.mean(ora) + 1.0, (gpu, ora)


def test_color_rejects_bad_arguments():
    g = G.queens(4, 4)
    with pytest.raises(qqa.QQAError):
        qqa.Coloring(g, 1, qqa.make_params(Params(S=8, steps=10)))
    with pytest.raises(qqa.QQAError):
        qqa.Coloring(g, 33, qqa.make_params(Params(S=8, steps=10)))
    c = qqa.Coloring(g, 4, qqa.make_params(Params(S=8, steps=10)))
    bad = np.full((g.n, 4, 8), 0.5, np.float32)
    bad[0, 0, 0] = 1.5
    z = np.zeros_like(bad)
    with pytest.raises(qqa.QQAError):
        c.set_state(bad, z, z, 0)
    assert c.steps(100) == 10 and c.t == 10 and c.steps(5) == 0
