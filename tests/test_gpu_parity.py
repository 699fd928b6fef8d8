"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
identical seeded inputs. Single steps are compared element by element within
the propagated FP32 / BF16 bound of tests/parity.py; integer costs, feasibility
and best replicas must be bit-exact."""
import numpy as np
import pytest

import oracle
import paper_2409_02135_gb300 as qqa
from parity import as_f32, assert_within, make_run, step_tolerance, RTOL
from qqa_inputs import graphs as G
from qqa_inputs.workloads import MIS, MAXCUT, MAXCLIQUE, FP32, BF16, Params

pytestmark = pytest.mark.gpu

KIND_NAMES = {MIS: "mis", MAXCUT: "cut", MAXCLIQUE: "clique"}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_02135_gb300 import _build
    _build.build()
    import torch
    assert torch.cuda.is_available()


def _graph(kind, n, p, seed, weighted=False):
    g = G.erdos_renyi(n, p, seed)
    if weighted:
        rng = np.random.default_rng(seed)
        u, v, _ = g.upper_edges()
        g = G.from_edges(n, u, v, rng.integers(-2, 5, size=u.size))
    return g


def _check_step(kind, g, p, prec, run, slot=0, rows=None):
    """GPU step from the run's current state vs the oracle step from the same state."""
    X0, m0, v0, t = run.get_state(slot)
    grad = run.step_debug(slot)
    X1, m1, v1, t1 = run.get_state(slot)
    assert t1 == t + 1
    po = as_f32(p)
    Xd = X0.astype(np.float64)
    if rows is None:
        out = oracle.step(kind, g, po, t, Xd, m0.astype(np.float64), v0.astype(np.float64))
        sel = slice(None)
    else:
        out = oracle.step(kind, g, po, t, Xd, m0[rows].astype(np.float64), v0[rows].astype(np.float64), rows=rows)
        sel = rows
    tg, tm, tv, tp = step_tolerance(po, prec, t, X0[sel].astype(np.float64), m0[sel].astype(np.float64),
                                    v0[sel].astype(np.float64), out)
    r = {}
    r["g"] = assert_within("gradient", grad[sel], out.grad, tg)
    r["m"] = assert_within("m", m1[sel], out.m, tm)
    r["v"] = assert_within("v", v1[sel], out.v, tv)
    r["p"] = assert_within("p", X1[sel], out.X, tp)
    return r


# ------------------------------------------------------------ init -------
@pytest.mark.parametrize("S", [13, 1])
@pytest.mark.parametrize("prec", [FP32, BF16])
def test_init_state_is_the_oracle_draw(prec, S):
    """Initial p are the same Philox uniforms on both sides (exact in FP32);
    S = 1 uses the one-value-per-node layout."""
    g = _graph(MIS, 77, 0.1, 1)
    p = Params(S=S, steps=10, seed=0xABCDEF12345, precision=prec)
    run = make_run(MIS, g, p)
    X, m, v, t = run.get_state(0)
    want = oracle.init_state(g.n, p.S, p.seed)
    assert t == 0
    np.testing.assert_array_equal(X.astype(np.float64), want)
    assert not m.any() and not v.any()


# --------------------------------------------------------- single step ---
@pytest.mark.parametrize("seed", [7, 0xFFFFFFFF00000001])
def test_noise_field_matches_oracle(seed):
    """Two steps from one state that differ only in the temperature differ by
    sqrt(2 lr T) xi (Eq. 11): the kernel's Gaussians against the oracle's Box-Muller
    draws, element by element. 192k draws include about a hundred uniforms within
    2^-10 of 1, where the radius takes its series branch."""
    n, S, t = 3000, 64, 4
    g = G.erdos_renyi(n, 0.002, 3)
    pT = Params(S=S, steps=10, lr=0.1, temperature=1e-3, alpha_comm=0.0, seed=seed, precision=FP32)
    X0 = np.full((n, S), 0.5, np.float32)
    zeros = np.zeros((n, S), np.float32)
    out = []
    for p in (pT, pT.with_(temperature=0.0)):
        run = make_run(MIS, g, p)
        run.set_state(0, X0, zeros, zeros, t)
        run.steps(1)
        out.append(run.get_state(0)[0].astype(np.float64))
    assert out[0].min() > 0.0 and out[0].max() < 1.0          # no clamping: the difference is the noise
    sigma = float(np.float32(np.sqrt(2.0 * float(np.float32(0.1)) * float(np.float32(1e-3)))))
    xi_gpu = (out[0] - out[1]) / sigma
    xi = oracle.noise_field(n, S, seed, t)
    # the fused q + sigma xi rounds once (half an ulp of [1/4, 1) is at most 2^-25), plus the
    # FP32 radius and the hardware sine/cosine (absolute error ~4e-7 times the radius)
    tol = 1.05 * 2.0 ** -25 / sigma + 1e-6 * (1.0 + 2.0 * np.abs(xi))
    assert_within("xi", xi_gpu, xi, tol)
    assert abs(xi.mean()) < 0.02 and abs(xi.std() - 1.0) < 0.01


@pytest.mark.parametrize("prec", [FP32, BF16])
@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
@pytest.mark.parametrize("S", [8, 37, 128])
def test_single_step_matches_oracle(kind, prec, S):
    g = _graph(kind, 150, 0.08, 10 + kind, weighted=(kind == MAXCUT))
    p = Params(S=S, steps=400, alpha_comm=0.3, lr=0.1, seed=3, precision=prec,
               gamma_min=-5.0 if kind == MAXCUT else -2.0)
    run = make_run(kind, g, p)
    _check_step(kind, g, p, prec, run)           # t = 0 (cold moments)
    run.steps(98)
    _check_step(kind, g, p, prec, run)           # t = 99 (warm moments)


def _interior_state(n, S, seed):
    """A state away from the clamp (p in [0.05, 0.95]) with warm moments."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.05, 0.95, size=(n, S)).astype(np.float32)
    m = rng.normal(0.0, 0.3, size=(n, S)).astype(np.float32)
    v = rng.uniform(0.01, 0.5, size=(n, S)).astype(np.float32)
    return X, m, v


KERNEL_NAMES = {qqa.KERNEL_DIRECT: "direct", qqa.KERNEL_PIPE: "pipe", qqa.KERNEL_DENSE: "dense"}


@pytest.mark.parametrize("kernel", [qqa.KERNEL_DIRECT, qqa.KERNEL_PIPE, qqa.KERNEL_DENSE],
                         ids=lambda k: KERNEL_NAMES[k])
@pytest.mark.parametrize("prec", [FP32, BF16])
@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
def test_single_step_at_schedule_endpoints(kind, prec, kernel):
    """The schedule's ends (App. C.2): the last step t = K - 1, where gamma_t =
    gamma_max > 0 (the regime that drives p to integral points), from an interior
    state with warm moments; and a one-step schedule K = 1 (gamma_0 = gamma_min)
    from the initial draw. Direct, pipelined and tensor-core steps."""
    g = _graph(kind, 200, 0.5 if kind == MAXCLIQUE else (0.2 if kernel == qqa.KERNEL_DENSE else 0.05), 90 + kind,
               weighted=(kind == MAXCUT))
    cfg = qqa.LaunchConfig(kernel=kernel)
    gmin = -5.0 if kind == MAXCUT else -2.0
    K = 300
    p = Params(S=64, steps=K, alpha_comm=0.3, lr=0.3, seed=17, precision=prec, gamma_min=gmin, gamma_max=0.5)
    run = make_run(kind, g, p, config=cfg)
    assert run.config().kernel == kernel
    X, m, v = _interior_state(g.n, p.S, 5 + kind)
    run.set_state(0, X, m, v, K - 1)
    _check_step(kind, g, p, prec, run)
    assert run.slot_step(0) == K
    p1 = p.with_(steps=1, seed=18)
    run1 = make_run(kind, g, p1, config=cfg)
    _check_step(kind, g, p1, prec, run1)
    assert run1.slot_step(0) == 1


@pytest.mark.parametrize("prec", [FP32, BF16])
@pytest.mark.parametrize("a_ent,alpha", [(2, 0.0), (4, 0.0), (4, 1.0), (6, 0.5)])
def test_single_step_entropy_exponents_and_alpha(prec, a_ent, alpha):
    g = _graph(MIS, 90, 0.1, 5)
    p = Params(S=16, steps=50, a_ent=a_ent, alpha_comm=alpha, seed=9, precision=prec)
    run = make_run(MIS, g, p)
    run.steps(7)
    _check_step(MIS, g, p, prec, run)


@pytest.mark.parametrize("cfg", [(1, 4, 64), (2, 2, 128), (4, 1, 256), (8, 1, 32)])
def test_single_step_every_layout(cfg):
    """Every (lanes per row, vectors per lane, block) layout computes the same step."""
    G_, V_, B_ = cfg
    g = _graph(MIS, 130, 0.1, 6)
    p = Params(S=16, steps=50, alpha_comm=0.5, seed=2)
    run = make_run(MIS, g, p, config=qqa.LaunchConfig(G_, V_, B_, kernel=qqa.KERNEL_DIRECT))
    c = run.config()
    assert (c.group_lanes, c.vec_per_lane, c.block_threads) == cfg
    run.steps(3)
    _check_step(MIS, g, p, FP32, run)


@pytest.mark.parametrize("S,prec", [(1, FP32), (3, BF16), (100, FP32), (1000, FP32), (1000, BF16), (256, BF16)])
def test_single_step_replica_counts(S, prec):
    """Ragged replica counts (padding lanes), S = 1 (zero variance), and S = 1000 (paper scale)."""
    g = _graph(MIS, 60, 0.15, 7)
    p = Params(S=S, steps=20, alpha_comm=0.3, seed=4, precision=prec)
    run = make_run(MIS, g, p)
    run.steps(2)
    _check_step(MIS, g, p, prec, run)


def test_isolated_nodes_single_node_and_ragged_tiles():
    """Rows with no neighbours, a 1-node graph, and n not a multiple of the tile height."""
    u = np.array([0, 0, 2]); v = np.array([1, 5, 5])
    g = G.from_edges(263, u, v)                      # 260 isolated nodes
    p = Params(S=8, steps=20, alpha_comm=0.2, seed=1)
    run = make_run(MIS, g, p)
    _check_step(MIS, g, p, FP32, run)
    g1 = G.from_edges(1, [], [])
    run1 = make_run(MAXCUT, g1, p)
    _check_step(MAXCUT, g1, p, FP32, run1)


@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
@pytest.mark.parametrize("prec,S,layout", [(FP32, 128, (32, 1, 4)), (FP32, 128, (32, 1, 8)), (FP32, 200, (32, 2, 2)),
                                           (FP32, 30, (8, 1, 4)), (BF16, 256, (32, 1, 2)), (BF16, 100, (16, 1, 8)),
                                           (FP32, 64, (16, 1, 2)), (BF16, 24, (4, 1, 4))])
def test_staged_kernel_equals_direct_kernel(kind, prec, S, layout):
    """The TMA-staged kernel reads neighbour rows from shared memory in the same
    ascending order as the direct gather, so states are bit-identical (max-clique
    too: its column sums are formed in a fixed order after every step)."""
    G_, V_, R_ = layout
    g = _graph(kind, 357, 0.12, 50 + kind, weighted=(kind == MAXCUT))
    p = Params(S=S, steps=100, alpha_comm=0.3, seed=11, precision=prec, gamma_min=-5.0 if kind == MAXCUT else -2.0)
    a = make_run(kind, g, p, config=qqa.LaunchConfig(G_, V_, 256, kernel=qqa.KERNEL_STAGED, kernel_param=R_))
    b = make_run(kind, g, p, config=qqa.LaunchConfig(G_, V_, 256, kernel=qqa.KERNEL_DIRECT))
    assert a.config().kernel == qqa.KERNEL_STAGED and b.config().kernel == qqa.KERNEL_DIRECT
    a.steps(60)
    b.steps(60)
    Xa, ma, va, _ = a.get_state(0)
    Xb, mb, vb, _ = b.get_state(0)
    np.testing.assert_array_equal(Xa, Xb)
    np.testing.assert_array_equal(ma, mb)
    np.testing.assert_array_equal(va, vb)


@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
@pytest.mark.parametrize("prec,S,layout", [(BF16, 256, (32, 1, 8)), (BF16, 256, (32, 1, 4)), (FP32, 128, (32, 1, 8)),
                                           (FP32, 200, (32, 2, 4)), (FP32, 30, (8, 1, 8)), (BF16, 40, (8, 1, 4)),
                                           (FP32, 8, (2, 1, 8))])
def test_stream_kernel_equals_direct_kernel(kind, prec, S, layout):
    """The cp.async streaming kernel (prefetched and overflow neighbours in CSR
    order) gives the direct kernel's states bit for bit; graphs mix rows with
    fewer and more neighbours than the prefetch depth."""
    G_, V_, NB = layout
    g = G.barabasi_albert(413, 3, 70 + kind)
    if kind == MAXCUT:
        rng = np.random.default_rng(kind)
        u, v, _ = g.upper_edges()
        g = G.from_edges(g.n, u, v, rng.integers(-2, 5, size=u.size))
    p = Params(S=S, steps=100, alpha_comm=0.3, seed=12, precision=prec, gamma_min=-5.0 if kind == MAXCUT else -2.0)
    a = make_run(kind, g, p, config=qqa.LaunchConfig(G_, V_, 256, kernel=qqa.KERNEL_STREAM, kernel_param=NB))
    b = make_run(kind, g, p, config=qqa.LaunchConfig(G_, V_, 256, kernel=qqa.KERNEL_DIRECT))
    assert a.config().kernel == qqa.KERNEL_STREAM
    a.steps(60)
    b.steps(60)
    Xa, ma, va, _ = a.get_state(0)
    Xb, mb, vb, _ = b.get_state(0)
    np.testing.assert_array_equal(Xa, Xb)
    np.testing.assert_array_equal(ma, mb)
    np.testing.assert_array_equal(va, vb)


@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
@pytest.mark.parametrize("prec,S,layout", [(BF16, 256, (16, 2, 128)), (BF16, 256, (32, 1, 256)), (FP32, 128, (32, 1, 64)),
                                           (FP32, 200, (32, 2, 256)), (FP32, 30, (8, 1, 128)), (BF16, 40, (8, 1, 256)),
                                           (FP32, 8, (2, 1, 64)), (BF16, 8, (1, 1, 32))])
def test_pipe_kernel_equals_direct_kernel(kind, prec, S, layout):
    """The pipelined kernel (own rows bulk-copied to shared memory one tile
    ahead) runs the direct kernel's gather and epilogue, so states are bit for
    bit the same; 413 nodes leave a ragged last tile for every tile height."""
    G_, V_, B_ = layout
    g = G.barabasi_albert(413, 3, 80 + kind)
    if kind == MAXCUT:
        rng = np.random.default_rng(kind)
        u, v, _ = g.upper_edges()
        g = G.from_edges(g.n, u, v, rng.integers(-2, 5, size=u.size))
    p = Params(S=S, steps=100, alpha_comm=0.3, seed=13, precision=prec, gamma_min=-5.0 if kind == MAXCUT else -2.0)
    a = make_run(kind, g, p, config=qqa.LaunchConfig(G_, V_, B_, kernel=qqa.KERNEL_PIPE))
    b = make_run(kind, g, p, config=qqa.LaunchConfig(G_, V_, B_, kernel=qqa.KERNEL_DIRECT))
    assert a.config().kernel == qqa.KERNEL_PIPE and a.config().block_threads == B_
    a.steps(60)
    b.steps(60)
    Xa, ma, va, _ = a.get_state(0)
    Xb, mb, vb, _ = b.get_state(0)
    np.testing.assert_array_equal(Xa, Xb)
    np.testing.assert_array_equal(ma, mb)
    np.testing.assert_array_equal(va, vb)


@pytest.mark.parametrize("prec", [FP32, BF16])
def test_pipe_kernel_single_step_parity_and_finished_instances(prec):
    """Single steps of the pipelined kernel against the oracle, in a batch where
    instances finish at different steps (their tiles are skipped: no copy is
    started for them) while the others go on, automatic block size."""
    gs = [G.random_regular(600, 3, 5), G.erdos_renyi(257, 0.03, 6), G.barabasi_albert(333, 4, 7)]
    ps = [Params(S=64, steps=k, alpha_comm=0.2, seed=20 + k, precision=prec, gamma_min=-5.0)
          for k in (12, 40, 25)]
    run = make_run(MAXCUT, gs, ps, config=qqa.LaunchConfig(16, 1, 0, kernel=qqa.KERNEL_PIPE))
    assert run.config().kernel == qqa.KERNEL_PIPE
    for slot in range(3):                           # each check advances every instance one step
        _check_step(MAXCUT, gs[slot], ps[slot], prec, run, slot=slot)
    run.steps(30)                                   # instance 0 stops at 12, instance 2 at 25
    t = [run.get_state(k)[3] for k in range(3)]
    assert t == [12, 33, 25]
    _check_step(MAXCUT, gs[1], ps[1], prec, run, slot=1)
    ref = make_run(MAXCUT, gs, ps, config=qqa.LaunchConfig(16, 1, 0, kernel=qqa.KERNEL_DIRECT))
    for k in range(3):
        ref.step_debug(k)
    ref.steps(30)
    ref.step_debug(1)
    for k in range(3):
        np.testing.assert_array_equal(run.get_state(k)[0], ref.get_state(k)[0])


def test_stream_kernel_single_step_parity_sparse_graph():
    g = G.random_regular(2000, 3, 4)
    p = Params(S=256, steps=500, alpha_comm=0.3, seed=0, precision=BF16, gamma_min=-5.0)
    run = make_run(MAXCUT, g, p, config=qqa.LaunchConfig(kernel=qqa.KERNEL_STREAM))
    run.steps(20)
    _check_step(MAXCUT, g, p, BF16, run)


@pytest.mark.parametrize("prec", [FP32, BF16])
@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
@pytest.mark.parametrize("n,p_edge,S", [(750, 0.15, 128), (300, 0.2, 64), (129, 0.3, 100), (450, 0.1, 200)])
def test_dense_tensor_core_step_matches_oracle(kind, n, p_edge, S, prec):
    """tcgen05 step (fp16 adjacency, two fp16 planes of p - from the FP32
    master in BF16 runs - FP32 accumulation in TMEM): single steps from the
    same state as the oracle, cold and warm moments, ragged last tile, several
    K chunks, MMA widths 64/128/256."""
    g = _graph(kind, n, p_edge if kind != MAXCLIQUE else 0.5, 60 + kind, weighted=(kind == MAXCUT))
    p = Params(S=S, steps=300, alpha_comm=0.3, lr=1.0, seed=8, gamma_min=-5.0 if kind == MAXCUT else -2.0,
               precision=prec)
    run = make_run(kind, g, p, config=qqa.LaunchConfig(kernel=qqa.KERNEL_DENSE))
    c = run.config()
    assert c.kernel == qqa.KERNEL_DENSE and c.kernel_param in (64, 128, 256)
    _check_step(kind, g, p, prec, run)
    run.steps(40)
    _check_step(kind, g, p, prec, run)


def test_dense_step_follows_the_direct_step_and_resumes():
    """A short trajectory of the tensor-core step stays within FP32 rounding of
    the direct gather (summation order differs), and set_state refreshes the
    fp16 planes so a resumed run continues bit-exactly."""
    g = G.erdos_renyi(700, 0.15, 3)
    p = Params(S=128, steps=400, alpha_comm=0.1, lr=1.0, seed=4)
    a = make_run(MIS, g, p, config=qqa.LaunchConfig(kernel=qqa.KERNEL_DENSE))
    b = make_run(MIS, g, p, config=qqa.LaunchConfig(kernel=qqa.KERNEL_DIRECT))
    a.steps(5)
    b.steps(5)
    np.testing.assert_allclose(a.get_state(0)[0], b.get_state(0)[0], atol=2e-5)
    a.steps(45)
    X, m, v, t = a.get_state(0)
    a.steps(30)
    c = make_run(MIS, g, p, config=qqa.LaunchConfig(kernel=qqa.KERNEL_DENSE))
    c.set_state(0, X, m, v, t)
    c.steps(30)
    np.testing.assert_array_equal(a.get_state(0)[0], c.get_state(0)[0])


def test_dense_step_batch_of_uneven_instances_and_quality():
    """Several instances of different n in one dense run; final quality of a
    full anneal within 1% of the direct kernel's."""
    gs = [G.erdos_renyi(n, 0.15, 700 + k) for k, n in enumerate((700, 777, 540, 800))]
    ps = [Params(S=128, steps=600, lr=1.0, seed=k) for k in range(4)]
    cfg_d = qqa.LaunchConfig(kernel=qqa.KERNEL_DENSE)
    cfg_g = qqa.LaunchConfig(kernel=qqa.KERNEL_DIRECT)
    probs = [qqa.Problem(MIS, g) for g in gs]
    rd = qqa.anneal(probs, [qqa.make_params(p) for p in ps], config=cfg_d)
    rg = qqa.anneal(probs, [qqa.make_params(p) for p in ps], config=cfg_g)
    for k in range(4):
        a, b = rd.result(k), rg.result(k)
        assert a["best"] >= 0 and b["best"] >= 0
        assert abs(a["obj"][a["best"]] - b["obj"][b["best"]]) <= 1
        o, v, f, _ = oracle.cost_of_x(MIS, gs[k], 2.0, a["best_x"])
        assert f and o == a["obj"][a["best"]]


@pytest.mark.parametrize("use_graphs", [1, 0], ids=["graphs", "launches"])
@pytest.mark.parametrize("prec", [FP32, BF16])
def test_dense_chained_batch_equals_each_instance_alone(prec, use_graphs):
    """A tensor-core run of several instances launches them as up to four
    chains of whole instances, each on its own stream, whose steps depend only
    on the chain's own previous step: every instance (uneven n, some finishing
    early) ends bit-identical to itself run alone, with and without CUDA
    graphs, and the step launches a product and an update per chain."""
    gs = [G.erdos_renyi(n, 0.15, 900 + k) for k, n in enumerate((700, 300, 777, 540, 800, 129))]
    ps = [Params(S=128, steps=s, lr=1.0, seed=k, precision=prec) for k, s in enumerate((60, 25, 60, 40, 60, 60))]
    cfg = qqa.LaunchConfig(kernel=qqa.KERNEL_DENSE, use_graphs=use_graphs)
    batch = make_run(MIS, gs, ps, config=cfg)
    n0 = qqa.launch_count()
    batch.steps(50)
    per_step = (qqa.launch_count() - n0 - 2) / 50   # prepare and advance once per chunk
    assert per_step in (4, 6, 8), per_step   # a product and an update per chain, 2 to 4 chains
    batch.steps(10)
    assert [batch.slot_step(k) for k in range(len(gs))] == [60, 25, 60, 40, 60, 60]
    for k in range(len(gs)):
        alone = make_run(MIS, gs[k], ps[k], config=cfg)
        alone.steps(60)
        for a, b in zip(alone.get_state(0)[:3], batch.get_state(k)[:3]):
            np.testing.assert_array_equal(a, b)


def test_staged_kernel_single_step_parity_dense_graph():
    g = G.erdos_renyi(750, 0.15, 1000)
    p = Params(S=128, steps=3000, alpha_comm=0.3, seed=0)
    run = make_run(MIS, g, p, config=qqa.LaunchConfig(kernel=qqa.KERNEL_STAGED))
    assert run.config().kernel == qqa.KERNEL_STAGED
    run.steps(50)
    _check_step(MIS, g, p, FP32, run)


@pytest.mark.parametrize("prec,kernel", [(FP32, qqa.KERNEL_DIRECT), (BF16, qqa.KERNEL_PIPE)])
def test_non_finite_gradient_is_reported(prec, kernel):
    """A gradient that overflows (lambda = 1e30 makes g^2 infinite) is counted in
    the device status word and reported as QQA_ENONFINITE; the state stays in
    [0, 1]. Non-finite moments are refused on the way in."""
    g = _graph(MIS, 120, 0.1, 3)
    p = Params(S=16, steps=20, lam=1e30, seed=4, precision=prec)
    run = make_run(MIS, g, p, config=qqa.LaunchConfig(8, 1, 128, kernel=kernel))
    run.steps(2)
    with pytest.raises(qqa.QQAError) as err:
        run.sync()
    assert err.value.code == qqa.QQA_ENONFINITE
    X = run.get_state(0)[0]
    assert np.all((X >= 0) & (X <= 1))
    ok = make_run(MIS, g, p.with_(lam=2.0))
    X0, m0, v0, t0 = ok.get_state(0)
    for bad_m, bad_v in ((np.inf, 0.0), (np.nan, 0.0), (0.0, -1.0), (0.0, np.inf)):
        m1, v1 = m0.copy(), v0.copy()
        m1[3, 5] = bad_m
        v1[7, 1] = bad_v
        with pytest.raises(qqa.QQAError) as err:
            ok.set_state(0, X0, m1, v1, t0)
        assert err.value.code == qqa.QQA_EINVAL


# ---------------------------------------------------------- multi-step ---
@pytest.mark.parametrize("kind", [MIS, MAXCUT])
def test_graph_replay_equals_single_launches(kind):
    """Chunks replayed from CUDA graphs give bit-identical states to one launch per step."""
    g = _graph(kind, 200, 0.05, 8)
    p = Params(S=32, steps=300, seed=5)
    a = make_run(kind, g, p, config=qqa.LaunchConfig(use_graphs=1))
    b = make_run(kind, g, p, config=qqa.LaunchConfig(use_graphs=0))
    a.steps(120)
    for _ in range(120):
        b.steps(1)
    Xa, ma, va, ta = a.get_state(0)
    Xb, mb, vb, tb = b.get_state(0)
    assert ta == tb == 120
    np.testing.assert_array_equal(Xa, Xb)
    np.testing.assert_array_equal(ma, mb)
    np.testing.assert_array_equal(va, vb)


def test_each_step_of_a_trajectory_matches_oracle():
    """Re-anchored trajectory: every one of 30 consecutive GPU steps equals the
    oracle step taken from the GPU's own state (catches ping-pong or t errors)."""
    g = _graph(MAXCLIQUE, 80, 0.3, 12)
    p = Params(S=24, steps=60, alpha_comm=0.3, seed=6)
    run = make_run(MAXCLIQUE, g, p)
    for _ in range(30):
        _check_step(MAXCLIQUE, g, p, FP32, run)


@pytest.mark.parametrize("kind", [MIS, MAXCLIQUE])
def test_steps_stop_at_K_and_checkpoint_resume_is_exact(kind):
    g = _graph(kind, 100, 0.1 if kind == MIS else 0.5, 2)
    p = Params(S=16, steps=130, seed=8)
    a = make_run(kind, g, p)
    a.steps(70)
    X, m, v, t = a.get_state(0)
    a.steps(500)
    assert a.slot_step(0) == 130
    b = make_run(kind, g, p)
    b.set_state(0, X, m, v, t)
    b.steps(60)
    np.testing.assert_array_equal(a.get_state(0)[0], b.get_state(0)[0])


@pytest.mark.parametrize("kind", [MIS, MAXCLIQUE])
def test_alone_equals_in_batch(kind):
    """An instance's trajectory does not depend on what else shares the launch."""
    gs = [_graph(kind, 90 + 37 * k, 0.1 if kind == MIS else 0.5, 30 + k) for k in range(4)]
    ps = [Params(S=32, steps=80 + 10 * k, seed=k) for k in range(4)]
    cfg = qqa.LaunchConfig(8, 1, 128)
    batch = make_run(kind, gs, ps, config=cfg)
    batch.steps(100)
    for k in (0, 3):
        alone = make_run(kind, gs[k], ps[k], config=cfg)
        alone.steps(100)
        np.testing.assert_array_equal(alone.get_state(0)[0], batch.get_state(k)[0])
        assert batch.slot_step(k) == min(100, ps[k].steps)


# -------------------------------------------------------------- eval -----
@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
@pytest.mark.parametrize("prec", [FP32, BF16])
def test_round_eval_is_exact(kind, prec):
    """Rounded costs, feasibility, energies and the best replica equal the
    oracle's evaluation of the GPU state, and best_x has the reported cost."""
    g = _graph(kind, 120, 0.2 if kind == MAXCLIQUE else 0.06, 40, weighted=(kind == MAXCUT))
    p = Params(S=70, steps=200, seed=3, precision=prec, gamma_min=-5.0 if kind == MAXCUT else -2.0)
    run = make_run(kind, g, p)
    for k in (37, 163):
        run.steps(k)
        run.eval()
        run.sync()
        res = run.result(0)
        X = run.get_state(0)[0].astype(np.float64)
        want = oracle.round_eval(kind, g, np.float32(p.lam), X)
        np.testing.assert_array_equal(res["obj"], want.obj)
        np.testing.assert_array_equal(res["viol"], want.viol)
        np.testing.assert_array_equal(res["feasible"], want.feasible)
        np.testing.assert_array_equal(res["energy"], want.energy)
        assert res["best"] == want.best
        if want.best >= 0:
            o, vv, f, e = oracle.cost_of_x(kind, g, p.lam, res["best_x"])
            assert (o, f) == (want.obj[want.best], True)


@pytest.mark.parametrize("prec", [FP32, BF16])
@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
@pytest.mark.parametrize("n,p_edge,S,weighted", [(300, 0.15, 128, False), (1100, 0.05, 100, False),
                                                 (257, 0.3, 37, False), (200, 0.1, 64, True)])
def test_round_eval_on_the_tensor_core_step_is_exact(kind, n, p_edge, S, weighted, prec):
    """Tensor-core runs of unit-weight graphs count costs by popcount over
    adjacency and replica bitsets (weighted ones by the per-edge kernel): costs,
    feasibility, energies and the best replica equal the oracle's evaluation of
    the GPU state. n = 1100 spans two 32-word batches of a bitset row; 257 and
    S = 37 leave ragged words."""
    weighted = weighted and kind == MAXCUT
    g = _graph(kind, n, p_edge, 60 + kind, weighted=weighted)
    prm = Params(S=S, steps=200, seed=5, precision=prec, gamma_min=-5.0 if kind == MAXCUT else -2.0)
    run = make_run(kind, g, prm, config=qqa.LaunchConfig(kernel=qqa.KERNEL_DENSE))
    assert run.config().kernel == qqa.KERNEL_DENSE
    for k in (41, 120):
        run.steps(k)
        run.eval()
        run.sync()
        res = run.result(0)
        X = run.get_state(0)[0].astype(np.float64)
        want = oracle.round_eval(kind, g, np.float32(prm.lam), X)
        np.testing.assert_array_equal(res["obj"], want.obj)
        np.testing.assert_array_equal(res["viol"], want.viol)
        np.testing.assert_array_equal(res["feasible"], want.feasible)
        np.testing.assert_array_equal(res["energy"], want.energy)
        assert res["best"] == want.best


def test_history_and_anneal_entry_point():
    g = _graph(MIS, 100, 0.05, 0)
    p = Params(S=8, steps=1000, round_every=50, seed=0)
    run = qqa.anneal([qqa.Problem(MIS, g)], [qqa.make_params(p)])
    hist, at = run.history(0)
    assert list(at) == list(range(50, 1001, 50))
    res = run.result(0)
    assert hist[-1] == res["obj"][res["best"]]
    assert res["step"] == 1000


# ----------------------------------------------------------- quality -----
def test_quality_matches_oracle_er100():
    """ER G(100, 0.05) MIS, S = 8, 1000 steps, 16 seeds: the mean best feasible
    objective is within 1% of the oracle's, and every result is feasible."""
    g = G.erdos_renyi(100, 0.05, 0)
    gpu, cpu = [], []
    for seed in range(16):
        p = Params(S=8, steps=1000, seed=seed)
        run = qqa.anneal([qqa.Problem(MIS, g)], [qqa.make_params(p)])
        r = run.result(0)
        assert r["best"] >= 0
        gpu.append(r["obj"][r["best"]])
        o = oracle.anneal(MIS, g, as_f32(p))
        cpu.append(o.eval.obj[o.eval.best])
    assert abs(np.mean(gpu) - np.mean(cpu)) <= 0.01 * np.mean(cpu)


@pytest.mark.parametrize("kind,gen,S,steps", [(MIS, "cliques", 32, 1000), (MAXCUT, "regular3", 32, 1000)])
def test_batched_bf16_quality_matches_oracle(kind, gen, S, steps):
    """The batched BF16 path (FP32 master and arithmetic, one launch for all 16
    runs, autotuned shape) against the FP64 oracle on the same graphs: per seed
    the best final feasible objective, mean over 16 seeds within 1%, every
    rounded best replica feasible and bit-exactly re-evaluated."""
    if gen == "cliques":
        g = G.clique_blocks(300, 17)
    else:
        g = G.random_regular(400, 3, 17)
    ps = [Params(S=S, steps=steps, seed=seed, precision=BF16, lr=1.0,
                 gamma_min=-5.0 if kind == MAXCUT else -2.0) for seed in range(16)]
    probs = [qqa.Problem(kind, g) for _ in ps]
    cps = [qqa.make_params(p) for p in ps]
    cfg, _ = qqa.autotune(probs, cps, trial_steps=50)
    run = qqa.anneal(probs, cps, config=cfg)
    gpu, cpu = [], []
    for k, p in enumerate(ps):
        r = run.result(k)
        assert r["best"] >= 0
        gpu.append(r["obj"][r["best"]])
        assert oracle.cost_of_x(kind, g, 2.0, r["best_x"])[0] == r["obj"][r["best"]]
        o = oracle.anneal(kind, g, as_f32(p.with_(precision=FP32)))
        cpu.append(o.eval.obj[o.eval.best])
    assert abs(np.mean(gpu) - np.mean(cpu)) <= 0.01 * np.mean(cpu)


def test_rrg_single_replica_quality_matches_oracle():
    """MIS on a random 20-regular graph with one replica (S = 1, the paper's RRG
    setting; the communication term vanishes): 16 seeds batched in one launch,
    mean independence density within 1% of the oracle's on the same seeds, every
    result feasible."""
    g = G.random_regular(2000, 20, 11)
    ps = [Params(S=1, steps=3000, seed=seed, lr=1.0) for seed in range(16)]
    run = qqa.anneal([qqa.Problem(MIS, g) for _ in ps], [qqa.make_params(p) for p in ps])
    gpu, cpu = [], []
    for k, p in enumerate(ps):
        r = run.result(k)
        assert r["best"] == 0 and r["feasible"][0]
        gpu.append(r["obj"][0] / g.n)
        o = oracle.anneal(MIS, g, as_f32(p))
        assert o.eval.best == 0
        cpu.append(o.eval.obj[0] / g.n)
    assert abs(np.mean(gpu) - np.mean(cpu)) <= 0.01 * np.mean(cpu)
    assert 0.15 < np.mean(gpu) < 0.25   # near the independence ratio of random 20-regular graphs
