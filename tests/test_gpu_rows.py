"""GPU parity of the two row layouts beside the vector step kernels:

- long rows: rows whose degree exceeds max(64, 8 x the mean degree) (hubs of
  scale-free graphs) are summed in segments of 32 neighbours by the long-row
  kernel and combined in segment order. Every gather kernel leaves them to it,
  so the direct, pipelined, streaming and staged steps stay bit-identical, and
  single steps match the FP64 oracle within the propagated bound.
- one replica per node (S = 1, the paper's random-regular-graph setting): the
  state is one value per node and the scalar kernel sums a row's neighbours with
  L lanes; single steps and the rounding match the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_2409_02135_gb300 as qqa
from parity import as_f32, assert_within, make_run, step_tolerance
from qqa_inputs import graphs as G
from qqa_inputs.workloads import MIS, MAXCUT, MAXCLIQUE, FP32, BF16, Params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_02135_gb300 import _build
    _build.build()
    import torch
    assert torch.cuda.is_available()


def _long_threshold(g):
    mean_up = -(-g.nnz // g.n)
    return max(64, 8 * mean_up)


def _hub_graph(kind, seed, n=3000):
    """BA(n, 4) plus one node joined to 900 others: a few rows of 65-200
    neighbours (3-7 segments) and one of about 900 (29 segments). Max-cut gets
    integer weights in [-2, 4]; max-clique the complement-like dense variant is
    not needed, the same sparse graph is used."""
    g = G.barabasi_albert(n, 4, seed)
    u, v, _ = g.upper_edges()
    have = set(zip(u.tolist(), v.tolist()))
    hub = 7
    extra = [(min(hub, j), max(hub, j)) for j in range(1000, 1900) if (min(hub, j), max(hub, j)) not in have]
    uu = np.concatenate([u, np.array([a for a, _ in extra])])
    vv = np.concatenate([v, np.array([b for _, b in extra])])
    w = None
    if kind == MAXCUT:
        w = np.random.default_rng(seed).integers(-2, 5, size=uu.size)
    g = G.from_edges(n, uu, vv, w)
    deg = g.degrees()
    assert deg.max() > 32 * 20 and (deg > _long_threshold(g)).sum() >= 5
    return g


def _check_step(kind, g, p, prec, run, slot=0):
    X0, m0, v0, t = run.get_state(slot)
    grad = run.step_debug(slot)
    X1, m1, v1, t1 = run.get_state(slot)
    assert t1 == t + 1
    po = as_f32(p)
    out = oracle.step(kind, g, po, t, X0.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64))
    tg, tm, tv, tp = step_tolerance(po, prec, t, X0.astype(np.float64), m0.astype(np.float64),
                                    v0.astype(np.float64), out)
    assert_within("gradient", grad, out.grad, tg)
    assert_within("m", m1, out.m, tm)
    assert_within("v", v1, out.v, tv)
    assert_within("p", X1, out.X, tp)


# -------------------------------------------------------------- long rows ---
@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
@pytest.mark.parametrize("prec,S,layout", [(BF16, 256, (16, 2)), (BF16, 256, (32, 1)), (FP32, 128, (32, 1)),
                                           (FP32, 30, (8, 1)), (BF16, 24, (4, 1))])
def test_long_rows_every_gather_kernel_is_bit_identical(kind, prec, S, layout):
    """Direct, pipelined, streaming and staged steps on a graph with hubs: the
    long rows go through the long-row kernel in every case, so 40 steps leave
    bit-identical p, m and v."""
    G_, V_ = layout
    g = _hub_graph(kind, 3 + kind)
    p = Params(S=S, steps=200, alpha_comm=0.3, seed=5, precision=prec, gamma_min=-5.0 if kind == MAXCUT else -2.0)
    ref = make_run(kind, g, p, config=qqa.LaunchConfig(G_, V_, 128, kernel=qqa.KERNEL_DIRECT))
    ref.steps(40)
    want = ref.get_state(0)
    for kernel, bt, kp in ((qqa.KERNEL_PIPE, 128, 0), (qqa.KERNEL_STREAM, 256, 4), (qqa.KERNEL_STAGED, 256, 2)):
        try:
            run = make_run(kind, g, p, config=qqa.LaunchConfig(G_, V_, bt, kernel=kernel, kernel_param=kp))
        except qqa.QQAError as err:   # the streaming and staged kernels are built for fewer shapes
            assert err.code == qqa.QQA_EINVAL and kernel != qqa.KERNEL_PIPE
            continue
        assert run.config().kernel == kernel
        run.steps(40)
        got = run.get_state(0)
        for a, b in zip(got[:3], want[:3]):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("kernel", [qqa.KERNEL_DIRECT, qqa.KERNEL_PIPE])
@pytest.mark.parametrize("prec", [FP32, BF16])
@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
def test_long_rows_single_step_matches_oracle(kind, prec, kernel):
    """Single steps (t = 0 and t = 30) with the hub rows summed in segments:
    every element of gradient, m, v and p within the propagated bound."""
    g = _hub_graph(kind, 11 + kind)
    p = Params(S=64, steps=300, alpha_comm=0.3, lr=0.3, seed=9, precision=prec,
               gamma_min=-5.0 if kind == MAXCUT else -2.0)
    run = make_run(kind, g, p, config=qqa.LaunchConfig(kernel=kernel))
    _check_step(kind, g, p, prec, run)
    run.steps(29)
    _check_step(kind, g, p, prec, run)


def test_long_rows_in_a_batch_with_finished_instances():
    """Hub instances of different lengths in one run: an instance that has
    finished skips its segments while the others go on, and each instance
    equals itself run alone (the arrival counters are per slot and reset by the
    last segment of every row)."""
    gs = [_hub_graph(MAXCUT, 21), _hub_graph(MAXCUT, 22, n=2500), G.random_regular(800, 3, 5)]
    ps = [Params(S=32, steps=k, seed=30 + k, precision=BF16, gamma_min=-5.0) for k in (15, 60, 40)]
    cfg = qqa.LaunchConfig(8, 1, 128, kernel=qqa.KERNEL_PIPE)
    batch = make_run(MAXCUT, gs, ps, config=cfg)
    batch.steps(50)
    assert [batch.slot_step(k) for k in range(3)] == [15, 50, 40]
    for k in range(3):
        alone = make_run(MAXCUT, gs[k], ps[k], config=cfg)
        alone.steps(50)
        np.testing.assert_array_equal(alone.get_state(0)[0], batch.get_state(k)[0])
    batch.eval()
    batch.sync()
    for k in range(3):
        res = batch.result(k)
        X = batch.get_state(k)[0].astype(np.float64)
        want = oracle.round_eval(MAXCUT, gs[k], np.float32(2.0), X)
        np.testing.assert_array_equal(res["obj"], want.obj)
        assert res["best"] == want.best


# -------------------------------------------------------- one replica -----
@pytest.mark.parametrize("L", [4, 8, 16, 32])
@pytest.mark.parametrize("prec", [FP32, BF16])
@pytest.mark.parametrize("kind", [MIS, MAXCUT, MAXCLIQUE])
def test_one_replica_single_step_matches_oracle(kind, prec, L):
    """S = 1 in the one-value-per-node layout: t = 0 and t = 40 single steps for
    every lanes-per-row choice, on a random 20-regular graph (MIS, clique) or a
    weighted graph with uneven degrees (max-cut); 1000 nodes leave a ragged
    last warp of rows."""
    if kind == MAXCUT:
        g0 = G.barabasi_albert(1000, 3, 4)
        u, v, _ = g0.upper_edges()
        g = G.from_edges(g0.n, u, v, np.random.default_rng(4).integers(-2, 5, size=u.size))
    else:
        g = G.random_regular(1000, 20, 6 + kind)
    p = Params(S=1, steps=300, lr=1.0, seed=13, precision=prec, gamma_min=-5.0 if kind == MAXCUT else -2.0)
    run = make_run(kind, g, p, config=qqa.LaunchConfig(kernel=qqa.KERNEL_SCALAR, kernel_param=L))
    c = run.config()
    assert c.kernel == qqa.KERNEL_SCALAR and c.kernel_param == L
    _check_step(kind, g, p, prec, run)
    run.steps(39)
    _check_step(kind, g, p, prec, run)
    run.eval()
    run.sync()
    res = run.result(0)
    X = run.get_state(0)[0].astype(np.float64)
    want = oracle.round_eval(kind, g, np.float32(p.lam), X)
    np.testing.assert_array_equal(res["obj"], want.obj)
    np.testing.assert_array_equal(res["viol"], want.viol)
    assert res["best"] == want.best


def test_one_replica_runs_take_the_scalar_kernel_only():
    """Runs of S = 1 always use the scalar layout; asking for a vector kernel is
    refused, and a batch of uneven instances equals each instance alone."""
    g = G.random_regular(500, 20, 1)
    p = Params(S=1, steps=50, seed=2)
    with pytest.raises(qqa.QQAError) as err:
        make_run(MIS, g, p, config=qqa.LaunchConfig(kernel=qqa.KERNEL_DIRECT))
    assert err.value.code == qqa.QQA_EINVAL
    assert make_run(MIS, g, p).config().kernel == qqa.KERNEL_SCALAR
    gs = [G.random_regular(300 + 77 * k, 20, 40 + k) for k in range(3)]
    ps = [Params(S=1, steps=30 + 5 * k, seed=k) for k in range(3)]
    cfg = qqa.LaunchConfig(kernel=qqa.KERNEL_SCALAR, kernel_param=8)
    batch = make_run(MIS, gs, ps, config=cfg)
    batch.steps(40)
    for k in range(3):
        alone = make_run(MIS, gs[k], ps[k], config=cfg)
        alone.steps(40)
        np.testing.assert_array_equal(alone.get_state(0)[0], batch.get_state(k)[0])
