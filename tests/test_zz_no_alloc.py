"""Evaluation without device allocation.

qqa_round_eval_noalloc serves callers that must not allocate device memory
while they evaluate (a serving loop that budgets HBM up front and cannot let a
request fail on, or stall behind, an allocation; a framework that owns every
device byte itself): they pass device pointers for the graph, the state and
the outputs, and the library works in a static scratch array. These tests
check that it returns exactly what the allocating qqa_round_eval returns for
the same state, on two calls in a row (the scratch keeps the previous call's
contents, so the second call shows that it clears what must start at zero).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _eval_both(qqa, torch, kind, g, run, lam, ld_pad=0):
    run.eval()
    run.sync()
    want = run.result(0, with_x=False)
    X = run.get_state(0)[0]
    n, S = X.shape
    ld = S + ld_pad
    Xd = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    Xd[:, :S] = torch.from_numpy(X).cuda()
    rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr, dtype=np.int32)).cuda()
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).cuda()
    w = None if g.w is None else torch.from_numpy(np.ascontiguousarray(g.w, dtype=np.int32)).cuda()
    obj = torch.full((S,), -7, dtype=torch.int64, device="cuda")
    viol = torch.full((S,), -7, dtype=torch.int64, device="cuda")
    feas = torch.full((S,), 7, dtype=torch.uint8, device="cuda")
    energy = torch.full((S,), float("nan"), dtype=torch.float64, device="cuda")
    best = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    qqa.round_eval_noalloc(kind, n, g.nnz, rp, col, w, S, ld, Xd, lam, obj, viol, feas, energy, best, stream=stream)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(obj.cpu().numpy(), want["obj"])
    np.testing.assert_array_equal(viol.cpu().numpy(), want["viol"])
    np.testing.assert_array_equal(feas.cpu().numpy().astype(bool), want["feasible"])
    np.testing.assert_array_equal(energy.cpu().numpy(), want["energy"])
    assert int(best.item()) == want["best"]


@pytest.mark.parametrize("kind_name", ["mis", "maxcut_weighted", "maxclique"])
def test_noalloc_eval_equals_allocating_eval_twice_in_a_row(kind_name):
    import torch

    from paper_2409_02135_gb300 import _build
    _build.build()
    import paper_2409_02135_gb300 as qqa
    from qqa_inputs import graphs as G
    from qqa_inputs.workloads import MAXCLIQUE, MAXCUT, MIS, Params

    assert torch.cuda.is_available()
    kind = {"mis": MIS, "maxcut_weighted": MAXCUT, "maxclique": MAXCLIQUE}[kind_name]
    g = G.erdos_renyi(301, 0.3 if kind == MAXCLIQUE else 0.05, 17)
    if kind == MAXCUT:
        rng = np.random.default_rng(3)
        u, v, _ = g.upper_edges()
        g = G.from_edges(g.n, u, v, rng.integers(-2, 6, size=u.size))
    p = Params(S=77, steps=300, seed=5, lr=1.0, gamma_min=-5.0 if kind == MAXCUT else -2.0)
    prob = qqa.Problem(kind, g)
    run = qqa.Run.create([prob], [qqa.make_params(p)])
    run.steps(40)
    _eval_both(qqa, torch, kind, g, run, p.lam)               # first call
    run.steps(200)
    _eval_both(qqa, torch, kind, g, run, p.lam, ld_pad=5)     # second call, padded row stride


def test_noalloc_eval_rejects_sizes_beyond_the_static_scratch():
    import torch

    import paper_2409_02135_gb300 as qqa

    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(qqa.QQAError, match="static scratch"):
        qqa.round_eval_noalloc(0, 2_000_000, 0, dummy, dummy, None, 1024, 1024, dummy, 2.0,
                               dummy, dummy, dummy, dummy, dummy)
    with pytest.raises(qqa.QQAError, match="1024"):
        qqa.round_eval_noalloc(0, 10, 0, dummy, dummy, None, 2048, 2048, dummy, 2.0,
                               dummy, dummy, dummy, dummy, dummy)
