"""Pins for the FP64 oracle: each check compares it with something other than
itself -- published known-answer vectors, closed forms the paper derives,
finite differences of its own objective, a library optimizer, or brute force
on tiny graphs -- so that a dropped term, a wrong sign or index, or a
transposed operand in any part of the oracle fails at least one test.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from qqa_inputs import graphs as G
from qqa_inputs.workloads import MIS, MAXCUT, MAXCLIQUE, Params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KINDS = [MIS, MAXCUT, MAXCLIQUE]


def _weighted(g, seed):
    rng = np.random.default_rng(seed)
    u, v, _ = g.upper_edges()
    return G.from_edges(g.n, u, v, rng.integers(-3, 6, size=u.size))


# ---------------------------------------------------------------- RNG ----
def test_philox_known_answers(oracle_lib):
    """Philox4x32-10 equals the published known-answer vectors (Salmon et al., SC'11)."""
    rows = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        lhs, rhs = line.split("|")
        a = [int(x, 16) for x in lhs.split()]
        want = [int(x, 16) for x in rhs.split()]
        got = oracle.philox4x32_10(a[:4], a[4:6])
        assert [int(x) for x in got] == want
        rows += 1
    assert rows == 3


def test_uniform_is_philox_mapping_and_in_range(oracle_lib):
    """Init uniforms are ((r>>8)+1)/2^24 of the Philox word for (i, s/4, t=0, tag=0)."""
    seed = 0x1234_5678_9ABC
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for (i, s) in [(0, 0), (5, 3), (17, 6), (1000, 255)]:
        r = oracle.philox4x32_10([i, s // 4, 0, 0], key)[s % 4]
        assert oracle.uniform(seed, i, s) == ((int(r) >> 8) + 1) / 2**24
    X = oracle.init_state(300, 64, seed=11)
    assert X.min() > 0.0 and X.max() <= 1.0
    assert abs(X.mean() - 0.5) < 5 * math.sqrt(1 / 12 / X.size)


def test_gaussian_is_box_muller_with_unit_moments(oracle_lib):
    """Noise xi is the Box-Muller transform of the Philox uniforms (tag 1) and
    has mean 0 and variance 1 within 5 sigma over 1e6 draws."""
    seed, t = 77, 9
    key = [seed, 0]
    for (i, s) in [(0, 0), (0, 1), (3, 2), (3, 3), (40, 13)]:
        r = oracle.philox4x32_10([i, s // 4, t, 1], key)
        pair = (s % 4) // 2
        u1 = ((int(r[2 * pair]) >> 8) + 1) / 2**24
        u2 = ((int(r[2 * pair + 1]) >> 8) + 1) / 2**24
        rad = math.sqrt(-2 * math.log(u1))
        want = rad * (math.cos(2 * math.pi * u2) if s % 2 == 0 else math.sin(2 * math.pi * u2))
        assert oracle.gaussian(seed, i, s, t) == pytest.approx(want, abs=1e-14)
    xi = oracle.noise_field(1000, 1000, seed, t)
    n = xi.size
    assert abs(xi.mean()) < 5 / math.sqrt(n)
    assert abs(xi.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(np.mean(xi ** 4) - 3.0) < 0.05          # Gaussian kurtosis
    # different steps give independent fields
    xi2 = oracle.noise_field(1000, 1000, seed, t + 1)
    assert abs(np.corrcoef(xi.ravel(), xi2.ravel())[0, 1]) < 5 / math.sqrt(n)


# ------------------------------------------------------- schedule ------
def test_gamma_schedule_endpoints_and_linearity(oracle_lib):
    """gamma goes linearly from gamma_min (first step) to gamma_max (last step) (Sec. 5, App. C.2)."""
    p = Params(steps=3000, gamma_min=-2.0, gamma_max=0.1)
    gs = [oracle.gamma(MIS, p, t) for t in range(p.steps)]
    assert gs[0] == -2.0
    assert gs[-1] == pytest.approx(0.1, abs=1e-15)
    d = np.diff(gs)
    assert np.allclose(d, 2.1 / 2999, rtol=1e-9)
    assert oracle.gamma(MIS, p.with_(steps=1), 0) == -2.0


# -------------------------------------------------------- entropy ------
@pytest.mark.parametrize("a", [2, 4, 6])
def test_alpha_entropy_closed_forms(oracle_lib, a):
    """s vanishes on {0,1}^N, equals N at p = 1/2, is symmetric about 1/2, and for
    gamma < 0 the term gamma*s is minimised at 1/2 (Eq. 7; Sec. 3.2)."""
    rng = np.random.default_rng(a)
    x = rng.integers(0, 2, size=50).astype(float)
    assert oracle.entropy(x, a) == 0.0
    assert oracle.entropy(np.full(37, 0.5), a) == 37.0
    p = rng.random(40)
    assert oracle.entropy(p, a) == pytest.approx(oracle.entropy(1 - p, a), rel=1e-14)
    grid = np.linspace(0, 1, 2001)
    vals = np.array([-1.5 * oracle.entropy(np.array([q]), a) for q in grid])
    assert vals[1000] == vals.min() == -1.5           # grid[1000] = 1/2
    assert np.all(vals[np.abs(grid - 0.5) > 0.05] > -1.5)
    # s(p) = 1 - (2p-1)^a elementwise, checked at one point against the power
    assert oracle.entropy(np.array([0.8]), a) == pytest.approx(1 - 0.6 ** a, rel=1e-14)


# ------------------------------------------------------- energies ------
def _dense_energy(kind, A, x, lam):
    """Energies of App. D.1 written with a dense adjacency matrix."""
    if kind == MIS:
        return -x.sum() + lam * x @ A @ x / 2
    if kind == MAXCLIQUE:
        return -x.sum() + lam / 2 * (x.sum() * (x.sum() - 1) - x @ A @ x)
    z = 2 * x - 1
    return -np.sum(np.triu(A * (1 - np.outer(z, z)) / 2, 1))


@pytest.mark.parametrize("kind", KINDS)
def test_relaxed_equals_discrete_on_binary_points(oracle_lib, kind):
    """l^(x) = l(x) on {0,1}^N (Sec. 3.1), and both equal the dense-matrix energy."""
    rng = np.random.default_rng(kind)
    g = G.erdos_renyi(40, 0.2, 3)
    if kind == MAXCUT:
        g = _weighted(g, 5)
    A = g.dense().astype(float)
    for _ in range(20):
        x = rng.integers(0, 2, size=g.n)
        rel = oracle.relaxed_loss(kind, g, 2.0, x.astype(float))
        obj, viol, feas, en = oracle.cost_of_x(kind, g, 2.0, x)
        assert rel == pytest.approx(en, abs=1e-9)
        assert en == pytest.approx(_dense_energy(kind, A, x.astype(float), 2.0), abs=1e-9)


def test_discrete_costs_match_definitions(oracle_lib):
    """Integer costs: MIS conflicts = adjacent selected pairs, clique missing
    edges = non-adjacent selected pairs, cut = weight across the partition."""
    rng = np.random.default_rng(4)
    g = _weighted(G.erdos_renyi(25, 0.3, 8), 9)
    gu = G.erdos_renyi(25, 0.3, 8)
    A = gu.dense()
    W = g.dense()
    for _ in range(30):
        x = rng.integers(0, 2, size=25)
        sel = np.flatnonzero(x)
        pairs = list(itertools.combinations(sel.tolist(), 2))
        adj = sum(A[i, j] for i, j in pairs)
        o, v, f, _ = oracle.cost_of_x(MIS, gu, 2.0, x)
        assert (o, v, f) == (len(sel), adj, adj == 0)
        o, v, f, _ = oracle.cost_of_x(MAXCLIQUE, gu, 2.0, x)
        assert (o, v, f) == (len(sel), len(pairs) - adj, len(pairs) == adj)
        cut = sum(W[i, j] for i in range(25) for j in range(i + 1, 25) if x[i] != x[j])
        o, v, f, e = oracle.cost_of_x(MAXCUT, g, 2.0, x)
        assert (o, v, f, e) == (cut, 0, True, -cut)


# ------------------------------------------------------- gradient ------
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("a_ent", [2, 4])
@pytest.mark.parametrize("alpha", [0.0, 0.7])
def test_gradient_matches_finite_differences(oracle_lib, kind, a_ent, alpha):
    """dR/dp (all terms: energy, gamma*entropy, communication) equals central
    finite differences of R itself (Eq. 6, Eq. 10) to 1e-7 relative."""
    g = G.erdos_renyi(14, 0.3, 21 + kind)
    if kind == MAXCUT:
        g = _weighted(g, 2)
    p = Params(S=5, a_ent=a_ent, alpha_comm=alpha, comm_eps=1e-8, lam=2.0)
    rng = np.random.default_rng(100 + kind)
    X = 0.05 + 0.9 * rng.random((g.n, p.S))
    gam = -1.3
    Gm = oracle.gradient(kind, g, p, gam, X)
    h = 1e-5
    worst = 0.0
    for i in range(g.n):
        for s in range(p.S):
            Xp = X.copy(); Xp[i, s] += h
            Xm = X.copy(); Xm[i, s] -= h
            fd = (oracle.objective(kind, g, p, gam, Xp) - oracle.objective(kind, g, p, gam, Xm)) / (2 * h)
            worst = max(worst, abs(fd - Gm[i, s]) / max(1.0, abs(Gm[i, s])))
    assert worst < 1e-7


def test_communication_term_closed_forms(oracle_lib):
    """STD term (Eq. 10): with K zeros and S-K ones in every row, the term equals
    -S alpha N sqrt(K(S-K)/S^2 + eps); the maximum over K is 1/4 for even S and
    (S^2-1)/(4S^2) for odd S (Prop. in App. A.2); and the gradient vanishes
    when all S values of a row are equal."""
    g = G.erdos_renyi(6, 0.0, 0)  # no edges: only the entropy (0 on binaries) and STD terms remain
    for S in (6, 7):
        best = 0.0
        for K in range(S + 1):
            X = np.zeros((g.n, S))
            X[:, K:] = 1.0
            p1 = Params(S=S, alpha_comm=0.4, comm_eps=0.0)
            p0 = p1.with_(alpha_comm=0.0)
            comm = oracle.objective(MIS, g, p1, 0.3, X) - oracle.objective(MIS, g, p0, 0.3, X)
            var = K * (S - K) / S ** 2
            assert comm == pytest.approx(-S * 0.4 * g.n * math.sqrt(var), abs=1e-12)
            best = max(best, var)
        want = 0.25 if S % 2 == 0 else (S * S - 1) / (4 * S * S)
        assert best == pytest.approx(want, rel=1e-15)
    X = np.full((g.n, 8), 0.3)
    p = Params(S=8, alpha_comm=0.9, comm_eps=1e-8)
    Gm = oracle.gradient(MIS, g, p, 0.0, X)
    assert np.all(Gm == -1.0)          # only -c remains: comm gradient exactly 0


# --------------------------------------------------------- AdamW -------
@pytest.mark.parametrize("kind", KINDS)
def test_step_is_torch_adamw_on_the_gradient(oracle_lib, kind):
    """With T = 0 and interior points, a step equals torch.optim.AdamW (FP64)
    applied to the oracle's gradient (Sec. 3.4: the update is replaced by AdamW;
    decoupled weight decay App. C.3)."""
    torch = pytest.importorskip("torch")
    g = G.erdos_renyi(30, 0.2, 40 + kind)
    p = Params(S=6, steps=50, lr=2e-3, temperature=0.0, alpha_comm=0.5, weight_decay=0.01,
               beta1=0.85, beta2=0.995, adam_eps=1e-8)
    rng = np.random.default_rng(7)
    X = 0.3 + 0.4 * rng.random((g.n, p.S))
    xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.AdamW([xt], lr=p.lr, betas=(p.beta1, p.beta2), eps=p.adam_eps,
                            weight_decay=p.weight_decay, foreach=False)
    m = np.zeros_like(X)
    v = np.zeros_like(X)
    for t in range(6):
        gam = oracle.gamma(kind, p, t)
        grad = oracle.gradient(kind, g, p, gam, X)
        xt.grad = torch.tensor(grad, dtype=torch.float64)
        opt.step()
        out = oracle.step(kind, g, p, t, X, m, v)
        assert np.allclose(out.grad, grad, rtol=0, atol=0)
        X, m, v = out.X, out.m, out.v
        assert 0.0 < X.min() and X.max() < 1.0
        np.testing.assert_allclose(X, xt.detach().numpy(), rtol=1e-13, atol=1e-15)
        st = opt.state[xt]
        np.testing.assert_allclose(m, st["exp_avg"].numpy(), rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(v, st["exp_avg_sq"].numpy(), rtol=1e-13, atol=1e-18)


def test_noise_is_added_after_adamw_before_clamp(oracle_lib):
    """The Langevin term sqrt(2 lr T) xi (Eq. 11) is the only difference between
    T > 0 and T = 0 steps at interior points, and the clamp keeps p in [0, 1]."""
    g = G.erdos_renyi(20, 0.2, 3)
    rng = np.random.default_rng(1)
    X = 0.3 + 0.4 * rng.random((g.n, 4))
    m = np.zeros_like(X)
    v = np.zeros_like(X)
    p0 = Params(S=4, steps=10, lr=0.01, temperature=0.0, seed=5)
    p1 = p0.with_(temperature=0.02)
    t = 3
    a = oracle.step(MIS, g, p0, t, X, m, v)
    b = oracle.step(MIS, g, p1, t, X, m, v)
    xi = oracle.noise_field(g.n, 4, 5, t)
    np.testing.assert_allclose(b.X - a.X, math.sqrt(2 * 0.01 * 0.02) * xi, atol=1e-14)
    big = p1.with_(lr=50.0, temperature=5.0)
    c = oracle.step(MIS, g, big, t, X, m, v)
    assert c.X.min() >= 0.0 and c.X.max() <= 1.0
    assert np.any(c.X == 0.0) and np.any(c.X == 1.0)


def test_step_reads_only_the_old_state(oracle_lib):
    """Jacobi update: computing a subset of rows gives the same values as the full step."""
    g = G.erdos_renyi(60, 0.1, 2)
    p = Params(S=8, steps=100, alpha_comm=0.3)
    X = oracle.init_state(g.n, p.S, 3)
    m = np.zeros_like(X); v = np.zeros_like(X)
    full = oracle.step(MAXCLIQUE, g, p, 4, X, m, v)
    rows = np.array([59, 0, 17, 33])
    part = oracle.step(MAXCLIQUE, g, p, 4, X, m[rows], v[rows], rows=rows)
    np.testing.assert_array_equal(part.X, full.X[rows])
    np.testing.assert_array_equal(part.m, full.m[rows])


# ------------------------------------------------- rounding / eval -----
def test_round_eval_matches_cost_of_x_and_best_rule(oracle_lib):
    """x = [p > 1/2] strictly; best = feasible replica with max objective, ties -> lowest s."""
    g = G.erdos_renyi(30, 0.15, 6)
    rng = np.random.default_rng(0)
    X = rng.random((g.n, 16))
    X[0, :] = 0.5          # exactly 1/2 rounds to 0
    r = oracle.round_eval(MIS, g, 2.0, X)
    best, best_obj = -1, None
    for s in range(16):
        x = (X[:, s] > 0.5).astype(int)
        assert x[0] == 0
        o, v, f, e = oracle.cost_of_x(MIS, g, 2.0, x)
        assert (r.obj[s], r.viol[s], bool(r.feasible[s]), r.energy[s]) == (o, v, f, e)
        if f and (best < 0 or o > best_obj):
            best, best_obj = s, o
    assert r.best == best
    X2 = np.zeros((g.n, 3)); X2[:, 1] = 1.0
    r2 = oracle.round_eval(MIS, g, 2.0, X2)     # replicas 0 and 2 tie (empty set); 1 infeasible
    assert r2.best == 0 and not r2.feasible[1]


# ------------------------------------------------ brute-force pins -----
def _all_x(n):
    return ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)


def _brute(kind, g, lam=2.0):
    A = g.dense()
    Xs = _all_x(g.n)
    size = Xs.sum(1)
    inside = np.einsum("ki,ij,kj->k", Xs, (A != 0).astype(np.int64), Xs) // 2
    if kind == MIS:
        feas = inside == 0
        energy = -size + lam * inside
        return int(size[feas].max()), float(energy.min())
    if kind == MAXCLIQUE:
        missing = size * (size - 1) // 2 - inside
        feas = missing == 0
        energy = -size + lam * missing
        return int(size[feas].max()), float(energy.min())
    cut = np.einsum("ki,ij,kj->k", Xs, A, 1 - Xs)
    return int(cut.max()), float(-cut.max())


def test_penalty_two_makes_energy_minimisers_feasible(oracle_lib):
    """With lambda = 2 (App. D.1), min over {0,1}^N of the penalised energy
    equals minus the optimum of the constrained problem (MIS and clique)."""
    for seed in range(6):
        g = G.erdos_renyi(12, 0.3, seed)
        for kind in (MIS, MAXCLIQUE):
            opt, emin = _brute(kind, g)
            assert emin == -opt


@pytest.mark.parametrize("kind", KINDS)
def test_whole_run_reaches_brute_force_optimum(oracle_lib, kind):
    """The full anneal (init, 1000 steps, S = 8, final rounding) finds the
    exhaustive-search optimum on at least 90% of random graphs with n <= 16."""
    hits, total = 0, 0
    for seed in range(25):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(8, 17))
        g = G.erdos_renyi(n, float(rng.uniform(0.15, 0.45)), 500 + seed)
        opt, _ = _brute(kind, g)
        p = Params(S=8, steps=1000, seed=seed, gamma_min=-2.0 if kind != MAXCUT else -5.0)
        out = oracle.anneal(kind, g, p)
        total += 1
        assert out.eval.best >= 0
        got = out.eval.obj[out.eval.best]
        assert got <= opt
        hits += int(got == opt)
    assert hits >= 0.9 * total


def test_annealing_ends_almost_binary(oracle_lib):
    """After the gamma sweep to gamma_max > 0 the relaxed variables are almost
    binary (Sec. 5 'Implementation'; Thm. 1's gamma -> +inf limit)."""
    g = G.erdos_renyi(80, 0.1, 1)
    p = Params(S=8, steps=1500, seed=3)
    out = oracle.anneal(MIS, g, p)
    assert np.mean(np.abs(out.X - 0.5) > 0.45) > 0.98
    # and a large negative gamma keeps the state near 1/2 (Thm. 1's gamma -> -inf limit)
    p2 = Params(S=8, steps=300, gamma_min=-1e5, gamma_max=-1e5, seed=3, temperature=0.0)
    out2 = oracle.anneal(MIS, g, p2)
    assert np.max(np.abs(out2.X - 0.5)) < 0.05


def test_periodic_history_is_monotone_prefix(oracle_lib):
    """A shorter run is a prefix of the full run (same schedule); the final
    evaluation is the last history entry."""
    g = G.erdos_renyi(40, 0.15, 12)
    p = Params(S=8, steps=400, round_every=50, seed=2)
    full = oracle.anneal(MIS, g, p)
    half = oracle.anneal(MIS, g, p, steps=200)
    assert len(full.history) == 8 and len(half.history) == 4
    np.testing.assert_array_equal(full.history[:3], half.history[:3])
    assert full.history[-1] == full.eval.obj[full.eval.best]


# ------------------------------------------- categorical colouring (NEXT) ---
def _color_graphs():
    rows = []
    with open(os.path.join(GOLDEN, "paper_color_graphs.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, gen, nodes, edges, colours, conflicts = line.split()
                rows.append((name, gen, int(nodes), int(edges), int(colours), int(conflicts)))
    return rows


def _make_color_graph(gen):
    parts = gen.split(":")
    return G.mycielski(int(parts[1])) if parts[0] == "mycielski" else G.queens(int(parts[1]), int(parts[2]))


def test_color_graph_generators_match_the_papers_table():
    """Queens and Mycielski graphs built from their definitions have the node and
    edge counts of the paper's Table 9."""
    for name, gen, nodes, edges, _, _ in _color_graphs():
        g = _make_color_graph(gen)
        assert (g.n, g.nnz // 2) == (nodes, edges), name


@pytest.mark.parametrize("a", [2, 4, 6])
def test_categorical_entropy_reduces_to_the_binary_one_at_K2(oracle_lib, a):
    """Proposition of App. B: s_2(sigma) with sigma_i = (p_i, 1 - p_i) equals the
    alpha-entropy s(p) of Eq. 7."""
    rng = np.random.default_rng(a)
    p = rng.random(40)
    sig = np.stack([p, 1 - p], axis=1)
    assert oracle.color_entropy(sig, a) == pytest.approx(oracle.entropy(p, a), rel=1e-14, abs=1e-12)


@pytest.mark.parametrize("K,a", [(3, 2), (5, 4), (7, 4)])
def test_categorical_entropy_closed_forms(oracle_lib, K, a):
    """s_K is 0 at every one-hot row (App. B: the minimisers are the discrete
    points), N at the uniform row 1/K (its maximum), and invariant under a
    permutation of the colours."""
    rng = np.random.default_rng(K)
    n = 25
    one_hot = np.eye(K)[rng.integers(0, K, size=n)]
    assert oracle.color_entropy(one_hot, a) == pytest.approx(0.0, abs=1e-12)
    assert oracle.color_entropy(np.full((n, K), 1.0 / K), a) == pytest.approx(n, rel=1e-14)
    sig = rng.random((n, K))
    sig /= sig.sum(axis=1, keepdims=True)
    perm = rng.permutation(K)
    assert oracle.color_entropy(sig[:, perm], a) == pytest.approx(oracle.color_entropy(sig, a), rel=1e-13)
    assert oracle.color_entropy(sig, a) < n


def test_relaxed_conflicts_equal_discrete_conflicts_on_one_hot_points(oracle_lib):
    """At one-hot sigma the relaxed energy equals the number of conflicting
    edges, and both equal a count over the dense adjacency matrix."""
    g = G.erdos_renyi(30, 0.25, 8)
    A = np.zeros((g.n, g.n), dtype=np.int64)
    for i in range(g.n):
        A[i, g.col[g.row_ptr[i]:g.row_ptr[i + 1]]] = 1
    rng = np.random.default_rng(2)
    for K in (2, 3, 6):
        for _ in range(5):
            x = rng.integers(0, K, size=g.n)
            same = (x[:, None] == x[None, :]).astype(np.int64)
            want = int(np.sum(np.triu(A * same, 1)))
            assert oracle.color_conflicts(g, x) == want
            assert oracle.color_relaxed_conflicts(g, np.eye(K)[x]) == pytest.approx(want, abs=1e-12)


@pytest.mark.parametrize("K", [3, 5])
@pytest.mark.parametrize("a_ent", [2, 4])
@pytest.mark.parametrize("alpha", [0.0, 0.7])
def test_color_gradient_matches_finite_differences(oracle_lib, K, a_ent, alpha):
    """dR/dW through the Clamp-normalise map (App. C.4) equals central finite
    differences of R (conflicts + gamma s_K - S alpha sum STD) to 1e-7 relative."""
    g = G.erdos_renyi(9, 0.4, 30 + K)
    p = Params(S=4, a_ent=a_ent, alpha_comm=alpha, comm_eps=1e-8)
    rng = np.random.default_rng(K * 10 + a_ent)
    W = 0.1 + 0.8 * rng.random((g.n, K, p.S))
    gam = -0.8
    Gm = oracle.color_gradient(g, K, p, gam, W)
    h = 1e-5
    worst = 0.0
    for idx in np.ndindex(W.shape):
        Wp = W.copy(); Wp[idx] += h
        Wm = W.copy(); Wm[idx] -= h
        fd = (oracle.color_objective(g, K, p, gam, Wp) - oracle.color_objective(g, K, p, gam, Wm)) / (2 * h)
        worst = max(worst, abs(fd - Gm[idx]) / max(1.0, abs(Gm[idx])))
    assert worst < 1e-7


def test_color_step_is_torch_adamw_and_noise_then_projection(oracle_lib):
    """A colouring step is torch.optim.AdamW (FP64) on the oracle's dR/dW, plus
    sqrt(2 lr T) xi with xi the Gaussian of counter row i*K + k, then the
    projection of W to [0, 1]."""
    torch = pytest.importorskip("torch")
    g = G.erdos_renyi(12, 0.3, 4)
    K = 4
    p = Params(S=5, steps=40, lr=2e-3, temperature=0.0, alpha_comm=0.3, weight_decay=0.01, seed=9)
    rng = np.random.default_rng(3)
    W = 0.3 + 0.4 * rng.random((g.n, K, p.S))
    wt = torch.tensor(W, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.AdamW([wt], lr=p.lr, betas=(p.beta1, p.beta2), eps=p.adam_eps,
                            weight_decay=p.weight_decay, foreach=False)
    m = np.zeros_like(W)
    v = np.zeros_like(W)
    for t in range(5):
        grad = oracle.color_gradient(g, K, p, oracle.gamma(MIS, p, t), W)
        wt.grad = torch.tensor(grad, dtype=torch.float64)
        opt.step()
        out = oracle.color_step(g, K, p, t, W, m, v)
        W, m, v = out.X, out.m, out.v
        assert 0.0 < W.min() and W.max() < 1.0
        np.testing.assert_allclose(W, wt.detach().numpy(), rtol=1e-13, atol=1e-15)
    pT = p.with_(temperature=0.01)
    a = oracle.color_step(g, K, p, 2, W, m, v)
    b = oracle.color_step(g, K, pT, 2, W, m, v)
    xi = np.array([[[oracle.gaussian(p.seed, i * K + k, s, 2) for s in range(p.S)] for k in range(K)]
                   for i in range(g.n)])
    np.testing.assert_allclose(b.X - a.X, math.sqrt(2 * p.lr * 0.01) * xi, atol=1e-14)
    big = oracle.color_step(g, K, p.with_(lr=30.0, temperature=4.0), 2, W, m, v)
    assert big.X.min() >= 0.0 and big.X.max() <= 1.0 and np.any(big.X == 0.0) and np.any(big.X == 1.0)


def test_color_init_and_rounding_rules(oracle_lib):
    """W starts as the U(0,1] draw of counter row i*K + k; rounding takes the
    colour of the largest sigma (lowest colour on ties) and the best replica has
    the fewest conflicts (lowest index on ties)."""
    g = G.erdos_renyi(10, 0.4, 5)
    K, S = 3, 4
    W = oracle.color_init(g.n, K, S, 77)
    for (i, k, s) in [(0, 0, 0), (3, 2, 1), (9, 1, 3)]:
        assert W[i, k, s] == oracle.uniform(77, i * K + k, s, 0, 0)
    W2 = np.zeros((g.n, K, S))
    W2[:, 1, :] = 0.5
    W2[:, 2, :] = 0.5          # tie between colours 1 and 2 -> 1
    W2[0, :, 0] = 0.0          # a zero row is uniform -> colour 0
    x, conf, best = oracle.color_round(g, K, W2)
    assert x[0, 0] == 0 and np.all(x[1:, 0] == 1) and np.all(x[:, 1:] == 1)
    assert conf[1] == g.nnz // 2 and best == int(np.argmin(conf))


def test_color_anneal_matches_brute_force_on_tiny_graphs(oracle_lib):
    """On 20 random graphs of 7 nodes, the oracle anneal (S = 8, 600 steps)
    reaches the brute-force minimum number of conflicts with 3 colours on at
    least 90% of them."""
    hits = 0
    for seed in range(20):
        g = G.erdos_renyi(7, 0.55, 300 + seed)
        best_bf = min(oracle.color_conflicts(g, np.array(x)) for x in itertools.product(range(3), repeat=g.n))
        conf, best, _, _ = oracle.color_anneal(g, 3, Params(S=8, steps=600, seed=seed, lr=0.1))
        hits += int(conf[best] == best_bf)
    assert hits >= 18


@pytest.mark.parametrize("name", ["queen5-5", "queen6-6", "myciel5"])
def test_color_anneal_reaches_the_papers_conflicts(oracle_lib, name):
    """The oracle anneal reaches the conflict count PQQA reports in Table 6 (a
    proper colouring with the colours of Table 9)."""
    row = [r for r in _color_graphs() if r[0] == name][0]
    g = _make_color_graph(row[1])
    conf, best, _, _ = oracle.color_anneal(g, row[4], Params(S=32, steps=2000, seed=1, lr=0.1))
    assert conf[best] <= row[5]
