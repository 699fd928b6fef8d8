"""Seeded input generators: valid symmetric CSR, reproducible, right shapes."""
import numpy as np
import pytest

from qqa_inputs import graphs as G
from qqa_inputs import workloads as W


def _check_csr(g):
    assert g.row_ptr.dtype == np.int32 and g.col.dtype == np.int32
    assert g.row_ptr[0] == 0 and np.all(np.diff(g.row_ptr) >= 0)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    assert np.all(g.col >= 0) and np.all(g.col < g.n)
    assert not np.any(rows == g.col)
    for i in range(0, g.n, max(1, g.n // 50)):
        seg = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
        assert np.all(np.diff(seg) > 0)
    fwd = set(zip(rows.tolist(), g.col.tolist()))
    assert all((b, a) in fwd for (a, b) in list(fwd)[:5000])


def test_erdos_renyi_density_and_reproducible():
    g = G.erdos_renyi(750, 0.15, 3)
    _check_csr(g)
    pairs = 750 * 749 / 2
    assert abs(g.num_edges - 0.15 * pairs) < 5 * np.sqrt(pairs * 0.15 * 0.85)
    g2 = G.erdos_renyi(750, 0.15, 3)
    assert np.array_equal(g.col, g2.col)
    big = G.erdos_renyi_avg_degree(20000, 10, 1)
    _check_csr(big)
    assert abs(big.nnz / big.n - 10) < 0.2


def test_random_regular_degrees():
    for d in (3, 6):
        g = G.random_regular(2000, d, 5)
        _check_csr(g)
        assert np.all(g.degrees() == d)


def test_barabasi_albert_edges():
    g = G.barabasi_albert(1100, 4, 2)
    _check_csr(g)
    assert g.num_edges == 4 + (1100 - 5) * 4     # star on m+1 nodes, then m edges per node
    assert g.degrees().min() >= 4
    assert g.degrees().max() > 40                # heavy tail


def test_clique_blocks_contains_cliques():
    g = G.clique_blocks(500, 3)
    _check_csr(g)
    A = g.dense()
    # the first block is a clique of 5..25 nodes starting at node 0
    k = 1
    while k < 500 and all(A[k, j] for j in range(k)):
        k += 1
    assert 5 <= k <= 26


def test_disjoint_union_offsets():
    a = G.erdos_renyi(30, 0.2, 1)
    b = G.erdos_renyi(40, 0.2, 2)
    u = G.disjoint_union([a, b])
    _check_csr(u)
    assert u.n == 70 and u.nnz == a.nnz + b.nnz
    assert np.array_equal(u.col[u.row_ptr[30]:], b.col + 30)


def test_workload_shapes():
    w = W.er_mis_small()
    assert w.instances[0].graph.n == 100 and w.instances[0].params.S == 8
    w2 = W.er_mis_paper(num_graphs=3)
    assert all(700 <= i.graph.n <= 800 for i in w2.instances)
    tr = W.serving_trace(num=50)
    assert len(tr) == 50 and all(tr[k][0] < tr[k + 1][0] for k in range(49))
    assert {p.S for _, _, p in tr} <= {32, 64, 128, 256}


def test_from_edges_rejects_bad_input():
    with pytest.raises(ValueError):
        G.from_edges(3, [0], [0])
    with pytest.raises(ValueError):
        G.from_edges(3, [0, 1], [1, 0])
    with pytest.raises(ValueError):
        G.from_edges(3, [0], [5])
