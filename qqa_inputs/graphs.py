"""Seeded random-graph generators returning symmetric CSR adjacency.

Every generator takes an integer seed and uses numpy's PCG64 generator, which
gives the same stream on x86 and Arm. The CSR is int32, each row sorted
ascending, no self-loops, no duplicate entries, and symmetric (both directions
of every undirected edge are stored).

Shapes follow the paper's synthetic workloads (App. D.2, Table 7): Erdos-Renyi
graphs for MIS and max-cut, Barabasi-Albert graphs for max-cut, random regular
graphs for MIS (Sec. 5.1), and an RB-model-like clique-block generator standing
in for the constraint-structured MIS/clique instances.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSRGraph:
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray      # int32 [nnz]
    w: np.ndarray | None = None  # int32 [nnz] edge weights, None = unit

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def num_edges(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def upper_edges(self):
        """(u, v, w) arrays with u < v, one entry per undirected edge."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        cols = self.col.astype(np.int64)
        keep = rows < cols
        w = None if self.w is None else self.w[keep]
        return rows[keep], cols[keep], w

    def dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n), dtype=np.int64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        a[rows, self.col] = 1 if self.w is None else self.w
        return a


def from_edges(n: int, u, v, w=None) -> CSRGraph:
    """Build a symmetric CSR from undirected edges (u_k, v_k); u_k != v_k, no repeats."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if u.size:
        if np.any(u == v):
            raise ValueError("self-loop in edge list")
        if u.min() < 0 or v.min() < 0 or max(u.max(), v.max()) >= n:
            raise ValueError("edge endpoint out of range")
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    ww = None
    if w is not None:
        w = np.asarray(w, dtype=np.int64)
        ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    if ww is not None:
        ww = ww[order]
    if src.size > 1:
        dup = (src[1:] == src[:-1]) & (dst[1:] == dst[:-1])
        if np.any(dup):
            raise ValueError("duplicate edge in edge list")
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    return CSRGraph(n=n, row_ptr=row_ptr.astype(np.int32), col=dst.astype(np.int32),
                    w=None if ww is None else ww.astype(np.int32))


def _dedupe_pairs(n: int, a: np.ndarray, b: np.ndarray):
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    keep = lo != hi
    key = np.unique(lo[keep] * n + hi[keep])
    return key // n, key % n


def erdos_renyi(n: int, p: float, seed: int) -> CSRGraph:
    """G(n, p): each of the n(n-1)/2 pairs is an edge independently with probability p."""
    rng = np.random.default_rng(np.random.SeedSequence([0x45524E59, int(seed)]))
    if n <= 4096:
        iu, ju = np.triu_indices(n, k=1)
        mask = rng.random(iu.size) < p
        return from_edges(n, iu[mask], ju[mask])
    # large sparse case: draw the edge count, then distinct uniform pairs
    pairs = n * (n - 1) // 2
    m = int(rng.binomial(pairs, p))
    have_u = np.zeros(0, dtype=np.int64)
    have_v = np.zeros(0, dtype=np.int64)
    while have_u.size < m:
        need = m - have_u.size
        k = int(need * 1.1) + 16
        a = rng.integers(0, n, size=k, dtype=np.int64)
        b = rng.integers(0, n, size=k, dtype=np.int64)
        u, v = _dedupe_pairs(n, np.concatenate([have_u, a]), np.concatenate([have_v, b]))
        have_u, have_v = u, v
    sel = np.sort(rng.choice(have_u.size, size=m, replace=False))
    return from_edges(n, have_u[sel], have_v[sel])


def erdos_renyi_avg_degree(n: int, avg_degree: float, seed: int) -> CSRGraph:
    """G(n, p) with p = avg_degree / (n - 1)."""
    return erdos_renyi(n, min(1.0, avg_degree / max(1, n - 1)), seed)


def random_regular(n: int, d: int, seed: int, max_tries: int = 1000) -> CSRGraph:
    """Uniform simple d-regular graph by the pairing (configuration) model.

    Stubs are paired uniformly; a pairing with a self-loop or a repeated edge
    is repaired by random double-edge swaps that remove the defect (for d <= 4
    plain rejection succeeds quickly, larger d relies on the swaps).
    """
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    rng = np.random.default_rng(np.random.SeedSequence([0x52524721, int(seed), int(d)]))
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n, dtype=np.int64), d)
        rng.shuffle(stubs)
        a = stubs[0::2].copy()
        b = stubs[1::2].copy()
        if d <= 4:
            lo, hi = np.minimum(a, b), np.maximum(a, b)
            if np.any(lo == hi):
                continue
            key = lo * n + hi
            if np.unique(key).size != key.size:
                continue
            return from_edges(n, lo, hi)
        ok = _repair_pairing(n, a, b, rng)
        if ok:
            return from_edges(n, np.minimum(a, b), np.maximum(a, b))
    raise RuntimeError("random_regular: no simple pairing found")


def _repair_pairing(n, a, b, rng, max_rounds=200):
    """Double-edge swaps until the multigraph (a_k, b_k) is simple."""
    m = a.size
    for _ in range(max_rounds):
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        key = lo * n + hi
        order = np.argsort(key, kind="stable")
        sk = key[order]
        dup = np.zeros(m, dtype=bool)
        dup[order[1:][sk[1:] == sk[:-1]]] = True
        bad = np.flatnonzero((a == b) | dup)
        if bad.size == 0:
            return True
        present = set(key.tolist())
        for e in bad.tolist():
            for _try in range(50):
                f = int(rng.integers(0, m))
                if f == e:
                    continue
                u, v, x, y = int(a[e]), int(b[e]), int(a[f]), int(b[f])
                # rewire (u,v),(x,y) -> (u,x),(v,y)
                if u == x or v == y:
                    continue
                k1 = min(u, x) * n + max(u, x)
                k2 = min(v, y) * n + max(v, y)
                if k1 in present or k2 in present or k1 == k2:
                    continue
                present.discard(min(x, y) * n + max(x, y))
                present.add(k1)
                present.add(k2)
                a[e], b[e], a[f], b[f] = u, x, v, y
                break
    return False


def barabasi_albert(n: int, m: int, seed: int) -> CSRGraph:
    """Preferential attachment: start from a star on m+1 nodes, then each new
    node links to m distinct existing nodes chosen with probability proportional
    to their degree."""
    if n <= m:
        raise ValueError("need n > m")
    rng = np.random.default_rng(np.random.SeedSequence([0x42412121, int(seed), int(m)]))
    src = list(range(1, m + 1))
    dst = [0] * m
    # every edge endpoint once: sampling uniformly from it is degree-proportional
    ends = np.empty(2 * (m + (n - m - 1) * m), dtype=np.int64)
    ends[: 2 * m] = np.array(src + dst, dtype=np.int64)
    filled = 2 * m
    us, vs = [np.array(src, dtype=np.int64)], [np.array(dst, dtype=np.int64)]
    for node in range(m + 1, n):
        targets = set()
        while len(targets) < m:
            picks = ends[rng.integers(0, filled, size=2 * m)]
            for t in picks.tolist():
                targets.add(t)
                if len(targets) == m:
                    break
        tg = np.fromiter(targets, dtype=np.int64, count=m)
        tg.sort()
        us.append(np.full(m, node, dtype=np.int64))
        vs.append(tg)
        ends[filled: filled + m] = node
        ends[filled + m: filled + 2 * m] = tg
        filled += 2 * m
    return from_edges(n, np.concatenate(vs), np.concatenate(us))


def clique_blocks(n: int, seed: int, size_lo: int = 5, size_hi: int = 25, p_inter: float = 0.02) -> CSRGraph:
    """Constraint-structured graph: nodes split into consecutive cliques whose
    sizes are uniform in [size_lo, size_hi] (the last one takes the remainder),
    complete inside each clique, plus Erdos-Renyi edges with probability
    p_inter between nodes of different cliques."""
    rng = np.random.default_rng(np.random.SeedSequence([0x43424C4B, int(seed)]))
    sizes = []
    left = n
    while left > 0:
        s = int(rng.integers(size_lo, size_hi + 1))
        s = min(s, left)
        sizes.append(s)
        left -= s
    block = np.repeat(np.arange(len(sizes)), sizes)
    us, vs = [], []
    start = 0
    for s in sizes:
        iu, ju = np.triu_indices(s, k=1)
        us.append(iu + start)
        vs.append(ju + start)
        start += s
    # inter-block ER edges, sampled as G(n, p_inter) restricted to different blocks
    if n <= 4096:
        iu, ju = np.triu_indices(n, k=1)
        mask = (rng.random(iu.size) < p_inter) & (block[iu] != block[ju])
        us.append(iu[mask])
        vs.append(ju[mask])
    else:
        er = erdos_renyi(n, p_inter, int(rng.integers(0, 2**31)))
        a, b, _ = er.upper_edges()
        keep = block[a] != block[b]
        us.append(a[keep])
        vs.append(b[keep])
    return from_edges(n, np.concatenate(us), np.concatenate(vs))


def disjoint_union(graphs) -> CSRGraph:
    """Block-diagonal union of graphs (node ids offset in order)."""
    us, vs, ws = [], [], []
    off = 0
    weighted = any(g.w is not None for g in graphs)
    for g in graphs:
        a, b, w = g.upper_edges()
        us.append(a + off)
        vs.append(b + off)
        if weighted:
            ws.append(w if w is not None else np.ones(a.size, dtype=np.int64))
        off += g.n
    return from_edges(off, np.concatenate(us), np.concatenate(vs),
                      np.concatenate(ws) if weighted else None)


def queens(rows: int, cols: int) -> CSRGraph:
    """Queens graph of a rows x cols board: one node per square (row-major), two
    squares adjacent when they share a row, a column or a diagonal (the COLOR
    benchmark family queen<r>_<c>)."""
    us, vs = [], []
    for a in range(rows * cols):
        ra, ca = divmod(a, cols)
        for b in range(a + 1, rows * cols):
            rb, cb = divmod(b, cols)
            if ra == rb or ca == cb or abs(ra - rb) == abs(ca - cb):
                us.append(a)
                vs.append(b)
    return from_edges(rows * cols, np.array(us, dtype=np.int64), np.array(vs, dtype=np.int64))


def mycielski(level: int) -> CSRGraph:
    """Mycielski graph of the COLOR family myciel<level>: the 5-cycle is
    myciel2, and each level applies the Mycielski construction (nodes v_i of G,
    copies u_i adjacent to the neighbours of v_i, and one node w adjacent to every
    u_i), which keeps the graph triangle-free and raises the chromatic number by one
    (myciel<l> has chromatic number l + 1)."""
    if level < 2:
        raise ValueError("level >= 2 (myciel2 is the 5-cycle)")
    n = 5
    edges = [(i, (i + 1) % 5) for i in range(5)]
    for _ in range(level - 2):
        new = list(edges)
        for (a, b) in edges:          # u_a ~ v_b and u_b ~ v_a
            new.append((n + a, b))
            new.append((n + b, a))
        w = 2 * n
        for i in range(n):
            new.append((n + i, w))
        edges, n = new, 2 * n + 1
    u = np.array([min(a, b) for a, b in edges], dtype=np.int64)
    v = np.array([max(a, b) for a, b in edges], dtype=np.int64)
    return from_edges(n, u, v)
