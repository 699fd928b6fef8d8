"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
anneals its own instances (no data-path collective), every instance of the
job on exactly one rank, a rank's result equal to the same computation in one
process; the timed region ends with a barrier, and the whole-job figures are
the max of the ranks' times and the sum of their work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup(world)
    assert (w, r) == (world, rank)
    bench.barrier(w)
    t = bench.max_over_ranks(0.5 + rank, w)
    total = bench.sum_over_ranks(100.0 * (rank + 1), w)
    wl = bench.build_workload("mis_er700_800", r)
    sig = [int(i.graph.nnz) for i in wl.instances[:3]]
    # every instance of this rank's shard, by content
    keys = [_graph_key(i.graph) for i in wl.instances]
    # a small anneal of this rank's own small instance on the oracle (what a rank computes)
    import oracle
    small = bench.build_workload("mis_er100", r).instances[0]
    res = oracle.anneal(small.kind, small.graph, small.params, steps=60)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, t, total, sig, len(wl.instances), keys, res.eval.obj.tolist(), int(res.eval.best)))


def _graph_key(g):
    import hashlib
    h = hashlib.sha256()
    h.update(g.row_ptr.tobytes())
    h.update(g.col.tobytes())
    return h.hexdigest()[:16]


def test_two_ranks_shard_instances_and_reduce_timings():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, sig0, n0, k0, o0, b0), (r1, t1, s1, sig1, n1, k1, o1, b1) = out
    assert t0 == t1 == 1.5                 # max over ranks
    assert s0 == s1 == 300.0               # sum over ranks
    assert n0 == n1 == 16                  # weak scaling: same work per rank
    assert sig0 != sig1                    # different graphs on each rank
    # every instance of the job is annealed exactly once: no graph on two ranks,
    # none twice on one rank, and each rank's shard is exactly the one a single
    # process builds for that rank
    assert len(set(k0)) == len(k0) and len(set(k1)) == len(k1) and not set(k0) & set(k1)
    sys.path.insert(0, ROOT)
    import bench
    assert k0 == [_graph_key(i.graph) for i in bench.build_workload("mis_er700_800", 0).instances]
    assert k1 == [_graph_key(i.graph) for i in bench.build_workload("mis_er700_800", 1).instances]
    # and a rank's result equals the same computation in a single process
    import oracle
    for rank, obj, best in ((0, o0, b0), (1, o1, b1)):
        small = bench.build_workload("mis_er100", rank).instances[0]
        res = oracle.anneal(small.kind, small.graph, small.params, steps=60)
        assert obj == res.eval.obj.tolist() and best == int(res.eval.best)
