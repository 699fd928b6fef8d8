"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
anneals its own instances (no data-path collective), the timed region ends
with a barrier, and the whole-job figures are the max of the ranks' times and
the sum of their work."""
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
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, t, total, sig, len(wl.instances)))


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
    (r0, t0, s0, sig0, n0), (r1, t1, s1, sig1, n1) = out
    assert t0 == t1 == 1.5                 # max over ranks
    assert s0 == s1 == 300.0               # sum over ranks
    assert n0 == n1 == 16                  # weak scaling: same work per rank
    assert sig0 != sig1                    # different graphs on each rank
