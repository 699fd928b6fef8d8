"""Serving path: continuous batching with admission by HBM budget.

Requests that arrive while others run join the class runs between chunks;
each result is bit-identical to the same request served alone (one launch
shape per replica class, no cross-instance arithmetic in MIS / max-cut)."""
import ctypes

import numpy as np
import pytest

import paper_2409_02135_gb300 as qqa
from qqa_inputs import graphs as G
from qqa_inputs.workloads import MAXCUT, MIS, Params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_02135_gb300 import _build
    _build.build()


def _requests():
    out = []
    for k in range(7):
        kind = MIS if k % 2 == 0 else MAXCUT
        n = [150, 420, 90, 333, 777, 60, 512][k]
        g = G.erdos_renyi_avg_degree(n, 6.0, 100 + k)
        S = [32, 64, 32, 128, 64, 100, 32][k]
        steps = [150, 320, 90, 210, 400, 120, 260][k]
        p = Params(S=S, steps=steps, seed=40 + k, lr=1.0, gamma_min=-5.0 if kind == MAXCUT else -2.0)
        out.append((kind, g, p))
    return out


def _serve(reqs, budget=1 << 34, arrive_every=2, chunk=30):
    srv = qqa.Server(budget, chunk_steps=chunk, slots_per_class=4)
    ids = {}
    pending = list(range(len(reqs)))
    pumps = 0
    while pending or any(srv.poll(i)["state"] in (qqa.REQ_QUEUED, qqa.REQ_RUNNING) for i in ids.values()):
        if pending and pumps % arrive_every == 0:
            k = pending.pop(0)
            kind, g, p = reqs[k]
            ids[k] = srv.submit(kind, g, qqa.make_params(p))
        srv.pump()
        pumps += 1
        assert pumps < 10_000
    return srv, ids


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = _requests()
    srv, ids = _serve(reqs, arrive_every=2)
    overlapped = False
    infos = {k: srv.poll(i) for k, i in ids.items()}
    for a in infos.values():
        for b in infos.values():
            if a is not b and a["t_admit"] < b["t_done"] and b["t_admit"] < a["t_done"]:
                overlapped = True
    assert overlapped, "requests never ran at the same time"
    for k, (kind, g, p) in enumerate(reqs):
        assert infos[k]["state"] == qqa.REQ_DONE
        mixed = srv.result(ids[k])
        alone_srv, alone_ids = _serve([reqs[k]], arrive_every=1)
        alone = alone_srv.result(alone_ids[0])
        np.testing.assert_array_equal(mixed["obj"], alone["obj"])
        np.testing.assert_array_equal(mixed["viol"], alone["viol"])
        np.testing.assert_array_equal(mixed["energy"], alone["energy"])
        assert mixed["best"] == alone["best"]
        np.testing.assert_array_equal(mixed["history"], alone["history"])
        alone_srv.close()


CLASS_FIXED = 4 * 512 + 8192   # fixed buffers of a class run of 4 slots


def _charges(reqs):
    """Device bytes the server charges each request (read back from a server
    that only queues them)."""
    probe = qqa.Server(1 << 40, chunk_steps=30, slots_per_class=4)
    out = [probe.poll(probe.submit(kind, g, qqa.make_params(p)))["bytes"] for kind, g, p in reqs]
    probe.close()
    return out


def test_admission_respects_the_hbm_budget_and_rejects_oversize():
    reqs = _requests()
    sizes = _charges(reqs)
    for (kind, g, p), b in zip(reqs, sizes):
        assert b >= qqa.request_bytes(g.n, g.nnz, p.S, qqa.FP32)   # the estimate leaves out granules and history
    budget = max(sizes) + min(sizes) + 3 * CLASS_FIXED   # the largest and the smallest fit, little else
    srv = qqa.Server(budget, chunk_steps=30, slots_per_class=4)
    ids = [srv.submit(kind, g, qqa.make_params(p)) for kind, g, p in reqs]
    huge = G.erdos_renyi_avg_degree(50_000, 4.0, 1)
    big_id = srv.submit(MIS, huge, qqa.make_params(Params(S=256, steps=10)))
    assert srv.poll(big_id)["state"] == qqa.REQ_FAILED and srv.poll(big_id)["error"] == qqa.QQA_ENOMEM
    for _ in range(10_000):
        running, queued, _ = srv.pump()
        used, _ = srv.stats()
        assert used <= budget
        if running == 0 and queued == 0:
            break
    assert all(srv.poll(i)["state"] == qqa.REQ_DONE for i in ids)


def test_cancel_frees_the_slot_and_others_finish():
    reqs = _requests()
    srv = qqa.Server(1 << 34, chunk_steps=30, slots_per_class=1)
    ids = [srv.submit(kind, g, qqa.make_params(p)) for kind, g, p in reqs]
    srv.pump()
    running = [i for i in ids if srv.poll(i)["state"] == qqa.REQ_RUNNING]
    assert running
    srv.cancel(running[0])
    assert srv.poll(running[0])["state"] == qqa.REQ_CANCELLED
    for _ in range(10_000):
        r, q, _ = srv.pump()
        if r == 0 and q == 0:
            break
    assert all(srv.poll(i)["state"] == qqa.REQ_DONE for i in ids if i != running[0])


def test_allocation_failure_fails_only_that_request():
    """An allocator that refuses once: the request being admitted fails with
    QQA_ENOMEM, the others complete."""
    import torch
    state = {"fail_at": None, "count": 0}

    def _alloc(nbytes, stream, ctx):
        state["count"] += 1
        if state["fail_at"] is not None and state["count"] == state["fail_at"]:
            return None
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))

    def _free(ptr, stream, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    alloc = qqa.qqa_allocator(qqa.ALLOC_FN(_alloc), qqa.FREE_FN(_free), None)
    reqs = _requests()[:4]
    srv = qqa.Server(1 << 34, chunk_steps=30, slots_per_class=4, allocator=alloc)
    ids = [srv.submit(kind, g, qqa.make_params(p)) for kind, g, p in reqs[:2]]
    srv.pump()
    state["fail_at"] = state["count"] + 5      # a state buffer of the next admitted request
    ids += [srv.submit(kind, g, qqa.make_params(p)) for kind, g, p in reqs[2:]]
    for _ in range(10_000):
        r, q, _ = srv.pump()
        if r == 0 and q == 0:
            break
    states = [srv.poll(i) for i in ids]
    failed = [s for s in states if s["state"] == qqa.REQ_FAILED]
    assert len(failed) == 1 and failed[0]["error"] == qqa.QQA_ENOMEM
    assert sum(s["state"] == qqa.REQ_DONE for s in states) == 3
    used, classes = srv.stats()
    assert used == classes * CLASS_FIXED      # only the class runs' fixed buffers remain charged
    srv.close()


def test_device_memory_stays_within_the_budget():
    """A counting allocator sees every byte the server's runs and graphs take:
    with a budget that admits only part of a mixed trace at a time, the live
    bytes never exceed the budget, and every request completes."""
    import torch
    live = {"bytes": 0, "peak": 0}
    sizes_of = {}

    def _alloc(nbytes, stream, ctx):
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        sizes_of[int(ptr)] = int(nbytes)
        live["bytes"] += int(nbytes)
        live["peak"] = max(live["peak"], live["bytes"])
        return ptr

    def _free(ptr, stream, ctx):
        if ptr:
            live["bytes"] -= sizes_of.pop(int(ptr))
            torch.cuda.caching_allocator_delete(int(ptr))

    alloc = qqa.qqa_allocator(qqa.ALLOC_FN(_alloc), qqa.FREE_FN(_free), None)
    reqs = _requests()
    hub = G.barabasi_albert(3000, 4, 9)       # long rows: their tables and partial sums are charged too
    reqs.append((MAXCUT, hub, Params(S=64, steps=200, seed=77, lr=1.0, gamma_min=-5.0)))
    sizes = _charges(reqs)
    budget = max(sizes) + int(0.3 * (sum(sizes) - max(sizes))) + 3 * CLASS_FIXED
    srv = qqa.Server(budget, chunk_steps=30, slots_per_class=4, allocator=alloc)
    ids = [srv.submit(kind, g, qqa.make_params(p)) for kind, g, p in reqs]
    for _ in range(10_000):
        r, q, _ = srv.pump()
        used, _ = srv.stats()
        assert used <= budget and live["bytes"] <= used
        if r == 0 and q == 0:
            break
    assert all(srv.poll(i)["state"] == qqa.REQ_DONE for i in ids)
    assert live["peak"] <= budget
    srv.close()
