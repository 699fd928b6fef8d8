"""Python binding of libqqa: GB300 (sm_103a) CUDA implementation of the per-step
replica update of Parallel Quasi-Quantum Annealing (Ichikawa & Arai, arXiv 2409.02135).

Every step of the method runs in the CUDA kernels behind the C ABI declared in
include/qqa.h; this module only marshals numpy arrays and stream handles.
There is no CPU fallback: without the built library or a CUDA device, calls
raise.

    import paper_2409_02135_gb300 as qqa
    prob = qqa.Problem(qqa.MIS, graph)                # graph: n, row_ptr, col, w
    run = qqa.anneal([prob], [params])                # init + K steps + evaluation
    res = run.result(0)                               # objective, feasibility, best replica
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import (  # noqa: F401
    BF16, FP32, KERNEL_AUTO, KERNEL_DENSE, KERNEL_DIRECT, KERNEL_PIPE, KERNEL_SCALAR, KERNEL_STAGED, KERNEL_STREAM, MAXCLIQUE, MAXCUT, MIS, QQA_EBUSY, QQA_ECUDA, QQA_EINVAL, QQA_ENOMEM, QQA_ENONFINITE, QQA_ETIMEOUT, QQA_OK,
    QQAError, check, load, qqa_allocator, qqa_launch_config, qqa_params, qqa_request_info, ALLOC_FN, FREE_FN,
    SIGNATURES, REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED,
)

__all__ = ["Problem", "Run", "Server", "anneal", "autotune", "make_params", "LaunchConfig", "QQAError", "MIS",
           "MAXCUT", "MAXCLIQUE", "FP32", "BF16", "launch_count", "torch_allocator", "stream_handle",
           "request_bytes", "round_eval_noalloc", "Coloring", "color_anneal"]


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def stream_handle(stream) -> int:
    """cudaStream_t of a torch.cuda.Stream, an int handle, or None (legacy default stream)."""
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def launch_count() -> int:
    return int(load().qqa_launch_count())


def version() -> str:
    return load().qqa_version().decode()


def make_params(src=None, **kw) -> qqa_params:
    """qqa_params from the library defaults, an object with the same attribute
    names (S, steps, round_every, a_ent, lr, weight_decay, beta1, beta2,
    adam_eps, gamma_min, gamma_max, alpha_comm, comm_eps, temperature, lam,
    seed, precision) and/or keyword overrides."""
    p = qqa_params()
    load().qqa_default_params(ctypes.byref(p))
    names = [f[0] for f in qqa_params._fields_ if f[0] != "reserved"]
    if src is not None:
        for name in names:
            if hasattr(src, name):
                setattr(p, name, getattr(src, name))
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def LaunchConfig(group_lanes=0, vec_per_lane=0, block_threads=0, grid_blocks=0, use_graphs=1, kernel=0,
                 kernel_param=0, rows_per_warp=None) -> qqa_launch_config:
    """kernel: 0 auto, 1 direct gather, 2 TMA-staged (kernel_param = row groups per warp),
    3 cp.async streaming (kernel_param = neighbour rows prefetched per row)."""
    if rows_per_warp is not None:
        kernel_param = rows_per_warp
    return qqa_launch_config(group_lanes, vec_per_lane, block_threads, grid_blocks, use_graphs, kernel,
                             kernel_param, 0)


_keep_alive = []


def torch_allocator():
    """qqa_allocator that takes device memory from PyTorch's caching allocator."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # out of memory is reported to the caller as QQA_ENOMEM
            return None

    def _free(ptr, stream, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    a = qqa_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    _keep_alive.append(a)
    return a


class Problem:
    """Device copy of one graph (qqa_create_problem)."""

    def __init__(self, kind: int, graph, stream=None, allocator=None):
        self.kind = int(kind)
        self.n = int(graph.n)
        rp = np.ascontiguousarray(graph.row_ptr, dtype=np.int32)
        col = np.ascontiguousarray(graph.col, dtype=np.int32)
        w = None if getattr(graph, "w", None) is None else np.ascontiguousarray(graph.w, dtype=np.int32)
        self.nnz = int(rp[-1])
        self._alloc = allocator
        h = ctypes.c_void_p()
        check(load().qqa_create_problem(self.kind, self.n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                        _ptr(w, ctypes.c_int32), ctypes.byref(allocator) if allocator else None,
                                        stream_handle(stream), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().qqa_destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Run:
    """Replica state of one or more instances (qqa_run_*)."""

    def __init__(self, handle, problems, params, stream=None, allocator=None):
        self.handle = handle
        self.problems = {}
        self.params = {}
        self.stream = stream
        self._alloc = allocator
        for k, (pb, pr) in enumerate(zip(problems, params)):
            self.problems[k] = pb
            self.params[k] = pr

    # -- construction ----------------------------------------------------
    @classmethod
    def create(cls, problems, params, config=None, stream=None, allocator=None):
        ps = (qqa_params * len(problems))(*params)
        hs = (ctypes.c_void_p * len(problems))(*[p.handle for p in problems])
        h = ctypes.c_void_p()
        check(load().qqa_run_create(hs, ps, len(problems), ctypes.byref(config) if config else None,
                                    ctypes.byref(allocator) if allocator else None, stream_handle(stream),
                                    ctypes.byref(h)))
        return cls(h, problems, list(params), stream, allocator)

    @classmethod
    def empty(cls, capacity: int, S_max: int, precision: int = FP32, config=None, stream=None, allocator=None):
        h = ctypes.c_void_p()
        check(load().qqa_run_create_empty(capacity, S_max, precision, ctypes.byref(config) if config else None,
                                          ctypes.byref(allocator) if allocator else None, stream_handle(stream),
                                          ctypes.byref(h)))
        return cls(h, [], [], stream, allocator)

    def add(self, problem: Problem, params: qqa_params) -> int:
        slot = ctypes.c_int32()
        check(load().qqa_run_add(self.handle, problem.handle, ctypes.byref(params), stream_handle(self.stream),
                                 ctypes.byref(slot)))
        self.problems[slot.value] = problem
        self.params[slot.value] = params
        return slot.value

    def reset(self, seed: int, slot: int = -1):
        """Restart one slot (or all, slot = -1) from a fresh initial state drawn with seed."""
        check(load().qqa_run_reset(self.handle, int(slot), int(seed), stream_handle(self.stream)))
        for k, p in self.params.items():
            if slot in (-1, k):
                p.seed = int(seed)

    def remove(self, slot: int):
        check(load().qqa_run_remove(self.handle, slot, stream_handle(self.stream)))
        self.problems.pop(slot, None)
        self.params.pop(slot, None)

    def close(self):
        if getattr(self, "handle", None):
            load().qqa_run_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stepping ----------------------------------------------------------
    def config(self) -> qqa_launch_config:
        c = qqa_launch_config()
        check(load().qqa_run_config(self.handle, ctypes.byref(c)))
        return c

    def steps(self, nsteps: int):
        check(load().qqa_run_steps(self.handle, int(nsteps), stream_handle(self.stream)))

    def eval(self):
        check(load().qqa_run_eval(self.handle, stream_handle(self.stream)))

    def sync(self):
        check(load().qqa_run_sync(self.handle, stream_handle(self.stream)))

    def slot_step(self, slot: int) -> int:
        t = ctypes.c_int32()
        check(load().qqa_run_slot_step(self.handle, slot, ctypes.byref(t)))
        return t.value

    # -- results -----------------------------------------------------------
    def result(self, slot: int, with_x: bool = True) -> dict:
        S = int(self.params[slot].S)
        n = self.problems[slot].n
        obj = np.zeros(S, np.int64)
        viol = np.zeros(S, np.int64)
        feas = np.zeros(S, np.uint8)
        en = np.zeros(S, np.float64)
        best = ctypes.c_int32()
        step = ctypes.c_int32()
        bx = np.zeros((n + 31) // 32, np.uint32) if with_x else None
        check(load().qqa_run_result(self.handle, slot, _ptr(obj, ctypes.c_int64), _ptr(viol, ctypes.c_int64),
                                    _ptr(feas, ctypes.c_uint8), _ptr(en, ctypes.c_double), ctypes.byref(best),
                                    _ptr(bx, ctypes.c_uint32), ctypes.byref(step)))
        out = {"obj": obj, "viol": viol, "feasible": feas.astype(bool), "energy": en, "best": best.value,
               "step": step.value}
        if with_x:
            bits = np.unpackbits(bx.view(np.uint8), bitorder="little")[:n]
            out["best_x"] = bits.astype(np.uint8)
        return out

    def history(self, slot: int):
        cap = int(self.params[slot].steps) + 2
        best = np.zeros(cap, np.int64)
        at = np.zeros(cap, np.int32)
        cnt = ctypes.c_int32()
        check(load().qqa_run_history(self.handle, slot, cap, _ptr(best, ctypes.c_int64), _ptr(at, ctypes.c_int32),
                                     ctypes.byref(cnt)))
        m = min(cnt.value, cap)
        return best[:m], at[:m]

    # -- state ---------------------------------------------------------------
    def get_state(self, slot: int):
        S = int(self.params[slot].S)
        n = self.problems[slot].n
        X = np.zeros((n, S), np.float32)
        m = np.zeros((n, S), np.float32)
        v = np.zeros((n, S), np.float32)
        t = ctypes.c_int32()
        check(load().qqa_run_get_state(self.handle, slot, stream_handle(self.stream), _ptr(X, ctypes.c_float),
                                       _ptr(m, ctypes.c_float), _ptr(v, ctypes.c_float), ctypes.byref(t)))
        return X, m, v, t.value

    def set_state(self, slot: int, X, m, v, t: int):
        X = np.ascontiguousarray(X, dtype=np.float32)
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        check(load().qqa_run_set_state(self.handle, slot, stream_handle(self.stream), _ptr(X, ctypes.c_float),
                                       _ptr(m, ctypes.c_float), _ptr(v, ctypes.c_float), int(t)))

    def step_debug(self, slot: int):
        S = int(self.params[slot].S)
        n = self.problems[slot].n
        g = np.zeros((n, S), np.float32)
        check(load().qqa_run_step_debug(self.handle, slot, stream_handle(self.stream), _ptr(g, ctypes.c_float)))
        return g

    def debug_set_status(self, nonfinite: int = 0, timeouts: int = 0):
        """Test hook: overwrite the device status word that sync() reports."""
        check(load().qqa_run_debug_set_status(self.handle, int(nonfinite), int(timeouts), stream_handle(self.stream)))


def autotune(problems, params, trial_steps: int = 100, stream=None, allocator=None):
    """qqa_autotune: the fastest launch shape for these instances (cached per
    workload signature). Returns (qqa_launch_config, microseconds per step)."""
    ps = (qqa_params * len(problems))(*params)
    hs = (ctypes.c_void_p * len(problems))(*[p.handle for p in problems])
    cfg = qqa_launch_config()
    us = ctypes.c_float()
    check(load().qqa_autotune(hs, ps, len(problems), int(trial_steps),
                              ctypes.byref(allocator) if allocator else None, stream_handle(stream),
                              ctypes.byref(cfg), ctypes.byref(us)))
    return cfg, float(us.value)


def round_eval_noalloc(kind: int, n: int, nnz: int, row_ptr, col, w, S: int, ld: int, X, lam: float,
                       obj, viol, feasible, energy, best_s, stream=None):
    """qqa_round_eval_noalloc: evaluate a state held in caller-owned device
    memory without any device allocation (for callers that must not allocate
    while they evaluate). All array arguments are device addresses (ints) or
    objects with data_ptr(); w may be None."""
    def addr(a):
        if a is None:
            return None
        return int(a.data_ptr()) if hasattr(a, "data_ptr") else int(a)
    rc = load().qqa_round_eval_noalloc(int(kind), int(n), int(nnz), addr(row_ptr), addr(col), addr(w), int(S),
                                       int(ld), addr(X), float(lam), addr(obj), addr(viol), addr(feasible),
                                       addr(energy), addr(best_s), stream_handle(stream))
    if rc != QQA_OK:
        raise QQAError(rc, load().qqa_noalloc_last_error().decode(errors="replace"))


def anneal(problems, params, config=None, stream=None, allocator=None) -> Run:
    """Whole anneal (qqa_anneal): init, K steps with periodic rounding, final evaluation."""
    ps = (qqa_params * len(problems))(*params)
    hs = (ctypes.c_void_p * len(problems))(*[p.handle for p in problems])
    h = ctypes.c_void_p()
    check(load().qqa_anneal(hs, ps, len(problems), ctypes.byref(config) if config else None,
                            ctypes.byref(allocator) if allocator else None, stream_handle(stream), ctypes.byref(h)))
    return Run(h, problems, list(params), stream, allocator)


def request_bytes(n: int, nnz: int, S: int, precision: int = FP32, weighted: bool = False) -> int:
    """Device bytes the server charges a request (state, evaluation buffers, graph)."""
    return int(load().qqa_request_bytes(int(n), int(nnz), int(S), int(precision), int(bool(weighted))))


class Server:
    """Continuous-batching solve server (qqa_server_*): FIFO admission by HBM
    budget into per-replica-class runs, one chunk of steps per pump."""

    def __init__(self, budget_bytes: int, chunk_steps: int = 50, slots_per_class: int = 64, precision: int = FP32,
                 config=None, allocator=None):
        h = ctypes.c_void_p()
        self._alloc = allocator
        check(load().qqa_server_create(int(budget_bytes), int(chunk_steps), int(slots_per_class), int(precision),
                                       ctypes.byref(config) if config else None,
                                       ctypes.byref(allocator) if allocator else None, ctypes.byref(h)))
        self.handle = h
        self.meta = {}

    def submit(self, kind: int, graph, params: qqa_params) -> int:
        rp = np.ascontiguousarray(graph.row_ptr, dtype=np.int32)
        col = np.ascontiguousarray(graph.col, dtype=np.int32)
        w = None if getattr(graph, "w", None) is None else np.ascontiguousarray(graph.w, dtype=np.int32)
        rid = ctypes.c_int64()
        check(load().qqa_server_submit(self.handle, int(kind), int(graph.n), _ptr(rp, ctypes.c_int32),
                                       _ptr(col, ctypes.c_int32), _ptr(w, ctypes.c_int32), ctypes.byref(params),
                                       ctypes.byref(rid)))
        self.meta[rid.value] = (int(graph.n), int(params.S))
        return rid.value

    def pump(self):
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(load().qqa_server_pump(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def poll(self, rid: int) -> dict:
        info = qqa_request_info()
        check(load().qqa_server_poll(self.handle, int(rid), ctypes.byref(info)))
        return {f[0]: getattr(info, f[0]) for f in qqa_request_info._fields_ if f[0] != "reserved"}

    def result(self, rid: int) -> dict:
        n, S = self.meta[rid]
        info = self.poll(rid)
        obj = np.zeros(S, np.int64)
        viol = np.zeros(S, np.int64)
        feas = np.zeros(S, np.uint8)
        en = np.zeros(S, np.float64)
        bx = np.zeros((n + 31) // 32, np.uint32)
        hist = np.zeros(max(info["evaluations"], 1), np.int64)
        check(load().qqa_server_result(self.handle, int(rid), _ptr(obj, ctypes.c_int64), _ptr(viol, ctypes.c_int64),
                                       _ptr(feas, ctypes.c_uint8), _ptr(en, ctypes.c_double),
                                       _ptr(bx, ctypes.c_uint32), _ptr(hist, ctypes.c_int64)))
        return {"obj": obj, "viol": viol, "feasible": feas.astype(bool), "energy": en, "best": info["best_s"],
                "best_x": np.unpackbits(bx.view(np.uint8), bitorder="little")[:n].astype(np.uint8),
                "history": hist[:info["evaluations"]], "info": info}

    def cancel(self, rid: int):
        check(load().qqa_server_cancel(self.handle, int(rid)))

    def stats(self):
        used = ctypes.c_int64()
        classes = ctypes.c_int32()
        check(load().qqa_server_stats(self.handle, ctypes.byref(used), ctypes.byref(classes)))
        return used.value, classes.value

    def close(self):
        if getattr(self, "handle", None):
            load().qqa_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Coloring:
    """Categorical PQQA for graph colouring with K colours (qqa_color_*):
    state W[n][K][S] in [0, 1], relaxation sigma = W / sum_k W (App. B, C.4)."""

    def __init__(self, graph, K: int, params, stream=None):
        self.n, self.K = int(graph.n), int(K)
        rp = np.ascontiguousarray(graph.row_ptr, dtype=np.int32)
        col = np.ascontiguousarray(graph.col, dtype=np.int32)
        self.params = make_params(params) if not isinstance(params, qqa_params) else params
        self.S = int(self.params.S)
        self._stream = stream
        h = ctypes.c_void_p()
        check(load().qqa_color_create(self.n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32), self.K,
                                      ctypes.byref(self.params), stream_handle(stream), ctypes.byref(h)))
        self.handle = h

    def steps(self, nsteps: int) -> int:
        done = ctypes.c_int32()
        check(load().qqa_color_steps(self.handle, int(nsteps), ctypes.byref(done)))
        return int(done.value)

    def sync(self):
        check(load().qqa_color_sync(self.handle))

    def step_debug(self):
        g = np.empty((self.n, self.K, self.S), np.float32)
        check(load().qqa_color_step_debug(self.handle, _ptr(g, ctypes.c_float)))
        return g

    def debug_set_status(self, nonfinite: int = 0, timeouts: int = 0):
        """Test hook: overwrite the device counters that sync() reports."""
        check(load().qqa_color_debug_set_status(self.handle, int(nonfinite), int(timeouts)))

    def get_state(self):
        W, m, v = (np.empty((self.n, self.K, self.S), np.float32) for _ in range(3))
        t = ctypes.c_int32()
        check(load().qqa_color_get_state(self.handle, _ptr(W, ctypes.c_float), _ptr(m, ctypes.c_float),
                                         _ptr(v, ctypes.c_float), ctypes.byref(t)))
        return W, m, v, int(t.value)

    def set_state(self, W, m, v, t: int):
        arrs = [np.ascontiguousarray(a, dtype=np.float32).reshape(self.n, self.K, self.S) for a in (W, m, v)]
        check(load().qqa_color_set_state(self.handle, *(_ptr(a, ctypes.c_float) for a in arrs), int(t)))

    def round(self, with_x: bool = True) -> dict:
        conf = np.empty(self.S, np.int64)
        best = ctypes.c_int32()
        x = np.empty((self.n, self.S), np.uint8) if with_x else None
        check(load().qqa_color_round(self.handle, _ptr(conf, ctypes.c_int64), ctypes.byref(best),
                                     _ptr(x, ctypes.c_uint8)))
        return {"conflicts": conf, "best_s": int(best.value), "x": x}

    @property
    def t(self) -> int:
        t = ctypes.c_int32()
        check(load().qqa_color_info(self.handle, None, None, None, ctypes.byref(t)))
        return int(t.value)

    def close(self):
        if getattr(self, "handle", None):
            load().qqa_color_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def color_anneal(graph, K: int, params, stream=None) -> tuple[Coloring, dict]:
    """Initial draw, the full schedule of params.steps steps, and the rounding."""
    c = Coloring(graph, K, params, stream=stream)
    c.steps(c.params.steps)
    return c, c.round()
