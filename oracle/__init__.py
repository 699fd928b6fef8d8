"""FP64 CPU oracle for Parallel Quasi-Quantum Annealing (arXiv 2409.02135).

TEST INFRASTRUCTURE ONLY. This package is the reference that the CUDA path is
checked against. It may be imported only by tests/, __graft_entry__.smoke()
and bench.py's cpu_baseline / reference legs. It shares no code with the CUDA
library (paper_2409_02135_gb300), and that library never imports it.

The arithmetic lives in qqa_oracle.c (plain loops in double precision, one
element at a time, in the order the paper states the method); this module
only marshals numpy arrays to it. Every function here is pinned by
tests/test_oracle_pins.py against what the paper and the mathematics fix.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qqa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MIS, MAXCUT, MAXCLIQUE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP over nodes, no FMA contraction so
    x86 and Arm round identically)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _OracleParams(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("S", ctypes.c_int32), ("K", ctypes.c_int32), ("a_ent", ctypes.c_int32),
        ("lr", ctypes.c_double), ("weight_decay", ctypes.c_double), ("beta1", ctypes.c_double),
        ("beta2", ctypes.c_double), ("adam_eps", ctypes.c_double),
        ("gamma_min", ctypes.c_double), ("gamma_max", ctypes.c_double),
        ("alpha_comm", ctypes.c_double), ("comm_eps", ctypes.c_double),
        ("temperature", ctypes.c_double), ("lam", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        D = ctypes.POINTER(ctypes.c_double)
        I32 = ctypes.POINTER(ctypes.c_int32)
        I64 = ctypes.POINTER(ctypes.c_int64)
        U8 = ctypes.POINTER(ctypes.c_uint8)
        U32 = ctypes.POINTER(ctypes.c_uint32)
        P = ctypes.POINTER(_OracleParams)
        i32, u64, dbl = ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        sig = {
            "oracle_philox4x32_10": (None, [U32, U32, U32]),
            "oracle_uniform": (dbl, [u64, i32, i32, i32, i32]),
            "oracle_gaussian": (dbl, [u64, i32, i32, i32]),
            "oracle_gamma": (dbl, [P, i32]),
            "oracle_entropy": (dbl, [i32, D, i32]),
            "oracle_relaxed_loss": (dbl, [i32, i32, I32, I32, I32, dbl, D]),
            "oracle_objective": (dbl, [P, i32, I32, I32, I32, dbl, D]),
            "oracle_gradient_rows": (None, [P, i32, I32, I32, I32, dbl, D, I32, i32, D, D]),
            "oracle_step_rows": (None, [P, i32, I32, I32, I32, i32, D, I32, i32, D, D, D, D, D]),
            "oracle_init": (None, [i32, i32, u64, D]),
            "oracle_noise_field": (None, [i32, i32, u64, i32, D]),
            "oracle_cost_of_x": (ctypes.c_int, [i32, i32, I32, I32, I32, dbl, U8, I64, I64, D]),
            "oracle_round_eval": (i32, [i32, i32, I32, I32, I32, dbl, i32, D, I64, I64, U8, D]),
            "oracle_anneal": (i32, [P, i32, I32, I32, I32, i32, i32, I64, I64, U8, D, I32, I64, i32, D]),
            "oracle_num_threads": (i32, []),
            "oracle_color_entropy": (dbl, [i32, i32, D, i32]),
            "oracle_color_relaxed_conflicts": (dbl, [i32, i32, I32, I32, D]),
            "oracle_color_conflicts": (ctypes.c_int64, [i32, I32, I32, I32]),
            "oracle_color_objective": (dbl, [P, i32, i32, I32, I32, dbl, D]),
            "oracle_color_gradient": (None, [P, i32, i32, I32, I32, dbl, D, D, D]),
            "oracle_color_step": (None, [P, i32, i32, I32, I32, i32, D, D, D, D, D]),
            "oracle_color_init": (None, [i32, i32, i32, u64, D]),
            "oracle_color_round": (i32, [i32, i32, i32, I32, I32, D, I32, I64]),
            "oracle_color_anneal": (i32, [P, i32, i32, I32, I32, i32, I64, I32, D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _graph_arrays(graph):
    rp = np.ascontiguousarray(graph.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(graph.col, dtype=np.int32)
    w = None if graph.w is None else np.ascontiguousarray(graph.w, dtype=np.int32)
    return rp, col, w


def _params(kind: int, p) -> _OracleParams:
    return _OracleParams(kind=kind, S=p.S, K=p.steps, a_ent=p.a_ent, lr=p.lr, weight_decay=p.weight_decay,
                         beta1=p.beta1, beta2=p.beta2, adam_eps=p.adam_eps, gamma_min=p.gamma_min,
                         gamma_max=p.gamma_max, alpha_comm=p.alpha_comm, comm_eps=p.comm_eps,
                         temperature=p.temperature, lam=p.lam, seed=p.seed)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def uniform(seed: int, i: int, s: int, t: int = 0, tag: int = 0) -> float:
    return float(_load().oracle_uniform(seed, i, s, t, tag))


def gaussian(seed: int, i: int, s: int, t: int) -> float:
    return float(_load().oracle_gaussian(seed, i, s, t))


def gamma(kind: int, p, t: int) -> float:
    pp = _params(kind, p)
    return float(_load().oracle_gamma(ctypes.byref(pp), t))


def entropy(pvec, a_ent: int) -> float:
    x = np.ascontiguousarray(pvec, dtype=np.float64)
    return float(_load().oracle_entropy(x.size, _ptr(x, ctypes.c_double), a_ent))


def relaxed_loss(kind: int, graph, lam: float, pvec) -> float:
    rp, col, w = _graph_arrays(graph)
    x = np.ascontiguousarray(pvec, dtype=np.float64)
    return float(_load().oracle_relaxed_loss(kind, graph.n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                             _ptr(w, ctypes.c_int32), lam, _ptr(x, ctypes.c_double)))


def objective(kind: int, graph, p, gamma_value: float, X) -> float:
    rp, col, w = _graph_arrays(graph)
    Xc = np.ascontiguousarray(X, dtype=np.float64)
    assert Xc.shape == (graph.n, p.S)
    pp = _params(kind, p)
    return float(_load().oracle_objective(ctypes.byref(pp), graph.n, _ptr(rp, ctypes.c_int32),
                                          _ptr(col, ctypes.c_int32), _ptr(w, ctypes.c_int32), gamma_value,
                                          _ptr(Xc, ctypes.c_double)))


def gradient(kind: int, graph, p, gamma_value: float, X, rows=None, with_scale: bool = False):
    rp, col, w = _graph_arrays(graph)
    Xc = np.ascontiguousarray(X, dtype=np.float64)
    assert Xc.shape == (graph.n, p.S)
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    nr = graph.n if r is None else r.size
    Gm = np.zeros((nr, p.S), dtype=np.float64)
    Gs = np.zeros((nr, p.S), dtype=np.float64)
    pp = _params(kind, p)
    _load().oracle_gradient_rows(ctypes.byref(pp), graph.n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                 _ptr(w, ctypes.c_int32), gamma_value, _ptr(Xc, ctypes.c_double),
                                 _ptr(r, ctypes.c_int32), nr, _ptr(Gm, ctypes.c_double), _ptr(Gs, ctypes.c_double))
    return (Gm, Gs) if with_scale else Gm


@dataclass
class StepOut:
    X: np.ndarray     # [nrows, S] new state of the listed rows
    m: np.ndarray
    v: np.ndarray
    grad: np.ndarray
    grad_scale: np.ndarray


def step(kind: int, graph, p, t: int, X, m, v, rows=None) -> StepOut:
    """One annealing step t from state (X, m, v); m and v are the moments of
    the listed rows ([nrows, S]) and are not modified."""
    rp, col, w = _graph_arrays(graph)
    Xc = np.ascontiguousarray(X, dtype=np.float64)
    assert Xc.shape == (graph.n, p.S)
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    nr = graph.n if r is None else r.size
    mm = np.array(m, dtype=np.float64, copy=True).reshape(nr, p.S)
    vv = np.array(v, dtype=np.float64, copy=True).reshape(nr, p.S)
    Xn = np.zeros((nr, p.S), dtype=np.float64)
    Gm = np.zeros((nr, p.S), dtype=np.float64)
    Gs = np.zeros((nr, p.S), dtype=np.float64)
    pp = _params(kind, p)
    _load().oracle_step_rows(ctypes.byref(pp), graph.n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                             _ptr(w, ctypes.c_int32), t, _ptr(Xc, ctypes.c_double), _ptr(r, ctypes.c_int32), nr,
                             _ptr(Xn, ctypes.c_double), _ptr(mm, ctypes.c_double), _ptr(vv, ctypes.c_double),
                             _ptr(Gm, ctypes.c_double), _ptr(Gs, ctypes.c_double))
    return StepOut(Xn, mm, vv, Gm, Gs)


def init_state(n: int, S: int, seed: int) -> np.ndarray:
    X = np.zeros((n, S), dtype=np.float64)
    _load().oracle_init(n, S, seed, _ptr(X, ctypes.c_double))
    return X


def noise_field(n: int, S: int, seed: int, t: int) -> np.ndarray:
    xi = np.zeros((n, S), dtype=np.float64)
    _load().oracle_noise_field(n, S, seed, t, _ptr(xi, ctypes.c_double))
    return xi


def cost_of_x(kind: int, graph, lam: float, x):
    rp, col, w = _graph_arrays(graph)
    xb = np.ascontiguousarray(np.asarray(x) != 0, dtype=np.uint8)
    obj = np.zeros(1, np.int64)
    viol = np.zeros(1, np.int64)
    en = np.zeros(1, np.float64)
    feas = _load().oracle_cost_of_x(kind, graph.n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                    _ptr(w, ctypes.c_int32), lam, _ptr(xb, ctypes.c_uint8), _ptr(obj, ctypes.c_int64),
                                    _ptr(viol, ctypes.c_int64), _ptr(en, ctypes.c_double))
    return int(obj[0]), int(viol[0]), bool(feas), float(en[0])


@dataclass
class EvalOut:
    obj: np.ndarray
    viol: np.ndarray
    feasible: np.ndarray
    energy: np.ndarray
    best: int


def round_eval(kind: int, graph, lam: float, X) -> EvalOut:
    rp, col, w = _graph_arrays(graph)
    Xc = np.ascontiguousarray(X, dtype=np.float64)
    S = Xc.shape[1]
    obj = np.zeros(S, np.int64)
    viol = np.zeros(S, np.int64)
    feas = np.zeros(S, np.uint8)
    en = np.zeros(S, np.float64)
    best = _load().oracle_round_eval(kind, graph.n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                     _ptr(w, ctypes.c_int32), lam, S, _ptr(Xc, ctypes.c_double),
                                     _ptr(obj, ctypes.c_int64), _ptr(viol, ctypes.c_int64),
                                     _ptr(feas, ctypes.c_uint8), _ptr(en, ctypes.c_double))
    return EvalOut(obj, viol, feas.astype(bool), en, int(best))


@dataclass
class AnnealOut:
    eval: EvalOut
    history: np.ndarray   # best feasible objective after each periodic evaluation (INT64_MIN: none)
    X: np.ndarray


def anneal(kind: int, graph, p, steps: int | None = None, round_every: int | None = None) -> AnnealOut:
    """Init + `steps` (default p.steps) annealing steps + evaluation. The gamma
    schedule always spans p.steps, so a shorter run is a prefix of the full one."""
    rp, col, w = _graph_arrays(graph)
    S = p.S
    re = p.round_every if round_every is None else round_every
    nsteps = p.steps if steps is None else steps
    cap = (nsteps // re + 2) if re > 0 else 2
    obj = np.zeros(S, np.int64)
    viol = np.zeros(S, np.int64)
    feas = np.zeros(S, np.uint8)
    en = np.zeros(S, np.float64)
    best = np.zeros(1, np.int32)
    hist = np.zeros(cap, np.int64)
    X = np.zeros((graph.n, S), np.float64)
    pp = _params(kind, p)
    nh = _load().oracle_anneal(ctypes.byref(pp), graph.n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                               _ptr(w, ctypes.c_int32), re, nsteps, _ptr(obj, ctypes.c_int64),
                               _ptr(viol, ctypes.c_int64), _ptr(feas, ctypes.c_uint8), _ptr(en, ctypes.c_double),
                               _ptr(best, ctypes.c_int32), _ptr(hist, ctypes.c_int64), cap,
                               _ptr(X, ctypes.c_double))
    return AnnealOut(EvalOut(obj, viol, feas.astype(bool), en, int(best[0])), hist[:nh], X)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))


# ---------------------------------------------------------------------------
# Categorical PQQA for graph colouring (App. B, App. C.4). W has shape
# [n, K, S] (node, colour, replica); sigma arrays passed to the entropy and
# relaxed-conflict functions have shape [n, K] (one replica).
# ---------------------------------------------------------------------------
COLORING = 3


def color_entropy(sig, a_ent: int) -> float:
    sg = np.ascontiguousarray(sig, dtype=np.float64)
    n, K = sg.shape
    return float(_load().oracle_color_entropy(n, K, _ptr(sg, ctypes.c_double), a_ent))


def color_relaxed_conflicts(graph, sig) -> float:
    rp, col, _ = _graph_arrays(graph)
    sg = np.ascontiguousarray(sig, dtype=np.float64)
    return float(_load().oracle_color_relaxed_conflicts(graph.n, sg.shape[1], _ptr(rp, ctypes.c_int32),
                                                        _ptr(col, ctypes.c_int32), _ptr(sg, ctypes.c_double)))


def color_conflicts(graph, x) -> int:
    rp, col, _ = _graph_arrays(graph)
    xx = np.ascontiguousarray(x, dtype=np.int32)
    return int(_load().oracle_color_conflicts(graph.n, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                              _ptr(xx, ctypes.c_int32)))


def color_sigma(W) -> np.ndarray:
    """Clamp-normalise over the colour axis of W[n, K, S] (plain numpy, for tests)."""
    Wc = np.clip(np.asarray(W, dtype=np.float64), 0.0, 1.0)
    tot = Wc.sum(axis=1, keepdims=True)
    K = Wc.shape[1]
    return np.where(tot > 0, Wc / np.where(tot > 0, tot, 1.0), 1.0 / K)


def color_objective(graph, K: int, p, gamma_value: float, W) -> float:
    rp, col, _ = _graph_arrays(graph)
    Wc = np.ascontiguousarray(W, dtype=np.float64)
    assert Wc.shape == (graph.n, K, p.S)
    pp = _params(COLORING, p)
    return float(_load().oracle_color_objective(ctypes.byref(pp), graph.n, K, _ptr(rp, ctypes.c_int32),
                                                _ptr(col, ctypes.c_int32), gamma_value, _ptr(Wc, ctypes.c_double)))


def color_gradient(graph, K: int, p, gamma_value: float, W, with_scale: bool = False):
    rp, col, _ = _graph_arrays(graph)
    Wc = np.ascontiguousarray(W, dtype=np.float64)
    assert Wc.shape == (graph.n, K, p.S)
    G = np.zeros_like(Wc)
    Gs = np.zeros_like(Wc)
    pp = _params(COLORING, p)
    _load().oracle_color_gradient(ctypes.byref(pp), graph.n, K, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                  gamma_value, _ptr(Wc, ctypes.c_double), _ptr(G, ctypes.c_double),
                                  _ptr(Gs, ctypes.c_double))
    return (G, Gs) if with_scale else G


def color_step(graph, K: int, p, t: int, W, m, v) -> StepOut:
    """One annealing step t of the colouring state (W, m, v) [n, K, S]; inputs are not modified."""
    rp, col, _ = _graph_arrays(graph)
    Wn = np.array(W, dtype=np.float64, copy=True)
    mm = np.array(m, dtype=np.float64, copy=True)
    vv = np.array(v, dtype=np.float64, copy=True)
    assert Wn.shape == (graph.n, K, p.S) == mm.shape == vv.shape
    G = np.zeros_like(Wn)
    Gs = np.zeros_like(Wn)
    pp = _params(COLORING, p)
    _load().oracle_color_step(ctypes.byref(pp), graph.n, K, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32), t,
                              _ptr(Wn, ctypes.c_double), _ptr(mm, ctypes.c_double), _ptr(vv, ctypes.c_double),
                              _ptr(G, ctypes.c_double), _ptr(Gs, ctypes.c_double))
    return StepOut(Wn, mm, vv, G, Gs)


def color_init(n: int, K: int, S: int, seed: int) -> np.ndarray:
    W = np.zeros((n, K, S), dtype=np.float64)
    _load().oracle_color_init(n, K, S, seed, _ptr(W, ctypes.c_double))
    return W


def color_round(graph, K: int, W):
    """(x [n, S] colours, conflicts [S], best replica) of the rounding argmax_k sigma."""
    rp, col, _ = _graph_arrays(graph)
    Wc = np.ascontiguousarray(W, dtype=np.float64)
    S = Wc.shape[2]
    x = np.zeros((graph.n, S), dtype=np.int32)
    conf = np.zeros(S, dtype=np.int64)
    best = _load().oracle_color_round(graph.n, K, S, _ptr(rp, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                      _ptr(Wc, ctypes.c_double), _ptr(x, ctypes.c_int32), _ptr(conf, ctypes.c_int64))
    return x, conf, int(best)


def color_anneal(graph, K: int, p, steps: int | None = None):
    """Init + steps (default p.steps) + rounding: (conflicts [S], best replica, x [n, S], W [n, K, S])."""
    rp, col, _ = _graph_arrays(graph)
    S = p.S
    conf = np.zeros(S, dtype=np.int64)
    x = np.zeros((graph.n, S), dtype=np.int32)
    W = np.zeros((graph.n, K, S), dtype=np.float64)
    pp = _params(COLORING, p)
    best = _load().oracle_color_anneal(ctypes.byref(pp), graph.n, K, _ptr(rp, ctypes.c_int32),
                                       _ptr(col, ctypes.c_int32), -1 if steps is None else steps,
                                       _ptr(conf, ctypes.c_int64), _ptr(x, ctypes.c_int32), _ptr(W, ctypes.c_double))
    return conf, int(best), x, W
