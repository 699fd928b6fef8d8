"""Helpers shared by the GPU parity tests: building runs through the C ABI,
running the oracle on the same inputs, and the error bound a single step may
show.

Tolerance of one step (condition-aware). The GPU computes in FP32 (optionally
with BF16 storage), the oracle in FP64, from the same state. With rtol the
relative accuracy of one FP32 (BF16) evaluation and gabs the oracle's sum of
absolute values of the gradient's terms, first-order propagation through the
AdamW update gives
    |dg| <= rtol * gabs
    |dm| <= rtol * (b1 |m0| + (1-b1) gabs) + st |m|
    |dv| <= rtol b2 v0 + (1-b2) (rtol g^2 + 2 |g| |dg| + |dg|^2) + st v
    den   = sqrt(v) / sqrt(bc2) + eps
    |dp| <= rtol |p0| + (lr / bc1) (|dm| / den + |m| |dv| / (2 sqrt(v bc2) den^2)) + rtol |sigma xi| + 2^-23
where st is the relative rounding of stored moments (0 in FP32, 2^-8 in BF16)
and the clamp to [0, 1] is 1-Lipschitz. Elements where Adam's first step
divides a tiny gradient by its own magnitude get a large bound automatically.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
import paper_2409_02135_gb300 as qqa
from qqa_inputs.workloads import Params, FP32, BF16

RTOL = {FP32: 1e-5, BF16: 1e-2}
STORE = {FP32: 0.0, BF16: 2.0 ** -8}


def f32(x: float) -> float:
    return float(np.float32(x))


def as_f32(p: Params) -> Params:
    """The parameters the GPU actually uses (rounded to FP32), for the oracle."""
    kw = {}
    for name in ("lr", "weight_decay", "beta1", "beta2", "adam_eps", "gamma_min", "gamma_max", "alpha_comm",
                 "comm_eps", "temperature", "lam"):
        kw[name] = f32(getattr(p, name))
    return p.with_(**kw)


def make_run(kind, graphs, params, config=None, stream=None):
    if not isinstance(graphs, (list, tuple)):
        graphs = [graphs]
    if not isinstance(params, (list, tuple)):
        params = [params] * len(graphs)
    probs = [qqa.Problem(kind, g, stream=stream) for g in graphs]
    cps = [qqa.make_params(p) for p in params]
    run = qqa.Run.create(probs, cps, config=config, stream=stream)
    run._keep = probs
    return run


def step_tolerance(p: Params, prec: int, t: int, X0, m0, v0, out: oracle.StepOut):
    rtol, st = RTOL[prec], STORE[prec]
    b1, b2 = p.beta1, p.beta2
    g, gabs = out.grad, out.grad_scale
    tol_g = rtol * gabs
    tol_m = rtol * (b1 * np.abs(m0) + (1 - b1) * gabs) + st * np.abs(out.m)
    tol_v = rtol * b2 * v0 + (1 - b2) * (rtol * g * g + 2 * np.abs(g) * tol_g + tol_g * tol_g) + st * out.v
    bc1 = 1 - b1 ** (t + 1)
    bc2 = 1 - b2 ** (t + 1)
    den = np.sqrt(out.v) / math.sqrt(bc2) + p.adam_eps
    step = p.lr / bc1
    sig = math.sqrt(2 * p.lr * p.temperature)
    tol_p = (rtol * np.abs(X0) + step * (tol_m / den + np.abs(out.m) * tol_v / (2 * np.sqrt(out.v * bc2) * den ** 2 + 1e-300))
             + rtol * sig * 6.0 + 2.0 ** -23)
    return tol_g, tol_m, tol_v, tol_p


def assert_within(name, got, want, tol):
    err = np.abs(np.asarray(got, np.float64) - np.asarray(want, np.float64))
    bad = err > tol
    if np.any(bad):
        idx = np.argwhere(bad)[:5]
        detail = ", ".join(f"{tuple(i)}: got {got[tuple(i)]:.9g} want {want[tuple(i)]:.9g} tol {tol[tuple(i)]:.3g}"
                           for i in idx)
        raise AssertionError(f"{name}: {int(bad.sum())} of {bad.size} elements outside tolerance; {detail}")
    return float(np.max(err / np.maximum(tol, 1e-300))) if err.size else 0.0
