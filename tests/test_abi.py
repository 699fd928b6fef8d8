"""The C-ABI library loads and exports every symbol include/qqa.h declares, and
its host-side argument checks reject malformed input before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qqa.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qqa_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_02135_gb300 import _build, _lib
    _build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("qqa_create_problem", "qqa_anneal", "qqa_round_eval", "qqa_run_steps", "qqa_run_eval"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2409_02135_gb300._lib import SIGNATURES
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in SIGNATURES, f"binding does not declare {name}"


def test_struct_layouts_match_header(lib):
    from paper_2409_02135_gb300._lib import qqa_params, qqa_launch_config
    assert ctypes.sizeof(qqa_params) == 80
    assert ctypes.sizeof(qqa_launch_config) == 32
    p = qqa_params()
    lib.qqa_default_params(ctypes.byref(p))
    assert (p.S, p.a_ent, p.lam, p.gamma_min, p.gamma_max) == (128, 4, 2.0, -2.0, pytest.approx(0.1))
    assert p.weight_decay == pytest.approx(0.01) and p.temperature == pytest.approx(1e-3)


def _create(lib, kind, n, rp, col, w=None):
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    wp = None if w is None else np.ascontiguousarray(w, dtype=np.int32)
    h = ctypes.c_void_p()
    P = ctypes.POINTER(ctypes.c_int32)
    rc = lib.qqa_create_problem(kind, n, rp.ctypes.data_as(P), col.ctypes.data_as(P),
                                None if wp is None else wp.ctypes.data_as(P), None, None, ctypes.byref(h))
    return rc, lib.qqa_last_error().decode()


@pytest.mark.parametrize("case,rp,col,w,kind,msg", [
    ("asymmetric", [0, 1, 1], [1], None, 0, "reverse"),
    ("self-loop", [0, 1, 1], [0], None, 0, "self-loop"),
    ("unsorted", [0, 2, 3, 4], [2, 1, 0, 0], None, 0, "increasing"),
    ("duplicate", [0, 2, 4], [1, 1, 0, 0], None, 0, "increasing"),
    ("out-of-range", [0, 1, 2], [5, 0], None, 0, "out of range"),
    ("bad row_ptr", [1, 1, 1], [], None, 0, "row_ptr"),
    ("weights on MIS", [0, 1, 2], [1, 0], [1, 1], 0, "max-cut"),
    ("asymmetric weights", [0, 1, 2], [1, 0], [1, 2], 1, "weight"),
    ("bad kind", [0, 1, 2], [1, 0], None, 7, "kind"),
])
def test_create_problem_rejects_malformed_graphs(lib, case, rp, col, w, kind, msg):
    rc, err = _create(lib, kind, len(rp) - 1, rp, col if col else [0], w)
    assert rc == -1, case
    assert msg in err, (case, err)


def test_run_create_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.qqa_run_create_empty(0, 8, 0, None, None, None, ctypes.byref(h)) == -1
    assert lib.qqa_run_create_empty(4, 5000, 0, None, None, None, ctypes.byref(h)) == -1
    assert lib.qqa_run_create_empty(4, 8, 3, None, None, None, ctypes.byref(h)) == -1


def test_request_bytes_accounting(lib):
    """Budget accounting of the server: state (FP32: X twice, m, v = 16 B per
    padded element; BF16: 12 B), evaluation buffers and the CSR."""
    import paper_2409_02135_gb300 as qqa
    n, nnz, S = 1000, 8000, 100
    elems = n * 100
    fp32 = qqa.request_bytes(n, nnz, S, qqa.FP32)
    assert fp32 == elems * 16 + n * 4 * 4 + 100 * 56 + 32 * 4 + 4096 + 4 * (n + 1) + 4 * nnz
    bf16 = qqa.request_bytes(n, nnz, S, qqa.BF16, weighted=True)
    elems16 = n * 104
    assert bf16 == elems16 * 12 + n * 4 * 4 + 104 * 56 + 32 * 4 + 4096 + 4 * (n + 1) + 8 * nnz


def _color_create(lib, n, rp, col, K, **kw):
    from paper_2409_02135_gb300._lib import qqa_params
    p = qqa_params()
    lib.qqa_default_params(ctypes.byref(p))
    p.S, p.steps = 8, 10
    for k, v in kw.items():
        setattr(p, k, v)
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col if col else [0], dtype=np.int32)
    P = ctypes.POINTER(ctypes.c_int32)
    h = ctypes.c_void_p()
    rc = lib.qqa_color_create(n, rp.ctypes.data_as(P), col.ctypes.data_as(P), K, ctypes.byref(p), None,
                              ctypes.byref(h))
    return rc, lib.qqa_last_error().decode()


@pytest.mark.parametrize("case,rp,col,K,kw,msg", [
    ("one colour", [0, 1, 2], [1, 0], 1, {}, "K must be"),
    ("too many colours", [0, 1, 2], [1, 0], 33, {}, "K must be"),
    ("no replicas", [0, 1, 2], [1, 0], 3, {"S": 0}, "S must be"),
    ("no steps", [0, 1, 2], [1, 0], 3, {"steps": 0}, "steps must be"),
    ("odd entropy exponent", [0, 1, 2], [1, 0], 3, {"a_ent": 3}, "a_ent"),
    ("BF16", [0, 1, 2], [1, 0], 3, {"precision": 1}, "FP32"),
    ("asymmetric", [0, 1, 1], [1], 3, {}, "reverse"),
    ("self-loop", [0, 1, 1], [0], 3, {}, "self-loop"),
])
def test_color_create_rejects_bad_arguments(lib, case, rp, col, K, kw, msg):
    """qqa_color_create checks its arguments and the graph on the host, before
    any device work."""
    rc, err = _color_create(lib, len(rp) - 1, rp, col, K, **kw)
    assert rc == -1, case
    assert msg in err, (case, err)
