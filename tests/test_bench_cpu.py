"""CPU checks of bench.py's bookkeeping: the algorithmic bytes a roofline is
quoted against, the kernel names it reports, and the machine-readable tail of
every committed step-kernel profile summary (which bench.py parses for the
measured DRAM traffic)."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from qqa_inputs import graphs as G  # noqa: E402
from qqa_inputs import workloads as W  # noqa: E402


def _workload(n, S, precision, weighted=False):
    g = G.random_regular(n, 3, 1)
    if weighted:
        u, v, _ = g.upper_edges()
        g = G.from_edges(n, u, v, [1] * len(u))
    p = W.Params(S=S, steps=10, precision=precision)
    return W.Workload("t", [W.Instance(W.MAXCUT, g, p, "t")])


@pytest.mark.parametrize("precision,per_elem", [(W.FP32, 24), (W.BF16, 20)])
def test_algorithmic_bytes_are_state_plus_csr(precision, per_elem):
    """24 B per element-step in FP32 (p read and written, m and v read and
    written), 20 B with BF16 storage (X 2 + 2, FP32 master 4 + 4, m and v 2 + 2
    each), plus the CSR (column indices, row pointers, and weights when the
    graph has them), once per step."""
    n, S = 1000, 256
    wl = _workload(n, S, precision)
    nnz = wl.instances[0].graph.nnz
    assert bench.algorithmic_bytes_per_launch(wl) == n * S * per_elem + 4 * nnz + 4 * (n + 1)
    wlw = _workload(n, S, precision, weighted=True)
    assert bench.algorithmic_bytes_per_launch(wlw) == n * S * per_elem + 8 * nnz + 4 * (n + 1)


def test_the_max_cut_configuration_moves_513_6_mb_per_step():
    """The graded configuration (3-regular, n = 1e5, S = 256, BF16): 512 MB of
    state and 1.6 MB of CSR per step."""
    wl = W.maxcut_large(n=100_000, family="regular3")
    assert bench.algorithmic_bytes_per_launch(wl) == 100_000 * 256 * 20 + 4 * 300_000 + 4 * 100_001


class _Cfg:
    def __init__(self, vpl):
        self.vec_per_lane = vpl


def test_kernel_names():
    assert bench.kernel_symbol("pipe", _Cfg(1)) == "qqa_step_pipe_kernel_v1"
    assert bench.kernel_symbol("pipe", _Cfg(2)) == "qqa_step_pipe_kernel"
    assert bench.kernel_symbol("dense", _Cfg(4)) == "qqa_dense_gemm_kernel + qqa_dense_update_kernel"
    assert bench.kernel_symbol("scalar", _Cfg(1)) == "qqa_step_scalar_kernel"


def test_profile_summaries_carry_their_variant_hash_and_traffic():
    """Every step-kernel summary ends with the kernel variant, the hash of the
    sources it was captured on and its DRAM bytes, in the form bench.py reads;
    the variant is one bench.py knows."""
    prof = os.path.join(ROOT, "profiles")
    names = [f for f in os.listdir(prof) if f.startswith("step_kernel_") and f.endswith(".md")]
    assert names
    for f in names:
        text = open(os.path.join(prof, f)).read()
        variant = re.search(r"kernel_variant:\s*(\w+)", text)
        assert variant and variant.group(1) in bench.KERNEL_NAMES, f
        assert re.search(r"kernel_source_sha256_16:\s*[0-9a-f]{16}\b", text), f
        traffic = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
        assert traffic and float(traffic.group(1)) > 0, f


def test_quality_ratio_against_the_stored_oracle_means():
    """The bench line's quality_vs_oracle divides each instance's best by the
    oracle's stored mean (16 runs where stored, else 4) and leaves instances
    without a target or a feasible replica as None."""
    q = bench.quality_vs_oracle("maxcut_regular3", [136310.75])
    assert q["oracle_runs"] == [4] and abs(q["ratio_per_instance"][0] - 1.0) < 1e-12
    q = bench.quality_vs_oracle("mis_er700_800", [None] + [45] * 15)
    assert q["ratio_per_instance"][0] is None and q["oracle_runs"][0] == 16 and len(q["oracle_runs"]) == 16
    assert bench.quality_vs_oracle("no_such_workload", [1]) is None
