"""Failure reporting through the C ABI without a failing kernel: the device
status words that the step kernels write (non-finite second moments, bounded
mbarrier waits that ran out) are planted with the debug hook, and the host
calls that read them must return the matching error codes. The device side of
the bounded waits is not forced to run out on the GPU (that would leave bulk
copies in flight); only this host-side mapping is tested."""
import numpy as np
import pytest

import paper_2409_02135_gb300 as qqa
from parity import make_run
from qqa_inputs import graphs as G
from qqa_inputs.workloads import MIS, FP32, BF16, Params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_02135_gb300 import _build
    _build.build()
    import torch
    assert torch.cuda.is_available()


@pytest.mark.parametrize("prec", [FP32, BF16])
def test_run_sync_reports_timeouts_then_non_finite_values(prec):
    g = G.erdos_renyi(120, 0.05, 1)
    run = make_run(MIS, g, Params(S=16, steps=40, seed=2, precision=prec))
    run.steps(5)
    run.sync()                                   # clean status
    run.debug_set_status(timeouts=3)
    with pytest.raises(qqa.QQAError) as err:
        run.sync()
    assert err.value.code == qqa.QQA_ETIMEOUT
    run.debug_set_status(nonfinite=2, timeouts=1)    # a timeout is reported first
    with pytest.raises(qqa.QQAError) as err:
        run.sync()
    assert err.value.code == qqa.QQA_ETIMEOUT
    run.debug_set_status(nonfinite=2)
    with pytest.raises(qqa.QQAError) as err:
        run.sync()
    assert err.value.code == qqa.QQA_ENONFINITE
    run.debug_set_status()
    run.sync()
    run.steps(5)
    run.eval()
    run.sync()
    assert run.result(0)["step"] == 10


def test_round_eval_reports_timeouts():
    g = G.erdos_renyi(90, 0.08, 3)
    prob = qqa.Problem(MIS, g)
    run = qqa.Run.create([prob], [qqa.make_params(Params(S=8, steps=20, seed=1))])
    run.steps(20)
    run.debug_set_status(timeouts=1)
    with pytest.raises(qqa.QQAError) as err:
        run.sync()
    assert err.value.code == qqa.QQA_ETIMEOUT
    run.debug_set_status()
    run.eval()
    run.sync()
    assert run.result(0)["best"] >= -1


def test_color_sync_reports_timeouts_then_non_finite_values():
    c = qqa.Coloring(G.queens(6, 6), 7, qqa.make_params(Params(S=32, steps=50, lr=0.1, seed=3)))
    c.steps(4)
    c.sync()
    c.debug_set_status(timeouts=1)
    with pytest.raises(qqa.QQAError) as err:
        c.sync()
    assert err.value.code == qqa.QQA_ETIMEOUT
    c.debug_set_status(nonfinite=5)
    with pytest.raises(qqa.QQAError) as err:
        c.sync()
    assert err.value.code == qqa.QQA_ENONFINITE
    c.debug_set_status()
    c.sync()
    c.steps(4)
    c.sync()
    r = c.round(with_x=False)
    assert np.all(r["conflicts"] >= 0)
