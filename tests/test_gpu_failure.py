"""Failure detection on the GPU without a fault: the bounded mbarrier waits of the
tensor-core kernel give up on a phase that nothing completes, the status word reaches
the host as MF_ERR_TIMEOUT, and the device context stays usable afterwards."""
import time

import numpy as np
import pytest

from paper_2308_14258_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_14258_gb300 import mosaicflow
    return mosaicflow


def test_bounded_wait_gives_up_and_reports_timeout(m):
    t0 = time.perf_counter()
    status, gave_up = m.check_wait_timeout(20.0)
    dt = time.perf_counter() - t0
    assert status == m.MF_ERR_TIMEOUT
    assert gave_up == 64
    assert 0.02 <= dt < 5.0, dt          # waited at least the limit, and not much longer
    assert "timed out" in m.load().mf_last_error().decode()


def test_context_usable_after_timeout(m):
    m.check_wait_timeout(5.0)
    w = I.tiny()
    net = m.SDNet(w.weights(bias_scale=0.1), w.shape.width, w.shape.depth)
    g = m.Grid(2, 2, w.problems[0].bc)
    for prec in ("fp32", "bf16"):
        out = g.sweep(net, 2, "M", prec)
        assert out.sweeps_done == 2 and np.isfinite(out.delta)
    assert np.all(np.isfinite(g.download()))


def test_invalid_limit(m):
    status, _ = m.check_wait_timeout(0.0)
    assert status == m.MF_ERR_INVALID_ARG
    status, _ = m.check_wait_timeout(5000.0)
    assert status == m.MF_ERR_INVALID_ARG
