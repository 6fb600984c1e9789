"""Execution contexts (mf_ctx_create / mf_ctx_destroy) and per-device state, through
the C ABI: handles live on their context's device, calls leave the caller's current
device as it was, and the launch set-up (shared-memory attributes, grid caps) is kept
per device, so a second GPU in the same process runs the same kernels."""
import ctypes as C

import numpy as np
import pytest

from oracle import mosaic_flow as orc
from paper_2308_14258_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_14258_gb300 import mosaicflow
    return mosaicflow


def test_context_reports_its_device(m):
    import torch
    ctx = m.Context(0)
    assert ctx.device == 0
    assert ctx.sm_count == torch.cuda.get_device_properties(0).multi_processor_count
    n = torch.cuda.device_count()
    with pytest.raises(m.MFError) as e:
        m.Context(n)
    assert e.value.status == m.MF_ERR_INVALID_ARG


def test_handles_on_their_context_and_caller_device_kept(m):
    import torch
    torch.cuda.set_device(0)
    ctx = m.Context(0)
    w = I.xavier_sdnet(I.SDNetShape(64, 3), 3)
    net = m.SDNet(w, 64, 3, ctx=ctx)
    bc = I.bc_values(2, 2, I.mode_field(I.mode_coeffs(4), 2, 2))
    g = m.Grid(2, 2, bc, ctx=ctx)
    out = g.sweep(net, 2, "M", "bf16")
    assert out.status == m.MF_OK and out.sweeps_done == 2
    assert torch.cuda.current_device() == 0
    # a context destroyed before its handles leaves them usable
    del ctx
    g.sweep(net, 1, "M", "fp32")
    assert np.isfinite(g.download()).all()


def test_result_status_reports_divergence(m):
    """A network whose output overflows FP32 makes delta infinite: the call returns
    MF_ERR_DIVERGED and the result's status field holds the same code."""
    width, depth = 64, 2
    w = np.zeros(I.SDNetShape(width, depth).n_params, dtype=np.float32)
    w[width * 130 + width + width * width + width:][:width] = 3e38   # w_out: 64 x 3e38 overflows
    w[128] = 1.0                                                      # unit 0 sees x
    o = width * 130 + width
    w[o:o + width * width] = 0.0
    w[o + width * width:o + width * width + width] = 1.0              # hidden bias -> tanh(1)
    net = m.SDNet(w, width, depth)
    bc = I.bc_values(2, 2, I.mode_field(I.mode_coeffs(4), 2, 2))
    g = m.Grid(2, 2, bc)
    opts = m.SweepOpts(1, 0, 0, 0, 0.0, 1, 0, 0.0, 0, 0)
    res = m.SweepResult()
    st = m.load().mf_sweep(g._h, net._h, C.byref(opts), C.byref(res), None)
    assert st == m.MF_ERR_DIVERGED
    assert res.status == m.MF_ERR_DIVERGED
    opts_ok = m.SweepOpts(0, 0, 0, 0, 0.0, 1, 0, 0.0, 0, 0)
    assert m.load().mf_sweep(g._h, net._h, C.byref(opts_ok), C.byref(res), None) == m.MF_OK
    assert res.status == m.MF_OK


def test_two_devices_share_one_process(m):
    """Same sweep on devices 0 and 1 (skipped with one visible GPU): the launch set-up
    recorded for device 0 must not be reused on device 1."""
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    w = I.xavier_sdnet(I.SDNetShape(128, 6), 5, bias_scale=0.1)
    bc = I.bc_values(3, 2, I.mode_field(I.mode_coeffs(6), 3, 2))
    outs = []
    for dev in (0, 1):
        ctx = m.Context(dev)
        net = m.SDNet(w, 128, 6, ctx=ctx)
        g = m.Grid(3, 2, bc, ctx=ctx)
        for prec in ("bf16", "fp32"):
            g.sweep(net, 1, "M", prec)
        outs.append(g.download())
    assert np.array_equal(outs[0], outs[1])
    ref = orc.make_grid(3, 2, bc)
    assert outs[0].shape == ref.shape
