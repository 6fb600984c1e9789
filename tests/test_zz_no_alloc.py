"""mf_sweep_noalloc, the sweep entry point that allocates no device memory, against
mf_sweep on the same state, through the C ABI.

Callers that cannot allocate (their device memory belongs to another allocator's pool,
or a cudaMalloc would synchronise a latency-critical loop) keep their own grid buffer
and call mf_sweep_noalloc, whose scratch is a fixed array inside the library. Two calls
in a row must both match the allocating entry point, which also checks that the shared
scratch left behind by the first call does not leak into the second. This file is named
to be collected last.
"""
import numpy as np
import pytest

from oracle import mosaic_flow as orc
from paper_2308_14258_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16": 3e-2}


@pytest.fixture(scope="module")
def m():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_14258_gb300 import mosaicflow
    return mosaicflow


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("lx,ly,width,depth", [(2, 3, 128, 6), (5, 4, 64, 4)])
def test_noalloc_matches_allocating_sweep_twice(m, prec, lx, ly, width, depth):
    import torch
    weights = I.xavier_sdnet(I.SDNetShape(width, depth), 11, bias_scale=0.1)
    bc = I.bc_values(lx, ly, I.mode_field(I.mode_coeffs(12), lx, ly))
    u0 = orc.make_grid(lx, ly, bc)
    u0[1:-1, 1:-1] = I.Stream(13, I.TAG_TEST).normal((u0.shape[0] - 2) * (u0.shape[1] - 2)).reshape(
        u0.shape[0] - 2, u0.shape[1] - 2) * 0.3
    u0 = u0.astype(np.float32)

    net = m.SDNet(weights, width, depth)
    grid = m.Grid(lx, ly, bc)
    grid.upload(u0)
    mine = torch.from_numpy(u0.copy()).cuda()
    for call in range(2):
        ref = grid.sweep(net, 1, "M", prec)
        expect = grid.download().astype(np.float64)
        d = m.sweep_noalloc(mine, lx, ly, net, 1, prec)
        torch.cuda.synchronize()
        got = mine.cpu().numpy().astype(np.float64)
        err = np.abs(got - expect).max() / np.abs(expect).max()
        assert err <= TOL[prec], (call, err)
        assert abs(d - ref.delta) <= 1e-6 * max(ref.delta, 1e-30), (call, d, ref.delta)


def test_noalloc_rejects_grids_beyond_its_scratch(m):
    import torch
    net = m.SDNet(I.xavier_sdnet(I.SDNetShape(64, 2), 1), 64, 2)
    big = torch.zeros((32 * 33 + 1, 32 * 2 + 1), dtype=torch.float32, device="cuda")
    with pytest.raises(m.MFError) as e:
        m.sweep_noalloc(big, 2, 33, net, 1, "fp32")
    assert e.value.status == m.MF_ERR_INVALID_ARG
    assert "32" in str(e.value)
