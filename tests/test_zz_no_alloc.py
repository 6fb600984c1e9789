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
# mf_sweep precision that runs the same kernel as the allocation-free sweep: its FP32
# path is the CUDA-core kernel (mf_sweep's MF_PREC_FP32 runs the tensor-core FP32 kernel
# for these SDNets, which agrees with it to about 3e-6, not bit for bit)
SAME_KERNEL = {"fp32": "fp32_simt", "bf16": "bf16"}


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
        ref = grid.sweep(net, 1, "M", SAME_KERNEL[prec])
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


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_at_its_size_limit(m, prec):
    """lx = ly = 32, the largest grid the fixed scratch holds (3969 subdomains, grid
    1025 x 1025): every scratch region is used at its full size, twice in a row."""
    import torch
    lx = ly = 32
    weights = I.xavier_sdnet(I.SDNetShape(128, 6), 14, bias_scale=0.1)
    bc = I.bc_values(lx, ly, I.mode_field(I.mode_coeffs(15), lx, ly))
    u0 = orc.make_grid(lx, ly, bc)
    u0[1:-1, 1:-1] = I.Stream(16, I.TAG_TEST).normal((u0.shape[0] - 2) * (u0.shape[1] - 2)).reshape(
        u0.shape[0] - 2, u0.shape[1] - 2) * 0.3
    u0 = u0.astype(np.float32)
    net = m.SDNet(weights, 128, 6)
    grid = m.Grid(lx, ly, bc)
    grid.upload(u0)
    mine = torch.from_numpy(u0.copy()).cuda()
    for call in range(2):
        ref = grid.sweep(net, 1, "M", SAME_KERNEL[prec])
        expect = grid.download().astype(np.float64)
        d = m.sweep_noalloc(mine, lx, ly, net, 1, prec)
        got = mine.cpu().numpy().astype(np.float64)
        assert np.abs(got - expect).max() / np.abs(expect).max() <= TOL[prec], call
        assert abs(d - ref.delta) <= 1e-6 * ref.delta, (call, d, ref.delta)


def test_noalloc_zero_sweeps_leaves_grid(m):
    import torch
    net = m.SDNet(I.xavier_sdnet(I.SDNetShape(64, 3), 2), 64, 3)
    bc = I.bc_values(2, 2, I.mode_field(I.mode_coeffs(3), 2, 2))
    u = torch.from_numpy(orc.make_grid(2, 2, bc).astype(np.float32)).cuda()
    u[1:-1, 1:-1] = 0.5
    before = u.clone()
    d = m.sweep_noalloc(u, 2, 2, net, 0, "bf16")
    torch.cuda.synchronize()
    assert d == -1.0
    assert torch.equal(u, before)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_several_sweeps_on_a_side_stream(m, prec):
    """Three sweeps in one call on a caller's non-default stream, against mf_sweep's
    three sweeps on the same stream: grid and the last sweep's delta agree."""
    import torch
    lx, ly = 4, 3
    weights = I.xavier_sdnet(I.SDNetShape(128, 6), 17, bias_scale=0.1)
    bc = I.bc_values(lx, ly, I.mode_field(I.mode_coeffs(18), lx, ly))
    u0 = orc.make_grid(lx, ly, bc).astype(np.float32)
    net = m.SDNet(weights, 128, 6)
    grid = m.Grid(lx, ly, bc)
    side = torch.cuda.Stream()
    ref = grid.sweep(net, 3, "M", SAME_KERNEL[prec], stream=side)
    expect = grid.download(stream=side).astype(np.float64)
    with torch.cuda.stream(side):
        mine = torch.from_numpy(u0.copy()).to("cuda", non_blocking=False)
    side.synchronize()
    d = m.sweep_noalloc(mine, lx, ly, net, 3, prec, stream=side)
    got = mine.cpu().numpy().astype(np.float64)
    assert np.abs(got - expect).max() / np.abs(expect).max() <= TOL[prec]
    assert abs(d - ref.delta) <= 1e-6 * ref.delta, (d, ref.delta)
