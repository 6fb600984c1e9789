"""Batched sweeps over independent problems of uneven sizes, against the oracle run on
each problem alone (problems never interact, so the batch must equal the parts)."""
import numpy as np
import pytest

from oracle import mosaic_flow as orc
from paper_2308_14258_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16": 3e-2, "f16": 5e-3}
SIZES = [(1, 1), (2, 3), (3, 2), (2, 2), (4, 1), (1, 3)]


@pytest.fixture(scope="module")
def m():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_14258_gb300 import mosaicflow
    return mosaicflow


def states(sizes, seed):
    bcs, us = [], []
    for q, (lx, ly) in enumerate(sizes):
        bc = I.bc_values(lx, ly, I.mode_field(I.mode_coeffs(seed + q), lx, ly))
        u = orc.make_grid(lx, ly, bc)
        ny, nx = u.shape
        u[1:-1, 1:-1] = I.Stream(seed + 50 + q, I.TAG_TEST).normal((ny - 2) * (nx - 2)).reshape(ny - 2, nx - 2) * 0.3
        bcs.append(bc)
        us.append(u.astype(np.float32))
    return bcs, us


def rel_err(got, ref):
    return float(np.abs(got.astype(np.float64) - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("prec", ["fp32", "bf16", "f16"])
@pytest.mark.parametrize("query", ["full", "centre"])
def test_batch_sweep_equals_each_problem(m, prec, query):
    w = I.xavier_sdnet(I.SDNetShape(128, 6), 31, bias_scale=0.1)
    net = m.SDNet(w, 128, 6)
    bcs, us = states(SIZES, 40)
    b = m.Batch(SIZES, bcs)
    for q, u in enumerate(us):
        b.upload(q, u)
    out = b.sweep(net, 1, prec, query=query)
    assert out.sweeps_done == 1
    solver = orc.Solver(orc.unpack_sdnet(w, 128, 6))
    num = den = 0.0
    for q, (lx, ly) in enumerate(SIZES):
        ref = orc.sweep_multiplicative(us[q].astype(np.float64), lx, ly, solver, query=query.replace("centre", "center"))
        got = b.download(q)
        assert rel_err(got, ref) <= TOL[prec], q
        num += float(np.sum((got.astype(np.float64) - us[q]) ** 2))
        den += float(np.sum(us[q].astype(np.float64) ** 2))
    # delta covers all problems together
    assert abs(out.delta - np.sqrt(num / den)) <= 1e-5 * np.sqrt(num / den)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "f16"])
def test_graph_replay_matches_plain_sweeps(m, prec):
    w = I.xavier_sdnet(I.SDNetShape(64, 4), 32, bias_scale=0.1)
    net = m.SDNet(w, 64, 4)
    bcs, us = states(SIZES, 60)
    b1, b2 = m.Batch(SIZES, bcs), m.Batch(SIZES, bcs)
    for q, u in enumerate(us):
        b1.upload(q, u)
        b2.upload(q, u)
    b1.sweep(net, 1, prec)                      # first sweep runs the kernels uncaptured
    o1 = b1.sweep(net, 4, prec, graph=True)     # then replayed from the captured graph
    b2.sweep(net, 5, prec)
    assert o1.graph_sweeps == 4
    for q in range(len(SIZES)):
        assert np.array_equal(b1.download(q), b2.download(q))


def test_batch_residual_and_validation(m):
    bcs, us = states(SIZES[:2], 70)
    b = m.Batch(SIZES[:2], bcs)
    b.upload(1, us[1])
    r_max, r_rms = b.residual(1)
    o_max, o_rms = orc.residual(us[1].astype(np.float64))
    assert abs(r_max - o_max) <= 1e-6 * o_max and abs(r_rms - o_rms) <= 1e-6 * o_rms
    net = m.SDNet(I.xavier_sdnet(I.SDNetShape(64, 2), 1), 64, 2)
    import ctypes as C
    opts = m.SweepOpts(1, 1, 0, 0, 0.0, 1, 0, 0.0, 0, 0)  # additive schedule is rejected
    assert m.load().mf_batch_sweep(b._h, net._h, C.byref(opts), None, None) == m.MF_ERR_INVALID_ARG


def test_batched_workload_sampled(m):
    """The 256-problem batch (sides 2..32 units, 71.7 M grid points, SDNet 6x128) in the
    benchmark's configuration: one BF16 sweep of the whole batch, then the oracle on a
    sample of its problems from the same initial state."""
    wl = I.batched(256)
    w = wl.weights()
    net = m.SDNet(w, 128, 6)
    sizes = [(p.lx, p.ly) for p in wl.problems]
    b = m.Batch(sizes, [p.bc for p in wl.problems])
    b.sweep(net, 1, "bf16")
    pick = [q for q, p in enumerate(wl.problems) if p.lx <= 4][:6] + \
           [next(q for q, p in enumerate(wl.problems) if p.lx == 16)]
    pre = {q: b.download(q) for q in pick}
    b.sweep(net, 1, "bf16")
    solver = orc.Solver(orc.unpack_sdnet(w, 128, 6))
    for q in pick:
        lx, ly = sizes[q]
        ref = orc.sweep_multiplicative(pre[q].astype(np.float64), lx, ly, solver)
        assert rel_err(b.download(q), ref) <= TOL["bf16"], q
