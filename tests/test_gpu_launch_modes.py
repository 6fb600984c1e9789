"""Launch modes of the multiplicative sweep, through the C ABI: one cooperative launch
per sweep (gather, SDNet and scatter of all colours with device-wide barriers between
them), CUDA-graph replay and the autotuner must leave exactly the grid the per-colour
launches leave. Every mode runs the same arithmetic in the same order (the in-kernel
gather forms B = W1 g + b0 with the boundary gather kernel's summation order), so the
comparison is bit for bit."""
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


def state(lx, ly, seed):
    bc = I.bc_values(lx, ly, I.mode_field(I.mode_coeffs(seed), lx, ly))
    u = orc.make_grid(lx, ly, bc)
    ny, nx = u.shape
    u[1:-1, 1:-1] = I.Stream(seed + 1, I.TAG_TEST).normal((ny - 2) * (nx - 2)).reshape(ny - 2, nx - 2) * 0.3
    return bc, u.astype(np.float32)


@pytest.mark.parametrize("lx,ly,width,depth,act,query", [
    (1, 1, 128, 6, "tanh", "full"),
    (2, 3, 128, 6, "tanh", "full"),
    (3, 2, 64, 4, "tanh", "full"),
    (4, 4, 128, 3, "gelu", "full"),
    (5, 3, 128, 6, "tanh", "centre"),
    (2, 2, 64, 2, "tanh", "centre"),
])
def test_whole_sweep_launch_equals_per_colour(m, lx, ly, width, depth, act, query):
    w = I.xavier_sdnet(I.SDNetShape(width, depth, act), 61, bias_scale=0.1)
    net = m.SDNet(w, width, depth, act)
    bc, u0 = state(lx, ly, 62)
    ga, gb = m.Grid(lx, ly, bc), m.Grid(lx, ly, bc)
    ga.upload(u0)
    gb.upload(u0)
    ra = ga.sweep(net, 3, "M", "bf16", query=query)
    rb = gb.sweep(net, 3, "M", "bf16", query=query, launch_mode="sweep")
    assert rb.launch_mode == "sweep" and rb.mlp_launches == 3
    assert np.array_equal(ga.download(), gb.download())
    assert ra.delta == rb.delta


def test_whole_sweep_launch_in_mixed_precision(m):
    """MF_PREC_MIXED with the whole-sweep launch: BF16 sweeps as one launch each, the FP32
    refinement per colour; same result as the per-colour launches."""
    w = I.xavier_sdnet(I.SDNetShape(128, 6), 63)
    net = m.SDNet(w, 128, 6)
    bc = I.bc_values(4, 4, I.mode_field(I.mode_coeffs(64), 4, 4))
    ga, gb = m.Grid(4, 4, bc), m.Grid(4, 4, bc)
    ra = ga.sweep(net, 80, "M", "mixed", eps=1e-6, eps_coarse=1e-2)
    rb = gb.sweep(net, 80, "M", "mixed", eps=1e-6, eps_coarse=1e-2, launch_mode="sweep")
    assert (ra.sweeps_done, ra.sweeps_bf16) == (rb.sweeps_done, rb.sweeps_bf16)
    assert np.array_equal(ga.download(), gb.download())


def test_whole_sweep_launch_full_size(m):
    """The 2049 x 2049 benchmark grid (16,129 subdomains, 6 x 128): one whole-sweep
    launch per sweep against the per-colour launches, two sweeps."""
    w = I.large()
    p = w.problems[0]
    net = m.SDNet(w.weights(), 128, 6)
    ga, gb = m.Grid(p.lx, p.ly, p.bc), m.Grid(p.lx, p.ly, p.bc)
    ra = ga.sweep(net, 2, "M", "bf16")
    rb = gb.sweep(net, 2, "M", "bf16", launch_mode="sweep")
    assert np.array_equal(ga.download(), gb.download())
    assert ra.delta == rb.delta


SMALL = [(2, 2)] * 40 + [(1, 1)] * 8 + [(2, 1), (1, 2), (3, 2), (2, 3)] * 4


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_batch_launch_modes_agree(m, prec):
    """Many small problems (the regime where launches, not arithmetic, dominate): every
    launch mode and the autotuner's choice give the per-colour result bit for bit."""
    w = I.xavier_sdnet(I.SDNetShape(128, 6), 65, bias_scale=0.1)
    net = m.SDNet(w, 128, 6)
    bcs, us = [], []
    for q, (lx, ly) in enumerate(SMALL):
        bc, u = state(lx, ly, 100 + q)
        bcs.append(bc)
        us.append(u)
    modes = ["per_colour", "graph", "auto"] + (["sweep"] if prec == "bf16" else [])
    outs, tuned = {}, None
    for mode in modes:
        b = m.Batch(SMALL, bcs)
        for q, u in enumerate(us):
            b.upload(q, u)
        r = b.sweep(net, 3, prec, launch_mode=mode, check_every=3)
        if mode == "auto":
            tuned = r
            r2 = b.sweep(net, 1, prec, launch_mode="auto")      # the choice is kept
            assert (r2.launch_mode, r2.gather_block) == (r.launch_mode, r.gather_block)
            outs[mode] = [b.download(q) for q in range(len(SMALL))]
            b2 = m.Batch(SMALL, bcs)
            for q, u in enumerate(us):
                b2.upload(q, u)
            b2.sweep(net, 4, prec)
            outs["per_colour_4"] = [b2.download(q) for q in range(len(SMALL))]
            continue
        outs[mode] = [b.download(q) for q in range(len(SMALL))]
    assert tuned.launch_mode in (["per_colour", "graph", "sweep"] if prec == "bf16" else ["per_colour", "graph"])
    assert tuned.gather_block in (4, 8, 16)
    for mode in modes:
        if mode == "auto":
            ref = outs["per_colour_4"]
        else:
            ref = outs["per_colour"]
        for q in range(len(SMALL)):
            assert np.array_equal(outs[mode][q], ref[q]), (mode, q)


def test_launch_mode_validation(m):
    w = I.xavier_sdnet(I.SDNetShape(64, 3), 66)
    net = m.SDNet(w, 64, 3)
    bc = I.bc_values(2, 2, I.mode_field(I.mode_coeffs(67), 2, 2))
    g = m.Grid(2, 2, bc)
    for mode, prec, code in (("sweep", "fp32", m.MF_ERR_UNSUPPORTED), ("graph", "bf16", m.MF_ERR_INVALID_ARG),
                             ("auto", "bf16", m.MF_ERR_INVALID_ARG), ("sweep", "f16", m.MF_ERR_UNSUPPORTED)):
        with pytest.raises(m.MFError) as e:
            g.sweep(net, 1, "M", prec, launch_mode=mode)
        assert e.value.status == code
    with pytest.raises(m.MFError) as e:
        g.sweep(net, 1, "A", "bf16", launch_mode="sweep")
    assert e.value.status == m.MF_ERR_UNSUPPORTED
    vw = I.xavier_sdnet(I.SDNetShape(64, 3, "tanh", 4, 3), 68)
    vnet = m.SDNet(vw, 64, 3, "tanh", 4, 3)
    with pytest.raises(m.MFError) as e:
        g.sweep(vnet, 1, "M", "bf16", launch_mode="sweep")
    assert e.value.status == m.MF_ERR_UNSUPPORTED
    b = m.Batch([(2, 2)], [bc])
    with pytest.raises(m.MFError) as e:
        b.sweep(net, 1, "fp32", launch_mode="sweep")
    assert e.value.status == m.MF_ERR_UNSUPPORTED


@pytest.mark.parametrize("width,depth,query", [(64, 4, "full"), (128, 6, "centre"), (64, 3, "centre")])
def test_batch_whole_sweep_other_shapes(m, width, depth, query):
    """The whole-sweep launch over a batch (subdomain tables) for width-64 SDNets (two
    CTAs per SM) and for centre-line queries, against the per-colour launches."""
    sizes = [(2, 2), (1, 3), (3, 1), (2, 3), (1, 1)] * 3
    w = I.xavier_sdnet(I.SDNetShape(width, depth), 69, bias_scale=0.1)
    net = m.SDNet(w, width, depth)
    bcs, us = [], []
    for q, (lx, ly) in enumerate(sizes):
        bc, u = state(lx, ly, 200 + q)
        bcs.append(bc)
        us.append(u)
    outs = {}
    for mode in ("per_colour", "sweep"):
        b = m.Batch(sizes, bcs)
        for q, u in enumerate(us):
            b.upload(q, u)
        b.sweep(net, 2, "bf16", query=query, launch_mode=mode)
        outs[mode] = [b.download(q) for q in range(len(sizes))]
    for q in range(len(sizes)):
        assert np.array_equal(outs["sweep"][q], outs["per_colour"][q]), q
