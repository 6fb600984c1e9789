"""The FP32 path on the tensor cores (MF_PREC_FP32 for width-128 SDNets, tanh here and
GELU in the variant tests: every hidden product split in three F16 products with FP32
accumulation) against the FP64 oracle at the FP32 tolerance, and against the FP32 SIMT
kernel (MF_PREC_FP32_SIMT) on the same state. Shapes cover every split of the hidden weights between tensor memory
(layers 1-3) and shared memory (layers 4-5), ragged last tiles (rows not a multiple of
64), the additive schedule, centre-line queries and batches."""
import numpy as np
import pytest

from oracle import mosaic_flow as orc
from paper_2308_14258_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def m():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_14258_gb300 import mosaicflow
    return mosaicflow


def case(lx, ly, depth, seed, bias=0.1):
    w = I.xavier_sdnet(I.SDNetShape(128, depth), seed, bias_scale=bias)
    bc = I.bc_values(lx, ly, I.mode_field(I.mode_coeffs(seed + 1), lx, ly))
    u0 = orc.make_grid(lx, ly, bc)
    ny, nx = u0.shape
    u0[1:-1, 1:-1] = I.Stream(seed + 2, I.TAG_TEST).normal((ny - 2) * (nx - 2)).reshape(ny - 2, nx - 2) * 0.3
    return w, bc, u0.astype(np.float32)


def rel(got, ref):
    return float(np.abs(got.astype(np.float64) - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("lx,ly,depth,schedule,query", [
    (1, 1, 6, "M", "full"),      # 961 rows: 15 tiles of 64 + a ragged tail of 1
    (2, 3, 6, "M", "full"),
    (3, 2, 5, "M", "full"),      # hidden layers 1-3 in TMEM, 4 in shared memory
    (2, 2, 4, "M", "full"),      # layers 1-3 in TMEM only
    (4, 1, 3, "M", "full"),
    (1, 2, 2, "M", "full"),      # one hidden layer
    (3, 3, 6, "A", "full"),      # additive schedule (cover-weighted scatter)
    (3, 2, 6, "M", "centre"),    # 61 centre-cross rows per subdomain
])
def test_fp32_tensor_path_matches_oracle(m, lx, ly, depth, schedule, query):
    w, bc, u0 = case(lx, ly, depth, 70 + depth)
    net = m.SDNet(w, 128, depth)
    solver = orc.Solver(orc.unpack_sdnet(w, 128, depth))
    g = m.Grid(lx, ly, bc)
    g.upload(u0)
    g.sweep(net, 1, schedule, "fp32", query=query)
    got = g.download()
    if schedule == "M":
        ref = orc.sweep_multiplicative(u0.astype(np.float64), lx, ly, solver, query=query.replace("centre", "center"))
    else:
        ref = orc.sweep_additive(u0.astype(np.float64), lx, ly, solver)
    assert rel(got, ref) <= TOL
    g.upload(u0)
    g.sweep(net, 1, schedule, "fp32_simt", query=query)
    simt = g.download()
    assert rel(simt, ref) <= TOL
    # the two FP32 paths agree far inside the tolerance
    assert rel(got, simt.astype(np.float64)) <= 3e-6


def test_fp32_tensor_path_large_sampled(m):
    """The 2049 x 2049 benchmark grid, one colour at a time from a swept state: sampled
    subdomains against the oracle, every point outside the colour untouched."""
    w = I.large()
    p = w.problems[0]
    weights = w.weights()
    solver = orc.Solver(orc.unpack_sdnet(weights, 128, 6))
    net = m.SDNet(weights, 128, 6)
    rng = np.random.default_rng(3)
    g = m.Grid(p.lx, p.ly, p.bc)
    g.sweep(net, 1, "M", "bf16")
    for c in range(4):
        pre = g.download()
        g.sweep(net, 1, "M", "fp32", colours=1 << c)
        post = g.download()
        subs = orc.subdomains_of_colour(p.lx, p.ly, c)
        pick = [subs[i] for i in rng.choice(len(subs), 16, replace=False)] + [subs[0], subs[-1]]
        V = solver.solve_batch(np.stack([orc.gather(pre.astype(np.float64), a, b) for (a, b) in pick]))
        scale = np.abs(pre).max()
        for (a, b), v in zip(pick, V):
            blk = post[16 * b + 1:16 * b + 32, 16 * a + 1:16 * a + 32].astype(np.float64).ravel()
            assert np.abs(blk - v).max() / scale <= TOL, (c, a, b)
        mask = np.ones(pre.shape, dtype=bool)
        for (a, b) in subs:
            mask[16 * b + 1:16 * b + 32, 16 * a + 1:16 * a + 32] = False
        assert np.array_equal(pre[mask], post[mask])


def test_fp32_tensor_path_in_batches(m):
    sizes = [(1, 1), (2, 3), (3, 2), (2, 2)]
    w = I.xavier_sdnet(I.SDNetShape(128, 6), 77, bias_scale=0.1)
    net = m.SDNet(w, 128, 6)
    solver = orc.Solver(orc.unpack_sdnet(w, 128, 6))
    bcs, us = [], []
    for q, (lx, ly) in enumerate(sizes):
        _, bc, u = case(lx, ly, 6, 80 + q)
        bcs.append(bc)
        us.append(u)
    b = m.Batch(sizes, bcs)
    for q, u in enumerate(us):
        b.upload(q, u)
    b.sweep(net, 1, "fp32")
    for q, (lx, ly) in enumerate(sizes):
        ref = orc.sweep_multiplicative(us[q].astype(np.float64), lx, ly, solver)
        assert rel(b.download(q), ref) <= TOL, q


def test_out_of_f16_range_weights_fall_back(m):
    """A hidden weight beyond the F16 range: the SDNet gets no F16 images and FP32 sweeps
    run on the SIMT kernel, with the same result as MF_PREC_FP32_SIMT."""
    w, bc, u0 = case(2, 2, 3, 90)
    o = 128 * 130 + 128
    w[o + 5] = 7.0e4     # one hidden weight (layer 1), far outside the others
    net = m.SDNet(w, 128, 3)
    g = m.Grid(2, 2, bc)
    g.upload(u0)
    g.sweep(net, 1, "M", "fp32")
    a = g.download()
    g.upload(u0)
    g.sweep(net, 1, "M", "fp32_simt")
    assert np.array_equal(a, g.download())


def test_fp32_tensor_path_saturated_units(m):
    """Pre-activations of +-60 in every layer (biases), where e = exp(2 z) of the kernel's
    tanh overflows to infinity or flushes to zero: those units must give exactly +-1 and
    the sweep must still match the oracle and the SIMT kernel."""
    H, depth = 128, 4
    w, bc, u0 = case(2, 2, depth, 95)
    o = H * 130
    w[o:o + 16] = 60.0            # first layer: b0
    w[o + 16:o + 32] = -60.0
    o += H
    for _ in range(depth - 1):    # hidden layers: biases after W_l
        b = o + H * H
        w[b:b + 32] = 60.0
        w[b + 32:b + 64] = -60.0
        o = b + H
    net = m.SDNet(w, H, depth)
    solver = orc.Solver(orc.unpack_sdnet(w, H, depth))
    g = m.Grid(2, 2, bc)
    g.upload(u0)
    g.sweep(net, 1, "M", "fp32")
    got = g.download()
    assert np.isfinite(got).all()
    ref = orc.sweep_multiplicative(u0.astype(np.float64), 2, 2, solver)
    assert rel(got, ref) <= TOL
    g.upload(u0)
    g.sweep(net, 1, "M", "fp32_simt")
    assert rel(got, g.download().astype(np.float64)) <= 3e-6
