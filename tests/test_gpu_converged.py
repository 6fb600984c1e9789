"""The mid workload (961 subdomains, grid 513 x 513, SDNet 6 x 128) along its whole
trajectory from the zero interior, against the FP64 oracle run the same way
(Algorithm 2's loop):

* FP32: 20 sweeps, the field within 1e-5 of the oracle's and delta within 1e-5 of the
  oracle's delta after every checked sweep;
* MF_PREC_MIXED (BF16 sweeps until delta < 1e-2, then FP32 refinement until
  delta < 1e-6): the converged field within 1e-3 of the oracle's converged field;
* BF16 alone to its own fixed point: within the per-sweep BF16 bound 3e-2.

The random 6 x 128 network contracts (delta falls by about 5x per sweep), so after 20
sweeps the oracle's field is converged to about 1e-13."""
import numpy as np
import pytest

from oracle import mosaic_flow as orc
from paper_2308_14258_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N_SWEEPS = 20


@pytest.fixture(scope="module")
def m():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_14258_gb300 import mosaicflow
    return mosaicflow


@pytest.fixture(scope="module")
def mid_oracle():
    w = I.mid()
    p = w.problems[0]
    weights = w.weights()
    solver = orc.Solver(orc.unpack_sdnet(weights, 128, 6))
    u0 = orc.make_grid(p.lx, p.ly, p.bc.astype(np.float32).astype(np.float64))
    ref, hist = orc.run(u0, p.lx, p.ly, solver, N_SWEEPS)
    return p, weights, ref, hist


def rel(got, ref):
    return float(np.abs(got.astype(np.float64) - ref).max() / np.abs(ref).max())


def test_mid_fp32_trajectory(m, mid_oracle):
    p, weights, ref, hist = mid_oracle
    assert hist[-1] < 1e-11
    net = m.SDNet(weights, 128, 6)
    g = m.Grid(p.lx, p.ly, p.bc)
    deltas = []
    for _ in range(N_SWEEPS):
        deltas.append(g.sweep(net, 1, "M", "fp32").delta)
    assert rel(g.download(), ref) <= 1e-5
    # delta agrees while it is above the FP32 rounding floor of the field (~4e-7)
    for k, (d, r) in enumerate(zip(deltas, hist)):
        if r > 1e-4:
            assert abs(d - r) <= 1e-5 * r + 1e-5, (k, d, r)


@pytest.mark.parametrize("eps_coarse", [1e-2, 1e-9])
def test_mid_mixed_refinement_reaches_oracle_fixed_point(m, mid_oracle, eps_coarse):
    """eps_coarse = 1e-9 lies below the BF16 rounding floor of delta (about 3.4e-3 on
    this grid): the switch to FP32 then comes from the stall rule (a BF16 sweep that
    does not reduce delta)."""
    p, weights, ref, _ = mid_oracle
    net = m.SDNet(weights, 128, 6)
    g = m.Grid(p.lx, p.ly, p.bc)
    out = g.sweep(net, 200, "M", "mixed", eps=1e-6, eps_coarse=eps_coarse)
    assert 0 < out.sweeps_bf16 < out.sweeps_done < 200
    assert out.delta < 1e-6
    assert rel(g.download(), ref) <= 1e-3
    g2 = m.Grid(p.lx, p.ly, p.bc)
    g2.sweep(net, 40, "M", "bf16")
    assert rel(g2.download(), ref) <= 3e-2


def test_mid_f16_alone_reaches_oracle_fixed_point(m, mid_oracle):
    """F16 sweeps alone (MF_PREC_F16, no FP32 refinement) to their own fixed point: the
    field within 1e-3 of the FP64 oracle's converged field. F16 rounds activations and
    weights to 11 significant bits against BF16's 8, the error floor of BF16 sweeps
    alone being above 1e-3 on the benchmark grid."""
    p, weights, ref, _ = mid_oracle
    net = m.SDNet(weights, 128, 6)
    g = m.Grid(p.lx, p.ly, p.bc)
    out = g.sweep(net, 40, "M", "f16", eps=0.0)
    assert out.sweeps_done == 40
    err = rel(g.download(), ref)
    assert err <= 1e-3, err
