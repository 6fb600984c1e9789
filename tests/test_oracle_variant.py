"""Pins for the oracle's SDNet variant (Section 3.1): GELU activations and the boundary
embedding by circular 1-D convolutions."""
import numpy as np
import pytest

from oracle import mosaic_flow as orc
from paper_2308_14258_gb300 import inputs as I


def test_gelu_published_values():
    # GELU(x) = x Phi(x); Phi(1) = 0.8413447460685429 and Phi(2) = 0.9772498680518208 are
    # the standard normal distribution's tabulated values
    assert abs(orc.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(orc.gelu(np.array(2.0)) - 2 * 0.9772498680518208) < 1e-15
    assert orc.gelu(np.array(0.0)) == 0.0


def test_gelu_odd_part_identity():
    # x Phi(x) - (-x) Phi(-x) = x (Phi(x) + Phi(-x)) = x for every x
    x = I.Stream(3, I.TAG_TEST).normal(1000) * 3
    assert np.abs(orc.gelu(x) - orc.gelu(-x) - x).max() < 1e-14


def test_conv1d_matches_library_wrap_correlation():
    ndimage = pytest.importorskip("scipy.ndimage")
    st = I.Stream(4, I.TAG_TEST)
    for c_in, c_out, k in ((1, 4, 5), (3, 2, 3), (2, 2, 1), (4, 3, 9)):
        h = st.normal(c_in * 128).reshape(c_in, 128)
        W = st.normal(c_out * c_in * k).reshape(c_out, c_in, k)
        b = st.normal(c_out)
        full = np.stack([sum(ndimage.correlate1d(h[ci], W[co, ci], mode="wrap") for ci in range(c_in)) + b[co]
                         for co in range(c_out)])
        assert np.abs(orc.conv1d_circular(h, W, b, 1) - full).max() < 1e-12
        # stride 2 keeps the stride-1 outputs at even positions
        assert np.abs(orc.conv1d_circular(h, W, b, 2) - full[:, ::2]).max() < 1e-12


def test_embedding_is_shift_equivariant():
    # rotating the closed boundary curve by two samples rotates the stride-2 embedding by one
    shape = I.SDNetShape(64, 3, "gelu", 4, 5)
    P = orc.unpack_sdnet(I.xavier_sdnet(shape, 1, bias_scale=0.2), 64, 3, "gelu", 4, 5)
    g = I.Stream(5, I.TAG_TEST).normal(128)
    e0 = orc.embed_boundary(P, g).reshape(4, 64)
    e1 = orc.embed_boundary(P, np.roll(g, 2)).reshape(4, 64)
    assert np.abs(np.roll(e0, 1, axis=1) - e1).max() < 1e-13


def test_embedding_impulse_response():
    # one conv layer on a unit impulse at position m returns the kernel taps around m
    W = np.arange(1.0, 6.0).reshape(1, 1, 5)
    g = np.zeros((1, 128))
    g[0, 10] = 1.0
    out = orc.conv1d_circular(g, W, np.zeros(1), 1)[0]
    # out[i] = sum_t W[t] g[i + t - 2]: nonzero where i + t - 2 = 10, i.e. i = 12 - t
    expect = np.zeros(128)
    for t in range(5):
        expect[12 - t] = W[0, 0, t]
    assert np.array_equal(out, expect)
    # and across the wrap: an impulse at 0 reaches positions 126, 127, 0, 1, 2
    g[0, 10], g[0, 0] = 0.0, 1.0
    out = orc.conv1d_circular(g, W, np.zeros(1), 1)[0]
    assert [out[i] for i in (2, 1, 0, 127, 126)] == [1.0, 2.0, 3.0, 4.0, 5.0]


@pytest.mark.parametrize("c,k", [(4, 5), (8, 3)])
def test_variant_concat_equals_split_and_batched(c, k):
    shape = I.SDNetShape(64, 4, "gelu", c, k)
    P = orc.unpack_sdnet(I.xavier_sdnet(shape, 2, bias_scale=0.2), 64, 4, "gelu", c, k)
    X = orc.interior_coords()
    G = I.Stream(6, I.TAG_TEST).normal(3 * 128).reshape(3, 128)
    for g in G:
        assert np.abs(orc.sdnet(P, g, X, "split") - orc.sdnet(P, g, X, "concat")).max() < 1e-12
    batched = orc.sdnet_batched(P, G, X)
    seq = np.stack([orc.sdnet(P, g, X, "split") for g in G])
    assert np.abs(batched - seq).max() < 1e-13


def test_variant_reduces_to_tanh_net_without_options():
    # the default options leave the raw-boundary tanh network untouched
    w = I.xavier_sdnet(I.SDNetShape(64, 3), 0, bias_scale=0.1)
    P = orc.unpack_sdnet(w, 64, 3)
    g = I.Stream(7, I.TAG_TEST).normal(128)
    X = orc.interior_coords()[:5]
    h = np.tanh((g @ P["W1"].T + P["b0"])[None, :] + X @ P["W2"].T)
    for Wl, bl in P["hidden"]:
        h = np.tanh(h @ Wl.T + bl)
    assert np.abs(orc.sdnet(P, g, X) - (h @ P["wout"] + P["bout"])).max() < 1e-15


def _conv_pin_holds():
    ndimage = pytest.importorskip("scipy.ndimage")
    st = I.Stream(8, I.TAG_TEST)
    h = st.normal(2 * 128).reshape(2, 128)
    W = st.normal(3 * 2 * 5).reshape(3, 2, 5)
    b = st.normal(3)
    full = np.stack([sum(ndimage.correlate1d(h[ci], W[co, ci], mode="wrap") for ci in range(2)) + b[co]
                     for co in range(3)])
    return np.abs(orc.conv1d_circular(h, W, b, 2) - full[:, ::2]).max() < 1e-12


def test_mutation_reversed_taps_is_caught(monkeypatch):
    # plant a convolution (flipped taps) where the cross-correlation belongs
    real = orc.conv1d_circular

    def flipped(h, W, b, stride):
        return real(h, W[:, :, ::-1], b, stride)
    monkeypatch.setattr(orc, "conv1d_circular", flipped)
    assert not _conv_pin_holds()


def test_mutation_odd_stride_phase_is_caught(monkeypatch):
    # plant a stride-2 layer that keeps the odd positions
    real = orc.conv1d_circular

    def odd(h, W, b, stride):
        out = real(h, W, b, 1)
        return out[:, 1::2] if stride == 2 else out
    monkeypatch.setattr(orc, "conv1d_circular", odd)
    assert not _conv_pin_holds()


def test_mutation_gelu_scale_is_caught(monkeypatch):
    # plant erf(x) in place of erf(x / sqrt 2): the tabulated value Phi(1) is missed
    from scipy.special import erf
    monkeypatch.setattr(orc, "gelu", lambda x: 0.5 * x * (1.0 + erf(x)))
    assert abs(orc.gelu(np.array(1.0)) - 0.8413447460685429) > 1e-2
