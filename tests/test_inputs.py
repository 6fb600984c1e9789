"""Seeded input generators: published SplitMix64 values, shapes and the harmonic data."""
import math
import os

import numpy as np

from paper_2308_14258_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_splitmix():
    out = {}
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            seed, *vals = line.split()
            out[int(seed)] = [int(v, 16) for v in vals]
    return out


def test_splitmix64_published_values():
    for seed, vals in _golden_splitmix().items():
        got = [int(v) for v in I.splitmix64(seed, len(vals))]
        assert got == vals


def test_stream_is_counter_based():
    s = I.Stream(7, I.TAG_TEST)
    a = s.u64(5)
    b = s.u64(3)
    full = I.splitmix64(I.stream_state(7, I.TAG_TEST), 8)
    assert list(np.concatenate([a, b])) == list(full)


def test_uniform_and_normal_moments():
    s = I.Stream(11, I.TAG_TEST)
    u = s.uniform(200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005
    z = I.Stream(12, I.TAG_TEST).normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_xavier_shapes_and_bounds():
    for shape in (I.SDNetShape(64, 4), I.SDNetShape(128, 6)):
        w = I.xavier_sdnet(shape, 0)
        assert w.dtype == np.float32 and w.size == shape.n_params
        h = shape.width
        W0 = w[: h * 130]
        assert np.abs(W0).max() <= math.sqrt(6.0 / (130 + h)) + 1e-7
        b0 = w[h * 130: h * 131]
        assert np.all(b0 == 0)


def test_boundary_points_ccw():
    pts = I.boundary_points(5, 4)
    assert len(pts) == 2 * 4 + 2 * 3
    assert tuple(pts[0]) == (0, 0) and tuple(pts[4]) == (4, 0)
    assert tuple(pts[7]) == (4, 3) and tuple(pts[11]) == (0, 3)
    assert len({tuple(p) for p in pts}) == len(pts)


def test_mode_field_is_harmonic_and_matches_sinh_ratio():
    a = I.mode_coeffs(1)
    f = I.mode_field(a, 16.0, 16.0)
    x, y, e = 3.3, 7.1, 1e-3
    lap = (f(x + e, y) + f(x - e, y) + f(x, y + e) + f(x, y - e) - 4 * f(x, y)) / e ** 2
    assert abs(lap) < 1e-4
    direct = sum(ak * math.sin(k * math.pi * x / 16) * math.sinh(k * math.pi * y / 16) / math.sinh(k * math.pi)
                 for k, ak in enumerate(a, start=1))
    assert abs(f(x, y) - direct) < 1e-12
    # boundary behaviour: zero on the bottom, left and right edges, sum a_k sin on top
    assert abs(f(0.0, 5.0)) < 1e-12 and abs(f(16.0, 5.0)) < 1e-12 and abs(f(5.0, 0.0)) < 1e-15


def test_presets():
    t = I.tiny()
    assert t.problems[0].bc.shape == (4 * 64,)
    assert t.shape.width == 64 and t.shape.depth == 4
    b = I.batched(16)
    assert all(p.lx in (2, 4, 8, 16, 32) for p in b.problems)


def test_training_batch_shapes_and_harmonic_data():
    tb = I.training_batch(4, 16)
    assert tb.G.shape == (4, 128) and tb.Xc.shape == (4, 16, 2) and tb.Xb.shape == (4, 128, 2)
    assert np.all((tb.Xc > 0) & (tb.Xc < 1))
    assert np.array_equal(tb.Yb, tb.G)
    # the 8-mode field vanishes on the bottom, left and right edges of the unit square
    assert np.abs(tb.G[:, :32]).max() < 1e-12 and np.abs(tb.G[:, 96:]).max() < 1e-12


def test_harmonic_family_sides_and_harmonicity():
    import math
    f = I.harmonic_family(3, 5, n_modes=4)
    t = np.linspace(0.0, 1.0, 17)
    k = np.arange(1, 5)[:, None]
    sk = np.sin(math.pi * k * t)
    # each side carries its own sine series plus the bilinear part
    np.testing.assert_allclose(f(t, 0 * t), f.e[:, :1] + f.e[:, 1:2] * t + f.a[:, 1, :] @ sk, atol=1e-12)
    np.testing.assert_allclose(f(t, 0 * t + 1), f.e[:, :1] + f.e[:, 2:3] + (f.e[:, 1:2] + f.e[:, 3:4]) * t
                               + f.a[:, 0, :] @ sk, atol=1e-12)
    np.testing.assert_allclose(f(0 * t + 1, t), f.e[:, :1] + f.e[:, 1:2] + (f.e[:, 2:3] + f.e[:, 3:4]) * t
                               + f.a[:, 2, :] @ sk, atol=1e-12)
    np.testing.assert_allclose(f(0 * t, t), f.e[:, :1] + f.e[:, 2:3] * t + f.a[:, 3, :] @ sk, atol=1e-12)
    # harmonic: the 5-point Laplacian is O(h^2) at interior points
    h = 1e-3
    x, y = np.array([0.3, 0.71]), np.array([0.45, 0.2])
    lap = (f(x + h, y) + f(x - h, y) + f(x, y + h) + f(x, y - h) - 4 * f(x, y)) / h**2
    assert np.abs(lap).max() < 1e-2
    # scaling the domain keeps the function harmonic and maps the corners
    np.testing.assert_allclose(f(np.array([4.0]), np.array([4.0]), scale=4.0), f(np.array([1.0]), np.array([1.0])))
