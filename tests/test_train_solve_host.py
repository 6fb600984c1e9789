"""Host-side pieces of the train-then-solve script: the learning-rate schedule and the
boundary data of a scaled held-out function."""
import numpy as np

from paper_2308_14258_gb300 import inputs as I
from paper_2308_14258_gb300 import train_solve as ts


def test_learning_rate_schedule():
    steps, lr0, warm = 1000, 2e-3, 100
    lr = np.array([ts.lr_at(i, steps, lr0, warm) for i in range(steps + 1)])
    np.testing.assert_allclose(lr[:warm], lr0 * np.arange(1, warm + 1) / warm)   # linear warm-up
    assert abs(lr[warm] - lr0) < 1e-15                                          # peak
    assert np.all(np.diff(lr[warm:]) <= 0)                                      # cosine decay
    assert abs(lr[steps] - 0.01 * lr0) < 1e-15                                  # floor at 1 %


def test_scaled_boundary_data_match_the_field():
    fam = I.harmonic_family(3, 2)
    L = 4
    n = 32 * L + 1
    pts = I.boundary_points(n, n) / 32.0
    bc = fam(pts[:, 0], pts[:, 1], scale=L)
    X, Y = ts.unit_grid_xy(L)
    grid = fam(X, Y, scale=L).reshape(3, n, n)
    ix, iy = I.boundary_points(n, n).T
    np.testing.assert_allclose(bc, grid[:, iy, ix], rtol=0, atol=1e-12)
