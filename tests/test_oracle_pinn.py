"""Pins for the training-step oracle: autograd Laplacian against finite differences,
parameter gradients against finite differences of the loss, closed forms for a
constant network, and a hand-worked LAMB step."""
import numpy as np
import pytest
import torch

from oracle import pinn
from paper_2308_14258_gb300 import inputs as I


def small_problem(width=16, depth=3, F=3, Nc=5, Nb=6, seed=1):
    w = I.xavier_sdnet(I.SDNetShape(width, depth), seed, bias_scale=0.2)
    st = I.Stream(seed, I.TAG_TEST)
    G = st.normal(F * 128).reshape(F, 128) * 0.5
    Xc = st.uniform(F * Nc * 2).reshape(F, Nc, 2)
    Xb = st.uniform(F * Nb * 2).reshape(F, Nb, 2)
    Yb = st.normal(F * Nb).reshape(F, Nb)
    return w, G, Xc, Xb, Yb


def test_laplacian_matches_finite_differences():
    w, G, Xc, _, _ = small_problem()
    P = pinn.unpack(w, 16, 3, requires_grad=False)
    G = torch.as_tensor(G)
    X = torch.as_tensor(Xc)
    _, lap = pinn.laplacian(P, G, X)
    h = 1e-4
    f = lambda X: pinn.sdnet(P, G, X)
    ex, ey = torch.zeros_like(X), torch.zeros_like(X)
    ex[..., 0], ey[..., 1] = h, h
    fd = (f(X + ex) + f(X - ex) + f(X + ey) + f(X - ey) - 4 * f(X)) / h ** 2
    assert torch.max(torch.abs(lap - fd)) < 1e-6 * max(1.0, float(torch.max(torch.abs(lap))))


def test_gradients_match_finite_differences():
    w, G, Xc, Xb, Yb = small_problem()
    (tot, _, _), g = pinn.loss_and_grads(w, 16, 3, G, Xc, Xb, Yb)
    w64 = np.asarray(w, dtype=np.float64)
    rng = np.random.default_rng(0)
    idx = list(rng.choice(w64.size, 12, replace=False)) + [16 * 130 + 3, w64.size - 1, w64.size - 5]
    for i in idx:
        h = 1e-6
        wp, wm = w64.copy(), w64.copy()
        wp[i] += h
        wm[i] -= h
        lp = pinn.loss_and_grads(wp, 16, 3, G, Xc, Xb, Yb)[0][0]
        lm = pinn.loss_and_grads(wm, 16, 3, G, Xc, Xb, Yb)[0][0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g).max()), (i, fd, g[i])


def test_constant_network_closed_form():
    width, depth = 8, 3
    shape = I.SDNetShape(width, depth)
    w = np.zeros(shape.n_params)
    w[-1] = 0.75                                   # u = b_out everywhere
    _, G, Xc, Xb, Yb = small_problem(width, depth)
    (tot, ld, lp), g = pinn.loss_and_grads(w, width, depth, G, Xc, Xb, Yb)
    assert lp == 0.0
    assert abs(ld - np.mean((0.75 - Yb) ** 2)) < 1e-15
    assert abs(g[-1] - 2 * np.mean(0.75 - Yb)) < 1e-15
    assert np.all(g[:-1] == 0)


def test_lamb_first_step_by_hand():
    # one tensor group per shape entry; take width 1, depth 2 so every group is tiny
    width, depth = 1, 2
    n = I.SDNetShape(width, depth).n_params
    w = np.linspace(0.5, 1.5, n)
    g = np.linspace(-1.0, 2.0, n)
    w1, m1, v1 = pinn.lamb(w, g, np.zeros(n), np.zeros(n), 1, 0.1, width, depth, eps=0.0, wd=0.0)
    # step 1: m_hat = g, v_hat = g^2 -> r = sign(g); trust = ||w|| / ||sign(g)|| per group
    o = 0
    for _, shp in pinn.shapes(width, depth):
        k = int(np.prod(shp))
        sl = slice(o, o + k)
        r = np.sign(g[sl])
        trust = np.linalg.norm(w[sl]) / np.linalg.norm(r)
        assert np.allclose(w1[sl], w[sl] - 0.1 * trust * r, rtol=0, atol=1e-15)
        o += k
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_boundary_points_order():
    pts = pinn.unit_square_boundary()
    assert pts.shape == (128, 2)
    assert tuple(pts[0]) == (0.0, 0.0) and tuple(pts[32]) == (1.0, 0.0)
    assert tuple(pts[64]) == (1.0, 1.0) and tuple(pts[96]) == (0.0, 1.0)
