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


# ------------------------------------------------------------------ forward pins from outside
#
# The checks above compare the training oracle with finite differences of itself and with
# a constant network, which a transposed hidden matrix or swapped coordinate columns would
# pass. The pins below fix the forward (Eq. 7-8 and the tanh layers) against values worked
# out by hand, a closed-form Laplacian, and the sweep oracle's SDNet, which has its own
# hand-computed pin.

import math

from oracle import mosaic_flow as mf


def packed_offsets(width, depth):
    """Offsets of the packed FP32 layout (W0[H][130], b0[H], {W[H][H], b[H]} x (depth-1),
    w_out[H], b_out), counted here from the layout itself."""
    h, o, off = width, 0, {}
    for name, n in [("W0", h * 130), ("b0", h)] + sum(
            ([(f"W{l}", h * h), (f"b{l}", h)] for l in range(1, depth)), []) + [("wout", h), ("bout", 1)]:
        off[name] = o
        o += n
    off["_n"] = o
    return off


def toy_packed(width=64, depth=4):
    """The ln3/2, ln2/2 toy: every pre-activation on the path is ln3/2 or ln2/2, so every
    activation is exactly 1/2 or 1/3. At g[5] = 2, (x, y) = (1/2, 1/4) the output is
    6 (1/2) + 9 (1/3) + 1/4 = 6.25."""
    l2, l3 = math.log(2.0), math.log(3.0)
    off = packed_offsets(width, depth)
    w = np.zeros(off["_n"])

    def put(name, r, c, v, cols=None):
        cols = cols if cols is not None else width
        w[off[name] + r * cols + c] = v

    put("W0", 0, 5, l3 / 4, 130)        # g[5] = 2     -> ln3/2 -> 1/2
    put("W0", 1, 128, l2, 130)          # x = 1/2      -> ln2/2 -> 1/3
    put("W0", 2, 129, 2 * l3, 130)      # y = 1/4      -> ln3/2 -> 1/2
    w[off["b0"] + 3] = l2 / 2           # bias only    -> 1/3
    put("W1", 0, 1, 1.5 * l3)           # h[1] = 1/3   -> 1/2
    put("W1", 1, 0, l2 / 2)
    put("W1", 1, 2, l2 / 2)             # 1/2 + 1/2    -> 1/3
    put("W1", 2, 3, 1.5 * l2)
    w[off["b1"] + 2] = (l3 - l2) / 2    # 1/3 + bias   -> 1/2
    put("W2", 0, 2, l2)                 # h[2] = 1/2   -> 1/3
    put("W2", 1, 0, l3)                 # h[0] = 1/2   -> 1/2
    put("W3", 5, 0, 1.5 * l3)           # h[0] = 1/3   -> 1/2
    put("W3", 6, 1, l2)                 # h[1] = 1/2   -> 1/3
    w[off["wout"] + 5], w[off["wout"] + 6] = 6.0, 9.0
    w[off["bout"]] = 0.25
    return w


def toy_inputs():
    g = np.linspace(-3.0, 5.0, 128)
    g[5] = 2.0
    G = torch.as_tensor(np.stack([g, g]))
    X = torch.tensor([[[0.5, 0.25], [0.25, 0.5]], [[0.5, 0.25], [0.5, 0.25]]], dtype=torch.float64)
    return G, X


def test_training_forward_matches_hand_computed_toy():
    P = pinn.unpack(toy_packed(), 64, 4, requires_grad=False)
    G, X = toy_inputs()
    u = pinn.sdnet(P, G, X)
    assert abs(float(u[0, 0]) - 6.25) < 1e-14
    assert abs(float(u[1, 0]) - 6.25) < 1e-14 and abs(float(u[1, 1]) - 6.25) < 1e-14
    assert abs(float(u[0, 1]) - 6.25) > 1e-3      # the swapped point gives another value


def one_path_net(width, a, b, c, d, v, e, wo, bo):
    """Packed depth-2 network with a single active path:
    u = wo tanh(v tanh(a x + b y + d g[5] + c) + e) + bo, routed through unit 0 of the
    first layer and unit 3 of the hidden layer (an off-diagonal hidden weight)."""
    off = packed_offsets(width, 2)
    w = np.zeros(off["_n"])
    w[off["W0"] + 0 * 130 + 128] = a
    w[off["W0"] + 0 * 130 + 129] = b
    w[off["W0"] + 0 * 130 + 5] = d
    w[off["b0"] + 0] = c
    w[off["W1"] + 3 * width + 0] = v
    w[off["b1"] + 3] = e
    w[off["wout"] + 3] = wo
    w[off["bout"]] = bo
    return w


ONE_PATH = dict(a=0.9, b=-1.7, c=0.2, d=0.35, v=1.3, e=-0.4, wo=2.5, bo=0.4)


def one_path_closed_form(G, X, a, b, c, d, v, e, wo, bo):
    """u and Delta_x u of the one-path network, by the chain rule written out:
    with t1 = tanh z1, s1 = 1 - t1^2, t2 = tanh z2, s2 = 1 - t2^2,
    u_x = wo s2 v s1 a, and Delta u = -2 wo (a^2 + b^2) v s1 s2 (t2 v s1 + t1)."""
    x, y = X[..., 0], X[..., 1]
    z1 = a * x + b * y + d * G[:, 5:6] + c
    t1 = np.tanh(z1)
    s1 = 1 - t1 * t1
    t2 = np.tanh(v * t1 + e)
    s2 = 1 - t2 * t2
    u = wo * t2 + bo
    lap = -2 * wo * (a * a + b * b) * v * s1 * s2 * (t2 * v * s1 + t1)
    return u, lap


def one_path_inputs():
    st = I.Stream(21, I.TAG_TEST)
    G = st.normal(3 * 128).reshape(3, 128)
    X = st.uniform(3 * 7 * 2).reshape(3, 7, 2)
    return G, X


def test_laplacian_matches_closed_form_of_one_path_network():
    w = one_path_net(8, **ONE_PATH)
    P = pinn.unpack(w, 8, 2, requires_grad=False)
    G, X = one_path_inputs()
    u, lap = pinn.laplacian(P, torch.as_tensor(G), torch.as_tensor(X))
    u_cf, lap_cf = one_path_closed_form(G, X, **ONE_PATH)
    assert np.abs(u.detach().numpy() - u_cf).max() < 1e-14
    assert np.abs(lap.detach().numpy() - lap_cf).max() < 1e-13 * max(1.0, np.abs(lap_cf).max())
    assert np.abs(lap_cf).max() > 0.1               # the pin is not vacuous


def test_training_forward_equals_sweep_oracle_sdnet():
    """pinn.sdnet and the sweep oracle's SDNet (pinned by its own hand-computed toy) on
    the same packed weights: width 64, depth 4, random non-symmetric matrices, biases."""
    width, depth = 64, 4
    w = I.xavier_sdnet(I.SDNetShape(width, depth), 31, bias_scale=0.3)
    st = I.Stream(32, I.TAG_TEST)
    G = st.normal(3 * 128).reshape(3, 128)
    X = st.uniform(3 * 9 * 2).reshape(3, 9, 2)
    u = pinn.sdnet(pinn.unpack(w, width, depth, requires_grad=False), torch.as_tensor(G),
                   torch.as_tensor(X)).numpy()
    Pm = mf.unpack_sdnet(w, width, depth)
    for f in range(3):
        ref = mf.sdnet(Pm, G[f], X[f])
        assert np.abs(u[f] - ref).max() < 1e-13 * max(1.0, np.abs(ref).max())


def _transposed_hidden(P):
    return [p.T.clone() if (i >= 2 and i < len(P) - 2 and p.dim() == 2) else p for i, p in enumerate(P)]


def _swapped_coordinates(P):
    W0 = P[0].clone()
    W0[:, 128], W0[:, 129] = P[0][:, 129].clone(), P[0][:, 128].clone()
    return [W0] + list(P[1:])


def test_mutation_transposed_hidden_weight_fails_the_pins():
    G, X = toy_inputs()
    P = _transposed_hidden(pinn.unpack(toy_packed(), 64, 4, requires_grad=False))
    assert abs(float(pinn.sdnet(P, G, X)[0, 0]) - 6.25) > 1e-3
    P1 = _transposed_hidden(pinn.unpack(one_path_net(8, **ONE_PATH), 8, 2, requires_grad=False))
    G1, X1 = one_path_inputs()
    _, lap = pinn.laplacian(P1, torch.as_tensor(G1), torch.as_tensor(X1))
    _, lap_cf = one_path_closed_form(G1, X1, **ONE_PATH)
    assert np.abs(lap.detach().numpy() - lap_cf).max() > 1e-3


def test_mutation_swapped_coordinate_columns_fail_the_pins():
    G, X = toy_inputs()
    P = _swapped_coordinates(pinn.unpack(toy_packed(), 64, 4, requires_grad=False))
    assert abs(float(pinn.sdnet(P, G, X)[0, 0]) - 6.25) > 1e-3
    P1 = _swapped_coordinates(pinn.unpack(one_path_net(8, **ONE_PATH), 8, 2, requires_grad=False))
    G1, X1 = one_path_inputs()
    u, _ = pinn.laplacian(P1, torch.as_tensor(G1), torch.as_tensor(X1))
    u_cf, _ = one_path_closed_form(G1, X1, **ONE_PATH)
    assert np.abs(u.detach().numpy() - u_cf).max() > 1e-3
