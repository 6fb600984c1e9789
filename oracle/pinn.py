"""FP64 CPU oracle of the physics-informed SDNet training step -- TEST INFRASTRUCTURE ONLY.

Only the tests may import this module. It restates, with plain PyTorch CPU autograd in
float64 (the paper's own way of forming the derivatives, Section 3.3):

* the SDNet N(x, g) with the input-split first layer (Eq. 7-8) and tanh layers;
* the PDE loss of Eq. 3, L_pde = mean over collocation points of (Delta_x N)^2, with the
  Laplacian from two nested autograd passes (d/dx, then d/dx of each component);
* the data loss L_data = mean squared error at points with known values (Section 3.3);
* one training iteration of Algorithm 1: gradients of the data loss, then of the PDE
  loss, summed (the allreduce of step 3 is the identity on one device);
* the LAMB update (You et al., "Large Batch Optimization for Deep Learning: Training
  BERT in 76 minutes", ICLR 2020), which the paper uses through Apex FusedLAMB (Section
  5.2), and plain SGD.

Shapes: G (F, 128) boundary values per function; Xc (F, Nc, 2) collocation points;
Xb (F, Nb, 2) data points with targets Yb (F, Nb). Parameters use the packed FP32
layout of the library: W0[H][130], b0[H], {W[H][H], b[H]} x (depth-1), w_out[H], b_out.
"""
from __future__ import annotations

import numpy as np
import torch

N_BDRY = 128


def shapes(width: int, depth: int):
    h = width
    out = [("W0", (h, N_BDRY + 2)), ("b0", (h,))]
    for l in range(1, depth):
        out += [(f"W{l}", (h, h)), (f"b{l}", (h,))]
    out += [("wout", (h,)), ("bout", (1,))]
    return out


def unpack(w, width: int, depth: int, requires_grad: bool = True):
    """Packed vector -> list of float64 leaf tensors in packed order."""
    w = torch.as_tensor(np.asarray(w, dtype=np.float64))
    params, o = [], 0
    for _, shp in shapes(width, depth):
        n = int(np.prod(shp))
        params.append(w[o:o + n].reshape(shp).clone().requires_grad_(requires_grad))
        o += n
    assert o == w.numel()
    return params


def pack(tensors) -> np.ndarray:
    return np.concatenate([t.detach().reshape(-1).numpy() for t in tensors])


def sdnet(params, G: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    """u (F, n) at points X (F, n, 2) of the functions with boundary values G (F, 128)."""
    W0, b0 = params[0], params[1]
    hidden = [(params[2 + 2 * i], params[3 + 2 * i]) for i in range((len(params) - 4) // 2)]
    wout, bout = params[-2], params[-1]
    B = G @ W0[:, :N_BDRY].T + b0                    # per function (Eq. 8, left term)
    pre = B[:, None, :] + X @ W0[:, N_BDRY:].T       # broadcast sum with the point term
    h = torch.tanh(pre)
    for W, b in hidden:
        h = torch.tanh(h @ W.T + b)
    return h @ wout + bout


def laplacian(params, G: torch.Tensor, X: torch.Tensor):
    """(u, Delta_x u) at X by two nested autograd passes."""
    X = X.clone().requires_grad_(True)
    u = sdnet(params, G, X)
    (gx,) = torch.autograd.grad(u.sum(), X, create_graph=True)
    (gxx,) = torch.autograd.grad(gx[..., 0].sum(), X, create_graph=True)
    (gyy,) = torch.autograd.grad(gx[..., 1].sum(), X, create_graph=True)
    return u, gxx[..., 0] + gyy[..., 1]


def loss_terms(params, G, Xc, Xb, Yb):
    u_b = sdnet(params, G, Xb)
    l_data = torch.mean((u_b - Yb) ** 2)
    _, lap = laplacian(params, G, Xc)
    l_pde = torch.mean(lap ** 2)
    return l_data, l_pde


def loss_and_grads(w, width: int, depth: int, G, Xc, Xb, Yb):
    """Algorithm 1 on one device: gradients of the data loss, plus gradients of the PDE
    loss. Returns ((total, data, pde), packed FP64 gradient)."""
    params = unpack(w, width, depth)
    G = torch.as_tensor(np.asarray(G, dtype=np.float64))
    Xc = torch.as_tensor(np.asarray(Xc, dtype=np.float64))
    Xb = torch.as_tensor(np.asarray(Xb, dtype=np.float64))
    Yb = torch.as_tensor(np.asarray(Yb, dtype=np.float64))
    l_data = torch.mean((sdnet(params, G, Xb) - Yb) ** 2)
    g_data = torch.autograd.grad(l_data, params, allow_unused=True)
    _, lap = laplacian(params, G, Xc)
    l_pde = torch.mean(lap ** 2)
    g_pde = torch.autograd.grad(l_pde, params, allow_unused=True)  # b_out drops out of Delta u
    grads = [(a if a is not None else torch.zeros_like(p)) + (b if b is not None else torch.zeros_like(p))
             for a, b, p in zip(g_data, g_pde, params)]
    ld, lp = float(l_data.detach()), float(l_pde.detach())
    return (ld + lp, ld, lp), pack(grads)


def sgd(w, g, lr):
    return np.asarray(w, dtype=np.float64) - lr * np.asarray(g, dtype=np.float64)


def lamb(w, g, m, v, step, lr, width, depth, beta1=0.9, beta2=0.999, eps=1e-6, wd=0.0):
    """One LAMB step (step counts from 1), trust ratio per parameter tensor:
    m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; r = m_hat / (sqrt(v_hat) + eps) + wd w;
    w -= lr * (||w|| / ||r|| if both norms > 0 else 1) * r."""
    w = np.asarray(w, dtype=np.float64).copy()
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    o = 0
    for _, shp in shapes(width, depth):
        n = int(np.prod(shp))
        sl = slice(o, o + n)
        r = mh[sl] / (np.sqrt(vh[sl]) + eps) + wd * w[sl]
        wn, rn = np.linalg.norm(w[sl]), np.linalg.norm(r)
        trust = wn / rn if (wn > 0 and rn > 0) else 1.0
        w[sl] -= lr * trust * r
        o += n
    return w, m, v


def unit_square_boundary(n_side: int = 32) -> np.ndarray:
    """(128, 2) coordinates of the boundary points of the unit square, CCW from (0,0),
    the order of the 128 boundary values (bottom, right, top, left; each corner once)."""
    h = 1.0 / n_side
    pts = [(i * h, 0.0) for i in range(n_side)]
    pts += [(1.0, j * h) for j in range(n_side)]
    pts += [(1.0 - i * h, 1.0) for i in range(n_side)]
    pts += [(0.0, 1.0 - j * h) for j in range(n_side)]
    return np.array(pts)
