"""Train an SDNet with the physics-informed training step (Eq. 3, Algorithm 1), then solve
larger Laplace problems by Mosaic Flow sweeps with it (Algorithm 2) and compare them with
the exact harmonic solution.

Training data: random harmonic functions on the unit square with data on all four sides
(inputs.harmonic_family), a pool of functions drawn once; every step takes F of them at
random with F x Nc collocation points uniform in the square (torch's generator, seeded)
and the 128 boundary points as data points. LAMB with a linear warm-up and a cosine
decay of the learning rate. The SDNet is 6 x 128 (the benchmark shape) on the fused BF16
training engine.

Checks, all on the GPU through the library's calls:
  * held-out error: the trained SDNet on one unit subdomain (a 33 x 33 grid, one sweep)
    for functions outside the training pool, against their exact interior values;
  * Mosaic Flow: [0, L]^2 problems (L = 2, 4, 8) whose boundary data come from a
    held-out function scaled to the domain, swept until the relative change is below
    eps; the maximum error over the grid against the exact solution, for the trained
    and the untrained network.

    python -m paper_2308_14258_gb300.train_solve --steps 12000
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import inputs as I
from . import mosaicflow as mf

WIDTH, DEPTH = 128, 6


def unit_grid_xy(L: int):
    n = 32 * L + 1
    xs = np.arange(n) / 32.0
    return np.meshgrid(xs, xs, indexing="xy")  # X[iy, ix] = x


def held_out_error(net: mf.SDNet, fam: I.HarmonicFamily, n: int) -> float:
    """Relative L2 error of the SDNet's interior prediction over n unit subdomains."""
    xb = I.unit_square_boundary_points()
    G = fam(xb[:, 0], xb[:, 1])
    X, Y = unit_grid_xy(1)
    exact = fam(X, Y).reshape(-1, 33, 33)
    num = den = 0.0
    for i in range(n):
        grid = mf.Grid(1, 1, G[i])
        grid.sweep(net, 1, "M", "fp32")
        u = grid.download()
        num += float(((u[1:-1, 1:-1] - exact[i, 1:-1, 1:-1]) ** 2).sum())
        den += float((exact[i, 1:-1, 1:-1] ** 2).sum())
    return math.sqrt(num / den)


def mosaic_flow_error(net: mf.SDNet, fam: I.HarmonicFamily, j: int, L: int, precision: str,
                      max_sweeps: int, eps: float) -> dict:
    """Sweeps on [0, L]^2 with the boundary data of held-out function j scaled to the
    domain; max |u - exact| / max |exact| over the grid."""
    n = 32 * L + 1
    pts = I.boundary_points(n, n) / 32.0
    bc = fam(pts[:, 0], pts[:, 1], scale=L)[j]
    X, Y = unit_grid_xy(L)
    exact = fam(X, Y, scale=L)[j].reshape(n, n)
    grid = mf.Grid(L, L, bc)
    out = grid.sweep(net, max_sweeps, "M", precision, eps=eps)
    u = grid.download()
    scale = float(np.abs(exact).max())
    res_max, res_rms = grid.residual()
    return {"L": L, "precision": precision, "sweeps": int(out.sweeps_done), "delta": float(out.delta),
            "residual_max": res_max, "residual_rms": res_rms,
            "max_err_rel": float(np.abs(u - exact).max()) / scale,
            "zero_start_err_rel": float(np.abs(exact[1:-1, 1:-1]).max()) / scale}


def lr_at(it: int, steps: int, lr0: float, warmup: int) -> float:
    if it < warmup:
        return lr0 * (it + 1) / warmup
    t = (it - warmup) / max(1, steps - warmup)
    return lr0 * (0.01 + 0.99 * 0.5 * (1.0 + math.cos(math.pi * t)))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=12000)
    ap.add_argument("--functions", type=int, default=1024, help="functions per step")
    ap.add_argument("--points", type=int, default=1024, help="collocation points per function")
    ap.add_argument("--pool", type=int, default=65536, help="training functions")
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--eval-every", type=int, default=3000)
    ap.add_argument("--max-sweeps", type=int, default=400)
    ap.add_argument("--eps", type=float, default=1e-7)
    a = ap.parse_args(argv)

    dev = torch.device("cuda")
    F, Nc = a.functions, a.points
    pool = I.harmonic_family(a.pool, a.seed)
    test = I.harmonic_family(64, a.seed + 1)
    xb = I.unit_square_boundary_points()
    G_pool = torch.tensor(pool(xb[:, 0], xb[:, 1]), dtype=torch.float32, device=dev)
    Xb = torch.tensor(xb, dtype=torch.float32, device=dev).expand(F, 128, 2).contiguous()
    w0 = I.xavier_sdnet(I.SDNetShape(WIDTH, DEPTH), a.seed)
    tr = mf.Trainer(w0, WIDTH, DEPTH, "bf16", "lamb", max_functions=F, max_points=Nc)
    gen = torch.Generator(device=dev)
    gen.manual_seed(a.seed)

    hist, evals = [], []
    t0 = time.time()
    for it in range(a.steps + 1):
        if it % a.eval_every == 0 or it == a.steps:
            net = mf.SDNet(tr.weights(), WIDTH, DEPTH)
            evals.append({"step": it, "held_out_rel_l2": held_out_error(net, test, 16)})
        if it == a.steps:
            break
        idx = torch.randint(0, a.pool, (F,), device=dev, generator=gen)
        G = G_pool[idx]
        Xc = torch.rand(F, Nc, 2, device=dev, generator=gen)
        loss = tr.step(G, Xc, Xb, G, lr_at(it, a.steps, a.lr, a.warmup))
        if it % 500 == 0 or it == a.steps - 1:
            hist.append({"step": it, "loss": loss[0], "data": loss[1], "pde": loss[2]})
    train_s = time.time() - t0

    trained = mf.SDNet(tr.weights(), WIDTH, DEPTH)
    untrained = mf.SDNet(w0, WIDTH, DEPTH)
    runs = []
    for L in (2, 4, 8):
        for j in range(2):
            r = mosaic_flow_error(trained, test, j, L, "fp32", a.max_sweeps, a.eps)
            r.update({"net": "trained", "function": j})
            runs.append(r)
        r = mosaic_flow_error(trained, test, 0, L, "bf16", a.max_sweeps, 1e-5)
        r.update({"net": "trained", "function": 0})
        runs.append(r)
        r = mosaic_flow_error(untrained, test, 0, L, "fp32", a.max_sweeps, a.eps)
        r.update({"net": "untrained", "function": 0})
        runs.append(r)
    print(json.dumps({"steps": a.steps, "functions_per_step": F, "points_per_function": Nc, "pool": a.pool,
                      "train_seconds": train_s, "loss": hist, "held_out": evals, "mosaic_flow": runs}))


if __name__ == "__main__":
    main()
