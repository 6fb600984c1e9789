"""FP64 CPU oracle of the Mosaic Flow predictor sweep -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may import
this module. The product path (the CUDA library and its Python binding) never calls it.

It is a plain, slow, obviously correct NumPy restatement of what the paper computes,
in float64 throughout, with NumPy matmul as the only library primitive on the SDNet
path and scipy's sparse direct solver for the global finite-difference check:

* Problem (Section 2.1, Eq. 2): 2-D Laplace with Dirichlet data on [0,Lx] x [0,Ly].
* SDNet (Section 2.2; Section 3.1-3.2): N(x, g; theta), an MLP whose first layer reads
  the discretised boundary g (4N values, N = 32) and the coordinate x. Both the
  input-concat form (Eq. 5-6) and the input-split form (Eq. 7-8) are written out.
  Hidden activation tanh (the workloads fix it), or the paper's own variant (Section
  3.1): GELU activations and a boundary embedding by 1-D convolutions over g taken as a
  closed curve (two circular conv1d layers, the second with stride 2, each followed by
  GELU), whose output replaces g as the first layer's boundary input.
* Mosaic Flow predictor (Section 2.4, Figure 3; Section 4.1): overlapping unit
  subdomains on a lattice of spacing 1/2 (Section 4.2), atomic (non-overlapping)
  subdomains of one colour predicted as one batch, colours applied one after another
  (multiplicative Schwarz, Section 2.3 Eq. 4). The additive variant reads the old
  grid for all subdomains and averages predictions over overlaps (the averaging of
  Algorithm 2's final assembly).
* Convergence test delta = ||g_i - g_{i-1}|| / ||g_{i-1}|| (Algorithm 2), taken over
  every grid point, and the 5-point Laplace residual.
* Exact-solver mode: the SDNet is replaced by the exact 5-point finite-difference
  solve on the 33x33 subdomain, which turns the sweep into the classical alternating
  Schwarz method (Section 2.3) and must converge to the global FD solution.

Conventions (readings where the paper is silent):
* grid arrays are indexed u[iy, ix], x = ix/32, y = iy/32;
* subdomain (a, b) has its lower-left corner at grid (16a, 16b), spans 33x33 points,
  a in [0, 2Lx-2], b in [0, 2Ly-2]; colour c = (a mod 2) + 2 (b mod 2);
* the 128 boundary values are read counter-clockwise from the local corner (0,0):
  bottom i=0..31, right j=0..31, top i=32..1, left j=32..1 (each corner once);
* interior point p = py*31 + px (px, py in 0..30) at local coordinate
  ((px+1)/32, (py+1)/32) in the unit square of the subdomain.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

PTS = 32           # intervals per unit length
SUB = PTS + 1      # points per subdomain side
NI = PTS - 1       # interior points per subdomain side (31)
N_INT = NI * NI    # 961
HALF = PTS // 2    # lattice spacing of subdomain origins, in grid points
N_BDRY = 4 * PTS   # 128


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------

def grid_shape(lx: int, ly: int):
    return PTS * ly + 1, PTS * lx + 1  # (ny, nx)


def n_subdomains(lx: int, ly: int):
    return 2 * lx - 1, 2 * ly - 1


def colour(a: int, b: int) -> int:
    return (a % 2) + 2 * (b % 2)


def subdomains_of_colour(lx: int, ly: int, c: int):
    """Subdomains (a, b) of colour c in lexicographic (b, a) order."""
    nsx, nsy = n_subdomains(lx, ly)
    return [(a, b) for b in range(c // 2, nsy, 2) for a in range(c % 2, nsx, 2)]


def perimeter_local():
    """Local (i, j) of the 128 boundary points of a 33x33 subdomain, CCW from (0,0)."""
    pts = [(i, 0) for i in range(0, PTS)]
    pts += [(PTS, j) for j in range(0, PTS)]
    pts += [(i, PTS) for i in range(PTS, 0, -1)]
    pts += [(0, j) for j in range(PTS, 0, -1)]
    return pts


def interior_coords():
    """(961, 2) local coordinates of the interior points, p = py*31 + px."""
    px, py = np.meshgrid(np.arange(NI), np.arange(NI), indexing="xy")
    return np.stack([(px.ravel() + 1) / PTS, (py.ravel() + 1) / PTS], axis=1)


def centre_cross():
    """Interior indices p = py*31 + px of the centre lines px = 15 or py = 15 (61 points):
    the only lattice lines (x, y in multiples of 1/2) strictly inside a unit subdomain,
    i.e. the only interior points that are other subdomains' boundaries (Figure 3 caption,
    Algorithm 2). Order: the centre row px = 0..30, then the centre column py = 0..30
    without its middle point."""
    c = HALF - 1  # 15
    row = [c * NI + px for px in range(NI)]
    col = [py * NI + c for py in range(NI) if py != c]
    return np.array(row + col)


# ---------------------------------------------------------------------------
# Grid set-up (Eq. 2): boundary from Dirichlet data, interior zero.
# ---------------------------------------------------------------------------

def global_boundary_points(lx: int, ly: int):
    ny, nx = grid_shape(lx, ly)
    pts = [(ix, 0) for ix in range(0, nx - 1)]
    pts += [(nx - 1, iy) for iy in range(0, ny - 1)]
    pts += [(ix, ny - 1) for ix in range(nx - 1, 0, -1)]
    pts += [(0, iy) for iy in range(ny - 1, 0, -1)]
    return pts


def make_grid(lx: int, ly: int, bc_ccw) -> np.ndarray:
    ny, nx = grid_shape(lx, ly)
    u = np.zeros((ny, nx))
    pts = global_boundary_points(lx, ly)
    bc = np.asarray(bc_ccw, dtype=np.float64)
    assert bc.shape == (len(pts),)
    for (ix, iy), v in zip(pts, bc):
        u[iy, ix] = v
    return u


# ---------------------------------------------------------------------------
# Gather / scatter (the in-device form of Algorithm 2's boundary exchange).
# ---------------------------------------------------------------------------

_PERIM = perimeter_local()


def gather(u: np.ndarray, a: int, b: int) -> np.ndarray:
    ox, oy = HALF * a, HALF * b
    return np.array([u[oy + j, ox + i] for (i, j) in _PERIM])


def write_interior(u: np.ndarray, a: int, b: int, v: np.ndarray):
    ox, oy = HALF * a, HALF * b
    u[oy + 1:oy + PTS, ox + 1:ox + PTS] = np.asarray(v).reshape(NI, NI)


# ---------------------------------------------------------------------------
# SDNet (Section 3.2).
# ---------------------------------------------------------------------------

def gelu(x):
    """GELU (Hendrycks and Gimpel), the paper's activation (Section 3.1):
    x Phi(x) = x (1 + erf(x / sqrt 2)) / 2, with scipy's erf."""
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def conv1d_circular(h: np.ndarray, W: np.ndarray, b: np.ndarray, stride: int) -> np.ndarray:
    """Cross-correlation of the closed sequence h (C_in x n) with W (C_out x C_in x K),
    K odd, centred, wrapping around: out[c, i] = b[c] + sum_{c', t} W[c, c', t]
    h[c', (stride i + t - K//2) mod n], for i = 0 .. n/stride - 1."""
    c_in, n = h.shape
    c_out, _, k = W.shape
    m = n // stride
    out = np.tile(b[:, None], (1, m)).astype(np.float64)
    base = stride * np.arange(m)
    for t in range(k):
        idx = (base + t - k // 2) % n
        out += W[:, :, t] @ h[:, idx]
    return out


def embed_boundary(P: dict, g: np.ndarray) -> np.ndarray:
    """Boundary embedding of the variant: the 128 CCW values as a closed curve,
    act(conv1d 1 -> C, stride 1), then act(conv1d C -> C, stride 2), flattened
    channel-major (C x 64 values), act the network's activation (GELU in the paper).
    Without an embedding, g itself."""
    if not P.get("embed"):
        return g
    h1 = activation(P, conv1d_circular(g[None, :], P["cw1"], P["cb1"], 1))
    h2 = activation(P, conv1d_circular(h1, P["cw2"], P["cb2"], 2))
    return h2.reshape(-1)


def unpack_sdnet(w, width: int, depth: int, activation: str = "tanh", embed_channels: int = 0,
                 embed_kernel: int = 0) -> dict:
    """Packed FP32 vector -> FP64 parameters.

    Layout: [conv1 W[C][1][K], b[C], conv2 W[C][C][K], b[C] when embed_channels = C > 0],
    W0[H][n_in + 2] (boundary block W1 = the first n_in columns, n_in = 128 or C x 64,
    coordinate block W2 = the last two, as in Eq. 7), b0[H], then depth-1 hidden layers
    W[H][H], b[H], then w_out[H], b_out.
    """
    w = np.asarray(w, dtype=np.float64)
    h = width
    o = 0

    def take(n):
        nonlocal o
        out = w[o:o + n]
        o += n
        return out

    P = {"act": activation, "embed": embed_channels > 0}
    n_in = N_BDRY
    if embed_channels:
        c, k = embed_channels, embed_kernel
        P["cw1"] = take(c * k).reshape(c, 1, k)
        P["cb1"] = take(c)
        P["cw2"] = take(c * c * k).reshape(c, c, k)
        P["cb2"] = take(c)
        n_in = c * (N_BDRY // 2)
    W = take(h * (n_in + 2)).reshape(h, n_in + 2)
    b0 = take(h)
    hidden = []
    for _ in range(depth - 1):
        Wl = take(h * h).reshape(h, h)
        bl = take(h)
        hidden.append((Wl, bl))
    wout = take(h)
    bout = take(1)[0]
    assert o == w.size, (o, w.size)
    P.update({"W": W, "W1": W[:, :n_in], "W2": W[:, n_in:], "b0": b0,
              "hidden": hidden, "wout": wout, "bout": bout})
    return P


def activation(P: dict, x: np.ndarray) -> np.ndarray:
    return gelu(x) if P.get("act") == "gelu" else np.tanh(x)


def first_layer_concat(P: dict, g: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Eq. 5-6: I = [G X] with g (or its embedding) replicated per point; pre-activation
    I W^T + b0."""
    q = X.shape[0]
    z = embed_boundary(P, g)
    I = np.concatenate([np.tile(z[None, :], (q, 1)), X], axis=1)
    return I @ P["W"].T + P["b0"]


def first_layer_split(P: dict, g: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Eq. 7-8: g W1^T (g or its embedding) broadcast-summed with X W2^T (plus b0)."""
    return (embed_boundary(P, g) @ P["W1"].T + P["b0"])[None, :] + X @ P["W2"].T


def mlp_tail(P: dict, pre1: np.ndarray) -> np.ndarray:
    """Activation of the first layer, the hidden layers, then the linear output."""
    h = activation(P, pre1)
    for Wl, bl in P["hidden"]:
        h = activation(P, h @ Wl.T + bl)
    return h @ P["wout"] + P["bout"]


def sdnet(P: dict, g: np.ndarray, X: np.ndarray, form: str = "split") -> np.ndarray:
    """N(x, g; theta) for the q points X (q x 2) of one subdomain with boundary g."""
    pre = first_layer_split(P, g, X) if form == "split" else first_layer_concat(P, g, X)
    return mlp_tail(P, pre)


def sdnet_batched(P: dict, G: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Section 4.1: the atomic subdomains of one colour as one batch, input-split.

    G: (n, 128) boundaries, X: (q, 2) points. Returns (n, q)."""
    n, q = G.shape[0], X.shape[0]
    Z = np.stack([embed_boundary(P, g) for g in G]) if P.get("embed") else G
    B = Z @ P["W1"].T + P["b0"]            # per-subdomain boundary term (n, H)
    C = X @ P["W2"].T                      # per-point coordinate term  (q, H)
    pre = (B[:, None, :] + C[None, :, :]).reshape(n * q, -1)
    return mlp_tail(P, pre).reshape(n, q)


# ---------------------------------------------------------------------------
# Exact finite-difference subdomain solver (classical Schwarz, Section 2.3).
# ---------------------------------------------------------------------------

def harmonic_extension() -> np.ndarray:
    """H_sub (961 x 128): interior values of the 5-point discrete harmonic function on
    a 33x33 patch with the given boundary values, H_sub = A^{-1} M.

    A: 4 on the diagonal, -1 for each interior neighbour; M: +1 where an interior
    point's neighbour is boundary point k (CCW index)."""
    idx = {pt: k for k, pt in enumerate(_PERIM)}
    A = np.zeros((N_INT, N_INT))
    M = np.zeros((N_INT, N_BDRY))
    for py in range(NI):
        for px in range(NI):
            r = py * NI + px
            A[r, r] = 4.0
            i, j = px + 1, py + 1
            for (di, dj) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ni, nj = i + di, j + dj
                if 1 <= ni <= NI and 1 <= nj <= NI:
                    A[r, (nj - 1) * NI + (ni - 1)] = -1.0
                else:
                    M[r, idx[(ni, nj)]] += 1.0
    return np.linalg.solve(A, M)


# ---------------------------------------------------------------------------
# Sweeps.
# ---------------------------------------------------------------------------

class Solver:
    """Subdomain solver: SDNet (FP64) or the exact FD harmonic extension."""

    def __init__(self, params: dict | None = None, exact: bool = False):
        self.P = params
        self.exact = exact
        self.X = interior_coords()
        self.Hsub = harmonic_extension() if exact else None

    def solve_batch(self, G: np.ndarray, points=None) -> np.ndarray:
        """Predictions at the interior points `points` (indices p; default all 961)."""
        if points is None:
            points = np.arange(N_INT)
        if self.exact:
            return G @ self.Hsub[points].T
        return sdnet_batched(self.P, G, self.X[points])

    def solve_one(self, g: np.ndarray) -> np.ndarray:
        if self.exact:
            return self.Hsub @ g
        return sdnet(self.P, g, self.X, "split")


def write_points(u: np.ndarray, a: int, b: int, points, v: np.ndarray):
    ox, oy = HALF * a, HALF * b
    for p, val in zip(points, v):
        u[oy + 1 + p // NI, ox + 1 + p % NI] = val


def sweep_multiplicative(u: np.ndarray, lx: int, ly: int, solver: Solver,
                         colours=(0, 1, 2, 3), query: str = "full") -> np.ndarray:
    """One sweep, colours in order; each colour gathers from the grid as left by the
    previous colour, predicts its atomic subdomains as one batch and writes them.
    query="centre" (or "center") predicts only each subdomain's centre cross (the
    interface points, Algorithm 2's per-iteration work); query="full" predicts all
    interior points."""
    if query not in ("full", "centre", "center"):
        raise ValueError(f"unknown query {query!r}")
    u = u.copy()
    pts = centre_cross() if query in ("centre", "center") else None
    for c in colours:
        subs = subdomains_of_colour(lx, ly, c)
        if not subs:
            continue
        G = np.stack([gather(u, a, b) for (a, b) in subs])
        V = solver.solve_batch(G, pts)
        for (a, b), v in zip(subs, V):
            if pts is None:
                write_interior(u, a, b, v)
            else:
                write_points(u, a, b, pts, v)
    return u


def sweep_sequential(u: np.ndarray, lx: int, ly: int, solver: Solver) -> np.ndarray:
    """The baseline (unbatched) predictor: one subdomain at a time, colour-major order,
    each prediction written before the next subdomain gathers."""
    u = u.copy()
    for c in range(4):
        for (a, b) in subdomains_of_colour(lx, ly, c):
            write_interior(u, a, b, solver.solve_one(gather(u, a, b)))
    return u


def cover_count(lx: int, ly: int) -> np.ndarray:
    """Number of subdomains whose interior holds each grid point (brute force)."""
    ny, nx = grid_shape(lx, ly)
    cnt = np.zeros((ny, nx))
    nsx, nsy = n_subdomains(lx, ly)
    for b in range(nsy):
        for a in range(nsx):
            ox, oy = HALF * a, HALF * b
            cnt[oy + 1:oy + PTS, ox + 1:ox + PTS] += 1.0
    return cnt


def sweep_additive(u: np.ndarray, lx: int, ly: int, solver: Solver) -> np.ndarray:
    """Every subdomain reads the same old grid; each interior point becomes the
    average of the predictions of the subdomains that hold it (weights 1/cover)."""
    cnt = cover_count(lx, ly)
    acc = np.zeros_like(u)
    for c in range(4):
        subs = subdomains_of_colour(lx, ly, c)
        if not subs:
            continue
        G = np.stack([gather(u, a, b) for (a, b) in subs])
        V = solver.solve_batch(G)
        for (a, b), v in zip(subs, V):
            ox, oy = HALF * a, HALF * b
            acc[oy + 1:oy + PTS, ox + 1:ox + PTS] += v.reshape(NI, NI)
    out = u.copy()
    inner = cnt > 0
    out[inner] = acc[inner] / cnt[inner]
    return out


# ---------------------------------------------------------------------------
# Convergence (Algorithm 2) and residual.
# ---------------------------------------------------------------------------

def delta(u_new: np.ndarray, u_old: np.ndarray) -> float:
    """||u_new - u_old||_2 / ||u_old||_2 over every grid point; 0/0 -> 0, x/0 -> inf."""
    num = float(np.sqrt(np.sum((u_new - u_old) ** 2)))
    den = float(np.sqrt(np.sum(u_old ** 2)))
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return num / den


def residual(u: np.ndarray):
    """5-point residual r = u_E + u_W + u_N + u_S - 4u on interior points (grid units,
    no 1/h^2). Returns (max |r|, rms r)."""
    r = u[1:-1, 2:] + u[1:-1, :-2] + u[2:, 1:-1] + u[:-2, 1:-1] - 4.0 * u[1:-1, 1:-1]
    return float(np.max(np.abs(r))), float(np.sqrt(np.mean(r ** 2)))


def lattice_mask(lx: int, ly: int) -> np.ndarray:
    """Grid points on the lattice lines x or y in multiples of 1/2 (subdomain boundaries)."""
    ny, nx = grid_shape(lx, ly)
    iy, ix = np.mgrid[0:ny, 0:nx]
    return (ix % HALF == 0) | (iy % HALF == 0)


def run(u0: np.ndarray, lx: int, ly: int, solver: Solver, n_sweeps: int,
        eps: float = 0.0, schedule: str = "M", query: str = "full"):
    """Algorithm 2's loop on one device: sweep, then delta; stop when delta < eps."""
    u = u0.copy()
    hist = []
    for k in range(n_sweeps):
        if schedule == "M":
            u_new = sweep_multiplicative(u, lx, ly, solver, query=query)
        else:
            u_new = sweep_additive(u, lx, ly, solver)
        d = delta(u_new, u)
        u = u_new
        hist.append(d)
        if eps > 0 and d < eps:
            break
    return u, hist


# ---------------------------------------------------------------------------
# Global finite-difference solve (ground truth for the exact-solver pins).
# ---------------------------------------------------------------------------

def global_fd_solve(u_bc: np.ndarray) -> np.ndarray:
    """Solve the 5-point discrete Laplace equation on the whole grid with the boundary
    rows of u_bc as Dirichlet data (sparse direct solve)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    ny, nx = u_bc.shape
    mx, my = nx - 2, ny - 2
    n = mx * my
    rows, cols, vals = [], [], []
    rhs = np.zeros(n)
    for j in range(my):
        for i in range(mx):
            r = j * mx + i
            rows.append(r); cols.append(r); vals.append(4.0)
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ni, nj = i + di, j + dj
                if 0 <= ni < mx and 0 <= nj < my:
                    rows.append(r); cols.append(nj * mx + ni); vals.append(-1.0)
                else:
                    rhs[r] += u_bc[nj + 1, ni + 1]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    x = spla.spsolve(A.tocsc(), rhs)
    u = u_bc.copy()
    u[1:-1, 1:-1] = x.reshape(my, mx)
    return u
