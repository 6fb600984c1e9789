"""Pins that tie the FP64 oracle to what the paper and the mathematics fix.

* Alternating Schwarz with exact subdomain solves converges to the global solution
  (Section 2.3, Eq. 4): brute force against a sparse direct solve of the whole grid.
* Discrete-harmonic polynomials are fixed points of the exact-solver sweep.
* The SDNet forward matches a hand-computed toy (tanh(ln3/2) = 1/2, tanh(ln2/2) = 1/3).
* Input-concat (Eq. 6) equals input-split (Eq. 8).
* Batched atomic subdomains equal the sequential predictor (Section 4.1).
* Residual and delta match closed forms; the gather follows the stated CCW order.

The mutation tests at the end plant plausible mistakes in the oracle (on the CPU) and
check that at least one pin catches each of them.
"""
import math

import numpy as np
import pytest

from oracle import mosaic_flow as mf
from paper_2308_14258_gb300 import inputs as I

H = 1.0 / 32


def field_grid(lx, ly, f):
    ny, nx = mf.grid_shape(lx, ly)
    iy, ix = np.mgrid[0:ny, 0:nx]
    return f(ix * H, iy * H)


def boundary_only(u):
    v = np.zeros_like(u)
    v[0, :], v[-1, :], v[:, 0], v[:, -1] = u[0, :], u[-1, :], u[:, 0], u[:, -1]
    return v


# --------------------------------------------------------------------- geometry

def test_gather_ccw_order():
    ny, nx = mf.grid_shape(2, 2)
    iy, ix = np.mgrid[0:ny, 0:nx]
    u = (ix + 1000 * iy).astype(float)
    a, b = 1, 2
    g = mf.gather(u, a, b)
    ox, oy = 16 * a, 16 * b
    exp = ([ox + i + 1000 * oy for i in range(32)]
           + [ox + 32 + 1000 * (oy + j) for j in range(32)]
           + [ox + 32 - i + 1000 * (oy + 32) for i in range(32)]
           + [ox + 1000 * (oy + 32 - j) for j in range(32)])
    assert g.tolist() == exp


def test_colours_partition_and_disjoint_interiors():
    for lx, ly in ((2, 2), (2, 3), (4, 4)):
        nsx, nsy = mf.n_subdomains(lx, ly)
        seen = []
        for c in range(4):
            cnt = np.zeros(mf.grid_shape(lx, ly))
            for (a, b) in mf.subdomains_of_colour(lx, ly, c):
                seen.append((a, b))
                cnt[16 * b + 1:16 * b + 32, 16 * a + 1:16 * a + 32] += 1
            assert cnt.max() <= 1  # atomic subdomains of a colour do not overlap
        assert sorted(seen) == sorted((a, b) for a in range(nsx) for b in range(nsy))


def test_cover_counts():
    cnt = mf.cover_count(3, 2)
    inner = cnt[1:-1, 1:-1]
    assert set(np.unique(inner)) == {1.0, 2.0, 4.0}
    assert cnt[0, :].max() == 0 and cnt[:, 0].max() == 0
    assert cnt[16, 16] == 1 and cnt[8, 8] == 1 and cnt[24, 24] == 4 and cnt[16, 24] == 2


# ------------------------------------------------------------ exact solver pins

@pytest.fixture(scope="module")
def exact():
    return mf.Solver(exact=True)


def test_harmonic_extension_properties(exact):
    Hs = exact.Hsub
    assert np.allclose(Hs.sum(axis=1), 1.0, atol=1e-13)   # reproduces constants
    assert Hs.min() >= -1e-15                              # discrete maximum principle
    # a linear field is discrete-harmonic: interior reproduced exactly
    f = lambda x, y: 0.3 + 1.7 * x - 2.2 * y
    patch = np.array([[f(i * H, j * H) for i in range(33)] for j in range(33)])
    g = np.array([patch[j, i] for (i, j) in mf.perimeter_local()])
    assert np.allclose(Hs @ g, patch[1:32, 1:32].ravel(), atol=1e-13)


@pytest.mark.parametrize("f", [lambda x, y: x * x - y * y,
                               lambda x, y: x * y,
                               lambda x, y: x ** 3 - 3 * x * y * y])
@pytest.mark.parametrize("lx,ly", [(2, 2), (2, 3)])
def test_discrete_harmonic_fixed_point(exact, f, lx, ly):
    u = field_grid(lx, ly, f)
    r_max, _ = mf.residual(u)
    assert r_max < 1e-12
    for sweep in (mf.sweep_multiplicative, mf.sweep_additive):
        v = sweep(u, lx, ly, exact)
        assert np.abs(v - u).max() < 1e-12


@pytest.mark.parametrize("lx,ly", [(2, 2), (2, 3)])
@pytest.mark.parametrize("schedule", ["M", "A"])
def test_exact_solver_sweep_converges_to_global_fd(exact, lx, ly, schedule):
    p = I.Problem(lx, ly, I.bc_values(lx, ly, I.mode_field(I.mode_coeffs(5), lx, ly)))
    u0 = mf.make_grid(lx, ly, p.bc)
    ufd = mf.global_fd_solve(u0)
    u, hist = mf.run(u0, lx, ly, exact, 400, eps=1e-15, schedule=schedule)
    assert np.abs(u - ufd).max() <= 1e-12 * max(1.0, np.abs(ufd).max())
    assert hist[-1] < 1e-13


def test_global_fd_exact_for_cubic():
    f = lambda x, y: x ** 3 - 3 * x * y * y + 0.5 * x * y
    u = field_grid(2, 3, f)
    assert np.abs(mf.global_fd_solve(boundary_only(u)) - u).max() < 1e-11


def test_fixed_point_close_to_continuum(exact):
    """Second-order FD: the converged field is within O(h^2) of the closed form."""
    w = I.tiny()
    u0 = mf.make_grid(2, 2, w.problems[0].bc)
    u, _ = mf.run(u0, 2, 2, exact, 200, eps=1e-15)
    f = lambda x, y: np.sin(math.pi * x) * np.sinh(math.pi * y) / math.sinh(2 * math.pi)
    err = np.abs(u - field_grid(2, 2, f)).max()
    assert 1e-6 < err < 5.0 * H * H


# ---------------------------------------------------------------- SDNet pins

def toy_params(width=64, depth=4):
    """Hand-built weights whose pre-activations are ln3/2 or ln2/2 (tanh = 1/2, 1/3)."""
    l2, l3 = math.log(2.0), math.log(3.0)
    shape = I.SDNetShape(width, depth)
    P = mf.unpack_sdnet(np.zeros(shape.n_params), width, depth)
    W, b0 = P["W"], P["b0"]
    W[0, 5] = l3 / 4          # g[5] = 2      -> ln3/2 -> 1/2
    W[1, 128] = l2            # x = 1/2       -> ln2/2 -> 1/3
    W[2, 129] = 2 * l3        # y = 1/4       -> ln3/2 -> 1/2
    b0[3] = l2 / 2            # bias only     -> 1/3
    (W1, b1), (W2, _), (W3, _) = P["hidden"]
    W1[0, 1] = 1.5 * l3                     # (1/3)           -> 1/2
    W1[1, 0] = l2 / 2; W1[1, 2] = l2 / 2    # (1/2, 1/2)      -> 1/3
    W1[2, 3] = 1.5 * l2; b1[2] = (l3 - l2) / 2   # 1/3 + bias -> 1/2
    W2[0, 2] = l2                           # (1/2)           -> 1/3
    W2[1, 0] = l3                           # (1/2)           -> 1/2
    W3[5, 0] = 1.5 * l3                     # (1/3)           -> 1/2
    W3[6, 1] = l2                           # (1/2)           -> 1/3
    P["wout"][5], P["wout"][6] = 6.0, 9.0
    P["bout"] = 0.25
    P["W1"], P["W2"] = W[:, :128], W[:, 128:]
    return P


def toy_boundary():
    g = np.linspace(-3.0, 5.0, 128)
    g[5] = 2.0
    return g


def test_mlp_toy_hand_computed():
    P = toy_params()
    X = mf.interior_coords()
    p = 7 * 31 + 15                       # local point x = 1/2, y = 1/4
    assert tuple(X[p]) == (0.5, 0.25)
    out = mf.sdnet(P, toy_boundary(), X[p:p + 1])
    assert abs(out[0] - 6.25) < 1e-14     # 6*(1/2) + 9*(1/3) + 1/4
    # the same weights through the batched form (two identical subdomains)
    G = np.stack([toy_boundary(), toy_boundary()])
    outb = mf.sdnet_batched(P, G, X)
    assert abs(outb[1, p] - 6.25) < 1e-14


def coordinate_only_weights(width, depth, ax, by, c):
    """Packed weights of an SDNet that ignores its boundary input: unit 0 of the first
    layer sees ax x + by y, each hidden layer passes unit 0 on with weight 1, and the
    output is unit 0 plus c, so N(x, y) = tanh^depth(ax x + by y) + c exactly."""
    w = np.zeros(I.SDNetShape(width, depth).n_params)
    w[0 * 130 + 128], w[0 * 130 + 129] = ax, by       # W0[0][x], W0[0][y]
    o = width * 130 + width                            # past W0 and b0
    for _ in range(depth - 1):
        w[o] = 1.0                                     # W_l[0][0]
        o += width * width + width
    w[o] = 1.0                                         # w_out[0]
    w[o + width] = c                                   # b_out
    return w


@pytest.mark.parametrize("lx,ly", [(2, 3), (3, 2)])
def test_coordinate_only_sdnet_sweep_closed_form(lx, ly):
    """One multiplicative sweep (colours 0..3 in turn, Section 4.1) with a network that
    ignores the boundary: every interior grid point ends with N at its local coordinates
    in the last subdomain, in colour order, whose open interior holds it. The expected
    grid comes from the subdomain layout alone (origins 16a, 16b at half overlap, colour
    (a mod 2) + 2 (b mod 2)), not from the oracle's sweep, and pins the coordinate
    convention, the colour order and the scatter."""
    width, depth, ax, by, c = 64, 3, 1.3, -0.7, 0.25
    P = mf.unpack_sdnet(coordinate_only_weights(width, depth, ax, by, c), width, depth)
    ny, nx = mf.grid_shape(lx, ly)
    u0 = np.asarray(I.Stream(31, I.TAG_TEST).normal(ny * nx)).reshape(ny, nx)
    u1 = mf.sweep_multiplicative(u0, lx, ly, mf.Solver(P))

    def N(x, y):
        v = ax * x + by * y
        for _ in range(depth):
            v = math.tanh(v)
        return v + c

    nsx, nsy = 2 * lx - 1, 2 * ly - 1
    for iy in range(1, ny - 1):
        for ix in range(1, nx - 1):
            cover = [(a, b) for a in range(nsx) for b in range(nsy)
                     if 16 * a < ix < 16 * a + 32 and 16 * b < iy < 16 * b + 32]
            a, b = max(cover, key=lambda ab: (ab[0] % 2) + 2 * (ab[1] % 2))
            want = N((ix - 16 * a) / 32.0, (iy - 16 * b) / 32.0)
            assert abs(u1[iy, ix] - want) < 1e-14, (ix, iy)
    assert np.array_equal(boundary_only(u1), boundary_only(u0))


def test_mutation_colour_order_is_caught(monkeypatch):
    orig = mf.subdomains_of_colour
    monkeypatch.setattr(mf, "subdomains_of_colour", lambda lx, ly, c: orig(lx, ly, 3 - c))
    with pytest.raises(AssertionError):
        test_coordinate_only_sdnet_sweep_closed_form(2, 3)


def test_concat_equals_split():
    w = I.xavier_sdnet(I.SDNetShape(128, 6), 9, bias_scale=0.3)
    P = mf.unpack_sdnet(w, 128, 6)
    X = mf.interior_coords()
    g = I.Stream(3, I.TAG_TEST).normal(128)
    a = mf.first_layer_concat(P, g, X)
    b = mf.first_layer_split(P, g, X)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
    ya, yb = mf.sdnet(P, g, X, "concat"), mf.sdnet(P, g, X, "split")
    assert np.abs(ya - yb).max() <= 1e-13 * np.abs(ya).max()


def test_batched_equals_sequential():
    w = I.tiny()
    P = mf.unpack_sdnet(w.weights(bias_scale=0.1), 64, 4)
    sol = mf.Solver(P)
    u0 = mf.make_grid(2, 2, w.problems[0].bc)
    u0[1:-1, 1:-1] = I.Stream(4, I.TAG_TEST).normal(63 * 63).reshape(63, 63) * 0.1
    a = mf.sweep_multiplicative(u0, 2, 2, sol)
    b = mf.sweep_sequential(u0, 2, 2, sol)
    assert np.abs(a - b).max() <= 1e-13


# ------------------------------------------------------- delta and residual pins

def test_residual_closed_forms():
    ny, nx = mf.grid_shape(2, 2)
    iy, ix = np.mgrid[0:ny, 0:nx]
    r_max, r_rms = mf.residual((ix ** 2).astype(float))      # second difference = 2
    assert r_max == 2.0 and r_rms == 2.0
    u = np.zeros((ny, nx)); u[10, 20] = 1.0
    r_max, r_rms = mf.residual(u)
    assert r_max == 4.0
    assert abs(r_rms - math.sqrt((16 + 4) / (63 * 63))) < 1e-15


def test_delta_closed_form():
    a = np.zeros((3, 4)); a[0, 0] = 3.0; a[1, 2] = 4.0       # ||a|| = 5
    b = a.copy(); b[2, 3] = 1.0
    assert mf.delta(b, a) == 0.2
    assert mf.delta(a, a) == 0.0
    assert mf.delta(a, np.zeros_like(a)) == float("inf")


# --------------------------------------------------------------- mutation tests

def _exact_convergence_ok(exact):
    lx, ly = 2, 2
    p = I.bc_values(lx, ly, I.mode_field(I.mode_coeffs(5), lx, ly))
    u0 = mf.make_grid(lx, ly, p)
    ufd = mf.global_fd_solve(u0)
    u, _ = mf.run(u0, lx, ly, exact, 100, eps=1e-15)
    return np.abs(u - ufd).max() <= 1e-12


def test_mutation_scatter_offset_is_caught(exact, monkeypatch):
    def bad_write(u, a, b, v):
        ox, oy = 16 * a, 16 * b
        u[oy + 1:oy + 32, ox + 2:ox + 33] = np.asarray(v).reshape(31, 31)
    monkeypatch.setattr(mf, "write_interior", bad_write)
    assert not _exact_convergence_ok(exact)


def test_mutation_gather_edge_reversed_is_caught(monkeypatch):
    perim = mf.perimeter_local()
    bad = perim[:64] + perim[64:96][::-1] + perim[96:]
    monkeypatch.setattr(mf, "_PERIM", bad)
    ny, nx = mf.grid_shape(2, 2)
    iy, ix = np.mgrid[0:ny, 0:nx]
    g = mf.gather((ix + 1000 * iy).astype(float), 1, 2)
    assert g[64] != 48 + 1000 * 64   # the CCW pin (test_gather_ccw_order) fails


def test_mutation_transposed_hidden_weight_is_caught():
    P = toy_params()
    P["hidden"] = [(Wl.T.copy(), bl) for (Wl, bl) in P["hidden"]]
    X = mf.interior_coords()
    out = mf.sdnet(P, toy_boundary(), X[232:233])
    assert abs(out[0] - 6.25) > 1e-3


def test_mutation_swapped_coordinates_is_caught():
    P = toy_params()
    X = mf.interior_coords()[:, ::-1].copy()
    out = mf.sdnet(P, toy_boundary(), X[232:233])
    assert abs(out[0] - 6.25) > 1e-3


def test_mutation_dropped_bias_is_caught():
    P = toy_params()
    P["hidden"][0] = (P["hidden"][0][0], np.zeros_like(P["hidden"][0][1]))
    out = mf.sdnet(P, toy_boundary(), mf.interior_coords()[232:233])
    assert abs(out[0] - 6.25) > 1e-3


# ------------------------------------------------------- centre-line sweeps

def test_centre_cross_points():
    pts = mf.centre_cross()
    assert len(pts) == 61 and len(set(pts.tolist())) == 61
    X = mf.interior_coords()[pts]
    assert np.all((X[:, 0] == 0.5) | (X[:, 1] == 0.5))
    # exactly the interior points that lie on lattice lines of spacing 1/2
    ny, nx = mf.grid_shape(1, 1)
    lat = mf.lattice_mask(1, 1)[1:-1, 1:-1].ravel()
    assert sorted(np.nonzero(lat)[0].tolist()) == sorted(pts.tolist())


@pytest.mark.parametrize("solver_kind", ["exact", "sdnet"])
def test_centre_lines_reproduce_full_sweep_on_lattice(exact, solver_kind):
    """Gathers read only lattice lines, so predicting just the centre crosses gives the
    same lattice-line values as predicting whole interiors (Algorithm 2's interface-only
    iterations), sweep after sweep."""
    lx, ly = 3, 2
    if solver_kind == "exact":
        sol = exact
    else:
        sol = mf.Solver(mf.unpack_sdnet(I.xavier_sdnet(I.SDNetShape(64, 3), 3, 0.1), 64, 3))
    u0 = mf.make_grid(lx, ly, I.bc_values(lx, ly, I.mode_field(I.mode_coeffs(4), lx, ly)))
    uf, uc = u0.copy(), u0.copy()
    lat = mf.lattice_mask(lx, ly)
    for _ in range(4):
        uf = mf.sweep_multiplicative(uf, lx, ly, sol, query="full")
        uc = mf.sweep_multiplicative(uc, lx, ly, sol, query="center")
        assert np.abs(uf[lat] - uc[lat]).max() <= 1e-13 * max(1.0, np.abs(uf).max())
    # off the lattice the centre-line sweep leaves the initial values untouched
    assert np.array_equal(uc[~lat], u0[~lat])


def test_centre_lines_then_assembly_solve_laplace(exact):
    """Exact-solver centre-line iterations followed by the averaged full assembly (one
    additive sweep) reproduce the global FD solution."""
    lx, ly = 2, 3
    u0 = mf.make_grid(lx, ly, I.bc_values(lx, ly, I.mode_field(I.mode_coeffs(5), lx, ly)))
    u, _ = mf.run(u0, lx, ly, exact, 200, eps=1e-15, query="center")
    u = mf.sweep_additive(u, lx, ly, exact)
    assert np.abs(u - mf.global_fd_solve(u0)).max() <= 1e-11
