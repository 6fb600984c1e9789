"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the benchmark.

This module draws random numbers and evaluates the closed-form boundary data of the
synthetic workloads. It holds none of the Mosaic Flow arithmetic (no gather, no SDNet,
no scatter, no convergence test), so both the CUDA path and the CPU oracle can take
their inputs from it without sharing any of the method.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based generator:
draw k of a stream with initial state s is mix(s + k * GAMMA). Uniform doubles take the
top 53 bits; normals use the Box-Muller transform (cosine branch only).

Workload presets mirror the five synthetic configurations of the sweep engine
(tiny / mid / large single problems, a batch of problems, and the training batch). The
paper (Section 5.1) builds its boundary data from Gaussian-process samples solved by
pyAMG; that data is not available, so closed-form harmonic boundary data with the
paper's domain shapes stand in for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream tags: one independent SplitMix64 stream per purpose and seed.
TAG_WEIGHTS = 1
TAG_BC = 2
TAG_COLLOCATION = 3
TAG_SIDES = 4
TAG_TEST = 5
TAG_FAMILY = 6

POINTS_PER_UNIT = 32  # grid intervals per unit length (33 points per unit subdomain side)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(state: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset+1 .. offset+n of the SplitMix64 stream that starts at `state`."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state & 0xFFFFFFFFFFFFFFFF) + k * GAMMA
    return _mix(z)


def stream_state(seed: int, tag: int) -> int:
    return (int(seed) + (int(tag) << 32)) & 0xFFFFFFFFFFFFFFFF


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int, tag: int):
        self.state = stream_state(seed, tag)
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        out = splitmix64(self.state, n, self.pos)
        self.pos += n
        return out

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) from the top 53 bits of each draw."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals, Box-Muller, two uniforms per normal."""
        u = self.uniform(2 * n).reshape(n, 2)
        r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
        return r * np.cos(2.0 * math.pi * u[:, 1])

    def integers(self, n: int, k: int) -> np.ndarray:
        """n integers uniform in [0, k) (floor of k * uniform)."""
        return np.minimum((self.uniform(n) * k).astype(np.int64), k - 1)


# ---------------------------------------------------------------------------
# SDNet weights: packed FP32 layout shared by the library and the tests.
#   W0[H][130] (columns 0..127 boundary block, 128..129 coordinate block), b0[H],
#   then for each of the depth-1 hidden-to-hidden layers: W[H][H], b[H],
#   then w_out[H], b_out[1].
# ---------------------------------------------------------------------------
N_BDRY = 128
N_COORD = 2


@dataclass
class SDNetShape:
    width: int = 128  # H
    depth: int = 6    # number of activation layers (first layer + depth-1 hidden layers)
    activation: str = "tanh"  # "tanh" or "gelu"
    embed_channels: int = 0   # C > 0: two circular conv1d layers embed the boundary first
    embed_kernel: int = 0     # odd kernel size K of both conv1d layers

    @property
    def n_in(self) -> int:
        """Width of the boundary input of the first layer: 128 raw values or C x 64."""
        return self.embed_channels * (N_BDRY // 2) if self.embed_channels else N_BDRY

    @property
    def n_params(self) -> int:
        h, c, k = self.width, self.embed_channels, self.embed_kernel
        conv = (c * k + c) + (c * c * k + c) if c else 0
        return conv + h * (self.n_in + N_COORD) + h + (self.depth - 1) * (h * h + h) + h + 1


def xavier_sdnet(shape: SDNetShape, seed: int, bias_scale: float = 0.0) -> np.ndarray:
    """Xavier-uniform weights U(+-sqrt(6/(fan_in+fan_out))), drawn in packed order.

    Biases are zero unless bias_scale > 0 (then U(+-bias_scale), used by tests to
    exercise the bias paths). Values are rounded to FP32; the FP32 array is canonical.
    """
    h, d = shape.width, shape.depth
    st = Stream(seed, TAG_WEIGHTS)
    parts = []

    def mat(rows, cols):
        bound = math.sqrt(6.0 / (rows + cols))
        return (2.0 * st.uniform(rows * cols) - 1.0) * bound

    def conv(c_out, c_in, k):
        bound = math.sqrt(6.0 / (c_in * k + c_out * k))
        return (2.0 * st.uniform(c_out * c_in * k) - 1.0) * bound

    def bias(n):
        if bias_scale > 0:
            return (2.0 * st.uniform(n) - 1.0) * bias_scale
        return np.zeros(n)

    c, k = shape.embed_channels, shape.embed_kernel
    if c:
        # conv1d weights [C_out][C_in][K]: fan_in C_in K, fan_out C_out K
        parts.append(conv(c, 1, k))
        parts.append(bias(c))
        parts.append(conv(c, c, k))
        parts.append(bias(c))
    parts.append(mat(h, shape.n_in + N_COORD))
    parts.append(bias(h))
    for _ in range(d - 1):
        parts.append(mat(h, h))
        parts.append(bias(h))
    parts.append(mat(1, h))
    parts.append(bias(1))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == shape.n_params
    return w


# ---------------------------------------------------------------------------
# Boundary data (Dirichlet values on the global boundary), counter-clockwise from
# the corner (0, 0): bottom edge ix = 0..nx-2 (iy = 0), right edge iy = 0..ny-2
# (ix = nx-1), top edge ix = nx-1..1 (iy = ny-1), left edge iy = ny-1..1 (ix = 0).
# ---------------------------------------------------------------------------

def boundary_points(nx: int, ny: int) -> np.ndarray:
    """(ix, iy) of the global boundary points in counter-clockwise order."""
    pts = []
    pts += [(ix, 0) for ix in range(0, nx - 1)]
    pts += [(nx - 1, iy) for iy in range(0, ny - 1)]
    pts += [(ix, ny - 1) for ix in range(nx - 1, 0, -1)]
    pts += [(0, iy) for iy in range(ny - 1, 0, -1)]
    return np.array(pts, dtype=np.int64)


def mode_field(coeffs, lx: float, ly: float):
    """u(x,y) = sum_k a_k sin(k pi x/lx) sinh(k pi y/lx) / sinh(k pi ly/lx), harmonic.

    The sinh ratio is evaluated as exp(kpi(y-ly)/lx)(1-exp(-2kpi y/lx))/(1-exp(-2kpi ly/lx))
    so that large k*ly/lx does not overflow.
    """
    coeffs = np.asarray(coeffs, dtype=np.float64)

    def f(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros(np.broadcast(x, y).shape)
        for k, a in enumerate(coeffs, start=1):
            kp = k * math.pi / lx
            ratio = np.exp(kp * (y - ly)) * (-np.expm1(-2.0 * kp * y)) / (-math.expm1(-2.0 * kp * ly))
            out = out + a * np.sin(kp * x) * ratio
        return out

    return f


def bc_values(lx: int, ly: int, field_fn) -> np.ndarray:
    """FP64 boundary values of field_fn on the (32lx+1) x (32ly+1) grid, CCW order."""
    nx, ny = POINTS_PER_UNIT * lx + 1, POINTS_PER_UNIT * ly + 1
    pts = boundary_points(nx, ny)
    h = 1.0 / POINTS_PER_UNIT
    return np.asarray(field_fn(pts[:, 0] * h, pts[:, 1] * h), dtype=np.float64)


def mode_coeffs(seed: int, n_modes: int = 8) -> np.ndarray:
    return Stream(seed, TAG_BC).normal(n_modes)


# ---------------------------------------------------------------------------
# Workload presets.
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    lx: int
    ly: int
    bc: np.ndarray  # FP64 CCW boundary values
    name: str = ""


@dataclass
class Workload:
    name: str
    problems: list
    shape: SDNetShape
    weight_seed: int
    sweeps: int
    eps: float
    precision: str  # "fp32" or "bf16"
    extra: dict = field(default_factory=dict)

    def weights(self, bias_scale: float = 0.0) -> np.ndarray:
        return xavier_sdnet(self.shape, self.weight_seed, bias_scale)


def tiny() -> Workload:
    """Global [0,2]^2, 3x3 unit subdomains at half overlap, grid 65x65, SDNet 4x64,
    BC sin(pi x) sinh(pi y) / sinh(2 pi), 20 sweeps, FP32."""
    f = lambda x, y: np.sin(math.pi * x) * np.sinh(math.pi * y) / math.sinh(2 * math.pi)
    p = Problem(2, 2, bc_values(2, 2, f), "tiny")
    return Workload("tiny_L2_fp32", [p], SDNetShape(64, 4), 0, 20, 0.0, "fp32")


def mid() -> Workload:
    """Global [0,16]^2, 31x31 subdomains, grid 513x513, SDNet 6x128 seed 1,
    8-mode harmonic BC a_k ~ N(0,1) seed 1, up to 200 sweeps, stop at 1e-6."""
    p = Problem(16, 16, bc_values(16, 16, mode_field(mode_coeffs(1), 16, 16)), "mid")
    return Workload("mid_L16_fp32", [p], SDNetShape(128, 6), 1, 200, 1e-6, "fp32")


def large() -> Workload:
    """Global [0,64]^2 (4096x the unit subdomain area), 127x127 = 16129 subdomains,
    grid 2049x2049, SDNet 6x128 seed 2, 8-mode harmonic BC seed 2, BF16 with FP32
    refinement."""
    p = Problem(64, 64, bc_values(64, 64, mode_field(mode_coeffs(2), 64, 64)), "large")
    return Workload("large_L64_bf16", [p], SDNetShape(128, 6), 2, 200, 1e-6, "bf16")


def batched(n_problems: int = 256) -> Workload:
    """n independent square problems, sides uniform in {2,4,8,16,32} (seed 4),
    problem q with 8-mode BC seed 1000+q; shared SDNet 6x128 (seed 4)."""
    sides = np.array([2, 4, 8, 16, 32])[Stream(4, TAG_SIDES).integers(n_problems, 5)]
    probs = []
    for q, s in enumerate(sides):
        s = int(s)
        probs.append(Problem(s, s, bc_values(s, s, mode_field(mode_coeffs(1000 + q), s, s)), f"q{q}"))
    return Workload("batched_256", probs, SDNetShape(128, 6), 4, 200, 1e-6, "bf16")


@dataclass
class TrainBatch:
    G: np.ndarray    # (F, 128) boundary values of each function (CCW on the unit square)
    Xc: np.ndarray   # (F, Nc, 2) collocation points, uniform in the open unit square
    Xb: np.ndarray   # (F, Nb, 2) data points: the 128 boundary points
    Yb: np.ndarray   # (F, Nb) data targets: the boundary values


def unit_square_boundary_points() -> np.ndarray:
    """(128, 2) boundary points of the unit square at spacing 1/32, CCW from (0, 0)."""
    h = 1.0 / POINTS_PER_UNIT
    n = POINTS_PER_UNIT
    pts = [(i * h, 0.0) for i in range(n)] + [(1.0, j * h) for j in range(n)]
    pts += [(1.0 - i * h, 1.0) for i in range(n)] + [(0.0, 1.0 - j * h) for j in range(n)]
    return np.array(pts)


def training_batch(n_functions: int = 1024, n_colloc: int = 1024, seed: int = 3) -> TrainBatch:
    """Physics-informed SDNet training batch: n_functions random 8-mode harmonic functions
    on the unit square (a_k ~ N(0,1)), n_colloc uniform collocation points each for the
    PDE loss, the 128 boundary points with their values for the data loss."""
    coef = Stream(seed, TAG_BC).normal(8 * n_functions).reshape(n_functions, 8)
    xb = unit_square_boundary_points()
    G = np.stack([mode_field(coef[f], 1.0, 1.0)(xb[:, 0], xb[:, 1]) for f in range(n_functions)])
    Xc = Stream(seed, TAG_COLLOCATION).uniform(n_functions * n_colloc * 2).reshape(n_functions, n_colloc, 2)
    Xb = np.broadcast_to(xb, (n_functions, 128, 2)).copy()
    return TrainBatch(G=G, Xc=Xc, Xb=Xb, Yb=G.copy())


@dataclass
class HarmonicFamily:
    """Random harmonic functions on the unit square with data on all four sides:
    u = e0 + e1 x + e2 y + e3 x y + sum over sides and k = 1..K of a_k times the
    separable solution that is sin(k pi t) on that side and 0 on the other three,
    e.g. sin(k pi x) sinh(k pi y) / sinh(k pi) for the top side."""
    a: np.ndarray  # (F, 4, K): sides top, bottom, right, left
    e: np.ndarray  # (F, 4): bilinear part

    def __call__(self, x, y, scale: float = 1.0) -> np.ndarray:
        """Values (F, P) at the points (x, y) (P each) of u(x / scale, y / scale)."""
        x = np.asarray(x, dtype=np.float64).ravel() / scale
        y = np.asarray(y, dtype=np.float64).ravel() / scale
        K = self.a.shape[2]
        kp = math.pi * np.arange(1, K + 1)[:, None]
        sh = np.sinh(kp)
        sx, sy = np.sin(kp * x), np.sin(kp * y)
        top, bottom = sx * np.sinh(kp * y) / sh, sx * np.sinh(kp * (1.0 - y)) / sh
        right, left = sy * np.sinh(kp * x) / sh, sy * np.sinh(kp * (1.0 - x)) / sh
        out = self.e[:, :1] + self.e[:, 1:2] * x + self.e[:, 2:3] * y + self.e[:, 3:4] * (x * y)
        for side, basis in enumerate((top, bottom, right, left)):
            out = out + self.a[:, side, :] @ basis
        return out


def harmonic_family(n_functions: int, seed: int, n_modes: int = 6) -> HarmonicFamily:
    """a ~ N(0, 1) / k (smoother functions weigh more), e ~ N(0, 1/4)."""
    st = Stream(seed, TAG_FAMILY)
    a = st.normal(n_functions * 4 * n_modes).reshape(n_functions, 4, n_modes) / np.arange(1, n_modes + 1)
    e = 0.5 * st.normal(n_functions * 4).reshape(n_functions, 4)
    return HarmonicFamily(a=a, e=e)


WORKLOADS = {"tiny": tiny, "mid": mid, "large": large, "batched": batched}
