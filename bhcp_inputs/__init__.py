"""Seeded synthetic inputs for the backward heat conduction problem (BHCP).

This module produces *data only*: grids, initial temperatures z(., 0), the final
data g = z(., T) that the heat equation carries them to, and the noisy
measurement g_delta with its noise level delta.  It holds none of the
quasi-boundary-value arithmetic (no all-at-once system, no omega-circulant
diagonalisation, no solver); both the CPU oracle and the CUDA library take
what it returns as given inputs.

Problem statement: Section 1, eq. (1.1): z_t - Laplace(z) = 0 in Omega x (0, T),
z = 0 on the boundary, z(., T) = g; a measurement g_delta with
||g - g_delta|| <= delta is given.

Grid (Section 2): t_n = n tau, tau = T/N; M intervals per space dimension,
h = L/M, unknowns on the (M-1)^d interior nodes.  Throughout this package
``nt`` is the number of time levels N_t = N + 1 (Section 2 defines N_t = N + 1),
so tau = T/(nt - 1).  Spatial arrays have numpy shape (n_z, n_y, n_x) -- x is
the fastest (last) axis -- and all-at-once arrays have shape (nt, n_z, n_y, n_x).

Noise models:
  * Section 5: g_delta = g * (1 + eps * U(-1, 1)), delta := ||g_delta - g||.
  * additive Gaussian scaled so that ||g_delta - g|| = rel * ||g||.
Norms are the grid-weighted discrete L2 norm h^{d/2} ||v||_2 (the discrete
L2(Omega) norm of Section 5).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
from typing import Sequence

import numpy as np

__all__ = [
    "Grid", "Problem", "discrete_l2", "interior_coords", "sine_field",
    "forward_discrete", "add_noise_multiplicative", "add_noise_gaussian",
    "make_c1", "make_c2", "make_c3", "make_paper_ex1", "make_paper_ex2",
    "make_problem", "random_general_rhs", "batch_specs_c4", "alpha_training_batch",
]


@dataclass(frozen=True)
class Grid:
    """Uniform space-time grid of Section 2.

    dim: space dimension d (1, 2 or 3).
    M:   intervals per dimension, ordered (x, y, z); interior points n = M - 1.
    L:   side length of the cube (0, L)^d.
    T:   final time.
    nt:  number of time levels N_t = N + 1 (tau = T / (nt - 1)).
    """

    dim: int
    M: tuple
    L: float
    T: float
    nt: int

    def __post_init__(self):
        if self.dim not in (1, 2, 3):
            raise ValueError("dim must be 1, 2 or 3")
        if len(self.M) != self.dim:
            raise ValueError("M needs one entry per dimension")
        if min(self.M) < 2 or self.nt < 2:
            raise ValueError("need M >= 2 and nt >= 2")

    @property
    def n(self) -> tuple:
        """Interior points per dimension (x, y, z order)."""
        return tuple(m - 1 for m in self.M)

    @property
    def h(self) -> tuple:
        return tuple(self.L / m for m in self.M)

    @property
    def tau(self) -> float:
        return self.T / (self.nt - 1)

    @property
    def Nx(self) -> int:
        """Spatial unknowns per time level, N_x = prod(M_d - 1)."""
        return int(np.prod(self.n))

    @property
    def shape(self) -> tuple:
        """numpy shape of one time level: (n_z, n_y, n_x) truncated to dim."""
        return tuple(reversed(self.n))

    @property
    def full_shape(self) -> tuple:
        return (self.nt,) + self.shape

    @property
    def unknowns(self) -> int:
        return self.Nx * self.nt


@dataclass
class Problem:
    """One BHCP instance: grid, initial data, clean and noisy final data."""

    name: str
    grid: Grid
    z0: np.ndarray          # exact initial temperature on the interior nodes
    g: np.ndarray           # clean final data z(., T)
    g_delta: np.ndarray     # noisy measurement
    delta: float            # ||g_delta - g|| in the grid-weighted L2 norm
    seed: int
    meta: dict = field(default_factory=dict)


def discrete_l2(v: np.ndarray, grid: Grid) -> float:
    """Grid-weighted discrete L2(Omega) norm: sqrt(prod h_d) * ||v||_2."""
    w = math.sqrt(float(np.prod(grid.h)))
    return w * float(np.linalg.norm(np.asarray(v).ravel()))


def interior_coords(grid: Grid) -> list:
    """Interior node coordinates per axis, in numpy axis order (z, y, x)."""
    axes = [np.arange(1, m) * (grid.L / m) for m in grid.M]   # x, y, z
    return list(reversed(axes))


def sine_field(grid: Grid, modes: Sequence[Sequence[int]], amps: Sequence[float]) -> np.ndarray:
    """sum_m a_m prod_d sin(k_{m,d} pi x_d / L) on the interior nodes.

    ``modes`` rows are wave numbers in (x, y, z) order.
    """
    coords = interior_coords(grid)[::-1]                      # x, y, z
    out = np.zeros(grid.shape)
    for k, a in zip(modes, amps):
        term = np.ones(())
        for d in range(grid.dim):
            s = np.sin(k[d] * math.pi * coords[d] / grid.L)
            # broadcast axis d (x is the last numpy axis)
            shape = [1] * grid.dim
            shape[grid.dim - 1 - d] = s.size
            term = term * s.reshape(shape)
        out = out + a * term
    return out


def _sine_matrix(n: int) -> np.ndarray:
    j = np.arange(1, n + 1)
    return np.sin(np.pi * np.outer(j, j) / (n + 1))


def forward_discrete(grid: Grid, z0: np.ndarray, steps: int | None = None) -> np.ndarray:
    """Data synthesis: the backward-Euler forward heat solution after ``steps``
    steps (default N = nt - 1), i.e. (I - tau Lap_h)^{-steps} z0, evaluated in
    the sine eigenbasis of the Dirichlet finite-difference Laplacian
    (eigenvalues (4/h^2) sin^2(k pi / (2M)), a textbook fact).

    This is the "exact discrete forward solution at T" the data recipe asks
    for; it is the forward (well-posed) problem, not the regularised backward
    solve.
    """
    steps = grid.nt - 1 if steps is None else steps
    c = np.asarray(z0, dtype=np.float64).reshape(grid.shape)
    lam_total = np.zeros(grid.shape)
    for d in range(grid.dim):
        M = grid.M[d]
        h = grid.h[d]
        S = _sine_matrix(M - 1)
        ax = grid.dim - 1 - d
        c = np.moveaxis(np.tensordot(S, np.moveaxis(c, ax, 0), axes=(1, 0)), 0, ax)
        lam = (4.0 / h ** 2) * np.sin(np.arange(1, M) * math.pi / (2 * M)) ** 2
        shape = [1] * grid.dim
        shape[ax] = M - 1
        lam_total = lam_total + lam.reshape(shape)
    c = c * (1.0 + grid.tau * lam_total) ** (-float(steps))
    for d in range(grid.dim):
        M = grid.M[d]
        S = _sine_matrix(M - 1) * (2.0 / M)
        ax = grid.dim - 1 - d
        c = np.moveaxis(np.tensordot(S, np.moveaxis(c, ax, 0), axes=(1, 0)), 0, ax)
    return c


def add_noise_multiplicative(grid: Grid, g: np.ndarray, eps: float, rng: np.random.Generator):
    """Section 5 noise model: g * (1 + eps * U(-1, 1)); returns (g_delta, delta)."""
    gd = g * (1.0 + eps * rng.uniform(-1.0, 1.0, size=g.shape))
    return gd, discrete_l2(gd - g, grid)


def add_noise_gaussian(grid: Grid, g: np.ndarray, rel: float, rng: np.random.Generator):
    """Additive i.i.d. Gaussian noise scaled to ||noise|| = rel * ||g||."""
    eta = rng.standard_normal(g.shape)
    eta *= rel * np.linalg.norm(g.ravel()) / max(np.linalg.norm(eta.ravel()), 1e-300)
    gd = g + eta
    return gd, discrete_l2(gd - g, grid)


# ---------------------------------------------------------------- workloads

def make_c1(seed: int = 1) -> Problem:
    """1D, M=64 (63 interior points), nt=64, T=0.1, z0 = sin(pi x) + 0.5 sin(3 pi x),
    g = discrete forward solution at T, multiplicative uniform noise eps=1e-3."""
    grid = Grid(1, (64,), 1.0, 0.1, 64)
    z0 = sine_field(grid, [(1,), (3,)], [1.0, 0.5])
    g = forward_discrete(grid, z0)
    rng = np.random.default_rng(seed)
    gd, delta = add_noise_multiplicative(grid, g, 1e-3, rng)
    return Problem("c1_1d_63x64", grid, z0, g, gd, delta, seed)


def _decaying_sine_modes(rng, dim: int, count: int, kmax: int):
    """``count`` distinct wave-number tuples from {1..kmax}^dim, the lowest mode
    always included and the others drawn with weight 1/|k|^4 (at T = 0.1 a mode
    with |k|^2 = 40 has decayed by e^{-40}: uniform draws give data ~1e-8)."""
    pool = np.array(np.meshgrid(*[np.arange(1, kmax + 1)] * dim, indexing="ij")).reshape(dim, -1).T
    k2 = (pool.astype(np.float64) ** 2).sum(axis=1)
    first = int(np.argmin(k2))
    rest = np.array([i for i in range(len(pool)) if i != first])
    w = 1.0 / k2[rest] ** 2
    idx = rng.choice(rest, size=count - 1, replace=False, p=w / w.sum())
    modes = pool[np.concatenate([[first], idx])]
    amps = rng.uniform(0.5, 1.5, size=count) * rng.choice([-1.0, 1.0], size=count)
    amps = amps / (modes.astype(np.float64) ** 2).sum(axis=1)
    return modes, amps


def make_c2(seed: int = 2, M: int = 256, nt: int = 256) -> Problem:
    """2D unit square, (M-1)^2 interior points, nt levels, T=0.1; z0 = 16 random
    sine modes (k, l) in {1..8}^2 (weighted toward low |k|, (1,1) always present)
    with amplitudes U(0.5,1.5) * sign / (k^2 + l^2);
    g = discrete forward solution at T; 1% Gaussian noise relative to ||g||."""
    grid = Grid(2, (M, M), 1.0, 0.1, nt)
    rng = np.random.default_rng(seed)
    modes, amps = _decaying_sine_modes(rng, 2, 16, 8)
    z0 = sine_field(grid, modes, amps)
    g = forward_discrete(grid, z0)
    gd, delta = add_noise_gaussian(grid, g, 1e-2, rng)
    return Problem(f"c2_2d_{M-1}sq_x{nt}", grid, z0, g, gd, delta, seed,
                   {"modes": modes.tolist(), "amps": amps.tolist()})


def gaussian_bumps(grid: Grid, rng: np.random.Generator, count: int = 8) -> np.ndarray:
    """Smooth random bumps times the bubble 4^d prod x(1-x) so z0 = 0 on the boundary."""
    coords = interior_coords(grid)[::-1]     # x, y, z
    mesh = np.meshgrid(*[c / grid.L for c in coords], indexing="ij")   # x, y, z order
    z = np.zeros(mesh[0].shape)
    for _ in range(count):
        c = rng.uniform(0.25, 0.75, size=grid.dim)
        s = rng.uniform(0.05, 0.15)
        a = rng.uniform(0.5, 1.5)
        r2 = sum((mesh[d] - c[d]) ** 2 for d in range(grid.dim))
        z = z + a * np.exp(-r2 / (2 * s * s))
    bubble = np.ones_like(z)
    for d in range(grid.dim):
        bubble = bubble * 4.0 * mesh[d] * (1.0 - mesh[d])
    return np.transpose(z * bubble)            # to numpy (z, y, x) order


def make_c3(seed: int = 3, M: int = 128, nt: int = 128) -> Problem:
    """3D unit cube, (M-1)^3 interior points, nt levels, T=0.05; z0 = 8 Gaussian
    bumps times the bubble; g = discrete forward solution; 0.1% Gaussian noise."""
    grid = Grid(3, (M, M, M), 1.0, 0.05, nt)
    rng = np.random.default_rng(seed)
    z0 = gaussian_bumps(grid, rng, 8)
    g = forward_discrete(grid, z0)
    gd, delta = add_noise_gaussian(grid, g, 1e-3, rng)
    return Problem(f"c3_3d_{M-1}cube_x{nt}", grid, z0, g, gd, delta, seed)


def make_paper_ex1(M: int, N: int, eps: float, seed: int = 11, terms: int = 100) -> Problem:
    """Section 5.1 Example 1: Omega=(0,pi), T=1, triangular z(x,0); g from the
    exact series truncated to ``terms`` odd terms; mesh h=pi/M, tau=T/N."""
    grid = Grid(1, (M,), math.pi, 1.0, N + 1)
    x = interior_coords(grid)[0]
    z0 = np.where(x <= math.pi / 2, 2 * x, 2 * (math.pi - x))
    k = np.arange(1, 2 * terms, 2)
    g = (8 / math.pi) * (np.cos(np.outer(x, k) - k * math.pi / 2) / k ** 2 * np.exp(-k ** 2 * grid.T)).sum(axis=1)
    rng = np.random.default_rng(seed)
    gd, delta = add_noise_multiplicative(grid, g, eps, rng)
    return Problem(f"paper_ex1_{M}_{N}", grid, z0, g, gd, delta, seed, {"eps": eps})


def make_paper_ex2(M: int, N: int, eps: float, seed: int = 12) -> Problem:
    """Section 5.2 Example 2: Omega=(0,pi)^2, T=1, z = exp(-2t) sin x1 sin x2."""
    grid = Grid(2, (M, M), math.pi, 1.0, N + 1)
    z0 = sine_field(grid, [(1, 1)], [1.0])
    g = math.exp(-2 * grid.T) * z0
    rng = np.random.default_rng(seed)
    gd, delta = add_noise_multiplicative(grid, g, eps, rng)
    return Problem(f"paper_ex2_{M}_{N}", grid, z0, g, gd, delta, seed, {"eps": eps})


def make_problem(name: str, seed: int | None = None) -> Problem:
    table = {"c1": make_c1, "c2": make_c2, "c3": make_c3}
    fn = table[name]
    return fn() if seed is None else fn(seed)


def random_general_rhs(grid: Grid, seed: int, scale: float = 1.0) -> np.ndarray:
    """A general all-at-once right-hand side F (nt, *shape): smooth-in-space,
    random-in-time data used to exercise the general-RHS path."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(grid.full_shape)


def batch_specs_c4(seed: int = 4, count: int = 512):
    """Uneven batch of instances: one third 1D with M-1 in {63,...,2047}, two
    thirds 2D with M-1 in {63,127,255}^2, nt in {32,...,512}, relative noise
    log-uniform in [1e-4, 1e-2].  Returns a list of dicts (dim, M, nt, rel_noise, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nt = int(rng.choice([32, 64, 128, 256, 512]))
        rel = float(10 ** rng.uniform(-4, -2))
        if i % 3 == 0:
            M = (int(rng.choice([64, 128, 256, 512, 1024, 2048])),)
        else:
            M = (int(rng.choice([64, 128, 256])), int(rng.choice([64, 128, 256])))
        out.append({"dim": len(M), "M": M, "nt": nt, "rel_noise": rel, "seed": seed * 100003 + i})
    return out


def alpha_training_batch(count: int, seed: int, M: int = 128, nt: int = 128, T: float = 0.1,
                         rel_range=(1e-4, 1e-2), modes: int = 16, kmax: int = 8):
    """A batch of 2D instances on the unit square for the learned-alpha data:
    z0 = `modes` random decaying sine modes (as for the 2D workload), g the
    exact discrete forward solution at T, additive Gaussian noise with relative
    level log-uniform in rel_range.

    Returns (grid, z0, g_delta, delta) with z0 and g_delta of shape
    (count, M-1, M-1) (x fastest) and delta (count,), the grid-weighted noise
    norms.  Built mode by mode: with S_k the sine vectors of the grid,
    z0_b = Sy^T C_b Sx and g_b = Sy^T (C_b * r^N) Sx, r = 1/(1 + tau lambda).
    """
    grid = Grid(2, (M, M), 1.0, T, nt)
    rng = np.random.default_rng(seed)
    n = M - 1
    x = np.arange(1, M) / M
    ks = np.arange(1, kmax + 1)
    S = np.sin(np.pi * np.outer(ks, x))                       # (kmax, n)
    lam1 = (4.0 * M * M) * np.sin(ks * np.pi / (2 * M)) ** 2
    lam = lam1[:, None] + lam1[None, :]                       # (ky, kx)
    decay = (1.0 + grid.tau * lam) ** (-(nt - 1.0))
    C = np.zeros((count, kmax, kmax))
    for b in range(count):
        md, amps = _decaying_sine_modes(rng, 2, modes, kmax)
        for (kx, ky), a in zip(md, amps):
            C[b, ky - 1, kx - 1] += a
    z0 = np.einsum("yn,byx,xm->bnm", S, C, S, optimize=True)
    g = np.einsum("yn,byx,xm->bnm", S, C * decay, S, optimize=True)
    rel = 10.0 ** rng.uniform(np.log10(rel_range[0]), np.log10(rel_range[1]), size=count)
    eta = rng.standard_normal(g.shape)
    gn = np.sqrt((g * g).sum(axis=(1, 2)))
    en = np.sqrt((eta * eta).sum(axis=(1, 2)))
    eta *= (rel * gn / en)[:, None, None]
    delta = (1.0 / M) * np.sqrt((eta * eta).sum(axis=(1, 2)))
    return grid, z0, g + eta, delta
