"""Seeded synthetic inputs (initial values and workload descriptions).

This module holds no arithmetic of the method: it only draws seeded sine-mode
amplitudes and evaluates the resulting initial values on the interior grid points
x_i = i / (n + 1), i = 1..n.  Both the CUDA path and the oracle take their inputs
from here, so the two sides see identical data.  The paper's test problems are
sums of sine modes of the heat equation with zero Dirichlet walls (Sec. 4.1, 4.2);
the workloads below follow that recipe at the sizes this library is measured on.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def sine_sum(dim: int, n: int, modes, amps) -> np.ndarray:
    """sum_k a_k prod_axis sin(k_axis pi x_axis) on the n^dim interior points,
    dense layout [z][y][x] (x fastest); modes are (kx, ky, kz) tuples."""
    x = np.arange(1, n + 1, dtype=np.float64) / (n + 1)
    out = np.zeros((n,) * dim)
    for k, a in zip(modes, amps):
        fx = np.sin(k[0] * np.pi * x)
        if dim == 1:
            out += a * fx
        elif dim == 2:
            out += a * np.outer(np.sin(k[1] * np.pi * x), fx)
        else:
            out += a * np.einsum("k,j,i->kji", np.sin(k[2] * np.pi * x), np.sin(k[1] * np.pi * x), fx)
    return out.reshape(-1)


def random_modes(dim: int, count: int, kmax: int, seed: int, radius: float | None = None):
    """`count` distinct mode vectors from {1..kmax}^dim (|k|_2 <= radius if given),
    drawn uniformly without repetition, and N(0,1) amplitudes; fixed seed."""
    rng = np.random.default_rng(seed)
    grid = np.stack(np.meshgrid(*[np.arange(1, kmax + 1)] * dim, indexing="ij"), -1).reshape(-1, dim)
    if radius is not None:
        grid = grid[np.sqrt((grid ** 2).sum(1)) <= radius + 1e-12]
    pick = rng.choice(len(grid), size=count, replace=False)
    modes = [tuple(int(v) for v in grid[p]) + (1,) * (3 - dim) for p in pick]
    amps = rng.standard_normal(count)
    return modes, amps


@dataclass
class Workload:
    """One synthetic heat-equation workload for SDC / PFASST."""
    name: str
    dim: int
    n: int
    nu: float
    dt: float
    slices: int
    fine_nodes: int
    coarse_nodes: int
    nlevels: int
    smoother: int            # 0 Jacobi (omega 2/3), 1 red-black Gauss-Seidel (omega 1)
    vcycles: int
    precision: int           # 0 FP64, 1 mixed
    iterations: int          # PFASST iterations (or SDC sweeps per step)
    steps: int = 1           # consecutive blocks (time steps of length slices*dt)
    modes: list = field(default_factory=list)
    amps: list = field(default_factory=list)

    @property
    def omega(self):
        return 1.0 if self.smoother == 1 else 2.0 / 3.0

    def u0(self) -> np.ndarray:
        return sine_sum(self.dim, self.n, self.modes, self.amps)

    @property
    def dofs(self):
        return self.n ** self.dim


def heat1d_c1() -> Workload:
    """1D heat, nu = 1, 127 points, u0 = sin(pi x) + 0.5 sin(3 pi x), 3 Gauss-Lobatto
    nodes, single-level SDC, dt = 0.01 to T = 0.1, V(2,1) Jacobi, FP64."""
    return Workload("heat1d_n127_sdc3", 1, 127, 1.0, 0.01, 1, 3, 0, 1, 0, 2, 0, 50, steps=10,
                    modes=[(1, 1, 1), (3, 1, 1)], amps=[1.0, 0.5])


def heat2d_c2(vcycles: int = 2, precision: int = 0, n: int = 255, slices: int = 16) -> Workload:
    """2D heat, nu = 1, 255^2 fine / 127^2 coarse, two-level PFASST 5/3 Gauss-Lobatto
    nodes, 16 slices, dt = 0.005, 8 sine modes with N(0,1) amplitudes (seed 1407)."""
    modes, amps = random_modes(2, 8, 8, 1407)
    return Workload(f"heat2d_n{n}_pfasst5x3_P{slices}", 2, n, 1.0, 0.005, slices, 5, 3, 2, 0, vcycles, precision,
                    20, modes=modes, amps=list(amps))


def heat3d_c3(n: int = 255, slices: int = 32, precision: int = 1, iterations: int = 10) -> Workload:
    """3D heat, nu = 0.5, 255^3 fine / 127^3 coarse, two-level PFASST 5/3 Gauss-Lobatto
    nodes, 32 slices, dt = 0.002, 16 sine modes with |k| <= 8 (seed 6486), V(2,1)
    red-black Gauss-Seidel, 2 V-cycles, FP32 multigrid with FP64 SDC/FAS, 10 iterations."""
    modes, amps = random_modes(3, 16, 8, 6486, radius=8.0)
    return Workload(f"heat3d_n{n}_pfasst5x3_P{slices}", 3, n, 0.5, 0.002, slices, 5, 3, 2, 1, 2, precision,
                    iterations, modes=modes, amps=list(amps))


def gaussian_random_field(n: int, ell: float, seed: int) -> np.ndarray:
    """Seeded Gaussian random field on the n^3 interior points with zero walls, by
    spectral synthesis: u = sum_k a_k sin(k_x pi x) sin(k_y pi y) sin(k_z pi z) with
    independent N(0, 1) draws scaled by exp(-(pi |k| ell)^2 / 4), the square root of the
    spectral density of the Gaussian covariance exp(-r^2 / (2 ell^2)) at the wave number
    pi |k|; summed as a type-I sine transform (its basis is exactly sin(k pi i / (n+1)) on
    the interior points).  Scaled to max |u| = 1; dense layout [z][y][x]."""
    from scipy.fft import idstn
    rng = np.random.default_rng(seed)
    k = np.arange(1, n + 1, dtype=np.float64)
    kk = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    coef = rng.standard_normal((n, n, n)) * np.exp(-(np.pi ** 2) * kk * ell ** 2 / 4.0)
    u = idstn(coef, type=1, norm="forward")  # sum_k coef_k prod sin(k pi i / (n + 1))
    return (u / np.abs(u).max()).reshape(-1)


@dataclass
class Problem:
    """One member of an uneven batch (single-level SDC, one time step per run step)."""
    dim: int
    n: int
    nodes: int
    nu: float
    dt: float
    modes: list
    amps: list

    def u0(self) -> np.ndarray:
        return sine_sum(self.dim, self.n, self.modes, self.amps)

    @property
    def dofs(self):
        return self.n ** self.dim


def heat_uneven_c4(seed: int = 64, n2d=(63, 127, 255, 511), n3d=(31, 63, 127), count2d: int = 32,
                   count3d: int = 32):
    """Uneven batch: independent heat problems, 2D sizes drawn from n2d and 3D sizes from
    n3d, nu ~ U[0.1, 2], dt ~ U[1e-3, 1e-2], 3 or 5 Gauss-Lobatto nodes, u0 = 4 sine
    modes with k <= min(8, n/4) and N(0,1) amplitudes; fixed seed."""
    rng = np.random.default_rng(seed)
    out = []
    for dim, sizes, count in ((2, n2d, count2d), (3, n3d, count3d)):
        for _ in range(count):
            n = int(rng.choice(sizes))
            nodes = int(rng.choice([3, 5]))
            nu = float(rng.uniform(0.1, 2.0))
            dt = float(rng.uniform(1e-3, 1e-2))
            kmax = max(2, min(8, n // 4))
            grid = np.stack(np.meshgrid(*[np.arange(1, kmax + 1)] * dim, indexing="ij"), -1).reshape(-1, dim)
            pick = rng.choice(len(grid), size=min(4, len(grid)), replace=False)
            modes = [tuple(int(v) for v in grid[p]) + (1,) * (3 - dim) for p in pick]
            amps = list(rng.standard_normal(len(modes)))
            out.append(Problem(dim, n, nodes, nu, dt, modes, amps))
    return out
