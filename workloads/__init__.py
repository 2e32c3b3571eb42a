"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds input generation only: grid coordinates, Gaussian densities,
trap potentials, random draws.  It contains none of the method's arithmetic
(no quadrature, no NUFFT, no kernel symbols), so both sides can import it
without sharing any part of the computation they are compared on.

Grid convention (the paper leaves it implicit): on [-L, L) with n points per
axis, h = 2L/n and x_m = -L + m h, m = 0..n-1, so the origin is the grid point
m = n/2.  Arrays are C order with the last axis fastest: a[i, j, k] = f(x_i,
y_j, z_k).  The densities are the paper's test functions (Sec. 2.4, Examples
2.1-2.3; Sec. 3.2 Gaussian starts).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_TRAIN = 20141014
SEED_HELDOUT = 20141015


@dataclass(frozen=True)
class Grid:
    """Uniform grid: n[d] points on prod [-L_d, L_d)."""

    n: tuple
    L: tuple

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def h(self) -> tuple:
        return tuple(2.0 * L / n for n, L in zip(self.n, self.L))

    def axes(self):
        return [(-L + np.arange(n, dtype=np.float64) * (2.0 * L / n)) for n, L in zip(self.n, self.L)]

    def mesh(self):
        return np.meshgrid(*self.axes(), indexing="ij")


def cube(n: int, L: float, dim: int = 3) -> Grid:
    return Grid(tuple([n] * dim), tuple([float(L)] * dim))


def gaussian(grid: Grid, widths, center=None, amp: float = 1.0) -> np.ndarray:
    """rho = amp * exp(-sum_d (x_d - c_d)^2 / a_d^2)  (FP64)."""
    X = grid.mesh()
    if center is None:
        center = [0.0] * grid.dim
    q = np.zeros(grid.n, dtype=np.float64)
    for x, a, c in zip(X, widths, center):
        q += (x - c) ** 2 / (a * a)
    return amp * np.exp(-q)


def gaussian_sum(grid: Grid, centers, widths, amps=None) -> np.ndarray:
    """rho = sum_i amp_i exp(-|x - c_i|^2 / s_i^2) (isotropic terms)."""
    rho = np.zeros(grid.n, dtype=np.float64)
    if amps is None:
        amps = [1.0] * len(centers)
    for c, s, a in zip(centers, widths, amps):
        rho += gaussian(grid, [s] * grid.dim, c, a)
    return rho


def three_gaussians_2d(seed: int = SEED_TRAIN):
    """Centres uniform in [-4,4]^2, widths uniform in [0.5,2], unit amplitudes."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-4.0, 4.0, size=(3, 2))
    widths = rng.uniform(0.5, 2.0, size=3)
    return [tuple(c) for c in centers], [float(s) for s in widths]


def three_gaussians_1d(seed: int = SEED_TRAIN):
    """1D: centres uniform in [-4,4], widths uniform in [0.5,2], amplitudes uniform in [0.5,1.5]."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-4.0, 4.0, size=3)
    widths = rng.uniform(0.5, 2.0, size=3)
    amps = rng.uniform(0.5, 1.5, size=3)
    return [(float(c),) for c in centers], [float(s) for s in widths], [float(a) for a in amps]


def harmonic_trap(grid: Grid, gammas) -> np.ndarray:
    """V = sum_d gamma_d^2 x_d^2 / 2."""
    X = grid.mesh()
    V = np.zeros(grid.n, dtype=np.float64)
    for x, g in zip(X, gammas):
        V += 0.5 * (g * x) ** 2
    return V


def normalized_gaussian_start(grid: Grid, gammas) -> np.ndarray:
    """Gaussian initial datum phi_0 = prod (g/pi)^{1/4} exp(-g x^2/2), then rescaled
    so that the discrete norm h^d sum phi^2 is exactly 1 (GF start, Sec. 3.2)."""
    X = grid.mesh()
    phi = np.ones(grid.n, dtype=np.float64)
    for x, g in zip(X, gammas):
        phi *= (g / math.pi) ** 0.25 * np.exp(-0.5 * g * x * x)
    hv = float(np.prod(grid.h))
    return phi / math.sqrt(hv * float(np.sum(phi * phi)))


@dataclass
class BatchItem:
    n: int
    L: float
    widths: tuple
    kernel: str  # "coulomb3d" | "dipole3d"


def batch_spec(count: int = 64, seed: int = SEED_TRAIN, sizes=(64, 96, 128, 160, 192)):
    """Batched workload: per density n ~ U(sizes), a_x = 1, a_y, a_z = r with
    r ~ U[1,4], L = 6 * a_max, kernel Coulomb or dipolar-z with probability 1/2."""
    rng = np.random.default_rng(seed)
    items = []
    for _ in range(count):
        n = int(rng.choice(sizes))
        ry, rz = rng.uniform(1.0, 4.0, size=2)
        widths = (1.0, float(ry), float(rz))
        L = 6.0 * max(widths)
        kern = "coulomb3d" if rng.uniform() < 0.5 else "dipole3d"
        items.append(BatchItem(n, L, widths, kern))
    return items


def gf_params(count: int, seed: int):
    """(beta, gamma) draws for the ground-state workload: gamma ~ U[1,4],
    beta ~ log-uniform on [1, 1000]."""
    rng = np.random.default_rng(seed)
    gam = rng.uniform(1.0, 4.0, size=count)
    beta = np.exp(rng.uniform(0.0, math.log(1000.0), size=count))
    return [(float(b), float(g)) for b, g in zip(beta, gam)]


def gs_problems(count: int, seed: int):
    """(beta, gamma, kernel) draws for the learned-initial-guess workload: the (beta, gamma)
    of gf_params and the kernel drawn uniformly from Coulomb / dipolar."""
    rng = np.random.default_rng(seed + 1)
    kern = rng.integers(0, 2, size=count)
    return [(b, g, "coulomb3d" if k == 0 else "dipole3d") for (b, g), k in zip(gf_params(count, seed), kern)]


def random_density(grid: Grid, seed: int) -> np.ndarray:
    """Non-negative smooth random density (sum of 4 random Gaussians), for
    invariance and linearity tests."""
    rng = np.random.default_rng(seed)
    lim = 0.35 * min(grid.L)
    centers = rng.uniform(-lim, lim, size=(4, grid.dim))
    widths = rng.uniform(0.6, 1.4, size=4)
    amps = rng.uniform(0.5, 1.5, size=4)
    return gaussian_sum(grid, [tuple(c) for c in centers], list(widths), list(amps))
