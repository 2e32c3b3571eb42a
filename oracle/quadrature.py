"""Fourier-space quadrature for Eq. (ifft) (Sec. 2.1): spherical (3D) / polar (2D).

The Coulomb-type integrand U-hat(k) rho-hat(k) e^{ik.x} becomes smooth in
spherical/polar coordinates because the Jacobian |k|^{d-1} cancels the
singularity of U-hat (Sec. 2.1).  The paper asks only for "high order
quadratures"; the rule used here (reading, recorded in the design notes):
  radial   Gauss-Legendre, n_r nodes on [0, P]
  polar    Gauss-Legendre in u = cos(theta) on [-1, 1] (absorbs sin(theta)), n_theta even
  azimuth  periodic trapezoid, n_phi even, phi_c = 2 pi c / n_phi
The node set is symmetric under k -> -k (u -> -u, phi -> phi + pi).
"""
from __future__ import annotations

import math

import numpy as np


def gauss_legendre(n: int, a: float, b: float):
    """n-point Gauss-Legendre rule mapped to [a, b] (library primitive)."""
    x, w = np.polynomial.legendre.leggauss(int(n))
    half = 0.5 * (b - a)
    return a + half * (x + 1.0), half * w


def sphere_rule(P: float, n_r: int, n_theta: int, n_phi: int):
    """Nodes k_j (M x 3) and plain quadrature weights w_r w_u w_phi (M,)
    for the measure dr du dphi on |k| <= P.  Order: (r, u, phi), phi fastest."""
    r, wr = gauss_legendre(n_r, 0.0, P)
    u, wu = gauss_legendre(n_theta, -1.0, 1.0)
    ph = 2.0 * math.pi * np.arange(n_phi) / n_phi
    wph = np.full(n_phi, 2.0 * math.pi / n_phi)
    R, U, PH = np.meshgrid(r, u, ph, indexing="ij")
    S = np.sqrt(np.maximum(0.0, 1.0 - U * U))
    k = np.stack([R * S * np.cos(PH), R * S * np.sin(PH), R * U], axis=-1).reshape(-1, 3)
    w = (wr[:, None, None] * wu[None, :, None] * wph[None, None, :]).reshape(-1)
    return k, w, R.reshape(-1)


def polar_rule(P: float, n_r: int, n_phi: int):
    """Nodes k_j (M x 2) and weights w_r w_phi for the measure dr dphi."""
    r, wr = gauss_legendre(n_r, 0.0, P)
    ph = 2.0 * math.pi * np.arange(n_phi) / n_phi
    wph = np.full(n_phi, 2.0 * math.pi / n_phi)
    R, PH = np.meshgrid(r, ph, indexing="ij")
    k = np.stack([R * np.cos(PH), R * np.sin(PH)], axis=-1).reshape(-1, 2)
    w = (wr[:, None] * wph[None, :]).reshape(-1)
    return k, w, R.reshape(-1)


def _round16(x: float) -> int:
    return int(16 * math.ceil(x / 16.0))


def default_counts(L, P: float):
    """Default node counts (reading of "high order quadrature"): with R the
    half-diagonal of the box and Rp that of its first two axes,
    n_r = n_theta = roundup16(P R / 2 + 16), n_phi = roundup16(P Rp + 32)."""
    L = [float(v) for v in L]
    R = math.sqrt(sum(v * v for v in L))
    Rp = math.sqrt(L[0] ** 2 + L[1] ** 2)
    nr = _round16(P * R / 2.0 + 16.0)
    nph = _round16(P * Rp + 32.0)
    if len(L) == 3:
        return nr, nr, nph
    return nr, nph


def density_P(a_min: float, h_max: float, eps: float = 1e-16) -> float:
    """Truncation radius for Gaussian densities (reading of P = O(eps^{-1/n}),
    Sec. 2.1): rho-hat ~ exp(-a^2 k^2 / 4) falls below eps at 2 sqrt(ln 1/eps)/a;
    never beyond pi / h_max, the largest ball inside the grid's spectral box."""
    return min(math.pi / h_max, 2.0 * math.sqrt(math.log(1.0 / eps)) / a_min)
