"""Normalized gradient flow, backward Euler, Fourier pseudospectral (GF-NUFFT,
Sec. 3.1, Eqs. (gf-eq2)-(gffg33)).

One step, for phi^n with h^d sum |phi^n|^2 = 1:
    rho = |phi^n|^2,  Phi = U * rho (any evaluator of the potential),
    b = V + g rho + beta Phi,
    solve (1/tau - Delta/2 + b) phi^(1) = phi^n / tau            (backward Euler)
    phi^{n+1} = phi^(1) / ||phi^(1)||                             (Eq. (gffg33))
The paper omits how the linear system is solved.  Reading (stabilised
fixed point, Fourier-diagonal preconditioner): with alpha = (max b + min b)/2,
    G(x) = F^{-1}[ F[ phi^n/tau + (alpha - b) x ] / (1/tau + alpha + |mu|^2/2) ]
(periodic box, mu_p = pi p / L); the fixed point of G is the backward-Euler solution, and
G(x) - x is the residual preconditioned by M = 1/tau + alpha - Delta/2.  The eigenvalues of
M^{-1} (1/tau - Delta/2 + b) lie in [1 - q, 1 + q], q = max|b - alpha| / (1/tau + alpha) < 1,
so the iteration is accelerated by the Chebyshev semi-iteration on that interval (Saad,
Iterative Methods for Sparse Linear Systems, Alg. 12.1, centre 1, half-width q):
    x_1 = G(x_0),  d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / q)(G(x_k) - x_k),
    x_{k+1} = x_k + d_k,  rho_0 = q,  rho_k = 1/(2/q - rho_{k-1}),
from x_0 = phi^n until max|x_{k+1} - x_k| <= inner_tol (plain x_{k+1} = G(x_k) if q is
not in (0, 1)).
g rho is an optional local (contact) term; the paper's examples have g = 0.
Stopping rule of Sec. 3.2: max |phi^{n+1} - phi^n| / tau <= eps0.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import fft as sfft

WORKERS = -1   # scipy.fft thread count (library FFT; all host cores)


def wavenumbers2(grid):
    """|mu|^2 on the FFT layout of the grid (Fourier pseudospectral, periodic box)."""
    ks = [2.0 * math.pi * np.fft.fftfreq(n, d=h) for n, h in zip(grid.n, grid.h)]
    K = np.meshgrid(*ks, indexing="ij")
    return sum(k * k for k in K)


def norm2(phi, grid):
    return float(np.prod(grid.h)) * float(np.sum(np.abs(phi) ** 2))


class GradientFlow:
    def __init__(self, grid, V, beta, potential, tau=1e-2, g=0.0, inner_tol=1e-12, max_inner=1000):
        self.grid, self.V, self.beta, self.g = grid, np.asarray(V, dtype=np.float64), float(beta), float(g)
        self.pot = potential
        self.tau = float(tau)
        self.inner_tol, self.max_inner = float(inner_tol), int(max_inner)
        self.mu2 = wavenumbers2(grid)
        self.mu2r = self.mu2[..., : grid.n[-1] // 2 + 1]   # real-to-complex half spectrum
        self.last_inner = 0

    def step(self, phi):
        tau = self.tau
        rho = phi * phi
        Phi = self.pot(rho)
        b = self.V + self.g * rho + self.beta * Phi
        bmax, bmin = float(np.max(b)), float(np.min(b))
        alpha = 0.5 * (bmax + bmin)
        q = 0.5 * (bmax - bmin) / (1.0 / tau + alpha)
        cheb = 0.0 < q < 1.0
        denom = 1.0 / tau + alpha + 0.5 * self.mu2r
        rhs0 = phi / tau
        x = phi.copy()
        d = np.zeros_like(x)
        rho_prev, rho = 0.0, q
        it = 0
        n = self.grid.n
        for it in range(1, self.max_inner + 1):
            gx = sfft.irfftn(sfft.rfftn(rhs0 + (alpha - b) * x, workers=WORKERS) / denom, s=n,
                             workers=WORKERS)
            if it == 1 or not cheb:
                d = gx - x                                   # x_1 = G(x_0)
            else:
                d = rho * rho_prev * d + (2.0 * rho / q) * (gx - x)
            x = x + d
            if cheb:
                rho_prev, rho = rho, 1.0 / (2.0 / q - rho)
            diff = float(np.max(np.abs(d)))
            if diff <= self.inner_tol:
                break
        self.last_inner = it
        x = x / math.sqrt(norm2(x, self.grid))
        change = float(np.max(np.abs(x - phi))) / tau
        return x, change

    def energies(self, phi):
        """E_kin, E_pot, E_int and E, mu of Sec. 3.2 (mu = E + E_int)."""
        hv = float(np.prod(self.grid.h))
        N = phi.size
        ph = np.fft.fftn(phi)
        ekin = 0.5 * hv * float(np.sum(self.mu2 * np.abs(ph) ** 2)) / N
        rho = np.abs(phi) ** 2
        epot = hv * float(np.sum(self.V * rho))
        Phi = self.pot(rho)
        eint = 0.5 * hv * float(np.sum((self.g * rho + self.beta * Phi) * rho))
        E = ekin + epot + eint
        return dict(E=E, Ekin=ekin, Epot=epot, Eint=eint, mu=E + eint)

    def solve(self, phi0, eps0=1e-10, max_steps=100000):
        phi = phi0.copy()
        change = np.inf
        n = 0
        while n < max_steps:
            phi, change = self.step(phi)
            n += 1
            if change <= eps0:
                break
        return phi, n, change
