"""Normalized gradient flow, backward Euler, Fourier pseudospectral (GF-NUFFT,
Sec. 3.1, Eqs. (gf-eq2)-(gffg33)).

One step, for phi^n with h^d sum |phi^n|^2 = 1:
    rho = |phi^n|^2,  Phi = U * rho (any evaluator of the potential),
    b = V + g rho + beta Phi,
    solve (1/tau - Delta/2 + b) phi^(1) = phi^n / tau            (backward Euler)
    phi^{n+1} = phi^(1) / ||phi^(1)||                             (Eq. (gffg33))
The paper omits how the linear system is solved.  Reading (stabilised
fixed point, Fourier-diagonal preconditioner): with alpha = (max b + min b)/2,
    (1/tau + alpha + |mu|^2/2) phi^(1),m+1 = F[ phi^n/tau + (alpha - b) phi^(1),m ]
in Fourier space (periodic box, mu_p = pi p / L), from phi^(1),0 = phi^n, until
max|phi^(1),m+1 - phi^(1),m| <= inner_tol.  It converges because
|alpha - b| / (1/tau + alpha) < 1, and its fixed point is the backward-Euler solution.
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
        alpha = 0.5 * (float(np.max(b)) + float(np.min(b)))
        denom = 1.0 / tau + alpha + 0.5 * self.mu2r
        rhs0 = phi / tau
        x = phi.copy()
        it = 0
        n = self.grid.n
        for it in range(1, self.max_inner + 1):
            xn = sfft.irfftn(sfft.rfftn(rhs0 + (alpha - b) * x, workers=WORKERS) / denom, s=n,
                             workers=WORKERS)
            diff = float(np.max(np.abs(xn - x)))
            x = xn
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
