"""Time splitting Fourier pseudospectral (TS-NUFFT, Sec. 4.1, Eqs. (sps-eq65)-(sps-eq68)).

Kinetic part (sps-eq65) is integrated exactly in Fourier space:
    psi <- F^{-1}[ exp(-i s |mu|^2 / 2) F psi ].
Potential part (sps-eq66): |psi| is invariant, so Phi is frozen at Phi^n and
    psi <- exp(-i (V + g |psi|^2 + beta Phi^n) s) psi          (Eq. (sps-eq68)).
Second order (Strang): K(tau/2) P(tau) K(tau/2); the paper lists the kinetic
sub-problem first.  Fourth order: the symmetric triple composition of Yoshida,
S(w1 tau) S(w0 tau) S(w1 tau) with w1 = 1/(2 - 2^{1/3}), w0 = 1 - 2 w1.
"""
from __future__ import annotations

import numpy as np

from .gf import wavenumbers2

YOSHIDA_W1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
YOSHIDA_W0 = 1.0 - 2.0 * YOSHIDA_W1


class TimeSplitting:
    def __init__(self, grid, V, beta, potential, g=0.0):
        self.grid = grid
        self.V = np.asarray(V, dtype=np.float64)
        self.beta, self.g = float(beta), float(g)
        self.pot = potential
        self.mu2 = wavenumbers2(grid)

    def kinetic(self, psi, s):
        return np.fft.ifftn(np.exp(-0.5j * s * self.mu2) * np.fft.fftn(psi))

    def potential_step(self, psi, s):
        rho = np.abs(psi) ** 2
        Phi = self.pot(rho)
        return np.exp(-1j * s * (self.V + self.g * rho + self.beta * Phi)) * psi

    def strang(self, psi, tau):
        psi = self.kinetic(psi, 0.5 * tau)
        psi = self.potential_step(psi, tau)
        return self.kinetic(psi, 0.5 * tau)

    def step(self, psi, tau, order=2):
        if order == 2:
            return self.strang(psi, tau)
        if order == 4:
            psi = self.strang(psi, YOSHIDA_W1 * tau)
            psi = self.strang(psi, YOSHIDA_W0 * tau)
            return self.strang(psi, YOSHIDA_W1 * tau)
        raise ValueError("order must be 2 or 4")

    def mass(self, psi):
        return float(np.prod(self.grid.h)) * float(np.sum(np.abs(psi) ** 2))

    def energy(self, psi):
        """E of Eq. (energy): kinetic by Parseval, potential, (1/2)(g rho + beta Phi) rho."""
        hv = float(np.prod(self.grid.h))
        ph = np.fft.fftn(psi)
        ekin = 0.5 * hv * float(np.sum(self.mu2 * np.abs(ph) ** 2)) / psi.size
        rho = np.abs(psi) ** 2
        Phi = self.pot(rho)
        return ekin + hv * float(np.sum(self.V * rho)) + 0.5 * hv * float(np.sum((self.g * rho + self.beta * Phi) * rho))
