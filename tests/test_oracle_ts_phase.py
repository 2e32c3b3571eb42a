"""Phase-sensitive pins for the oracle's time splitting (Sec. 4.1, Eqs. (sps-eq65)-(sps-eq68)).

Mass conservation and the temporal order do not fix the sign of either sub-step: with real
initial data, running the potential step as exp(+i ...) or evolving the conjugate equation
(both signs flipped) leaves |psi| and the order unchanged.  These tests pin the signs of
i psi_t = (-Delta/2 + V + beta Phi) psi (the NLSE of Sec. 1) against facts the equation
itself fixes:

  * a free Gaussian packet exp(-|x|^2/2 + i k0.x) moves towards +k0 and has the closed form
    prod_d (1 + i t)^{-1/2} exp(-(x_d - k0_d t)^2 / (2 (1 + i t)) + i k0_d x_d - i k0_d^2 t / 2);
  * a displaced ground state of V = |x|^2/2 is a coherent state with the closed form
    prod_d pi^{-1/4} exp(-(x_d - c_d cos t)^2/2 - i x_d c_d sin t + i c_d^2 sin(2t)/4 - i t/2);
  * the energy E of Sec. 1 is conserved by the flow, so the splitting keeps it to O(tau^2)
    (Strang) or O(tau^4) (Yoshida), while a flipped potential sign flows with a different
    Hamiltonian and does not.

Each plausible slip (potential sign, kinetic sign, conjugate evolution) is planted in a
subclass of the oracle and must fail at least one pin.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import potential, ts


def free_packet(grid, k0, t):
    X = grid.mesh()
    psi = np.ones(grid.n, dtype=np.complex128)
    a = 1.0 + 1j * t
    for x, k in zip(X, k0):
        psi *= a ** -0.5 * np.exp(-(x - k * t) ** 2 / (2.0 * a) + 1j * k * x - 0.5j * k * k * t)
    return psi


def coherent_state(grid, c, t):
    X = grid.mesh()
    psi = np.ones(grid.n, dtype=np.complex128)
    for x, cd in zip(X, c):
        psi *= math.pi ** -0.25 * np.exp(-(x - cd * math.cos(t)) ** 2 / 2.0 - 1j * x * cd * math.sin(t)
                                         + 0.25j * cd * cd * math.sin(2.0 * t) - 0.5j * t)
    return psi


class PotentialSignFlipped(ts.TimeSplitting):
    """Planted mistake: potential sub-step exp(+i (V + ...) s)."""

    def potential_step(self, psi, s):
        return super().potential_step(psi, -s)


class KineticSignFlipped(ts.TimeSplitting):
    """Planted mistake: kinetic sub-step exp(+i s |mu|^2 / 2) in Fourier space."""

    def kinetic(self, psi, s):
        return super().kinetic(psi, -s)


class ConjugateEvolution(ts.TimeSplitting):
    """Planted mistake: both signs flipped (the conjugate equation)."""

    def potential_step(self, psi, s):
        return super().potential_step(psi, -s)

    def kinetic(self, psi, s):
        return super().kinetic(psi, -s)


MISTAKES = (PotentialSignFlipped, KineticSignFlipped, ConjugateEvolution)
GRID = W.cube(128, 16.0, 2)
K0 = (1.0, -0.5)
C0 = (2.0, -1.0)


def _zero_potential(rho):
    return np.zeros_like(rho)


def free_packet_error(cls):
    """max |psi - exact| at t = 1 for the free packet (V = 0, beta = 0), and the centre of mass."""
    S = cls(GRID, np.zeros(GRID.n), 0.0, _zero_potential)
    psi = free_packet(GRID, K0, 0.0)
    for _ in range(10):
        psi = S.step(psi, 0.1, 2)
    rho = np.abs(psi) ** 2
    centre = [float(np.sum(x * rho) / np.sum(rho)) for x in GRID.mesh()]
    return float(np.max(np.abs(psi - free_packet(GRID, K0, 1.0)))), centre


def coherent_error(cls, tau, order):
    S = cls(GRID, W.harmonic_trap(GRID, (1.0, 1.0)), 0.0, _zero_potential)
    psi = coherent_state(GRID, C0, 0.0)
    for _ in range(int(round(1.0 / tau))):
        psi = S.step(psi, tau, order)
    return float(np.max(np.abs(psi - coherent_state(GRID, C0, 1.0))))


_EG = W.cube(64, 8.0, 2)
_EOP = potential.ConvolutionOperator(_EG, "coulomb2d", math.pi / _EG.h[0])


def energy_drift(cls, tau, order):
    """max_t |E(t) - E(0)| / |E(0)| over t <= 1/2 for a moving packet in a trap with the 2D
    Coulomb potential (beta = 5)."""
    X, Y = _EG.mesh()
    psi = W.gaussian(_EG, [1.2, 1.2], center=(0.5, -0.3)) * np.exp(1j * (0.8 * X - 0.4 * Y))
    S = cls(_EG, W.harmonic_trap(_EG, (1.0, 1.0)), 5.0, _EOP)
    E0 = S.energy(psi)
    drift = 0.0
    for _ in range(int(round(0.5 / tau))):
        psi = S.step(psi, tau, order)
        drift = max(drift, abs(S.energy(psi) - E0))
    return drift / abs(E0)


def test_free_packet_matches_closed_form():
    err, centre = free_packet_error(ts.TimeSplitting)
    # the kinetic flow is exact in time for a trigonometric interpolant: only the spatial
    # truncation of the Gaussian on the box is left
    assert err < 1e-11, err
    assert np.allclose(centre, K0, atol=1e-9), centre


@pytest.mark.parametrize("order,tau,bound,ratio", [(2, 0.02, 2e-4, 4.0), (4, 0.05, 3e-6, 16.0)])
def test_coherent_state_matches_closed_form(order, tau, bound, ratio):
    e1 = coherent_error(ts.TimeSplitting, tau, order)
    e2 = coherent_error(ts.TimeSplitting, tau / 2, order)
    assert e1 < bound, e1
    assert 0.75 * ratio < e1 / e2 < 1.4 * ratio, (e1, e2)


@pytest.mark.parametrize("order,tau,bound,ratio", [(2, 0.02, 6e-5, 4.0), (4, 0.05, 5e-6, 16.0)])
def test_energy_conserved_to_the_splitting_order(order, tau, bound, ratio):
    d1 = energy_drift(ts.TimeSplitting, tau, order)
    d2 = energy_drift(ts.TimeSplitting, tau / 2, order)
    assert d1 < bound, d1
    assert 0.75 * ratio < d1 / d2 < 1.4 * ratio, (d1, d2)


@pytest.mark.parametrize("mistake", MISTAKES, ids=lambda c: c.__name__)
def test_planted_sign_mistakes_fail_a_pin(mistake):
    failed = []
    err, centre = free_packet_error(mistake)
    if err > 1e-3 or not np.allclose(centre, K0, atol=1e-3):
        failed.append("free packet")
    if coherent_error(mistake, 0.02, 2) > 1e-2:
        failed.append("coherent state")
    if energy_drift(mistake, 0.02, 2) > 1e-3:
        failed.append("energy")
    assert failed, mistake.__name__
    # the conjugate evolution conserves E (time reversal): only the closed forms catch it
    if mistake is ConjugateEvolution:
        assert "coherent state" in failed and "free packet" in failed
