"""Pins of the 1D Poisson oracle (Sec. 2.2, the 1D case) -- CPU only.

The oracle (oracle/poisson1d.py) is pinned to the continuum closed form of Gaussian
densities (itself checked against adaptive quadrature of the defining convolution), to the
defining properties of u_{1,1} and u_{1,2} (Eq. (1DPois)), to the k -> 0 limit that defines
W(0), and to superposition; three planted mistakes each fail a pin.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import poisson1d as p1


def _grid(n, L):
    return W.cube(n, L, dim=1).axes()[0]


@pytest.mark.parametrize("n,L,a,c", [(512, 16.0, 1.0, 0.0), (512, 16.0, 0.7, 1.3), (256, 16.0, 1.5, -2.0),
                                     (1024, 16.0, 0.5, 0.25), (64, 8.0, 1.0, 0.5)])
def test_gaussian_matches_closed_form(n, L, a, c):
    x = _grid(n, L)
    rho = np.exp(-((x - c) / a) ** 2)
    phi = p1.poisson1d(rho, L)
    ex = cf.poisson1d_gaussian(x, a, c)
    assert cf.rel_linf(phi, ex) < 1e-13


def test_closed_form_matches_quadrature_of_the_convolution():
    for a, c in [(1.0, 0.0), (0.7, 1.3), (2.0, -0.5)]:
        for x in (-5.0, -0.3, 0.0, 0.9, 4.0):
            assert abs(cf.poisson1d_gaussian(x, a, c) - cf.poisson1d_gaussian_quad(x, a, c)) < 1e-11 * a * a * (1 + abs(x))


def test_u11_u12_solve_the_auxiliary_problem():
    """-u11'' = G (unit-mass Gaussian), u12 = u11', u11 + |x|/2 -> 0 (Eq. (1DPois) with C0 = 1, M1 = 0)."""
    sigma = 0.37
    x = np.linspace(-3.0, 3.0, 61)
    d = 1e-3
    G = np.exp(-x * x / (2 * sigma * sigma)) / (math.sqrt(2 * math.pi) * sigma)
    d2 = (p1.u11(x + d, sigma) - 2 * p1.u11(x, sigma) + p1.u11(x - d, sigma)) / (d * d)
    assert np.max(np.abs(-d2 - G)) < 1e-5 * np.max(G)
    d1 = (p1.u11(x + d, sigma) - p1.u11(x - d, sigma)) / (2 * d)
    assert np.max(np.abs(d1 - p1.u12(x, sigma))) < 1e-6
    far = np.array([-20.0, -12.0, 12.0, 20.0]) * sigma
    assert np.max(np.abs(p1.u11(far, sigma) + 0.5 * np.abs(far))) < 1e-12
    # the far-field of u_1 = C0 u11 - M1 u12 is -(C0 |x| -/+ M1)/2
    C0, M1 = 1.7, -0.4
    for xx, s in ((25.0, 1), (-25.0, -1)):
        u1 = C0 * p1.u11(xx, sigma) - M1 * p1.u12(xx, sigma)
        assert abs(u1 + 0.5 * (C0 * abs(xx) - s * M1)) < 1e-12


@pytest.mark.parametrize("a,c", [(1.0, 0.0), (0.8, 1.5), (1.3, -2.0)])
def test_W0_is_the_limit_of_W(a, c):
    """With the analytic transform of exp(-(x-c)^2/a^2) and its exact moments M_j = int x^j rho,
    rho-hat(k) = C0 - i k M1 - k^2 M2/2 + i k^3 M3/6 + ..., so
    W(k) = W(0) + i k (M3/6 - sigma^2 M1/2) + O(k^2): the real part tends to W(0) and the
    imaginary part is linear in k with that slope."""
    C0 = a * math.sqrt(math.pi)
    M1 = c * C0
    M2 = (c * c + 0.5 * a * a) * C0
    M3 = (c ** 3 + 1.5 * c * a * a) * C0
    sigma = 0.3
    k = np.array([0.0, 1e-4, -1e-4, 3e-4])
    rhohat = C0 * np.exp(-0.25 * a * a * k * k) * np.exp(-1j * k * c)
    Wk = p1.W_of_k(rhohat, k, C0, M1, M2, sigma)
    W0 = Wk[0].real
    assert abs(W0 - (-0.5 * M2 + 0.5 * sigma * sigma * C0)) == 0.0
    assert np.max(np.abs(Wk[1:].real - W0)) < 1e-6 * abs(W0)
    slope = M3 / 6.0 - 0.5 * sigma * sigma * M1
    assert np.max(np.abs(Wk[1:].imag / k[1:] - slope)) < 1e-3 * max(1.0, abs(slope))


def test_three_gaussians_superposition():
    cs, ws, amps = W.three_gaussians_1d(W.SEED_TRAIN)
    n, L = 1024, 16.0
    x = _grid(n, L)
    rho = np.zeros(n)
    ex = np.zeros(n)
    for (c,), s, a in zip(cs, ws, amps):
        rho += a * np.exp(-((x - c) / s) ** 2)
        ex += a * cf.poisson1d_gaussian(x, s, c)
    assert cf.rel_linf(p1.poisson1d(rho, L), ex) < 1e-13


def test_linearity_and_translation():
    n, L = 256, 12.0
    x = _grid(n, L)
    h = 2 * L / n
    r1 = np.exp(-((x - 1.0) / 0.9) ** 2)
    r2 = np.exp(-((x + 2.0) / 1.4) ** 2)
    assert cf.rel_linf(p1.poisson1d(2 * r1 + r2, L), 2 * p1.poisson1d(r1, L) + p1.poisson1d(r2, L)) < 1e-13
    # shifting rho by one cell shifts phi by one cell (away from the box edge)
    phi = p1.poisson1d(r1, L)
    phis = p1.poisson1d(np.exp(-((x - 1.0 - h) / 0.9) ** 2), L)
    assert np.max(np.abs(phis[1:] - phi[:-1])) < 1e-12 * np.max(np.abs(phi))


def _gauss_err(monkeypatch=None):
    n, L, a, c = 512, 16.0, 0.8, 1.1
    x = _grid(n, L)
    return cf.rel_linf(p1.poisson1d(np.exp(-((x - c) / a) ** 2), L), cf.poisson1d_gaussian(x, a, c))


def test_planted_mistakes_fail(monkeypatch):
    assert _gauss_err() < 1e-13
    orig_W, orig_u11 = p1.W_of_k, p1.u11
    # (a) W(0) dropped
    def W_no0(rhohat, k, C0, M1, M2, sigma):
        w = orig_W(rhohat, k, C0, M1, M2, sigma)
        w[k == 0] = 0.0
        return w
    monkeypatch.setattr(p1, "W_of_k", W_no0)
    assert _gauss_err() > 1e-6
    # (b) sign of the first-moment term flipped
    monkeypatch.setattr(p1, "W_of_k", lambda rh, k, C0, M1, M2, s: orig_W(rh, k, C0, -M1, M2, s))
    assert _gauss_err() > 1e-6
    monkeypatch.setattr(p1, "W_of_k", orig_W)
    # (c) u_1 built with a Gaussian of another width than the one subtracted in W
    monkeypatch.setattr(p1, "u11", lambda x, s: orig_u11(x, 1.5 * s))
    assert _gauss_err() > 1e-6
