"""Pins for the oracle's quadrature, spreading function and plain NUFFT (CPU)."""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads as W
from oracle import es_kernel, nufft, quadrature


@pytest.mark.parametrize("n", [4, 9, 32, 144])
def test_gauss_legendre_exact_for_polynomials(n):
    # degree 2n-1 polynomials are integrated exactly: int_0^P t^m dt = P^{m+1}/(m+1)
    P = 3.7
    t, w = quadrature.gauss_legendre(n, 0.0, P)
    for m in range(0, 2 * n, max(1, (2 * n) // 12)):
        exact = P ** (m + 1) / (m + 1)
        assert abs(np.dot(w, t ** m) - exact) <= (1e-14 * (m + 1) + 1e-14) * exact  # t^m amplifies node rounding by m


def test_sphere_rule_measures_and_symmetry():
    P = 2.5
    k, w, r = quadrature.sphere_rule(P, 8, 6, 10)
    # sum of dr du dphi weights = P * 2 * 2pi ; with the Jacobian r^2: ball volume
    assert abs(w.sum() - P * 4.0 * math.pi) < 1e-12
    assert abs((w * r * r).sum() - 4.0 / 3.0 * math.pi * P ** 3) < 1e-12
    assert np.allclose(np.linalg.norm(k, axis=1), r, atol=1e-14)
    # symmetric under k -> -k: every node has its mirror with the same weight
    kw = {tuple(np.round(kk, 12)): ww for kk, ww in zip(k, w)}
    for kk, ww in zip(k, w):
        assert abs(kw[tuple(np.round(-kk, 12) + 0.0)] - ww) < 1e-15


def test_polar_rule_measures():
    P = 1.7
    k, w, r = quadrature.polar_rule(P, 12, 16)
    assert abs(w.sum() - 2.0 * math.pi * P) < 1e-12
    assert abs((w * r).sum() - math.pi * P * P) < 1e-12     # disc area with Jacobian r


@pytest.mark.parametrize("tol", [1e-6, 1e-12, 1e-14])
def test_es_fourier_transform_vs_adaptive_quadrature(tol):
    w, beta = es_kernel.es_params(tol)
    for xi in [0.0, 0.3, 1.2, math.pi / 2]:
        ref, _ = integrate.quad(lambda z: float(es_kernel.es_phi(np.array([z]), w, beta)[0]) * math.cos(xi * z),
                                -w / 2, w / 2, epsabs=1e-15, epsrel=1e-14, limit=200)
        got = float(es_kernel.es_ft(np.array([xi]), w, beta)[0])
        assert abs(got - ref) <= 1e-13 * abs(ref)


def _random_nodes(rng, M, d, h):
    # cover the whole periodic range including both ends (wrap-around taps)
    t = rng.uniform(-math.pi, math.pi, size=(M, d))
    t[:4] = math.pi * np.array([[1, -1, 1][:d], [-1, 1, -1][:d], [0.999999, 0, 0][:d], [0, 0, 0][:d]])
    return t / np.asarray(h)[None, :]


@pytest.mark.parametrize("d,n", [(2, (12, 10)), (3, (8, 10, 6))])
@pytest.mark.parametrize("tol", [1e-6, 1e-12])
def test_nufft_types_match_direct_sums(d, n, tol):
    rng = np.random.default_rng(1)
    h = tuple(0.3 + 0.1 * a for a in range(d))
    k = _random_nodes(rng, 300, d, h)
    rho = rng.standard_normal(n)
    a = nufft.direct_type2(rho, h, k)
    b = nufft.type2(rho, h, k, tol)
    scale = float(np.prod(h)) * np.abs(rho).sum()
    assert np.max(np.abs(a - b)) <= 10 * tol * scale
    c = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    g_ref = nufft.direct_type1_real(c, k, n, h)
    g = np.real(nufft.type1(c, k, n, h, tol))
    assert np.max(np.abs(g - g_ref)) <= 10 * tol * np.abs(c).sum()


def test_direct_type2_closed_form_single_mode():
    # rho = a single grid cosine: its trapezoid transform at k is a geometric sum
    n, L = 16, 3.0
    g = W.cube(n, L, 1)
    x = g.axes()[0]
    q = 3 * math.pi / L          # on the grid's Fourier lattice (pi p / L)
    rho = np.cos(q * x)
    kk = np.array([[q], [q + 0.37], [0.0]])
    got = nufft.direct_type2(rho, g.h, kk)
    h = g.h[0]
    for j, kv in enumerate(kk[:, 0]):
        ref = h * sum(np.cos(q * xi) * np.exp(-1j * kv * xi) for xi in x)
        assert abs(got[j] - ref) < 1e-13
    assert abs(got[0] - n * h / 2.0) < 1e-13    # orthogonality: sum cos^2 = n/2
