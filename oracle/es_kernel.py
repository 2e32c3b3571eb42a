"""Spreading function for the oracle's plain NUFFT.

The paper gives no NUFFT internals (it cites them).  The oracle uses the
"exponential of semicircle" function of Barnett, Magland & af Klinteberg
(SIAM J. Sci. Comput. 41, 2019), with upsampling factor 2:
    phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)),  |z| < w/2   (z in fine cells)
    w = ceil(log10(1/tol)) + 1,  beta = 2.30 w.
Its Fourier transform psi-hat(xi) = int phi(z) e^{-i xi z} dz is computed by
Gauss-Legendre quadrature (phi is even, so only the cosine part survives).
"""
from __future__ import annotations

import math

import numpy as np


def es_params(tol: float):
    w = int(math.ceil(math.log10(1.0 / tol))) + 1
    w = max(2, min(w, 16))
    return w, 2.30 * w


def es_phi(z, w: int, beta: float):
    x = 2.0 * np.asarray(z, dtype=np.float64) / w
    out = np.zeros_like(x)
    m = np.abs(x) < 1.0
    out[m] = np.exp(beta * (np.sqrt(1.0 - x[m] ** 2) - 1.0))
    return out


def es_ft(xi, w: int, beta: float, nq: int = 100):
    """psi-hat(xi) = int_{-w/2}^{w/2} phi(z) cos(xi z) dz.  With z = (w/2) sin(theta)
    the square-root endpoint behaviour of phi disappears:
        psi-hat(xi) = w int_0^{pi/2} exp(beta (cos theta - 1)) cos(xi (w/2) sin theta) cos theta dtheta,
    a smooth integrand, integrated by nq-point Gauss-Legendre."""
    x, wx = np.polynomial.legendre.leggauss(nq)
    th = 0.25 * math.pi * (x + 1.0)
    wth = 0.25 * math.pi * wx
    f = np.exp(beta * (np.cos(th) - 1.0)) * np.cos(th)
    xi = np.asarray(xi, dtype=np.float64)
    return w * np.cos(np.multiply.outer(xi, 0.5 * w * np.sin(th))) @ (wth * f)
