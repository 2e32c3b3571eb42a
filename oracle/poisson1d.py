"""1D Poisson potential (Sec. 2.2, the 1D case) -- oracle, test infrastructure only.

phi = U_Lap * rho with U_Lap(x) = -|x|/2 (Eq. (Kernal21d), d = 1), evaluated the way the
paper describes for 1D: a Gaussian G_1 carrying the mass and the first moment of rho is
split off, its potential u_1 is taken in closed form, and the remainder u_2, whose
Fourier integrand W(k) is smooth at k = 0, is integrated by the regular FFT quadrature.
Only tests/, the smoke check and bench.py's CPU baseline use this module.

Steps, in the paper's order (plain FP64, direct sums instead of FFTs):
  1. rho-hat(0) = C0, (x rho)-hat(0) = M1, (x^2 rho)-hat(0) = M2: trapezoid sums on the grid.
  2. u_1 = C0 u_{1,1} - M1 u_{1,2} (Eq. (1DPois) and its solution by convolution), with
       u_{1,1}(x) = -sigma/sqrt(2 pi) exp(-x^2/(2 sigma^2)) - (x/2) erf(x/(sqrt(2) sigma)),
       u_{1,2}(x) = u_{1,1}'(x) = -(1/2) erf(x/(sqrt(2) sigma)).
  3. W(k) = (rho-hat(k) - (C0 - i k M1) exp(-k^2 sigma^2/2)) / k^2 for k != 0 and
     W(0) = -M2/2 + sigma^2 C0/2 (rho-hat(k) by the trapezoid sum, rho-hat'(0) = -i M1).
  4. u_2(x) = (1/2 pi) int_{-P}^{P} W(k) exp(i k x) dk by the rectangle rule.
  5. phi = u_1 + u_2.

Readings (the paper gives the formulas, not the discretisation):
  - grid x_m = -L + m h, h = 2L/n (as in 2D/3D);
  - the "regular FFT method" of step 4 is the rectangle rule on the frequencies of the
    zero-padded 2n-point grid, k_l = l pi/(n h), l = -n..n-1 (spacing pi/(n h)); with P = pi/h
    (default) this is every such frequency, with a smaller P the terms |k_l| > P are dropped;
  - sigma = 6 sqrt(2)/P, the choice of the 2D case ("similar as in the 2D case").
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def u11(x, sigma):
    """U_Lap * G for the unit-mass Gaussian G of width sigma (the closed form after Eq. (1DPois))."""
    x = np.asarray(x, dtype=np.float64)
    return (-sigma / math.sqrt(2.0 * math.pi) * np.exp(-x * x / (2.0 * sigma * sigma))
            - 0.5 * x * special.erf(x / (math.sqrt(2.0) * sigma)))


def u12(x, sigma):
    """u_{1,1}'(x) = -(1/2) erf(x / (sqrt(2) sigma))."""
    x = np.asarray(x, dtype=np.float64)
    return -0.5 * special.erf(x / (math.sqrt(2.0) * sigma))


def params(n: int, L: float, P: float | None = None):
    """(h, P, sigma, k_l) of an n-point grid on [-L, L)."""
    h = 2.0 * L / n
    if P is None or P <= 0:
        P = math.pi / h
    P = min(P, math.pi / h)
    sigma = 6.0 * math.sqrt(2.0) / P
    k = np.arange(-n, n, dtype=np.float64) * (math.pi / (n * h))
    return h, P, sigma, k


def W_of_k(rhohat, k, C0, M1, M2, sigma):
    """Step 3: the smooth Fourier integrand of u_2."""
    W = np.empty(k.shape, dtype=np.complex128)
    nz = k != 0
    kk = k[nz]
    W[nz] = (rhohat[nz] - (C0 - 1j * kk * M1) * np.exp(-0.5 * kk * kk * sigma * sigma)) / (kk * kk)
    W[~nz] = -0.5 * M2 + 0.5 * sigma * sigma * C0
    return W


def poisson1d(rho, L: float, P: float | None = None, return_parts: bool = False):
    """phi on the grid x_m = -L + m h for the 1D density rho (length n)."""
    rho = np.asarray(rho, dtype=np.float64)
    n = rho.shape[0]
    h, P, sigma, k = params(n, L, P)
    x = -L + h * np.arange(n, dtype=np.float64)
    # 1. moments
    C0 = h * rho.sum()
    M1 = h * (x * rho).sum()
    M2 = h * (x * x * rho).sum()
    # 2. u_1 in closed form
    u1 = C0 * u11(x, sigma) - M1 * u12(x, sigma)
    # 3. W(k_l) from the trapezoid rho-hat (direct sum)
    rhohat = h * (np.exp(-1j * np.outer(k, x)) @ rho)
    W = W_of_k(rhohat, k, C0, M1, M2, sigma)
    W[np.abs(k) > P] = 0.0
    # 4. u_2 by the rectangle rule in k (direct sum)
    dk = math.pi / (n * h)
    u2 = (dk / (2.0 * math.pi)) * np.real(np.exp(1j * np.outer(x, k)) @ W)
    phi = u1 + u2
    if return_parts:
        return phi, dict(u1=u1, u2=u2, C0=C0, M1=M1, M2=M2, sigma=sigma, P=P, W=W, k=k)
    return phi
