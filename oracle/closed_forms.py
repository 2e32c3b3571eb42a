"""Continuum closed forms for Gaussian densities (oracle tier O3).

  3D Coulomb, rho = exp(-|x|^2/s^2):      Eq. (DensGaus) first line (erf form).
  3D Coulomb, rho = exp(-sum x_a^2/a_a^2): generalisation of Eq. (DensGaus) second
      line to three widths (substitute s = sigma^2 t there):
      u = (a1 a2 a3 / 4) int_0^inf exp(-sum x_a^2/(a_a^2+s)) / sqrt(prod (a_a^2+s)) ds.
  3D dipolar (axis n), reading U-hat = 3(n.k)^2/|k|^2 - 1:  u = -rho - 3 d_nn u_Cou,
      d_nn taken under the integral sign.
  2D Coulomb, rho = exp(-|x|^2/s^2):      Eq. (2.5D-clb-exact) first line (I0 form, via i0e).
  2D Poisson, rho = exp(-|x|^2/s^2):      Eq. (eg-2d-Exact) (E1 form).
  1D Poisson (U = -|x|/2, Sec. 2.2, 1D case), rho = exp(-(x-c)^2/a^2): integrating
      -(1/2) int |x - y| rho(y) dy (its second derivative is -rho, its first is
      -(a sqrt(pi)/2) erf((x-c)/a)) gives -(a^2/2) [t sqrt(pi) erf(t) + exp(-t^2)], t = (x-c)/a.
Sums of shifted Gaussians follow by superposition.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special

EULER_GAMMA = 0.57721566490153286061


def coulomb3d_iso(r, s):
    """sigma^3 sqrt(pi) erf(r/sigma) / (4 r); value sigma^2/2 at r = 0."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    nz = r > 0
    out[nz] = s ** 3 * math.sqrt(math.pi) * special.erf(r[nz] / s) / (4.0 * r[nz])
    out[~nz] = 0.5 * s * s
    return out


def _tri_integrand_t(t, X, a, aref, dn=None):
    """Integrand of the triaxial formula after s = aref^2 (1/t^2 - 1), t in (0,1]:
    ds / sqrt(prod(a^2+s)) = 2 aref^2 dt / prod sqrt(aref^2 + (a^2 - aref^2) t^2)."""
    c = [(aref * aref + (ai * ai - aref * aref) * t * t) for ai in a]   # (a^2+s) t^2
    q = sum(x * x * t * t / ci for x, ci in zip(X, c))
    base = 2.0 * aref * aref / math.sqrt(c[0] * c[1] * c[2]) if np.isscalar(t) else \
        2.0 * aref * aref / np.sqrt(c[0] * c[1] * c[2])
    e = np.exp(-q)
    if dn is None:
        return base * e
    # d_nn exp(-sum x^2/(a^2+s)) with a^2+s = c/t^2
    g = sum(nv * 2.0 * x * t * t / ci for nv, x, ci in zip(dn, X, c))
    lap = sum(nv * nv * 2.0 * t * t / ci for nv, ci in zip(dn, c))
    return base * e * (g * g - lap)


def coulomb3d_triaxial(X, Y, Z, a, nq=600, dn=None):
    """Triaxial formula by Gauss-Legendre in t (vectorised over points).
    With dn given, returns d_nn of the potential instead."""
    aref = min(a)
    t, wt = np.polynomial.legendre.leggauss(nq)
    t = 0.5 * (t + 1.0)
    wt = 0.5 * wt
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros_like(X)
    pre = a[0] * a[1] * a[2] / 4.0
    for ti, wi in zip(t, wt):
        out += wi * _tri_integrand_t(ti, (X, Y, Z), a, aref, dn)
    return pre * out


def coulomb3d_triaxial_quad(x, a, dn=None):
    """Same integral at one point by adaptive quadrature (scipy.integrate.quad)."""
    aref = min(a)
    f = lambda t: _tri_integrand_t(t, x, a, aref, dn)
    val, _ = integrate.quad(f, 0.0, 1.0, epsabs=1e-15, epsrel=1e-13, limit=400)
    return a[0] * a[1] * a[2] / 4.0 * val


def dipole3d_triaxial(X, Y, Z, a, axis=(0.0, 0.0, 1.0), nq=600):
    """u_dip = -rho - 3 d_nn u_Cou for rho = exp(-sum x^2/a^2)."""
    nv = np.asarray(axis, dtype=np.float64)
    nv = nv / np.linalg.norm(nv)
    rho = np.exp(-(X * X / a[0] ** 2 + Y * Y / a[1] ** 2 + Z * Z / a[2] ** 2))
    return -rho - 3.0 * coulomb3d_triaxial(X, Y, Z, a, nq=nq, dn=tuple(nv))


def coulomb2d_iso(r, s):
    """(sqrt(pi) s / 2) I0(r^2/2s^2) exp(-r^2/2s^2)."""
    r = np.asarray(r, dtype=np.float64)
    return 0.5 * math.sqrt(math.pi) * s * special.i0e(r * r / (2.0 * s * s))


def poisson2d_iso(r, s):
    """-(s^2/4) [E1(r^2/s^2) + 2 ln r]; value (s^2/4)(gamma - 2 ln s) at r = 0."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    nz = r > 0
    out[nz] = -0.25 * s * s * (special.exp1(r[nz] ** 2 / (s * s)) + 2.0 * np.log(r[nz]))
    out[~nz] = 0.25 * s * s * (EULER_GAMMA - 2.0 * math.log(s))
    return out


def rel_linf(u, ref):
    """Relative L-infinity error e_h of Eq. (error_infty)."""
    return float(np.max(np.abs(u - ref)) / np.max(np.abs(ref)))


def confined2d_W1(k, eps):
    """W_1(k) = |k| U-hat_Con(k) of the 2D confined Coulomb kernel (Eqs. (Kernal124d), (2Dw1)):
    (2/pi) int_0^inf exp(-eps^2 k^2 s^2 / 2) / (1 + s^2) ds = exp(a) erfc(sqrt(a)), a = eps^2 k^2 / 2,
    i.e. erfcx(eps |k| / sqrt 2) (the integral of exp(-a s^2)/(1 + s^2) is a classical one)."""
    return special.erfcx(eps * np.asarray(k, dtype=np.float64) / math.sqrt(2.0))


def confined2d_W1_quad(k, eps):
    """The same integral by adaptive quadrature (the paper's route, Gauss-Kronrod)."""
    from scipy import integrate
    f = lambda s: math.exp(-0.5 * (eps * k * s) ** 2) / (1.0 + s * s)
    return 2.0 / math.pi * integrate.quad(f, 0.0, np.inf, epsabs=1e-15, epsrel=1e-14, limit=400)[0]


def confined2d_gaussian(r, sigma, eps):
    """Confined Coulomb potential of rho = exp(-|x|^2 / sigma^2) in 2D, by the radial inverse
    transform phi(r) = (2 pi)^{-1} int_0^inf W_1(k) rho-hat(k) J_0(k r) dk with
    rho-hat(k) = pi sigma^2 exp(-sigma^2 k^2 / 4) (adaptive quadrature, one radius at a time)."""
    from scipy import integrate
    out = np.empty(np.shape(r))
    for i, rr in enumerate(np.ravel(r)):
        f = lambda k: float(confined2d_W1(k, eps)) * math.exp(-0.25 * sigma * sigma * k * k) * special.j0(k * rr)
        kmax = 2.0 * math.sqrt(math.log(1e18)) / sigma
        out.flat[i] = 0.5 * sigma * sigma * integrate.quad(f, 0.0, kmax, epsabs=1e-15, epsrel=1e-13, limit=800)[0]
    return out


def poisson1d_gaussian(x, a, c=0.0):
    """-(1/2) int |x - y| exp(-(y-c)^2/a^2) dy = -(a^2/2) [t sqrt(pi) erf(t) + exp(-t^2)], t = (x-c)/a."""
    t = (np.asarray(x, dtype=np.float64) - c) / a
    return -0.5 * a * a * (t * math.sqrt(math.pi) * special.erf(t) + np.exp(-t * t))


def poisson1d_gaussian_quad(x, a, c=0.0):
    """The same convolution by adaptive quadrature (split at the kink y = x)."""
    f = lambda y: abs(x - y) * math.exp(-((y - c) / a) ** 2)
    lo, hi = c - 40.0 * a, c + 40.0 * a
    pts = [p for p in (x,) if lo < p < hi]
    v = integrate.quad(f, lo, hi, points=pts or None, limit=400, epsabs=0, epsrel=1e-13)[0]
    return -0.5 * v
