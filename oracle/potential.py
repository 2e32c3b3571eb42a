"""phi = U * rho by the paper's quadrature (oracle tiers O1 and O2).

The quantity the method computes (Sec. 2.1, Eq. (ifft)), for grid points x_i:
    rho-hat_j = (prod h) sum_i rho_i exp(-i k_j . x_i)               (trapezoid)
    phi_i     = (2 pi)^{-d} Re sum_j w_j J(k_j) rho-hat_j exp(i k_j . x_i)
with {k_j, w_j} the spherical/polar rule of oracle.quadrature and J = |k|^{d-1}
U-hat(k) the Jacobian-weighted symbol:
    coulomb3d  U-hat = 1/|k|^2                 (Eq. (Kernal))      J = 1
    coulomb2d  U-hat = 1/|k|                   (Eq. (Kernal))      J = 1
    dipole3d   U-hat = 3 (n.k)^2/|k|^2 - 1      (reading: the paper only names
               the dipolar kernel; this is the standard form of the cited works)
               J = 3 (n.k)^2 - |k|^2
    poisson2d  U-hat = 1/|k|^2 in 2D: Algorithm 1 (Sec. 2.2, Eqs. (GG1)-(phi2fourier)).
    confined2d the 2D confined Coulomb kernel of Eq. (Kernal124d) with parameter eps:
               J = W_1(|k|) of Eq. (2Dw1) (closed_forms.confined2d_W1)
Real part: phi is real; with the symmetric node set the imaginary part is rounding.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import fft as sfft
from scipy import special

from . import nufft, quadrature

EULER_GAMMA = 0.57721566490153286061

KERNELS = ("coulomb3d", "dipole3d", "coulomb2d", "poisson2d", "confined2d")
DIM = {"coulomb3d": 3, "dipole3d": 3, "coulomb2d": 2, "poisson2d": 2, "confined2d": 2}


def node_set(kernel: str, P: float, counts, dipole_axis=(0.0, 0.0, 1.0), eps: float = 0.0):
    """Nodes k (M x d), plain weights wq, radii r, and Jacobian-weighted
    weights wq * J(k) (for poisson2d J is applied inside Algorithm 1)."""
    if DIM[kernel] == 3:
        k, wq, r = quadrature.sphere_rule(P, *counts)
        if kernel == "coulomb3d":
            J = np.ones_like(r)
        else:
            nv = np.asarray(dipole_axis, dtype=np.float64)
            nv = nv / np.linalg.norm(nv)
            J = 3.0 * (k @ nv) ** 2 - r * r
    else:
        k, wq, r = quadrature.polar_rule(P, *counts)
        if kernel == "confined2d":
            from .closed_forms import confined2d_W1
            J = confined2d_W1(r, eps)
        else:
            J = np.ones_like(r)
    return k, wq, r, wq * J


def _transforms(method: str, tol: float):
    if method == "direct":
        return (lambda rho, h, k: nufft.direct_type2(rho, h, k),
                lambda c, k, n, h: nufft.direct_type1_real(c, k, n, h))
    if method == "nufft":
        return (lambda rho, h, k: nufft.type2(rho, h, k, tol),
                lambda c, k, n, h: np.real(nufft.type1(c, k, n, h, tol)))
    raise ValueError(method)


def poisson2d_sigma(P: float) -> float:
    """Width of the auxiliary Gaussian G (Eq. (GG1)).  The printed choice
    sigma = 6/P does not give the stated 2e-16 at |k| = P for exp(-sigma^2 k^2/2);
    reading: sigma = 6 sqrt(2)/P, for which exp(-sigma^2 P^2/2) = e^{-36}."""
    return 6.0 * math.sqrt(2.0) / P


def u1_parts(X, Y, sigma: float):
    """u_{1,1} (Eq. (phi1_exct)) and u_{1,2} = grad u_{1,1} (Eq. (phi12_ext)) on the grid."""
    r2 = X * X + Y * Y
    u11 = np.empty_like(r2)
    u12x = np.zeros_like(r2)
    u12y = np.zeros_like(r2)
    nz = r2 > 0.0
    z = r2[nz] / (2.0 * sigma * sigma)
    u11[nz] = -(special.exp1(z) + np.log(r2[nz])) / (4.0 * math.pi)
    u11[~nz] = (EULER_GAMMA - math.log(2.0 * sigma * sigma)) / (4.0 * math.pi)
    f = -(1.0 - np.exp(-z)) / (2.0 * math.pi * r2[nz])
    u12x[nz] = f * X[nz]
    u12y[nz] = f * Y[nz]
    return u11, u12x, u12y


def poisson2d(rho, grid, P, counts, method="nufft", tol=1e-13, sigma=None, return_parts=False, partition=None,
              sigma_u1=None):
    """Algorithm 1 (Sec. 2.2): u = u_1 + u_2.
    Step 1: rho-hat(k_j) and the moments rho-hat(0) = C0, (x rho)-hat(0) = M1 (trapezoid).
    Step 2: u_1 = C0 u_{1,1} - M1 . u_{1,2}                      (Eqs. (u2u3), (phi1_exct), (phi12_ext)).
    Step 3: u_2 = (2pi)^{-2} int_0^P int_0^{2pi} W(k) e^{ik.x} d|k| dtheta with
            W = (rho-hat - (C0 - i k.M1) e^{-sigma^2|k|^2/2}) / |k|  (Eq. (phi2fourier) and the W that follows it).
    Step 4: u = u_1 + u_2.
    For the improved algorithm (evaluate_split) the integrand of step 3 carries a partition
    factor p(|k|) and u_1 is taken with the width sigma_u1 (see evaluate_split)."""
    t2, t1 = _transforms(method, tol)
    h = grid.h
    X, Y = grid.mesh()
    hv = h[0] * h[1]
    C0 = hv * float(np.sum(rho))
    M1 = np.array([hv * float(np.sum(X * rho)), hv * float(np.sum(Y * rho))])
    if sigma is None:
        sigma = poisson2d_sigma(P)
    k, wq, r, _ = node_set("poisson2d", P, counts)
    rh = t2(rho, h, k)
    G1 = (C0 - 1j * (k @ M1)) * np.exp(-0.5 * sigma * sigma * r * r)
    W = (rh - G1) / r
    c = wq * W / (2.0 * math.pi) ** 2
    if partition is not None:
        c = c * partition(r)
    u2 = t1(c, k, grid.n, h)
    u11, u12x, u12y = u1_parts(X, Y, sigma if sigma_u1 is None else sigma_u1)
    u1 = C0 * u11 - (M1[0] * u12x + M1[1] * u12y)
    if return_parts:
        return u1 + u2, dict(C0=C0, M1=M1, sigma=sigma, u1=u1, u2=u2)
    return u1 + u2


def evaluate(rho, grid, kernel, P, counts=None, method="nufft", tol=1e-13,
             dipole_axis=(0.0, 0.0, 1.0), eps=0.0):
    """phi = U * rho on the grid (Eq. (ifft) quadrature; Algorithm 1 for poisson2d)."""
    if counts is None:
        counts = quadrature.default_counts(grid.L, P)
    if kernel == "poisson2d":
        return poisson2d(rho, grid, P, counts, method=method, tol=tol)
    t2, t1 = _transforms(method, tol)
    d = grid.dim
    k, wq, r, wj = node_set(kernel, P, counts, dipole_axis, eps)
    rh = t2(rho, grid.h, k)
    c = wj * rh / (2.0 * math.pi) ** d
    return t1(c, k, grid.n, grid.h)


def split_params(grid, P: float, eps: float = 1e-16, kappa: float = 5.5, kernel: str = "coulomb3d"):
    """Parameters of the split of Sec. 2.1 (Eq. (3.9)).  Returns (s, k2): the scale s of the
    partition of unity and the radius k2 of the ball that carries I_2.
      3D kernels and poisson2d: p(k) = exp(-|k|^2 / a), s = a.  Reading: the x-space kernel of
        I_1 (3D Coulomb: erfc(sqrt(a) |x| / 2) / (4 pi |x|); 2D Laplace: E_1(a |x|^2 / 4) / (4 pi))
        must have decayed at the doubled grid's nearest image (distance >= 2 L_min):
        a = (kappa / L_min)^2; I_2 is needed where p >= eps: k2 = min(P, sqrt(a ln(1/eps))).
      coulomb2d: p(k) = erfc(|k| / l), s = l = kappa / L_min.  The x-space kernel of I_1 is
        erfc(l |x| / 2) / (2 pi |x|), so the same kappa gives the same decay at 2 L_min;
        k2 = min(P, l erfc^{-1}(eps))."""
    Lmin = min(grid.L)
    if kernel == "coulomb2d":
        ell = kappa / Lmin
        return ell, min(P, ell * float(special.erfcinv(eps)))
    a = (kappa / Lmin) ** 2
    return a, min(P, math.sqrt(a * math.log(1.0 / eps)))


def partition(kernel: str, r, s: float):
    """The partition of unity p(|k|) of Eq. (3.9) for this kernel (see split_params)."""
    r = np.asarray(r, dtype=np.float64)
    if kernel == "coulomb2d":
        return special.erfc(r / s)
    return np.exp(-r * r / s)


def split_multiplier(kernel: str, K, a: float, dipole_axis=(0.0, 0.0, 1.0)):
    """w(k) = (1 - p(k)) U-hat(k) at wave vectors K (list of d arrays), with its limit at k = 0:
      coulomb3d, poisson2d  (1 - exp(-|k|^2/a)) / |k|^2      -> 1/a      (an entire function of |k|^2)
      dipole3d              (1 - exp(-|k|^2/a)) (3 (n.k)^2/|k|^2 - 1)  -> 0
      coulomb2d             erf(|k| / l) / |k|  (a = l)          -> 2 / (l sqrt(pi))  (entire in |k|^2)"""
    k2 = sum(k * k for k in K)
    with np.errstate(divide="ignore", invalid="ignore"):
        if kernel in ("coulomb3d", "poisson2d"):
            one_m_p = -np.expm1(-k2 / a)
            w = np.where(k2 > 0, one_m_p / k2, 1.0 / a)
        elif kernel == "dipole3d":
            one_m_p = -np.expm1(-k2 / a)
            nv = np.asarray(dipole_axis, dtype=np.float64)
            nv = nv / np.linalg.norm(nv)
            nk = sum(c * k for c, k in zip(nv, K))
            w = np.where(k2 > 0, one_m_p * (3.0 * nk * nk / k2 - 1.0), 0.0)
        elif kernel == "coulomb2d":
            kr = np.sqrt(k2)
            w = np.where(k2 > 0, special.erf(kr / a) / kr, 2.0 / (a * math.sqrt(math.pi)))
        else:
            raise ValueError(kernel)
    return w


def evaluate_split(rho, grid, kernel, P, counts2=None, tol=1e-13, eps=1e-16, kappa=5.5,
                   dipole_axis=(0.0, 0.0, 1.0), return_parts=False):
    """The improved algorithm (Sec. 2.1, Eq. (3.9)): phi = I_1 + I_2.
    I_1 = (2pi)^{-d} int w(k) rho-hat(k) e^{ik.x} dk by the rectangle rule on the frequencies of
          the doubled grid (spacing pi/L per axis) with the trapezoid rho-hat: the aperiodic
          layout x = (i - n/2) h placed at index (i - n/2) mod 2n, plain FFTs;
    I_2 = the quadrature of Eq. (ifft) on the ball |k| <= k2 with node weights multiplied by
          p(k), plain NUFFT.
    poisson2d (U-hat = 1/|k|^2, d = 2): w = (1 - p)/|k|^2 is smooth, but p/|k|^2 is not
          integrable at k = 0 in polar coordinates, so I_2 follows Algorithm 1 (Sec. 2.2): with
          G_1 of Eq. (GG1), p rho-hat = p (rho-hat - G_1-hat) + p G_1-hat; the first term is
          step 3 of Algorithm 1 with the factor p, the second is the potential of G_1 with
          the Gaussian widened to sigma_u1^2 = sigma^2 + 2/a (p G_1-hat = G_1-hat at that
          width), i.e. step 2 of Algorithm 1 with sigma_u1."""
    d = grid.dim
    a, k2 = split_params(grid, P, eps, kappa, kernel)
    n, h = grid.n, grid.h
    big = np.zeros(tuple(2 * m for m in n))
    idx = np.ix_(*[(np.arange(m) - m // 2) % (2 * m) for m in n])
    big[idx] = rho
    ks = [2.0 * math.pi * np.fft.fftfreq(2 * m, d=hh) for m, hh in zip(n, h)]
    K = np.meshgrid(*ks, indexing="ij")
    w = split_multiplier(kernel, K, a, dipole_axis)
    I1 = np.real(np.fft.ifftn(w * np.fft.fftn(big)))[idx]
    if counts2 is None:
        counts2 = quadrature.default_counts(grid.L, k2)
    extra = {}
    if kernel == "poisson2d":
        sigma = poisson2d_sigma(k2)
        sigma_u1 = math.sqrt(sigma * sigma + 2.0 / a)
        I2 = poisson2d(rho, grid, k2, counts2, method="nufft", tol=tol, sigma=sigma,
                       partition=lambda r: partition(kernel, r, a), sigma_u1=sigma_u1)
        extra = dict(sigma=sigma, sigma_u1=sigma_u1)
    else:
        t2, t1 = _transforms("nufft", tol)
        k, wq, r, wj = node_set(kernel, k2, counts2, dipole_axis)
        rh = t2(rho, h, k)
        c = wj * partition(kernel, r, a) * rh / (2.0 * math.pi) ** d
        I2 = t1(c, k, n, h)
    if return_parts:
        return I1 + I2, dict(a=a, k2=k2, I1=I1, I2=I2, counts2=counts2, **extra)
    return I1 + I2


def eval_direct(rho, grid, kernel, P, counts=None, **kw):
    """O1: exact discrete definition by direct sums (small grids only)."""
    return evaluate(rho, grid, kernel, P, counts, method="direct", **kw)


def eval_nufft(rho, grid, kernel, P, counts=None, tol=1e-13, **kw):
    """O2: plain FP64 NUFFT of the same definition."""
    return evaluate(rho, grid, kernel, P, counts, method="nufft", tol=tol, **kw)


class ConvolutionOperator:
    """The discrete operator of Eq. (ifft) for translation-invariant kernels
    (coulomb3d, dipole3d, coulomb2d) written as the exact Toeplitz sum
        phi_i = sum_{i'} K(i - i') rho_{i'},
        K(m) = (2pi)^{-d} (prod h) sum_j w_j J(k_j) cos(k_j . m h),  m in [-n, n)^d,
    (expand rho-hat in the definition and swap the finite sums).  K is built
    once by a type-1 sum onto the doubled grid; applying it is an aperiodic
    convolution by FFT of size 2n (library primitive).  Used where many
    evaluations are needed (gradient flow, time splitting)."""

    def __init__(self, grid, kernel, P, counts=None, method="nufft", tol=1e-13,
                 dipole_axis=(0.0, 0.0, 1.0), eps=0.0):
        assert kernel != "poisson2d"
        if counts is None:
            counts = quadrature.default_counts(grid.L, P)
        d = grid.dim
        self.grid = grid
        k, wq, r, wj = node_set(kernel, P, counts, dipole_axis, eps)
        n2 = [2 * v for v in grid.n]
        c = wj * float(np.prod(grid.h)) / (2.0 * math.pi) ** d
        if method == "direct":
            K = nufft.direct_type1_real(c.astype(np.complex128), k, n2, grid.h)
        else:
            K = np.real(nufft.type1(c.astype(np.complex128), k, n2, grid.h, tol))
        # K is indexed by m + n (grid convention); move m = 0 to index 0
        K = np.fft.ifftshift(K)
        self.Khat = sfft.rfftn(K, workers=-1)
        self.n2 = n2

    def __call__(self, rho):
        n = self.grid.n
        pad = np.zeros(self.n2, dtype=np.float64)
        pad[tuple(slice(0, v) for v in n)] = rho
        out = sfft.irfftn(sfft.rfftn(pad, workers=-1) * self.Khat, s=self.n2, workers=-1)
        return out[tuple(slice(0, v) for v in n)]
