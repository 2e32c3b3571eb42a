"""Plain FP64 NUFFT, types 2 and 1 (oracle tier O2; Sec. 2.1 evaluates the
quadrature sum of Eq. (ifft) "via the NUFFT").

Grid points x_i = (i - n/2) h, i = 0..n-1 per axis.  With t = k h and the
upsampled grid nf = 2n (the paper's oversampling factor 2 per dimension, Sec. 2.1):

  type 2   f_j = sum_i c_i exp(-i t_j . i):
           deconvolve c_i / prod psi-hat(i 2pi/nf), zero-pad to nf^d (index i mod nf),
           forward FFT (library primitive), interpolate with phi at z_j = t_j nf / 2pi.
  type 1   g_i = sum_j c_j exp(+i t_j . i):
           spread c_j with phi, inverse FFT (unnormalized), deconvolve, crop.
"""
from __future__ import annotations

import math

import numpy as np

from . import native
from .es_kernel import es_ft, es_params


def _setup(n, h, k, tol):
    d = len(n)
    w, beta = es_params(tol)
    nf = [2 * int(v) for v in n]
    corr = []
    idx = []
    for a in range(d):
        i = np.arange(n[a]) - n[a] // 2
        corr.append(es_ft(i * (2.0 * math.pi / nf[a]), w, beta))
        idx.append(np.mod(i, nf[a]))
    z = np.empty((k.shape[0], d), dtype=np.float64)
    for a in range(d):
        z[:, a] = k[:, a] * h[a] * nf[a] / (2.0 * math.pi)
    return d, w, beta, nf, corr, idx, np.ascontiguousarray(z)


def _deconv(arr, corr):
    d = arr.ndim
    for a in range(d):
        shape = [1] * d
        shape[a] = -1
        arr = arr / corr[a].reshape(shape)
    return arr


def type2(rho: np.ndarray, h, k: np.ndarray, tol: float = 1e-13) -> np.ndarray:
    """rho-hat_j = (prod h) sum_i rho_i exp(-i k_j . x_i), complex (M,)."""
    n = rho.shape
    k = np.ascontiguousarray(k, dtype=np.float64)
    d, w, beta, nf, corr, idx, z = _setup(n, h, k, tol)
    F = np.zeros(nf, dtype=np.complex128)
    F[np.ix_(*idx)] = _deconv(np.asarray(rho, dtype=np.float64), corr)
    Fh = np.ascontiguousarray(np.fft.fftn(F))
    out = np.empty(2 * k.shape[0], dtype=np.float64)
    native.lib().orc_interp(d, native.ptr(native.i64arr(nf)), native.ptr(Fh.view(np.float64)),
                            k.shape[0], native.ptr(z), w, beta, native.ptr(out))
    return float(np.prod(h)) * (out[0::2] + 1j * out[1::2])


def type1(c: np.ndarray, k: np.ndarray, n, h, tol: float = 1e-13) -> np.ndarray:
    """g_i = sum_j c_j exp(+i k_j . x_i) on the n-grid, complex."""
    k = np.ascontiguousarray(k, dtype=np.float64)
    d, w, beta, nf, corr, idx, z = _setup(n, h, k, tol)
    cc = np.ascontiguousarray(np.stack([np.real(c), np.imag(c)], axis=-1).reshape(-1))
    G = np.zeros(nf, dtype=np.complex128)
    native.lib().orc_spread(d, native.ptr(native.i64arr(nf)), k.shape[0], native.ptr(z),
                            native.ptr(cc), w, beta, native.ptr(G.view(np.float64)))
    Gh = np.fft.ifftn(G) * float(np.prod(nf))
    return _deconv(Gh[np.ix_(*idx)], corr)


def direct_type2(rho: np.ndarray, h, k: np.ndarray) -> np.ndarray:
    """O1: rho-hat_j by the direct trapezoid sum."""
    k = np.ascontiguousarray(k, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.empty(2 * k.shape[0], dtype=np.float64)
    native.lib().orc_direct_type2(rho.ndim, native.ptr(native.i64arr(rho.shape)),
                                  native.ptr(native.f64arr(h)), native.ptr(rho),
                                  k.shape[0], native.ptr(k), native.ptr(out))
    return out[0::2] + 1j * out[1::2]


def direct_type1_real(c: np.ndarray, k: np.ndarray, n, h) -> np.ndarray:
    """O1: Re sum_j c_j exp(+i k_j . x_i) by direct summation."""
    k = np.ascontiguousarray(k, dtype=np.float64)
    cc = np.ascontiguousarray(np.stack([np.real(c), np.imag(c)], axis=-1).reshape(-1))
    out = np.empty(tuple(int(v) for v in n), dtype=np.float64)
    native.lib().orc_direct_type1(len(n), native.ptr(native.i64arr(n)), native.ptr(native.f64arr(h)),
                                  k.shape[0], native.ptr(k), native.ptr(cc), native.ptr(out))
    return out
