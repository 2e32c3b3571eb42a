"""Pins of the FP64 host model of the learned initial guess (oracle/surrogate.py).

The backward pass is pinned to central finite differences of the forward pass; the
building blocks to library routines (scipy.ndimage.correlate, numpy.kron).  A planted
mistake in the activation derivative must be caught by the finite-difference check.
"""
import math

import numpy as np
import pytest
from scipy import ndimage

from oracle import surrogate as S

SMALL = S.Arch(feat=4, feat_pad=8, hid=12, depth=2, C=2, g0=2, head_pad=24, n_conv=3)


def test_layout_sizes_full_network():
    lay, total = S.layout(S.FULL)
    names = [n for n, _, _ in lay]
    assert names[:4] == ["W0", "b0", "W1", "b1"] and names[-2:] == ["cw2", "cb2"]
    expect = 512 * 64 + 512 + 3 * (512 * 512 + 512) + 1792 * 512 + 1792 + 2 * (8 * 8 * 27 + 8) + 8 * 27 + 1
    assert total == expect
    assert S.FULL.g_out == 48


def test_conv3_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 5, 5, 5))
    w = rng.standard_normal((4, 3, 27))
    b = rng.standard_normal(4)
    out = S.conv3(x, w, b)
    for bb in range(2):
        for co in range(4):
            ref = np.full((5, 5, 5), b[co])
            for ci in range(3):
                ref += ndimage.correlate(x[bb, ci], w[co, ci].reshape(3, 3, 3), mode="constant", cval=0.0)
            assert np.max(np.abs(out[bb, co] - ref)) < 1e-12


def test_up2_matches_kron_and_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 2, 3, 3, 3))
    u = S.up2(x)
    for c in range(2):
        assert np.array_equal(u[0, c], np.kron(x[0, c], np.ones((2, 2, 2))))
    d = rng.standard_normal(u.shape)
    # <up2 x, d> = <x, up2^T d>
    assert abs(np.sum(u * d) - np.sum(x * S.up2_backward(d))) < 1e-12


def _fd_check(arch, theta, feats, target, coords, h=1e-6):
    """max over coords of |fd - g| / (|fd| + floor), floor = 1e-4 max|g|: coordinates whose
    gradient is a near-cancellation of much larger terms are judged on the gradient's scale."""
    _, g = S.loss_and_grad(theta, feats, target, arch)
    floor = 1e-4 * float(np.max(np.abs(g)))
    errs = []
    for i in coords:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp = float(np.mean((S.forward(tp, feats, arch) - target) ** 2))
        lm = float(np.mean((S.forward(tm, feats, arch) - target) ** 2))
        fd = (lp - lm) / (2 * h)
        errs.append(abs(fd - g[i]) / (abs(fd) + floor))
    return max(errs)


def _coords_every_tensor(arch, rng, per=3):
    lay, _ = S.layout(arch)
    out = []
    for name, off, shp in lay:
        n = int(np.prod(shp))
        if name == "W0":   # real (unpadded) columns only
            cols = rng.integers(0, arch.feat, size=per)
            rows = rng.integers(0, shp[0], size=per)
            out += [off + r * shp[1] + c for r, c in zip(rows, cols)]
        elif name in ("W%d" % arch.depth, "b%d" % arch.depth):
            lim = arch.C * arch.g0 ** 3
            idx = rng.integers(0, lim * (shp[1] if len(shp) > 1 else 1), size=per)
            out += [off + int(i) for i in idx]
        else:
            out += [off + int(i) for i in rng.integers(0, n, size=per)]
    return out


def _problem(arch, seed, B=3):
    rng = np.random.default_rng(seed)
    theta = S.init_params(seed, arch)
    feats = np.stack([S.features(b, g, k) for b, g, k in
                      [(3.0, 1.5, "coulomb3d"), (400.0, 3.2, "dipole3d"), (40.0, 2.0, "coulomb3d")][:B]])
    target = 0.05 * rng.standard_normal((B,) + (arch.g_out,) * 3)
    return theta, feats, target, rng


def test_backward_matches_finite_differences_small():
    theta, feats, target, rng = _problem(SMALL, 3)
    err = _fd_check(SMALL, theta, feats, target, _coords_every_tensor(SMALL, rng, per=4))
    assert err < 1e-6, err


def test_backward_matches_finite_differences_full_size():
    theta, feats, target, rng = _problem(S.FULL, 4, B=2)
    err = _fd_check(S.FULL, theta, feats, target, _coords_every_tensor(S.FULL, rng, per=1))
    assert err < 1e-5, err


def test_padding_gradients_are_zero():
    theta, feats, target, _ = _problem(SMALL, 5)
    _, g = S.loss_and_grad(theta, feats, target, SMALL)
    G = S.unpack(g, SMALL)
    assert np.all(G["W0"][:, SMALL.feat:] == 0.0)
    lim = SMALL.C * SMALL.g0 ** 3
    assert np.all(G["W%d" % SMALL.depth][lim:] == 0.0) and np.all(G["b%d" % SMALL.depth][lim:] == 0.0)


def test_planted_activation_mistake_is_caught(monkeypatch):
    theta, feats, target, rng = _problem(SMALL, 6)
    monkeypatch.setattr(S, "silu_grad", lambda v: 1.0 / (1.0 + np.exp(-v)))   # drops a term
    err = _fd_check(SMALL, theta, feats, target, _coords_every_tensor(SMALL, rng, per=4))
    assert err > 1e-3


def test_adamw_first_step_is_signed_lr():
    """Step 1 of Adam moves every coordinate with a nonzero gradient by lr * sign(g)
    (bias correction makes m_hat = g, v_hat = g^2), plus the decoupled decay lr wd theta."""
    rng = np.random.default_rng(7)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m, v = S.adamw(th, g, np.zeros(50), np.zeros(50), 1, lr=1e-2, wd=0.1, eps=0.0)
    assert np.allclose(new, th - 1e-2 * (np.sign(g) + 0.1 * th), rtol=0, atol=1e-15)


def test_resample_on_matching_grid_is_base_plus_symmetrised_correction():
    """On the cube's own grid the trilinear sample is the identity: the guess is the beta = 0
    amplitude plus the correction, averaged over reflections (checked by index arithmetic)."""
    rng = np.random.default_rng(8)
    g, Lb, gam = 8, 4.0, 1.7
    c = 0.01 * rng.standard_normal((g, g, g))
    phi = S.resample(c, Lb, (g, g, g), (Lb, Lb, Lb), gam)
    raw = np.maximum(S.base_cube(Lb, g, gam) + c, 0.0)
    ref = np.zeros_like(raw)
    for i in range(g):
        for j in range(g):
            for k in range(g):
                acc = 0.0
                for a in (i, (g - i) % g):
                    for b in (j, (g - j) % g):
                        for e in (k, (g - k) % g):
                            acc += raw[a, b, e]
                ref[i, j, k] = acc / 8
    ref /= math.sqrt(1.0 * np.sum(ref * ref))
    assert np.max(np.abs(phi - ref)) < 1e-14


def test_base_amplitude_is_normalised_ground_state():
    """b is the normalised ground state of -Delta/2 + V for beta = 0: unit L2 norm (Riemann
    sum of a rapidly decaying function) and, along z, (-d^2/dz^2 / 2 + gamma^2 z^2 / 2) b =
    (gamma / 2) b (second differences, h = 0.01)."""
    gam, h = 2.5, 0.05
    a = np.arange(-8, 8, h)
    X, Y, Z = np.meshgrid(a, a, a, indexing="ij")
    assert abs(np.sum(S.base_amplitude(X, Y, Z, gam) ** 2) * h ** 3 - 1.0) < 1e-10
    zz = np.arange(-6, 6, 0.01)
    fz = S.base_amplitude(0.0, 0.0, zz, gam)
    lap = (fz[2:] - 2 * fz[1:-1] + fz[:-2]) / 0.01 ** 2
    Hz = -0.5 * lap + 0.5 * gam ** 2 * zz[1:-1] ** 2 * fz[1:-1]
    assert np.max(np.abs(Hz - 0.5 * gam * fz[1:-1])) < 1e-4
