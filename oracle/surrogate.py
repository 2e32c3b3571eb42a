"""FP64 host model of the learned gradient-flow initial guess (test infrastructure only).

The network is not part of the paper: it maps (beta, gamma, kernel) features to an
amplitude on a cube grid, which then starts the normalized gradient flow of Sec. 3.1.
This module restates its forward pass and the backward pass (reverse-mode chain rule,
written out by hand) in plain numpy FP64, with the sizes as parameters so that small
instances can be checked against finite differences quickly.

Architecture (sizes of the library's network in brackets):
    x0 = features zero-padded to feat_pad [64]                       (rows = batch)
    x_{l+1} = silu(x_l W_l^T + b_l),  l = 0..depth-1                  [depth 4, hid 512]
    y = x_depth W_h^T + b_h  (W_h rows >= C g0^3 are padding)          [1792 rows, C 8, g0 6]
    z = y[:, :C g0^3] as [C][g0][g0][g0]
    repeat for each conv layer c: z <- conv_c(up2(z)), silu after every layer but the last
        (channels C -> C, ..., C -> 1)                                [3 layers: 12^3, 24^3, 48^3]
    out = z[:, 0]
    loss = mean((out - target)^2)

Flat parameter order (as documented for nlp_surrogate_*): W_l then b_l for every dense
layer (row-major [out][in]), then w_c [co][ci][27] and bias_c [co] for every conv layer,
tap d = 9 dz + 3 dy + dx reading input position p + (dz, dy, dx) - 1, zero padding.

Pins (tests/test_oracle_surrogate.py): conv3 against scipy.ndimage.correlate, up2 against
a Kronecker product, the backward pass against central finite differences of the forward
pass (every tensor), and AdamW against its textbook update written per element.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Arch:
    feat: int = 4
    feat_pad: int = 64
    hid: int = 512
    depth: int = 4          # hidden dense layers
    C: int = 8
    g0: int = 6
    head_pad: int = 1792
    n_conv: int = 3

    @property
    def g_out(self) -> int:
        return self.g0 * 2 ** self.n_conv


FULL = Arch()


def layout(a: Arch = FULL):
    """[(name, offset, shape)] in the flat parameter order."""
    ents = []
    ins = [a.feat_pad] + [a.hid] * (a.depth - 1) + [a.hid]
    outs = [a.hid] * a.depth + [a.head_pad]
    for l, (i, o) in enumerate(zip(ins, outs)):
        ents.append(("W%d" % l, (o, i)))
        ents.append(("b%d" % l, (o,)))
    for c in range(a.n_conv):
        co = 1 if c == a.n_conv - 1 else a.C
        ents.append(("cw%d" % c, (co, a.C, 27)))
        ents.append(("cb%d" % c, (co,)))
    out, off = [], 0
    for name, shp in ents:
        out.append((name, off, shp))
        off += int(np.prod(shp))
    return out, off


def unpack(theta: np.ndarray, a: Arch = FULL) -> dict:
    lay, total = layout(a)
    assert theta.size == total, (theta.size, total)
    return {name: np.asarray(theta[off:off + int(np.prod(shp))], dtype=np.float64).reshape(shp)
            for name, off, shp in lay}


def pack(params: dict, a: Arch = FULL) -> np.ndarray:
    lay, total = layout(a)
    out = np.zeros(total, dtype=np.float64)
    for name, off, shp in lay:
        out[off:off + int(np.prod(shp))] = params[name].ravel()
    return out


def init_params(seed: int, a: Arch = FULL) -> np.ndarray:
    """Random parameters (real entries U(-1/sqrt(fan_in), 1/sqrt(fan_in)), padding zero,
    small random biases so that the bias gradients are exercised)."""
    rng = np.random.default_rng(seed)
    P = {}
    lay, _ = layout(a)
    for name, off, shp in lay:
        if name.startswith("W"):
            fan = a.feat if name == "W0" else a.hid
            w = rng.uniform(-1, 1, size=shp) / math.sqrt(fan)
            if name == "W0":
                w[:, a.feat:] = 0.0
            if name == "W%d" % a.depth:
                w[a.C * a.g0 ** 3:, :] = 0.0
            P[name] = w
        elif name.startswith("cw"):
            P[name] = rng.uniform(-1, 1, size=shp) / math.sqrt(a.C * 27)
        else:
            b = 0.1 * rng.uniform(-1, 1, size=shp)
            if name == "b%d" % a.depth:
                b[a.C * a.g0 ** 3:] = 0.0
            P[name] = b
    return pack(P, a)


def features(beta: float, gamma: float, kernel: str) -> np.ndarray:
    """[log10(beta)/3, (gamma-1)/3, is Coulomb, is dipolar]."""
    return np.array([math.log10(beta) / 3.0, (gamma - 1.0) / 3.0,
                     1.0 if kernel == "coulomb3d" else 0.0, 1.0 if kernel == "dipole3d" else 0.0])


def silu(v):
    return v / (1.0 + np.exp(-v))


def silu_grad(v):
    s = 1.0 / (1.0 + np.exp(-v))
    return s * (1.0 + v * (1.0 - s))


def _taps():
    return [(d // 9, (d // 3) % 3, d % 3) for d in range(27)]


def conv3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [B][Ci][g][g][g], w [Co][Ci][27], b [Co]: zero-padded 3^3 cross-correlation."""
    B, Ci, g = x.shape[0], x.shape[1], x.shape[2]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.zeros((B, w.shape[0], g, g, g)) + b[None, :, None, None, None]
    for d, (dz, dy, dx) in enumerate(_taps()):
        out += np.einsum("oc,bcxyz->boxyz", w[:, :, d], xp[:, :, dz:dz + g, dy:dy + g, dx:dx + g])
    return out


def conv3_backward(x, w, dout):
    """Gradients of conv3 w.r.t. (x, w, b) given d loss / d out."""
    g = x.shape[2]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for d, (dz, dy, dx) in enumerate(_taps()):
        sl = (slice(None), slice(None), slice(dz, dz + g), slice(dy, dy + g), slice(dx, dx + g))
        dw[:, :, d] = np.einsum("boxyz,bcxyz->oc", dout, xp[sl])
        dxp[sl] += np.einsum("oc,boxyz->bcxyz", w[:, :, d], dout)
    return dxp[:, :, 1:-1, 1:-1, 1:-1], dw, dout.sum(axis=(0, 2, 3, 4))


def up2(x):
    """Nearest-neighbour upsampling by 2 along the last three axes."""
    return x.repeat(2, axis=-3).repeat(2, axis=-2).repeat(2, axis=-1)


def up2_backward(dout):
    B, C, G = dout.shape[0], dout.shape[1], dout.shape[2]
    g = G // 2
    return dout.reshape(B, C, g, 2, g, 2, g, 2).sum(axis=(3, 5, 7))


def forward(theta: np.ndarray, feats: np.ndarray, a: Arch = FULL, keep: bool = False):
    """out [B][g_out]^3 (and the intermediate values if keep)."""
    P = unpack(theta, a)
    B = feats.shape[0]
    x = np.zeros((B, a.feat_pad))
    x[:, :feats.shape[1]] = feats
    xs, pres = [x], []
    for l in range(a.depth + 1):
        pre = xs[-1] @ P["W%d" % l].T + P["b%d" % l]
        pres.append(pre)
        xs.append(silu(pre) if l < a.depth else pre)
    z = xs[-1][:, :a.C * a.g0 ** 3].reshape(B, a.C, a.g0, a.g0, a.g0)
    ups, cpres = [], []
    for c in range(a.n_conv):
        u = up2(z)
        ups.append(u)
        cp = conv3(u, P["cw%d" % c], P["cb%d" % c])
        cpres.append(cp)
        z = silu(cp) if c < a.n_conv - 1 else cp
    out = z[:, 0]
    if keep:
        return out, dict(xs=xs, pres=pres, ups=ups, cpres=cpres)
    return out


def loss_and_grad(theta: np.ndarray, feats: np.ndarray, target: np.ndarray, a: Arch = FULL):
    """Mean squared error and its gradient in the flat layout (reverse-mode, FP64)."""
    P = unpack(theta, a)
    out, K = forward(theta, feats, a, keep=True)
    B = feats.shape[0]
    diff = out - target
    loss = float(np.mean(diff * diff))
    G = {}
    dz = (2.0 / diff.size) * diff[:, None]                 # d loss / d (last conv output)
    for c in reversed(range(a.n_conv)):
        if c < a.n_conv - 1:
            dz = dz * silu_grad(K["cpres"][c])
        du, G["cw%d" % c], G["cb%d" % c] = conv3_backward(K["ups"][c], P["cw%d" % c], dz)
        dz = up2_backward(du)
    dy = np.zeros((B, a.head_pad))
    dy[:, :a.C * a.g0 ** 3] = dz.reshape(B, -1)
    for l in reversed(range(a.depth + 1)):
        dpre = dy * silu_grad(K["pres"][l]) if l < a.depth else dy
        G["W%d" % l] = dpre.T @ K["xs"][l]
        G["b%d" % l] = dpre.sum(axis=0)
        dy = dpre @ P["W%d" % l]
    return loss, pack(G, a)


def adamw(theta, grad, m, v, step: int, lr: float, wd: float, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW update (bias-corrected moments, decoupled weight decay), per element."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v


def base_amplitude(x, y, z, gamma: float):
    """beta = 0 ground state of V = (x^2 + y^2 + gamma^2 z^2)/2 (continuum normalisation):
    gamma^{1/4} pi^{-3/4} exp(-(x^2 + y^2 + gamma z^2)/2)."""
    return gamma ** 0.25 * math.pi ** -0.75 * np.exp(-0.5 * (x * x + y * y + gamma * z * z))


def base_cube(box_L: float, g: int, gamma: float) -> np.ndarray:
    a = -box_L + np.arange(g) * (2.0 * box_L / g)
    return base_amplitude(a[:, None, None], a[None, :, None], a[None, None, :], gamma)


def reflect_average(phi: np.ndarray) -> np.ndarray:
    """Average over the 8 grid reflections i -> (n - i) mod n of the three axes."""
    out = np.zeros_like(phi)
    for fz in (0, 1):
        for fy in (0, 1):
            for fx in (0, 1):
                v = phi
                for ax, f in ((0, fz), (1, fy), (2, fx)):
                    if f:
                        v = np.roll(np.flip(v, axis=ax), 1, axis=ax)
                out += v
    return out / 8.0


def resample(out48: np.ndarray, box_L: float, n, L, gamma: float) -> np.ndarray:
    """Initial guess on the grid x_i = -L + i 2L/n: the beta = 0 amplitude plus the trilinear
    sample of the cube correction (point j at -box_L + j 2 box_L / g; zero outside the cube),
    clamped at zero, averaged over the grid reflections, normalised to h^3 sum phi^2 = 1."""
    g = out48.shape[0]
    hs = 2.0 * box_L / g
    idx, frac, inside, xs = [], [], [], []
    for a in range(3):
        x = -L[a] + np.arange(n[a]) * (2.0 * L[a] / n[a])
        xs.append(x)
        u = (x + box_L) / hs
        ins = (u >= 0.0) & (u <= g - 1)
        lo = np.clip(np.floor(u).astype(int), 0, g - 2)
        idx.append(lo)
        frac.append(u - lo)
        inside.append(ins)
    corr = np.zeros(tuple(n))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                wz = frac[0] if dz else 1 - frac[0]
                wy = frac[1] if dy else 1 - frac[1]
                wx = frac[2] if dx else 1 - frac[2]
                vals = out48[np.ix_(idx[0] + dz, idx[1] + dy, idx[2] + dx)]
                corr += wz[:, None, None] * wy[None, :, None] * wx[None, None, :] * vals
    mask = inside[0][:, None, None] & inside[1][None, :, None] & inside[2][None, None, :]
    phi = base_amplitude(xs[0][:, None, None], xs[1][None, :, None], xs[2][None, None, :], gamma)
    phi = np.maximum(phi + np.where(mask, corr, 0.0), 0.0)
    phi = reflect_average(phi)
    hv = float(np.prod([2.0 * L[a] / n[a] for a in range(3)]))
    return phi / math.sqrt(hv * float(np.sum(phi * phi)))
