"""Learned initial guess for the normalized gradient flow: data generation, training and use.

The ground states the network learns from are computed by the library's own gradient
flow (nlp_gf_solve, Sec. 3.1 with the stopping rule of Sec. 3.2) and the network is trained
by its own kernels (nlp_surrogate_*).  The gradient flow started from the network's guess
still runs to the same stopping rule, so the guess changes only how long the solve takes.

Ground-state problems: V = (x^2 + y^2 + gamma^2 z^2)/2 on [-L, L)^3, and either the Coulomb
kernel with strength beta, or the dipolar kernel (axis z) with strength beta/2 plus a
contact term g = beta (dipolar strength below the contact strength keeps the energy bounded
below).  Device memory and streams come from torch; everything else is library calls.
"""
from __future__ import annotations

import concurrent.futures as cf
import math

import numpy as np

from . import _binding as B

BOX_L = 10.0
GRID = B.SURROGATE_GRID


def problem(beta: float, gamma: float, kernel: str) -> dict:
    """Interaction parameters of the ground-state problem (beta, gamma, kernel)."""
    if kernel == "coulomb3d":
        return {"kernel": kernel, "beta": float(beta), "g": 0.0}
    if kernel == "dipole3d":
        return {"kernel": kernel, "beta": 0.5 * float(beta), "g": float(beta)}
    raise ValueError(kernel)


def _axes(n, L):
    return [-L + np.arange(n) * (2.0 * L / n)] * 3


def trap(n: int, L: float, gamma: float) -> np.ndarray:
    """V = (x^2 + y^2 + gamma^2 z^2)/2 on the n^3 grid over [-L, L)^3 (FP64, host)."""
    x, y, z = _axes(n, L)
    return 0.5 * (x[:, None, None] ** 2 + y[None, :, None] ** 2 + (gamma * z[None, None, :]) ** 2)


def gaussian_start(n: int, L: float, gamma: float) -> np.ndarray:
    """The plain start: exp(-(x^2 + y^2 + gamma z^2)/2), normalised to h^3 sum phi^2 = 1."""
    x, y, z = _axes(n, L)
    phi = np.exp(-0.5 * (x[:, None, None] ** 2 + y[None, :, None] ** 2 + gamma * z[None, None, :] ** 2))
    h3 = (2.0 * L / n) ** 3
    return phi / math.sqrt(h3 * float(np.sum(phi * phi)))


class GroundStateSolver:
    """FP64 gradient flow on one grid, with one plan per kernel on one stream."""

    def __init__(self, n: int = GRID, L: float = BOX_L, stream=None, method: int = 1):
        import torch
        self.n, self.L = n, L
        self.stream = stream or torch.cuda.Stream()
        self.method = method
        self.plans = {}

    def plan(self, kernel: str) -> "B.Plan":
        if kernel not in self.plans:
            h = 2.0 * self.L / self.n
            kw = {"dipole_axis": (0.0, 0.0, 1.0)} if kernel == "dipole3d" else {}
            self.plans[kernel] = B.Plan((self.n,) * 3, (self.L,) * 3, kernel, "fp64", kmax=math.pi / h,
                                        method=self.method, stream=self.stream, **kw)
        return self.plans[kernel]

    def solve(self, beta: float, gamma: float, kernel: str, phi=None, stop_tol: float = 1e-10,
              max_steps: int = 20000, tau: float = 1e-2, inner_tol: float = 1e-12, max_inner: int = 400):
        """Runs the flow from phi (device FP64 tensor, updated in place; None = Gaussian start).
        Returns (phi, steps, device seconds of the flow, energies)."""
        import torch
        pr = problem(beta, gamma, kernel)
        plan = self.plan(kernel)
        with torch.cuda.stream(self.stream):
            V = torch.from_numpy(trap(self.n, self.L, gamma)).to("cuda", non_blocking=False)
            if phi is None:
                phi = torch.from_numpy(gaussian_start(self.n, self.L, gamma)).to("cuda")
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            self.stream.synchronize()
            t0.record(self.stream)
            steps, ch, E, st = B.nlp_gf_solve(plan.handle, phi, V, pr["beta"], pr["g"], tau, stop_tol, max_steps,
                                              inner_tol, max_inner, raise_on_nonconv=False)
            t1.record(self.stream)
            t1.synchronize()
        return phi, steps, t0.elapsed_time(t1) * 1e-3, dict(E, change=ch, converged=(st == B.NLP_OK))

    def close(self):
        for p in self.plans.values():
            p.close()
        self.plans = {}


def generate(params, stop_tol: float = 1e-6, workers: int = 12, n: int = GRID, L: float = BOX_L,
             inner_tol: float = 1e-9):
    """Ground states for [(beta, gamma, kernel), ...] on the n^3 grid over [-L, L)^3, computed
    by `workers` host threads, each driving its own plans on its own stream.
    Returns (targets [N][n][n][n] FP32 device tensor, features [N][4] FP32 device tensor,
    per-item info)."""
    import torch
    N = len(params)
    targets = torch.empty((N, n, n, n), dtype=torch.float32, device="cuda")
    feats = torch.from_numpy(np.stack([B.nlp_surrogate_features(*p) for p in params])).cuda()
    info = [None] * N
    chunks = [list(range(w, N, workers)) for w in range(workers)]

    def run(idx):
        solver = GroundStateSolver(n, L)
        try:
            for i in idx:
                beta, gamma, kernel = params[i]
                phi, steps, secs, E = solver.solve(beta, gamma, kernel, stop_tol=stop_tol, inner_tol=inner_tol)
                with torch.cuda.stream(solver.stream):
                    targets[i].copy_(phi)
                solver.stream.synchronize()
                info[i] = {"steps": steps, "seconds": secs, **E}
        finally:
            solver.close()

    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for f in [ex.submit(run, c) for c in chunks if c]:
            f.result()
    torch.cuda.synchronize()
    return targets, feats, info


def residual_targets(sur: "B.Surrogate", targets, params):
    """Training targets of the network: ground state minus the beta = 0 amplitude b (the
    network learns the correction; nlp_surrogate_initial_guess adds b back)."""
    import torch
    gam = torch.tensor([p[1] for p in params], dtype=torch.float32, device=targets.device)
    base = sur.base(gam)
    (sur.stream or torch.cuda.current_stream()).synchronize()
    return (targets - base).contiguous()


def train(sur: "B.Surrogate", feats, targets, steps: int, batch: int = 32, lr: float = 2e-3,
          lr_final: float = 1e-4, weight_decay: float = 0.0, seed: int = 0, log_every: int = 50):
    """AdamW on mean squared error with a cosine learning-rate decay; batches drawn from a
    seeded permutation of the training set.  Returns [(step, loss)] every log_every steps."""
    import torch
    N = feats.shape[0]
    rng = np.random.default_rng(seed)
    perm, pos = rng.permutation(N), 0
    hist = []
    stream = sur.stream or torch.cuda.current_stream()
    for s in range(steps):
        if pos + batch > N:
            perm, pos = rng.permutation(N), 0
        idx = torch.from_numpy(perm[pos:pos + batch]).cuda()
        pos += batch
        with torch.cuda.stream(stream):
            fb = feats.index_select(0, idx).contiguous()
            tb = targets.index_select(0, idx).contiguous()
        lr_s = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * s / max(1, steps - 1)))
        want = (s % log_every == 0) or s == steps - 1
        loss = sur.train_step(fb, tb, lr_s, weight_decay, want_loss=want)
        if want:
            hist.append((s, loss))
    return hist
