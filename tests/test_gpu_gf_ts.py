"""GPU parity of the gradient-flow and time-splitting steps (through the C-ABI) against
the FP64 oracle, and the GPU ground state against the paper's energy table."""
import math

import numpy as np
import pytest

import workloads as W
from conftest import load_golden
from oracle import gf, potential, ts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1410_3584_gb300 as m
    return m


COUNTS3 = (48, 48, 96)


def _setup3(n=32, L=8.0):
    g = W.cube(n, L)
    gam = (1.0, 1.0, 2.0)
    return g, gam, W.harmonic_trap(g, gam), math.pi / g.h[0]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_gf_step_parity(nl, prec, tol):
    import torch
    g, gam, V, P = _setup3()
    beta, gc, tau = 5.0, 0.7, 1e-2
    phi0 = W.normalized_gaussian_start(g, (1.3, 0.8, 1.5))
    op = potential.ConvolutionOperator(g, "coulomb3d", P, COUNTS3)
    G = gf.GradientFlow(g, V, beta, op, tau=tau, g=gc, inner_tol=1e-12 if prec == "fp64" else 1e-6)
    ref, ch_ref = G.step(phi0)
    E_ref = G.energies(ref)
    plan = nl.Plan(g.n, g.L, "coulomb3d", prec, kmax=P, counts=COUNTS3)
    dt = plan.torch_dtype
    tphi = torch.from_numpy(phi0).to("cuda", dt)
    tV = torch.from_numpy(V).to("cuda", dt)
    ch, it, E, st = nl.nlp_gf_step(plan.handle, tphi, tV, beta, gc, tau, 1e-12 if prec == "fp64" else 1e-6, 200,
                                   energies=True)
    out = tphi.double().cpu().numpy()
    plan.close()
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < tol
    assert abs(ch - ch_ref) < tol * 50 * max(1.0, ch_ref)
    for k in ("E", "Ekin", "Epot", "Eint", "mu"):
        assert abs(E[k] - E_ref[k]) < tol * max(1.0, abs(E_ref[k])), (k, E[k], E_ref[k])
    if prec == "fp64":
        assert abs(it - G.last_inner) <= 1


def test_gpu_ground_state_matches_paper_table(nl):
    """Example 3.1 (Table tab:virial:3d:sps), beta = 1: GF-NUFFT on the GPU to
    max|phi^{n+1} - phi^n|/tau <= 1e-8 on [-5,5)^3 with h = 1/3, FP64."""
    import torch
    g, gam, V, P = _setup3(30, 5.0)
    plan = nl.Plan(g.n, g.L, "coulomb3d", "fp64", kmax=P)
    tphi = torch.from_numpy(W.normalized_gaussian_start(g, gam)).cuda()
    tV = torch.from_numpy(V).cuda()
    for n in range(5000):
        ch, it, _, _ = nl.nlp_gf_step(plan.handle, tphi, tV, 1.0, 0.0, 1e-2, 1e-12, 200)
        if ch <= 1e-8:
            break
    E = nl.nlp_energies(plan.handle, tphi, tV, 1.0, 0.0)
    plan.close()
    rows = {float(r[0]): r[1:] for r in load_golden("paper_gs_energies_3d_coulomb.txt")}
    for key, txt in zip(("E", "mu", "Ekin", "Epot", "Eint"), rows[1.0]):
        mant, _, ex = txt.upper().partition("E")
        ulp = 10.0 ** (-len(mant.split(".")[1]) + (int(ex) if ex else 0))
        assert abs(E[key] - float(txt)) < ulp, (key, E[key], txt)
    assert abs(2 * E["Ekin"] - 2 * E["Epot"] + E["Eint"]) < 1e-6


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_ts_step_parity_and_mass(nl, order, prec, tol):
    import torch
    g = W.Grid((48, 40), (8.0, 7.0))
    V = W.harmonic_trap(g, (1.0, 1.3))
    P = math.pi / max(g.h)
    counts = (64, 128)
    op = potential.ConvolutionOperator(g, "coulomb2d", P, counts)
    psi0 = W.gaussian(g, [math.sqrt(2.0)] * 2, center=(0.5, -0.3)).astype(np.complex128)
    S = ts.TimeSplitting(g, V, 5.0, op, g=0.3)
    ref = psi0.copy()
    for _ in range(3):
        ref = S.step(ref, 0.01, order)
    plan = nl.Plan(g.n, g.L, "coulomb2d", prec, kmax=P, counts=counts)
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    tpsi = torch.from_numpy(psi0).to("cuda", cdt)
    tV = torch.from_numpy(V).to("cuda", plan.torch_dtype)
    for _ in range(3):
        nl.nlp_ts_step(plan.handle, tpsi, tV, 5.0, 0.3, 0.01, order)
    out = tpsi.cpu().numpy().astype(np.complex128)
    plan.close()
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < tol
    m0 = float(np.sum(np.abs(psi0) ** 2))
    assert abs(float(np.sum(np.abs(out) ** 2)) - m0) < (1e-12 if prec == "fp64" else 1e-5) * m0
