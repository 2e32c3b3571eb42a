"""GPU parity of the gradient-flow and time-splitting steps (through the C-ABI) against
the FP64 oracle, and the GPU ground state against the paper's energy table."""
import math

import numpy as np
import pytest

import workloads as W
from conftest import load_golden
from oracle import gf, potential, quadrature, ts

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


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
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
    err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
    print("gf_step %s rel L-inf vs oracle %.3e" % (prec, err))
    assert err < tol
    assert abs(ch - ch_ref) < tol * 50 * max(1.0, ch_ref)
    for k in ("E", "Ekin", "Epot", "Eint", "mu"):
        assert abs(E[k] - E_ref[k]) < tol * max(1.0, abs(E_ref[k])), (k, E[k], E_ref[k])
    if prec == "fp64":
        assert abs(it - G.last_inner) <= 1


@pytest.mark.parametrize("beta", [-10.0, -5.0, -1.0, 1.0, 5.0, 10.0])
def test_gpu_ground_state_matches_paper_table(nl, beta):
    """Example 3.1 (Table tab:virial:3d:sps), all six beta: GF-NUFFT on the GPU to
    max|phi^{n+1} - phi^n|/tau <= 1e-8 on [-5,5)^3 with h = 1/3, FP64."""
    import torch
    g, gam, V, P = _setup3(30, 5.0)
    plan = nl.Plan(g.n, g.L, "coulomb3d", "fp64", kmax=P)
    tphi = torch.from_numpy(W.normalized_gaussian_start(g, gam)).cuda()
    tV = torch.from_numpy(V).cuda()
    for n in range(5000):
        ch, it, _, _ = nl.nlp_gf_step(plan.handle, tphi, tV, beta, 0.0, 1e-2, 1e-12, 200)
        if ch <= 1e-8:
            break
    E = nl.nlp_energies(plan.handle, tphi, tV, beta, 0.0)
    plan.close()
    rows = {float(r[0]): r[1:] for r in load_golden("paper_gs_energies_3d_coulomb.txt")}
    for key, txt in zip(("E", "mu", "Ekin", "Epot", "Eint"), rows[beta]):
        mant, _, ex = txt.upper().partition("E")
        ulp = 10.0 ** (-len(mant.split(".")[1]) + (int(ex) if ex else 0))
        assert abs(E[key] - float(txt)) < ulp, (key, E[key], txt)
    assert abs(2 * E["Ekin"] - 2 * E["Epot"] + E["Eint"]) < 1e-6


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
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
    err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
    print("ts_step order %d %s rel L-inf vs oracle %.3e" % (order, prec, err))
    assert err < tol
    m0 = float(np.sum(np.abs(psi0) ** 2))
    assert abs(float(np.sum(np.abs(out) ** 2)) - m0) < (1e-12 if prec == "fp64" else 1e-5) * m0


@pytest.mark.parametrize("beta", [-10.0, -5.0, -1.0, 1.0, 5.0, 10.0])
def test_gpu_2d_coulomb_ground_states_match_paper_table(nl, beta):
    """Example 3.2 (Table virial_2d_Coulomb) at the paper's own mesh: V = (x^2 + 4 y^2)/2,
    h = 1/8 on [-8,8)^2, GF-NUFFT on the GPU (nlp_gf_solve, FP64) to the Sec. 3.2 stopping
    rule with eps0 = 1e-10; each printed energy to one unit in its last printed place, and
    the virial identity I^h of the table (|I| ~ 2e-10 there)."""
    import torch
    g = W.cube(128, 8.0, dim=2)
    gam = (1.0, 2.0)
    V = W.harmonic_trap(g, gam)
    plan = nl.Plan(g.n, g.L, "coulomb2d", "fp64", kmax=math.pi / g.h[0])
    tphi = torch.from_numpy(W.normalized_gaussian_start(g, gam)).cuda()
    tV = torch.from_numpy(V).cuda()
    steps, ch, E, st = nl.nlp_gf_solve(plan.handle, tphi, tV, beta, 0.0, 1e-2, 1e-10, 20000, 1e-12, 1000)
    plan.close()
    rows = {float(r[0]): r[1:] for r in load_golden("paper_gs_energies_2d_coulomb.txt")}
    for key, txt in zip(("E", "mu", "Ekin", "Epot", "Eint"), rows[beta]):
        mant, _, ex = txt.upper().partition("E")
        ulp = 10.0 ** (-len(mant.split(".")[1]) + (int(ex) if ex else 0))
        assert abs(E[key] - float(txt)) < ulp, (key, E[key], txt)
    assert abs(2 * E["Ekin"] - 2 * E["Epot"] + E["Eint"]) < 1e-8


def _dyn_run(nl, h, beta, method=1):
    """Example 4.1 on the GPU: psi_0 = exp(-|x|^2/2), V = |x|^2/2 on [-8,8)^3, fourth-order
    splitting with tau = 1e-3 to t = 1/8; returns (psi, phi = U * |psi|^2, mass before/after)."""
    import torch
    n = int(round(16.0 / h))
    g = W.cube(n, 8.0)
    V = W.harmonic_trap(g, (1.0, 1.0, 1.0))
    X, Y, Z = g.mesh()
    psi0 = np.exp(-0.5 * (X * X + Y * Y + Z * Z)).astype(np.complex128)
    P = quadrature.density_P(1.0, h)
    plan = nl.Plan(g.n, g.L, "coulomb3d", "fp64", kmax=P, counts=quadrature.default_counts(g.L, P), method=method)
    tpsi = torch.from_numpy(psi0).cuda()
    tV = torch.from_numpy(V).cuda()
    for _ in range(125):
        nl.nlp_ts_step(plan.handle, tpsi, tV, beta, 0.0, 1e-3, 4)
    rho = (tpsi.real ** 2 + tpsi.imag ** 2).contiguous()
    phi = plan.eval(rho)
    plan.sync()
    out, ph = tpsi.cpu().numpy(), phi.cpu().numpy()
    plan.close()
    hv = h ** 3
    return out, ph, hv * float(np.sum(np.abs(psi0) ** 2)), hv * float(np.sum(np.abs(out) ** 2))


@pytest.mark.parametrize("beta", [-5.0, 5.0])
def test_gpu_dynamics_example_4_1_error_levels(nl, beta):
    """Example 4.1 (Table dy_3d_Coulomb): TS-NUFFT at h = 1, 1/2, 1/4 against our own h = 1/8
    run (the paper's reference solution is not printed).  The printed wave-function errors at
    t = 1/8 are reproduced within a factor 3 at h = 1 and 1/2 (where the mesh error dominates
    the reference's own), and at h = 1/4 wave function and potential agree to the 1e-11 level
    of the table; mass is conserved by the splitting (unitary steps).  The potential error at
    h <= 1/2 is larger than printed because the truncation radius is capped at pi/h (the
    largest ball inside the grid's spectral box); it is only bounded here."""
    rows = {(r[0], float(r[1])): [float(v) for v in r[2:]] for r in load_golden("paper_dynamics_3d_coulomb_errors.txt")}
    ref_psi, ref_phi, m0, m1 = _dyn_run(nl, 1.0 / 8, beta)
    assert abs(m1 - m0) < 1e-12 * m0
    for k, h in enumerate((1.0, 0.5, 0.25)):
        psi, phi, a0, a1 = _dyn_run(nl, h, beta)
        assert abs(a1 - a0) < 1e-12 * a0
        s = int(round(h * 8))
        rp, rf = ref_psi[::s, ::s, ::s], ref_phi[::s, ::s, ::s]
        e_psi = float(np.max(np.abs(psi - rp)) / np.max(np.abs(rp)))
        e_phi = float(np.max(np.abs(phi - rf)) / np.max(np.abs(rf)))
        p_psi, p_phi = rows[("psi", beta)][k], rows[("phi", beta)][k]
        print("beta %g h %g: e_psi %.3e (paper %.3e), e_phi %.3e (paper %.3e)" % (beta, h, e_psi, p_psi, e_phi, p_phi))
        if h >= 0.5:
            assert p_psi / 3 < e_psi < 3 * p_psi
            assert e_phi < 10 * e_psi
        else:
            assert e_psi < 1e-10 and e_phi < 1e-10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_gf_step_parity_poisson2d(nl, prec, tol):
    """One gradient-flow step with the 2D Laplace kernel (potential through Algorithm 1)
    against the oracle's step with its own Algorithm 1 evaluation."""
    import torch
    g = W.Grid((48, 40), (8.0, 7.0))
    V = W.harmonic_trap(g, (1.0, 2.0))
    P = math.pi / max(g.h)
    counts = (64, 128)
    phi0 = W.normalized_gaussian_start(g, (1.2, 1.8))
    G = gf.GradientFlow(g, V, 5.0, lambda r: potential.eval_nufft(r, g, "poisson2d", P, counts), tau=1e-2,
                        inner_tol=1e-12 if prec == "fp64" else 1e-6)
    ref, ch_ref = G.step(phi0)
    plan = nl.Plan(g.n, g.L, "poisson2d", prec, kmax=P, counts=counts)
    tphi = torch.from_numpy(phi0).to("cuda", plan.torch_dtype)
    tV = torch.from_numpy(V).to("cuda", plan.torch_dtype)
    ch, it, E, st = nl.nlp_gf_step(plan.handle, tphi, tV, 5.0, 0.0, 1e-2, 1e-12 if prec == "fp64" else 1e-6, 200)
    out = tphi.double().cpu().numpy()
    plan.close()
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < tol


@pytest.mark.parametrize("beta", [-10.0, -5.0, -1.0, 1.0, 5.0, 10.0])
def test_gpu_2d_poisson_ground_states_match_paper_table(nl, beta):
    """Example 3.3 (Table virial_2d_Poisson): V = (x^2 + 4 y^2)/2, h = 1/8 on [-8,8)^2, the
    2D Laplace kernel through Algorithm 1, GF-NUFFT on the GPU (FP64) to eps0 = 1e-10; each
    printed energy to one unit in its last printed place; the virial identity of a
    logarithmic kernel, 2 E_kin - 2 E_pot + beta/(4 pi) = 0 (unit mass)."""
    import torch
    g = W.cube(128, 8.0, dim=2)
    gam = (1.0, 2.0)
    V = W.harmonic_trap(g, gam)
    plan = nl.Plan(g.n, g.L, "poisson2d", "fp64", kmax=math.pi / g.h[0])
    tphi = torch.from_numpy(W.normalized_gaussian_start(g, gam)).cuda()
    tV = torch.from_numpy(V).cuda()
    steps, ch, E, st = nl.nlp_gf_solve(plan.handle, tphi, tV, beta, 0.0, 1e-2, 1e-10, 20000, 1e-12, 1000)
    plan.close()
    rows = {float(r[0]): r[1:] for r in load_golden("paper_gs_energies_2d_poisson.txt")}
    for key, txt in zip(("E", "mu", "Ekin", "Epot", "Eint"), rows[beta]):
        mant, _, ex = txt.upper().partition("E")
        ulp = 10.0 ** (-len(mant.split(".")[1]) + (int(ex) if ex else 0))
        assert abs(E[key] - float(txt)) < ulp, (key, E[key], txt)
    assert abs(2 * E["Ekin"] - 2 * E["Epot"] + beta / (4 * math.pi)) < 1e-8


def _dyn2d_run(nl, kernel, h, beta):
    """Examples 4.2 / 4.3 on the GPU: psi_0 = exp(-|x|^2/2), V = |x|^2/2 on [-16,16)^2,
    fourth-order splitting with tau = 1e-4 to t = 0.5; returns (psi, phi = U * |psi|^2)."""
    import torch
    n = int(round(32.0 / h))
    g = W.cube(n, 16.0, dim=2)
    V = W.harmonic_trap(g, (1.0, 1.0))
    X, Y = g.mesh()
    psi0 = np.exp(-0.5 * (X * X + Y * Y)).astype(np.complex128)
    P = quadrature.density_P(1.0, h)
    plan = nl.Plan(g.n, g.L, kernel, "fp64", kmax=P, counts=quadrature.default_counts(g.L, P),
                   method=1 if kernel == "coulomb2d" else 0)
    tpsi = torch.from_numpy(psi0).cuda()
    tV = torch.from_numpy(V).cuda()
    for _ in range(5000):
        nl.nlp_ts_step(plan.handle, tpsi, tV, beta, 0.0, 1e-4, 4)
    rho = (tpsi.real ** 2 + tpsi.imag ** 2).contiguous()
    phi = plan.eval(rho)
    plan.sync()
    out, ph = tpsi.cpu().numpy(), phi.cpu().numpy()
    plan.close()
    m0, m1 = float(np.sum(np.abs(psi0) ** 2)), float(np.sum(np.abs(out) ** 2))
    assert abs(m1 - m0) < 1e-11 * m0
    return out, ph


@pytest.mark.parametrize("kernel", ["coulomb2d", "poisson2d"])
@pytest.mark.parametrize("beta", [-5.0, 5.0])
def test_gpu_dynamics_examples_4_2_4_3_error_levels(nl, kernel, beta):
    """Examples 4.2 (2D Coulomb, Table dy_2d_Coulomb) and 4.3 (2D Poisson through Algorithm 1,
    Table dy_2d_Poisson): TS-NUFFT at h = 1, 1/2, 1/4 against our own h = 1/8 run.  Printed
    wave-function errors above 1e-10 (where our reference's own error, ~1e-12 by the table,
    is negligible) are reproduced within a factor 3; smaller ones are bounded by 1e-9."""
    rows = {(r[0], r[1], float(r[2])): [float(v) for v in r[3:]] for r in load_golden("paper_dynamics_2d_errors.txt")}
    ref_psi, ref_phi = _dyn2d_run(nl, kernel, 1.0 / 8, beta)
    for k, h in enumerate((1.0, 0.5, 0.25)):
        psi, phi = _dyn2d_run(nl, kernel, h, beta)
        s = int(round(h * 8))
        rp, rf = ref_psi[::s, ::s], ref_phi[::s, ::s]
        e_psi = float(np.max(np.abs(psi - rp)) / np.max(np.abs(rp)))
        e_phi = float(np.max(np.abs(phi - rf)) / np.max(np.abs(rf)))
        p_psi, p_phi = rows[(kernel, "psi", beta)][k], rows[(kernel, "phi", beta)][k]
        print("%s beta %g h %g: e_psi %.3e (paper %.3e), e_phi %.3e (paper %.3e)"
              % (kernel, beta, h, e_psi, p_psi, e_phi, p_phi))
        if p_psi > 1e-10:
            assert p_psi / 3 < e_psi < 3 * p_psi
        else:
            assert e_psi < 1e-9
