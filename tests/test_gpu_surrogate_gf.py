"""The learned initial guess end to end on the GPU: ground states computed by the library's
gradient flow (several host threads, one stream each), the network trained on them by the
library's kernels, and on held-out problems the flow started from the network reaching the
plain flow's ground state (energy within 1e-9) in fewer device-seconds.

Scale: 48^3 grids over [-10, 10)^3 and a few dozen training states, so that the test runs in
about two minutes; the benchmark's surrogate workload runs the larger configuration."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

N_TRAIN = 64
N_HELDOUT = 3


@pytest.fixture(scope="module")
def nl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1410_3584_gb300 as m
    return m


def test_surrogate_start_reaches_plain_ground_state_faster(nl):
    import torch
    from paper_1410_3584_gb300 import surrogate as SG
    params = W.gs_problems(N_TRAIN, W.SEED_TRAIN)
    targets, feats, info = SG.generate(params, workers=12)
    assert all(i["converged"] for i in info)
    # the threaded generation equals a sequential solve of the same problem
    solver = SG.GroundStateSolver(48, 10.0)
    phi, _, _, _ = solver.solve(*params[0], stop_tol=1e-6, inner_tol=1e-9)
    assert float((targets[0].double() - phi).abs().max()) < 1e-6
    sur = nl.Surrogate(10.0, seed=W.SEED_TRAIN, mode=0)
    resid = SG.residual_targets(sur, targets, params)
    hist = SG.train(sur, feats, resid, steps=3000, batch=32, lr=2e-3, lr_final=5e-5)
    assert hist[-1][1] < 0.05 * hist[0][1], hist
    tot_plain = tot_sur = 0.0
    for beta, gamma, kernel in W.gs_problems(N_HELDOUT, W.SEED_HELDOUT):
        _, n_p, t_p, E_p = solver.solve(beta, gamma, kernel, stop_tol=1e-10)
        phi0 = torch.empty((48, 48, 48), dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sur.initial_guess(beta, gamma, kernel, (48,) * 3, (10.0,) * 3, phi0)
        e1.record()
        e1.synchronize()
        t_guess = e0.elapsed_time(e1) * 1e-3
        _, n_s, t_s, E_s = solver.solve(beta, gamma, kernel, phi=phi0, stop_tol=1e-10)
        print("beta %.1f gamma %.2f %s: plain %d steps %.2f s, surrogate %d steps %.2f s (+%.4f s guess), dE %.2e"
              % (beta, gamma, kernel, n_p, t_p, n_s, t_s, t_guess, abs(E_s["E"] - E_p["E"])))
        assert E_p["converged"] and E_s["converged"]
        assert abs(E_s["E"] - E_p["E"]) < 1e-9
        tot_plain += t_p
        tot_sur += t_s + t_guess
    solver.close()
    assert tot_sur < tot_plain, (tot_sur, tot_plain)
    # the held-out grid of the ground-state workload (96^3), one Coulomb and one dipolar problem:
    # the flow from the guess reaches the plain flow's energy (speed is the benchmark's to report)
    held = W.gs_problems(16, W.SEED_HELDOUT)
    picks = [next(p for p in held if p[2] == k) for k in ("coulomb3d", "dipole3d")]
    big = SG.GroundStateSolver(96, 10.0)
    for beta, gamma, kernel in picks:
        _, n_p, t_p, E_p = big.solve(beta, gamma, kernel, stop_tol=1e-10)
        phi0 = torch.empty((96, 96, 96), dtype=torch.float64, device="cuda")
        sur.initial_guess(beta, gamma, kernel, (96,) * 3, (10.0,) * 3, phi0)
        _, n_s, t_s, E_s = big.solve(beta, gamma, kernel, phi=phi0, stop_tol=1e-10)
        print("96^3 beta %.1f gamma %.2f %s: plain %d steps %.2f s, surrogate %d steps %.2f s, dE %.2e"
              % (beta, gamma, kernel, n_p, t_p, n_s, t_s, abs(E_s["E"] - E_p["E"])))
        assert E_p["converged"] and E_s["converged"]
        assert abs(E_s["E"] - E_p["E"]) < 1e-9
    big.close()
    sur.close()
