"""GPU parity of the 1D Poisson potential (NLP_POISSON_1D, Sec. 2.2, the 1D case) against
the FP64 oracle, through the C-ABI.  Bar: relative L-infinity <= 1e-10 (FP64 plans)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import poisson1d as p1

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def nl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1410_3584_gb300 as m
    return m


def rho_three(n, L, seed=W.SEED_TRAIN):
    x = W.cube(n, L, dim=1).axes()[0]
    cs, ws, amps = W.three_gaussians_1d(seed)
    rho = np.zeros(n)
    ex = np.zeros(n)
    for (c,), s, a in zip(cs, ws, amps):
        rho += a * np.exp(-((x - c) / s) ** 2)
        ex += a * cf.poisson1d_gaussian(x, s, c)
    return rho, ex


def gpu_eval(nl, n, L, rho, **kw):
    import torch
    plan = nl.Plan((n,), (L,), "poisson1d", "fp64", **kw)
    phi = plan.eval(torch.from_numpy(rho).to("cuda", torch.float64))
    torch.cuda.synchronize()
    out = phi.cpu().numpy()
    info = plan.info
    plan.close()
    return out, info


# smallest grid, several sizes with radix 2/3/5 FFT lengths (2n), the largest grid
@pytest.mark.parametrize("n,L", [(8, 8.0), (64, 16.0), (96, 12.0), (250, 16.0), (1000, 16.0), (1024, 16.0)])
def test_parity_with_oracle(nl, n, L):
    rho, _ = rho_three(n, L)
    phi, info = gpu_eval(nl, n, L, rho)
    ref = p1.poisson1d(rho, L)
    assert cf.rel_linf(phi, ref) <= TOL
    assert info["nf"][2] == 2 * n and info["dim"] == 1


def test_closed_form_at_full_size(nl):
    n, L = 1024, 16.0
    rho, ex = rho_three(n, L)
    phi, _ = gpu_eval(nl, n, L, rho)
    assert cf.rel_linf(phi, ex) <= 1e-12


def test_truncation_radius_option(nl):
    """kmax below pi/h drops the terms |k_l| > P and changes sigma = 6 sqrt(2)/P; same on both sides."""
    n, L = 512, 16.0
    rho, ex = rho_three(n, L)
    P = 0.6 * math.pi / (2 * L / n)
    phi, info = gpu_eval(nl, n, L, rho, kmax=P)
    assert abs(info["kmax"] - P) < 1e-12
    assert cf.rel_linf(phi, p1.poisson1d(rho, L, P)) <= TOL
    assert cf.rel_linf(phi, ex) <= 1e-9


def test_zero_density_and_repeat_determinism(nl):
    import torch
    n, L = 256, 10.0
    plan = nl.Plan((n,), (L,), "poisson1d", "fp64")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert float(plan.eval(z).abs().max()) == 0.0
    rho, _ = rho_three(n, L)
    r = torch.from_numpy(rho).cuda()
    a = plan.eval(r).cpu().numpy()
    b = plan.eval(r).cpu().numpy()
    assert np.array_equal(a, b)
    plan.close()


def test_host_entry_point_and_unsupported_calls(nl):
    import torch
    n, L = 128, 12.0
    rho, _ = rho_three(n, L)
    plan = nl.Plan((n,), (L,), "poisson1d", "fp64")
    out = np.empty(n)
    nl.nlp_eval_potential_host(plan.handle, np.ascontiguousarray(rho), out)
    assert cf.rel_linf(out, p1.poisson1d(rho, L)) <= TOL
    phi = torch.ones(n, dtype=torch.float64, device="cuda")
    V = torch.zeros(n, dtype=torch.float64, device="cuda")
    lib = nl.lib()
    import ctypes
    st = lib.nlp_gf_step(plan.handle, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(V.data_ptr()), 1.0, 0.0,
                         0.1, 1e-8, 10, None, None, None)
    assert st == nl.NLP_ERR_UNSUPPORTED
    psi = torch.ones(2 * n, dtype=torch.float64, device="cuda")
    assert lib.nlp_ts_step(plan.handle, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(V.data_ptr()), 1.0, 0.0,
                           0.1, 2) == nl.NLP_ERR_UNSUPPORTED
    plan.close()
