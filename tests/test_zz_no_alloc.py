"""nlp_energies_noalloc: energies for callers that cannot allocate device memory during
the call (stream capture, foreign allocators).  It must agree with nlp_energies on two
calls in a row (the static scratch keeps the previous call's contents), and reject grids
beyond its 32768-point limit.  Collected last so a failure here stops nothing else."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1410_3584_gb300 as m
    return m


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("shape,kernel", [((32, 32, 32), "coulomb3d"), ((24, 20, 16), "dipole3d"),
                                          ((128, 256), "coulomb2d")], ids=["32^3", "24x20x16", "128x256"])
def test_noalloc_matches_nlp_energies(nl, prec, tol, shape, kernel):
    import torch
    L = tuple(6.0 for _ in shape)
    g = W.Grid(shape, L)
    gam = (1.0, 1.0, 2.0)[: g.dim]
    phi = W.normalized_gaussian_start(g, gam)
    V = W.harmonic_trap(g, gam)
    plan = nl.Plan(g.n, g.L, kernel, prec, counts=(32, 32, 64) if g.dim == 3 else (48, 96))
    dt = plan.torch_dtype
    tphi = torch.from_numpy(phi).to("cuda", dt)
    tV = torch.from_numpy(V).to("cuda", dt)
    ref = nl.nlp_energies(plan.handle, tphi, tV, 5.0, 0.5)
    for call in range(2):
        got = nl.nlp_energies_noalloc(plan.handle, tphi, tV, 5.0, 0.5)
        for k in ref:
            assert abs(got[k] - ref[k]) <= tol * max(1.0, abs(ref[k])), (call, k, got[k], ref[k])
    plan.close()


def test_noalloc_rejects_grids_beyond_limit(nl):
    import torch
    g = W.cube(40, 6.0)          # 64000 points > 32768
    plan = nl.Plan(g.n, g.L, "coulomb3d", "fp64", counts=(16, 16, 32))
    t = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    with pytest.raises(nl.NlpError) as e:
        nl.nlp_energies_noalloc(plan.handle, t, t, 1.0, 0.0)
    assert e.value.status == nl.NLP_ERR_INVALID_ARG
    plan.close()
