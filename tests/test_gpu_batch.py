"""Batched persistent evaluation (one graph-replayed launch over many FP32 plans)."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import potential

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1410_3584_gb300 as m
    return m


SPECS = [  # (n, L, kernel, widths) -- mixed grids, kernels and dimensions
    ((24, 20, 16), (6.0, 5.0, 4.5), "coulomb3d", (1.0, 1.3, 0.8)),
    ((32, 32, 32), (7.0, 7.0, 7.0), "dipole3d", (1.0, 1.6, 2.2)),
    ((30, 24, 20), (7.0, 6.0, 5.0), "coulomb3d", (1.2, 1.0, 1.5)),
    ((64, 48), (8.0, 6.0), "coulomb2d", (1.0, 1.4)),
    ((20, 20, 20), (5.0, 5.0, 5.0), "dipole3d", (0.9, 0.9, 1.8)),
]


def _build(nl, torch, stream):
    plans, rhos, phis, refs, grids = [], [], [], [], []
    for n, L, kern, a in SPECS:
        g = W.Grid(n, L)
        rho = W.gaussian(g, a)
        P = math.pi / max(g.h)
        counts = (32, 32, 64) if g.dim == 3 else (64, 128)
        pl = nl.Plan(n, L, kern, "fp32", kmax=P, counts=counts, stream=stream)
        r = torch.from_numpy(rho).to("cuda", torch.float32)
        out = pl.eval(r)
        pl.sync()      # the plan works on its own stream
        single = out.double().cpu().numpy()
        plans.append(pl)
        rhos.append(r)
        phis.append(torch.zeros_like(r))
        refs.append(single)
        grids.append((g, rho, kern, P, counts))
    return plans, rhos, phis, refs, grids


def test_batch_matches_single_plans_and_oracle(nl):
    import torch
    stream = torch.cuda.Stream()
    plans, rhos, phis, refs, grids = _build(nl, torch, stream)
    b = nl.nlp_batch_create([p.handle for p in plans], stream=stream)
    info = nl.nlp_batch_get_info(b)
    assert info["tasks"] > 0 and info["grid"] >= 152
    for rep in range(2):   # replays of the same graph
        for ph in phis:
            ph.zero_()
        torch.cuda.synchronize()
        nl.nlp_batch_eval(b, rhos, phis)
        nl.nlp_batch_sync(b)
        for ph, ref in zip(phis, refs):
            out = ph.double().cpu().numpy()
            assert np.max(np.abs(out - ref)) <= 1e-6 * np.max(np.abs(ref))
    for i in (0, 1, 3):
        g, rho, kern, P, counts = grids[i]
        o = potential.eval_nufft(rho, g, kern, P, counts, tol=1e-13)
        assert cf.rel_linf(phis[i].double().cpu().numpy(), o) < 1e-5
    # new inputs through the same graph: scaled densities give scaled potentials
    scaled = [2.5 * r for r in rhos]
    nl.nlp_batch_eval(b, scaled, phis)
    nl.nlp_batch_sync(b)
    for ph, ref in zip(phis, refs):
        assert np.max(np.abs(ph.double().cpu().numpy() - 2.5 * ref)) <= 3e-6 * np.max(np.abs(2.5 * ref))
    nl.nlp_batch_destroy(b)
    for p in plans:
        p.close()


def test_batch_autotune_keeps_results(nl):
    """The batch autotuner picks a persistent grid (CTAs per SM from 1 to the occupancy limit)
    by timing; the results of the tuned graph equal the single-plan evaluations."""
    import torch
    stream = torch.cuda.Stream()
    plans, rhos, phis, refs, grids = _build(nl, torch, stream)
    b = nl.nlp_batch_create([p.handle for p in plans], stream=stream)
    grid, ms = nl.nlp_batch_autotune(b, rhos, phis)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    info = nl.nlp_batch_get_info(b)
    assert ms > 0
    if info["mode"] == "graph":
        assert grid == 0 and info["branches"] in (1, 2, 4)
    else:
        assert grid % sms == 0 and grid >= sms and info["grid"] == grid
    for ph in phis:
        ph.zero_()
    nl.nlp_batch_eval(b, rhos, phis)
    nl.nlp_batch_sync(b)
    for ph, ref in zip(phis, refs):
        assert np.max(np.abs(ph.double().cpu().numpy() - ref)) <= 1e-6 * np.max(np.abs(ref))
    nl.nlp_batch_destroy(b)
    for p in plans:
        p.close()


@pytest.mark.parametrize("branches", [1, 2, 3])
def test_batch_graph_form_equals_single_plans(nl, branches):
    """The graph form (the plans' own stage launches on parallel branches of one graph) gives
    exactly the single-plan results; other rho / phi pointers capture the graph again; a
    switch back to the persistent form keeps working."""
    import torch
    stream = torch.cuda.Stream()
    plans, rhos, phis, refs, grids = _build(nl, torch, stream)
    singles = [torch.from_numpy(r).to("cuda", torch.float32) for r in refs]
    b = nl.nlp_batch_create([p.handle for p in plans], stream=stream)
    nl.nlp_batch_set_mode(b, "graph", branches)
    info = nl.nlp_batch_get_info(b)
    assert info["mode"] == "graph" and info["branches"] == branches
    for rep in range(2):   # capture, then a replay of the same graph
        for ph in phis:
            ph.zero_()
        torch.cuda.synchronize()
        nl.nlp_batch_eval(b, rhos, phis)
        nl.nlp_batch_sync(b)
        for ph, ref in zip(phis, singles):
            assert torch.equal(ph, ref)
    scaled = [2.5 * r for r in rhos]
    out2 = [torch.zeros_like(r) for r in rhos]
    torch.cuda.synchronize()
    nl.nlp_batch_eval(b, scaled, out2)   # new pointers: captured again
    nl.nlp_batch_sync(b)
    for ph, ref in zip(out2, refs):
        assert np.max(np.abs(ph.double().cpu().numpy() - 2.5 * ref)) <= 3e-6 * np.max(np.abs(2.5 * ref))
    nl.nlp_batch_set_mode(b, "persistent")
    for ph in phis:
        ph.zero_()
    torch.cuda.synchronize()
    nl.nlp_batch_eval(b, rhos, phis)
    nl.nlp_batch_sync(b)
    for ph, ref in zip(phis, refs):
        assert np.max(np.abs(ph.double().cpu().numpy() - ref)) <= 1e-6 * np.max(np.abs(ref))
    with pytest.raises(nl.NlpError):
        nl.nlp_batch_set_mode(b, "graph", 0)
    nl.nlp_batch_destroy(b)
    for p in plans:
        p.close()


def test_batch_wait_timeout_is_reported_and_recoverable(nl):
    import torch
    stream = torch.cuda.Stream()
    plans, rhos, phis, refs, grids = _build(nl, torch, stream)
    b = nl.nlp_batch_create([p.handle for p in plans], stream=stream)
    # item 1, stage 2 (forward FFT along axis 0) never counts as complete: the stages after
    # it poll 2000 times and give up
    nl.nlp_batch_set_wait_limit(b, 2000, 1, 2)
    nl.nlp_batch_eval(b, rhos, phis)
    st = nl.nlp_batch_sync(b, raise_on_error=False)
    assert st == nl.NLP_ERR_TIMEOUT
    nl.nlp_batch_set_wait_limit(b, 1 << 24, -1, -1)
    nl.nlp_batch_eval(b, rhos, phis)
    nl.nlp_batch_sync(b)
    for ph, ref in zip(phis, refs):
        assert np.max(np.abs(ph.double().cpu().numpy() - ref)) <= 1e-6 * np.max(np.abs(ref))
    nl.nlp_batch_destroy(b)
    for p in plans:
        p.close()


def test_autotuner_picks_a_candidate_and_caches(nl, tmp_path):
    cache = str(tmp_path / "tune.txt")
    t1, ms1 = nl.nlp_autotune_tile((32, 32, 32), (7.0, 7.0, 7.0), "coulomb3d", "fp32", cache_path=cache,
                                   counts=(32, 32, 64))
    assert t1 in (4, 8, 16) and ms1 > 0
    assert os.path.exists(cache)
    t2, ms2 = nl.nlp_autotune_tile((32, 32, 32), (7.0, 7.0, 7.0), "coulomb3d", "fp32", cache_path=cache,
                                   counts=(32, 32, 64))
    assert (t2, ms2) == (t1, pytest.approx(ms1, rel=1e-5))
    t3, _ = nl.nlp_autotune_tile((64, 48), (8.0, 6.0), "coulomb2d", "fp32", counts=(64, 128))
    assert t3 in (8, 16, 32)


def _batch_item_setup(it):
    """A batched-workload item: grid, density, P where rho-hat falls below 1e-8 (never past
    pi/h) and the default quadrature counts."""
    from oracle import quadrature
    g = W.cube(it.n, it.L)
    P = quadrature.density_P(min(it.widths), max(g.h), eps=1e-8)
    return g, W.gaussian(g, it.widths), P, quadrature.default_counts(g.L, P)


def test_batch_largest_grids_vs_oracle(nl):
    """Items of the batched workload at its largest grids, 160^3 and 192^3 (fine grids 320^3
    and 384^3: FFT lengths with radix-5 and radix-3 factors on the long-line engine paths),
    beside a 64^3 and a 96^3 item: each as a single plan and inside one batch, against the
    FP64 oracle at full size (FP32 bar 1e-5), and batch == single plan."""
    import torch
    items = W.batch_spec(64)
    pick = [next(it for it in items if it.n == n) for n in (64, 96, 160, 192)]
    stream = torch.cuda.Stream()
    plans, rhos, phis, singles, refs = [], [], [], [], []
    for it in pick:
        g, rho, P, counts = _batch_item_setup(it)
        pl = nl.Plan(g.n, g.L, it.kernel, "fp32", kmax=P, counts=counts, tol=1e-6, stream=stream)
        r = torch.from_numpy(rho).to("cuda", torch.float32)
        out = pl.eval(r)
        pl.sync()
        singles.append(out.double().cpu().numpy())
        plans.append(pl)
        rhos.append(r)
        phis.append(torch.zeros_like(r))
        refs.append(potential.eval_nufft(rho, g, it.kernel, P, counts, tol=1e-10))
    b = nl.nlp_batch_create([p.handle for p in plans], stream=stream)
    for mode in ("persistent", "graph"):
        nl.nlp_batch_set_mode(b, mode, 2)
        for ph in phis:
            ph.zero_()
        torch.cuda.synchronize()
        nl.nlp_batch_eval(b, rhos, phis)
        nl.nlp_batch_sync(b)
        for it, ph, single, ref in zip(pick, phis, singles, refs):
            out = ph.double().cpu().numpy()
            e_single, e_batch = cf.rel_linf(single, ref), cf.rel_linf(out, ref)
            print("%d^3 %s: single plan %.3e, batch (%s) %.3e vs oracle" % (it.n, it.kernel, e_single, mode, e_batch))
            assert e_single < 1e-5 and e_batch < 1e-5
            assert np.max(np.abs(out - single)) <= 1e-6 * np.max(np.abs(single))
            if mode == "graph":
                assert np.array_equal(out, single)
    nl.nlp_batch_destroy(b)
    for p in plans:
        p.close()
