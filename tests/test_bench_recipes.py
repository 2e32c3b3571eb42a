"""The bench's workload recipes (grid, density, truncation radius P, quadrature counts) agree
with the documented readings as the oracle's quadrature module states them (CPU only)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import quadrature  # noqa: E402


def test_metric_workload_recipe():
    g, rho, P, counts = bench.workload()
    assert g.n == (128, 128, 128) and rho.shape == (128, 128, 128)
    assert abs(P - quadrature.density_P(min(bench.WIDTHS), max(g.h))) < 1e-12
    assert tuple(counts) == tuple(quadrature.default_counts(g.L, P)) == (144, 144, 240)


def test_2d_workload_recipe():
    g, rho, P, counts, cs, ws = bench.workload_2d()
    assert g.n == (1024, 1024) and rho.shape == (1024, 1024)
    assert abs(P - quadrature.density_P(min(ws), g.h[0])) < 1e-12
    assert tuple(counts) == tuple(quadrature.default_counts(g.L, P))


def test_batch_quadrature_recipe():
    import workloads as W
    items = W.batch_spec(8)
    assert len(items) == 8
    for it in items:
        g = W.cube(it.n, it.L)
        P, counts = bench.batch_quadrature(g, it.widths)
        assert abs(P - quadrature.density_P(min(it.widths), max(g.h), eps=1e-8)) < 1e-12
        assert tuple(counts) == tuple(quadrature.default_counts(g.L, P))
