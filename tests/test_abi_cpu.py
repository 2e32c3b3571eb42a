"""CPU checks of the C-ABI library: it loads, exports every declared symbol, and
rejects invalid arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "nlpot.h")).read()
    return sorted(set(re.findall(r"\b(nlp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def nl():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_1410_3584_gb300 as m
    return m


def test_exports_every_declared_symbol(nl):
    lib = ctypes.CDLL(nl.LIB_PATH)
    names = _declared()
    assert "nlp_eval_potential" in names and "nlp_gf_step" in names and "nlp_ts_step" in names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_version(nl):
    assert nl.nlp_status_string(0) == "ok"
    assert "invalid" in nl.nlp_status_string(1)
    assert "sm_103a" in nl.nlp_version()


@pytest.mark.parametrize("n,L,kernel,kw", [
    ((31, 32, 32), (8, 8, 8), "coulomb3d", {}),          # odd n
    ((32, 32, 14), (8, 8, 8), "coulomb3d", {}),          # 14 = 2 * 7: not 2^a 3^b 5^c
    ((32, 32), (8, 8), "coulomb3d", {}),                  # dim / kernel mismatch
    ((32, 32, 32), (8, 8, 8), "coulomb2d", {}),
    ((32, 32, 32), (8, -1, 8), "coulomb3d", {}),          # L <= 0
    ((512, 32, 32), (8, 8, 8), "coulomb3d", {}),          # too large in 3D
    ((32, 32, 32), (8, 8, 8), "coulomb3d", {"tol": 1e-20}),
    ((32, 32, 32), (8, 8, 8), "coulomb3d", {"counts": (32, 31, 64)}),   # odd n_theta
    ((32, 32, 32), (8, 8, 8), "coulomb3d", {"counts": (32, 32, 63)}),   # odd n_phi
    ((32, 32, 32), (8, 8, 8), "coulomb3d", {"tile": 64}),
    ((32, 32, 32), (8, 8, 8), "coulomb3d", {"spread_variant": 2}),
    ((32, 32, 32), (8, 8, 8), "coulomb3d", {"method": 3}),
    ((32, 32, 32), (8, 8, 8), "coulomb3d", {"kmax": -1.0}),
])
def test_invalid_arguments_rejected_before_launch(nl, n, L, kernel, kw):
    with pytest.raises(nl.NlpError) as e:
        nl.nlp_plan_create(n, L, kernel, "fp64", stream=0, **kw)
    assert e.value.status == nl.NLP_ERR_INVALID_ARG


def test_precomputed_kernel_rejects_poisson(nl):
    with pytest.raises(nl.NlpError) as e:
        nl.nlp_plan_create((64, 64), (8, 8), "poisson2d", "fp64", method=1, stream=0)
    assert e.value.status == nl.NLP_ERR_UNSUPPORTED


def test_null_handles_rejected(nl):
    lib = nl.lib()
    assert lib.nlp_eval_potential(None, None, None) == nl.NLP_ERR_INVALID_ARG
    assert lib.nlp_plan_get_info(None, None) == nl.NLP_ERR_INVALID_ARG
    assert lib.nlp_ts_step(None, None, None, 1.0, 0.0, 0.1, 2) == nl.NLP_ERR_INVALID_ARG
    lib.nlp_plan_destroy(None)   # no-op
    assert lib.nlp_batch_create(None, 0, None, None) == nl.NLP_ERR_INVALID_ARG
    assert lib.nlp_batch_eval(None, None, None) == nl.NLP_ERR_INVALID_ARG
    assert lib.nlp_batch_sync(None) == nl.NLP_ERR_INVALID_ARG
    assert lib.nlp_batch_autotune(None, None, None, None, None) == nl.NLP_ERR_INVALID_ARG
    assert lib.nlp_batch_get_order(None, None) == nl.NLP_ERR_INVALID_ARG
    assert lib.nlp_batch_set_mode(None, 1, 2) == nl.NLP_ERR_INVALID_ARG
    assert lib.nlp_batch_get_mode(None, None, None) == nl.NLP_ERR_INVALID_ARG
    lib.nlp_batch_destroy(None)
    assert lib.nlp_surrogate_set_timing(None, 1) == nl.NLP_ERR_INVALID_ARG
    assert lib.nlp_surrogate_get_kernel_times(None, None, None) == nl.NLP_ERR_INVALID_ARG


def test_split_method_rejects_confined2d(nl):
    """method = 2 (the improved algorithm) covers 3D Coulomb/dipolar and 2D Coulomb/Poisson; the
    confined 2D kernel has no partition here."""
    with pytest.raises(nl.NlpError) as e:
        nl.nlp_plan_create((64, 64), (8, 8), "confined2d", "fp64", method=2, eps=0.5, stream=0)
    assert e.value.status == nl.NLP_ERR_UNSUPPORTED


def test_confined2d_rejects_negative_eps_and_3d(nl):
    with pytest.raises(nl.NlpError) as e:
        nl.nlp_plan_create((64, 64), (8, 8), "confined2d", "fp64", eps=-0.1, stream=0)
    assert e.value.status == nl.NLP_ERR_INVALID_ARG
    with pytest.raises(nl.NlpError) as e:
        nl.nlp_plan_create((32, 32, 32), (8, 8, 8), "confined2d", "fp64", eps=0.1, stream=0)
    assert e.value.status == nl.NLP_ERR_INVALID_ARG


def test_poisson1d_argument_checks(nl):
    """NLP_POISSON_1D: 1D grids only, FP64 only, method 0 only; 1D grids take no other kernel."""
    bad = [((64,), (8,), "coulomb3d", "fp64", {}), ((64, 64), (8, 8), "poisson1d", "fp64", {}),
           ((63,), (8,), "poisson1d", "fp64", {}), ((2048,), (8,), "poisson1d", "fp64", {}),
           ((64,), (-1.0,), "poisson1d", "fp64", {})]
    for n, L, k, prec, kw in bad:
        with pytest.raises(nl.NlpError) as e:
            nl.nlp_plan_create(n, L, k, prec, stream=0, **kw)
        assert e.value.status == nl.NLP_ERR_INVALID_ARG, (n, k)
    for prec, kw in (("fp32", {}), ("fp64", {"method": 1}), ("fp64", {"method": 2})):
        with pytest.raises(nl.NlpError) as e:
            nl.nlp_plan_create((64,), (8,), "poisson1d", prec, stream=0, **kw)
        assert e.value.status == nl.NLP_ERR_UNSUPPORTED
