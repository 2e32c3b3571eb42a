"""GPU checks of the learned initial guess (through the C-ABI): the tcgen05 BF16 GEMM, the
forward and backward kernels against the FP64 host model (oracle/surrogate.py), AdamW, and
the sampling of the network output onto a gradient-flow grid."""
import math

import numpy as np
import pytest

from oracle import surrogate as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1410_3584_gb300 as m
    return m


def _bf16_round(x):
    import torch
    return torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 64, 128), (256, 512, 512), (128, 1792, 512),
                                   (512, 64, 128), (128, 512, 1792)])
def test_gemm_bf16_tensor_cores(nl, M, N, K):
    """C = A B^T on tcgen05 (FP32 accumulation) vs the exact product of the BF16-rounded inputs."""
    import torch
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K))
    Bm = rng.standard_normal((N, K))
    tA = torch.from_numpy(A).to("cuda", torch.bfloat16).contiguous()
    tB = torch.from_numpy(Bm).to("cuda", torch.bfloat16).contiguous()
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    nl.nlp_gemm_bf16(tA, tB, C)
    ref = _bf16_round(A) @ _bf16_round(Bm).T
    err = np.max(np.abs(C.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 1e-5, err


def _case(seed, B=3):
    rng = np.random.default_rng(seed)
    cases = [(3.0, 1.5, "coulomb3d"), (400.0, 3.2, "dipole3d"), (40.0, 2.0, "coulomb3d"),
             (900.0, 1.1, "dipole3d")][:B]
    feats = np.stack([S.features(*c) for c in cases]).astype(np.float32)
    target = (0.05 * rng.standard_normal((B, 48, 48, 48))).astype(np.float32)
    return feats, target


def _to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _per_tensor_errors(g_gpu, g_ref):
    errs = {}
    for name, off, shp in S.layout(S.FULL)[0]:
        n = int(np.prod(shp))
        a, b = g_gpu[off:off + n].astype(np.float64), g_ref[off:off + n]
        errs[name] = float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))
    return errs


@pytest.mark.parametrize("mode,tol", [(1, 1e-4), (0, 5e-2)])
def test_forward_and_gradients_vs_fp64_oracle(nl, mode, tol):
    """Mode 1 (FP32 CUDA-core GEMMs) within FP32 rounding of the FP64 host model; mode 0
    (BF16 tensor-core GEMMs) within BF16 rounding, and aligned with it as a whole."""
    sur = nl.Surrogate(10.0, seed=11, mode=mode)
    theta = sur.get_params().astype(np.float64)
    feats, target = _case(5)
    f, t = _to_dev(feats), _to_dev(target)
    out = sur.forward(f).cpu().numpy()
    ref_out = S.forward(theta, feats.astype(np.float64))
    assert np.max(np.abs(out - ref_out)) / np.max(np.abs(ref_out)) < tol / 5
    loss, g = sur.gradients(f, t)
    ref_loss, ref_g = S.loss_and_grad(theta, feats.astype(np.float64), target.astype(np.float64))
    sur.close()
    assert abs(loss - ref_loss) / ref_loss < (1e-6 if mode == 1 else 1e-2)
    errs = _per_tensor_errors(g, ref_g)
    assert max(errs.values()) < tol, errs
    cos = float(np.dot(g, ref_g) / (np.linalg.norm(g) * np.linalg.norm(ref_g)))
    assert cos > (1 - 1e-9 if mode == 1 else 0.999), cos


def test_padding_stays_zero_and_adamw_matches(nl):
    """One AdamW step (mode 1) equals the per-element update of the host model applied to
    the library's own gradient; padded weights stay exactly zero."""
    sur = nl.Surrogate(10.0, seed=12, mode=1)
    theta = sur.get_params().astype(np.float64)
    feats, target = _case(6, B=2)
    f, t = _to_dev(feats), _to_dev(target)
    _, g = sur.gradients(f, t)
    lr, wd = 1e-3, 1e-2
    sur.train_step(f, t, lr, wd)
    new = sur.get_params().astype(np.float64)
    sur.close()
    ref, _, _ = S.adamw(theta, g.astype(np.float64), np.zeros_like(theta), np.zeros_like(theta), 1, lr, wd)
    assert np.max(np.abs(new - ref)) < 1e-6 * lr + 1e-7 * np.max(np.abs(theta))
    P = S.unpack(new)
    assert np.all(P["W0"][:, 4:] == 0) and np.all(P["W4"][1728:] == 0) and np.all(P["b4"][1728:] == 0)


@pytest.mark.parametrize("n,L,prec", [(40, 9.0, "fp64"), (36, 10.0, "fp32"), (50, 12.0, "fp64"), (48, 10.0, "fp64")])
def test_initial_guess_sampling(nl, n, L, prec):
    """nlp_surrogate_initial_guess = beta = 0 amplitude + trilinear sample of the forward
    output, clamped at zero, reflection-averaged, normalised in FP64 (host model)."""
    import torch
    sur = nl.Surrogate(10.0, seed=13, mode=1)
    f = _to_dev(nl.nlp_surrogate_features(200.0, 2.5, "dipole3d")[None, :])
    out = sur.forward(f)[0].double().cpu().numpy()
    dt = torch.float64 if prec == "fp64" else torch.float32
    phi = torch.empty((n, n, n), dtype=dt, device="cuda")
    sur.initial_guess(200.0, 2.5, "dipole3d", (n, n, n), (L, L, L), phi, prec)
    got = phi.double().cpu().numpy()
    base = sur.base(torch.tensor([2.5], dtype=torch.float32, device="cuda"))[0].double().cpu().numpy()
    sur.close()
    ref = S.resample(out, 10.0, (n, n, n), (L, L, L), 2.5)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < (1e-12 if prec == "fp64" else 1e-6)
    h3 = (2 * L / n) ** 3
    assert abs(h3 * float(np.sum(got * got)) - 1.0) < (1e-12 if prec == "fp64" else 1e-5)
    assert np.max(np.abs(base - S.base_cube(10.0, 48, 2.5))) < 1e-6


def test_kernel_class_timers(nl):
    """The per-class timers of a training step: every launch is attributed (14 GEMMs: 5 forward,
    5 weight gradients, 4 input gradients; 3 convolutions each way, the two stages of a layer's
    weight gradient timed as one interval), the times are positive, and timing does not change
    the result."""
    import torch
    feats, target = _case(5, B=3)
    f, t = _to_dev(feats), _to_dev(target)
    a = nl.Surrogate(10.0, seed=3, mode=0)
    b = nl.Surrogate(10.0, seed=3, mode=0)
    b.set_timing(True)
    steps = 3
    for _ in range(steps):
        la = a.train_step(f, t, lr=1e-3)
        lb = b.train_step(f, t, lr=1e-3)
        assert la == lb
    torch.cuda.synchronize()
    kt = b.kernel_times()
    per = {c: n / steps for c, (_, n) in kt.items()}
    assert per["gemm"] == 14 and per["conv_fwd"] == 3 and per["conv_bwd_in"] == 3 and per["conv_bwd_w"] == 3
    assert per["loss"] == 1 and per["adamw"] == 1 and per["elementwise"] > 0
    assert all(ms > 0 for ms, n in kt.values() if n > 0)
    assert np.array_equal(a.get_params(), b.get_params())
    b.set_timing(False)
    assert all(n == 0 for _, n in b.kernel_times().values())
    a.close()
    b.close()
