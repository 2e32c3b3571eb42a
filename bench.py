"""Benchmark: phi = U * rho evaluations per second, 3D Coulomb on a 128^3 grid.

Workload: 128^3 over [-12,12)^3, rho = exp(-(x^2 + y^2/2 + z^2/4)) (anisotropic Gaussian of
the paper's test family, Example 2.1), truncation radius P from the density (rho-hat < 1e-16
beyond it), default quadrature counts, FP32 path at NUFFT tolerance 1e-6 (headline) and FP64
path at 1e-12, each with its relative L-infinity error against the FP64 oracle.

One step = one evaluation (deconvolve/pad + 3 forward FFT passes, fused interpolate/scale/
spread, 3 inverse FFT passes + deconvolve/crop) with rho resident in HBM.  L2 (126 MB) is
flushed between timed steps by writing a 512 MB buffer outside the timed events.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the evaluation does not shard);
value = evaluations of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

N_GRID, L_BOX = 128, 12.0
WIDTHS = (1.0, math.sqrt(2.0), 2.0)
METRIC = "phi=U*rho evals/s, 3D Coulomb 128^3, FP32 vs FP64 GPU at stated L-inf error"
WORKLOAD = ("3D Coulomb 128^3 over [-12,12)^3, rho=exp(-(x^2+y^2/2+z^2/4)), density-informed P, "
            "default spherical quadrature, FP32 NUFFT tol 1e-6 (headline) / FP64 tol 1e-12")


def workload():
    """Grid, density, truncation radius P (rho-hat below 1e-16 of its peak beyond P, never past
    pi/h) and quadrature counts n_r = n_theta = roundup16(P R/2 + 16), n_phi = roundup16(P Rp + 32)."""
    g = W.cube(N_GRID, L_BOX)
    rho = W.gaussian(g, WIDTHS)
    h = g.h[0]
    P = min(math.pi / h, 2.0 * math.sqrt(math.log(1e16)) / min(WIDTHS))
    R = math.sqrt(3.0) * L_BOX
    Rp = math.sqrt(2.0) * L_BOX
    nr = int(16 * math.ceil((P * R / 2.0 + 16.0) / 16.0))
    nph = int(16 * math.ceil((P * Rp + 32.0) / 16.0))
    return g, rho, P, (nr, nr, nph)


def workload_2d():
    """2D workload: 1024^2 over [-16,16)^2, three Gaussians (seed 20141014); P where rho-hat falls
    below 1e-16 (never past pi/h); n_r = roundup16(P R/2 + 16), n_phi = roundup16(P R + 32) with
    R the half-diagonal of the box."""
    g = W.cube(1024, 16.0, dim=2)
    cs, ws = W.three_gaussians_2d(W.SEED_TRAIN)
    rho = W.gaussian_sum(g, cs, ws)
    P = min(math.pi / g.h[0], 2.0 * math.sqrt(math.log(1e16)) / min(ws))
    R = math.sqrt(sum(L * L for L in g.L))
    counts = (int(16 * math.ceil((P * R / 2.0 + 16.0) / 16.0)), int(16 * math.ceil((P * R + 32.0) / 16.0)))
    return g, rho, P, counts, cs, ws


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over all ranks (the replicas' slowest time
    bounds the whole job); identity on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_rate(world_size: int, units_per_rank: int, t_max: float) -> float:
    """Throughput of N independent replicas: all ranks' units over the slowest rank's time."""
    return world_size * units_per_rank / t_max


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "nlpot_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nme, v in zip(names, p[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nme)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def run_precision(nl, torch, prec, g, rho, P, counts, steps, warmup, flush, stream, e2e=True, method=0,
                  kernel="coulomb3d", spread_variant=0):
    tol = 1e-6 if prec == "fp32" else 1e-12
    t_plan = time.perf_counter()
    plan = nl.Plan(g.n, g.L, kernel, prec, kmax=P, counts=counts, tol=tol, stream=stream, method=method,
                   spread_variant=spread_variant)
    t_plan = time.perf_counter() - t_plan
    dt = plan.torch_dtype
    with torch.cuda.stream(stream):
        r = torch.from_numpy(rho).to("cuda", dt)
        phi = torch.empty_like(r)
    stream.synchronize()
    for _ in range(warmup):
        nl.nlp_eval_potential(plan.handle, r, phi)
    stream.synchronize()
    nl.nlp_set_stage_timing(plan.handle, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stage_tot = {}
    launches = 0
    torch.cuda.synchronize()
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[k][0].record(stream)
        nl.nlp_eval_potential(plan.handle, r, phi)
        ev[k][1].record(stream)
        st = nl.nlp_get_stage_times(plan.handle)     # syncs on the last stage event
        for name, ms in st:
            stage_tot[name] = stage_tot.get(name, 0.0) + ms
        launches += len(st)   # one kernel launch per recorded stage
    torch.cuda.synchronize()
    nl.nlp_set_stage_timing(plan.handle, False)
    times = [a.elapsed_time(b) for a, b in ev]
    out = phi.double().cpu().numpy()
    info = plan.info
    if not e2e:
        plan.close()
        return dict(times=times, stages={k: v / steps for k, v in stage_tot.items()}, phi=out, info=info,
                    launches=launches, plan_s=t_plan)
    # end-to-end through the host entry point, pinned host buffers, copies inside the timing
    hr = torch.from_numpy(rho.astype(np.float64 if prec == "fp64" else np.float32)).pin_memory()
    hp = torch.empty_like(hr).pin_memory()
    nl.nlp_eval_potential_host(plan.handle, hr.numpy(), hp.numpy())
    t0 = time.perf_counter()
    e2e_steps = max(3, steps // 2)
    for _ in range(e2e_steps):
        nl.nlp_eval_potential_host(plan.handle, hr.numpy(), hp.numpy())
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    plan.close()
    return dict(times=times, stages={k: v / steps for k, v in stage_tot.items()}, phi=out, info=info,
                launches=launches, e2e_s=e2e_s, bytes_io=int(hr.numel() * hr.element_size()))


# DRAM bytes (read + write) per launch of the interpolation and spreading kernels from one ncu
# capture of the 128^3 Coulomb workload, keyed by (precision, stage), with a digest of the sources that decide the
# kernel's traffic: once any of them changes, the counters no longer describe the kernel and
# the line reports traffic null.
TRAFFIC_SOURCES = ("paper_1410_3584_gb300/csrc/spread_reg.cu", "paper_1410_3584_gb300/csrc/spread_dev.cuh",
                   "paper_1410_3584_gb300/csrc/spread_common.cuh", "paper_1410_3584_gb300/csrc/plan.cu")
CAPTURED_TRAFFIC = {("fp32", "interp"): (65_039_616 + 1_372_160, "fb2309dde0f03593"),
                    ("fp32", "interp_spread"): (62_658_048 + 38_548_480, "fb2309dde0f03593")}


def source_digest(files=TRAFFIC_SOURCES):
    """Digest of the code of the given sources: comments and whitespace removed, so that only a
    change of the code itself marks the captured counters as stale."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"//[^\n]*|/\*.*?\*/", "", text, flags=re.S)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def captured_traffic(prec, kernel):
    ent = CAPTURED_TRAFFIC.get((prec, kernel))
    if ent is None:
        return None
    return ent[0] if source_digest() == ent[1] else None


def roofline(res, prec, alu_peak, hbm_peak, hbm_source):
    """Dominant kernel: the stage with the largest average time."""
    st = res["stages"]
    name = max(st, key=st.get)
    info = res["info"]
    t = st[name] * 1e-3
    w = info["width"]
    elt = 8 if prec == "fp32" else 16          # complex element bytes
    n, nf = info["n"], info["nf"]
    nh = nf[2] // 2 + 1
    if name in ("interp", "interp_spread"):
        # algorithmic work per processed node and tap: interpolation 2 FMA (4 flop), spreading
        # 2 FMA (4 flop).  FP32 plans run them as two kernels ("interp", then "interp_spread"
        # for the spreading half); the FP64 kernel fuses them (8 flop per tap)
        split = "interp" in st
        flops = (4.0 if split else 8.0) * info["nodes_half"] * w ** 3
        ach = flops / t
        traffic = captured_traffic(prec, name)
        out = dict(kernel="interpolate" if name == "interp" else ("spread" if split else "interp_spread"),
                   bound="alu", achieved=ach / 1e12, peak=alu_peak / 1e12, unit="TFLOP/s", frac=ach / alu_peak,
                   traffic=traffic, peak_source="measured FMA microbenchmark (nlp_measure_alu_peak)")
        if traffic:
            out["hbm"] = {"achieved_gbs": traffic / t / 1e9, "frac": traffic / t / 1e9 / hbm_peak,
                          "peak_source": hbm_source}
        return out
    # FFT passes: algorithmic bytes = one read + one write of the pass's data
    spec = nf[0] * nf[1] * nh * elt
    if name == "fwd_last" or name == "inv_last":
        byt = n[0] * n[1] * n[2] * (elt // 2) + n[0] * n[1] * nh * elt
    elif name in ("fwd_mid", "inv_mid"):
        byt = n[0] * (n[1] + nf[1]) * nh * elt
    elif name in ("fwd_first", "inv_first"):
        byt = nf[1] * (n[0] + nf[0]) * nh * elt
    else:
        byt = spec
    ach = byt / t
    return dict(kernel=name, bound="hbm", achieved=ach / 1e9, peak=hbm_peak, unit="GB/s", frac=ach / 1e9 / hbm_peak,
                traffic=None, peak_source=hbm_source)


def gpu_arm(args):
    import torch
    import paper_1410_3584_gb300 as nl
    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    g, rho, P, counts = workload()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if args.profile:
        res = run_precision(nl, torch, args.profile, g, rho, P, counts, args.steps, args.warmup, flush, stream,
                            e2e=False)
        print(json.dumps({"profile": args.profile, "ms": res["times"], "stages_ms": res["stages"]}))
        return
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_source = "measured (MEASURED_PEAKS.json hbm_gbs)"
    else:
        peaks = {"hbm_gbs": 6800.0}
        hbm_source = "fallback 6800 GB/s (MEASURED_PEAKS.json absent)"
    alu = {p: nl.nlp_measure_alu_peak(p, stream) for p in ("fp32", "fp64")}
    clk = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    res32 = run_precision(nl, torch, "fp32", g, rho, P, counts, args.steps, args.warmup, flush, stream)
    res64 = run_precision(nl, torch, "fp64", g, rho, P, counts, max(3, args.steps // 4), min(args.warmup, 3), flush,
                          stream)
    # the same discrete operator through its precomputed kernel (plan option method = 1)
    resk64 = run_precision(nl, torch, "fp64", g, rho, P, counts, args.steps, args.warmup, flush, stream, e2e=False,
                           method=1)
    resk32 = run_precision(nl, torch, "fp32", g, rho, P, counts, args.steps, args.warmup, flush, stream, e2e=False,
                           method=1)
    # the paper's improved algorithm (plan option method = 2): FFT convolution + small-ball NUFFT
    ress64 = run_precision(nl, torch, "fp64", g, rho, P, None, args.steps, args.warmup, flush, stream, e2e=False,
                           method=2)
    ress32 = run_precision(nl, torch, "fp32", g, rho, P, None, args.steps, args.warmup, flush, stream, e2e=False,
                           method=2)
    # the dipolar kernel (axis z) on the same density, grid and quadrature
    resd32 = run_precision(nl, torch, "fp32", g, rho, P, counts, args.steps, args.warmup, flush, stream, e2e=False,
                           kernel="dipole3d")
    resd64 = run_precision(nl, torch, "fp64", g, rho, P, counts, max(3, args.steps // 4), min(args.warmup, 3),
                           flush, stream, e2e=False, kernel="dipole3d")
    clocks = clk.stop()
    torch.cuda.synchronize()
    t32 = sum(res32["times"]) / 1e3
    t64 = sum(res64["times"]) / 1e3
    e2e = res32["e2e_s"]
    if ws > 1:
        t32, t64, e2e = max_over_ranks([t32, t64, e2e], "cuda")
    if rank == 0:
        from oracle import closed_forms as cf
        from oracle import native, potential
        t0 = time.perf_counter()
        ref = potential.eval_nufft(rho, g, "coulomb3d", P, counts, tol=1e-13)
        t_or = time.perf_counter() - t0
        refd = potential.eval_nufft(rho, g, "dipole3d", P, counts, tol=1e-13)
        err32 = cf.rel_linf(res32["phi"], ref)
        err64 = cf.rel_linf(res64["phi"], ref)
        X, Y, Z = g.mesh()
        # closed form on a sample of grid lines (the full grid would take minutes)
        sl = (slice(None), slice(None), slice(0, None, 16))
        ex = cf.coulomb3d_triaxial(X[sl], Y[sl], Z[sl], WIDTHS)
        err_cf = float(np.max(np.abs(res64["phi"][sl] - ex)) / np.max(np.abs(ex)))
        sm = clocks.get("sm_mhz")
        r32 = roofline(res32, "fp32", alu["fp32"], peaks["hbm_gbs"], hbm_source)
        r64 = roofline(res64, "fp64", alu["fp64"], peaks["hbm_gbs"], hbm_source)
        K = args.steps
        line = {
            "metric": METRIC,
            "value": whole_job_rate(ws, K, t32),
            "unit": "evals/s",
            "n_gpus": ws,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": 1e3 * t32 / K,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [N_GRID] * 3, "L": L_BOX, "kernel": "coulomb3d",
                       "P": P, "quadrature": [res32["info"]["n_r"], res32["info"]["n_theta"], res32["info"]["n_phi"]],
                       "nodes": res32["info"]["nodes_total"], "width_fp32": res32["info"]["width"],
                       "spread_pieces_fp32": res32["info"]["segments"], "tile_fp32": res32["info"]["tile"],
                       "width_fp64": res64["info"]["width"], "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "rel_linf_vs_oracle": err32,
            "fp64": {"value": ws * len(res64["times"]) / t64, "unit": "evals/s",
                     "ms_per_step": 1e3 * t64 / len(res64["times"]), "steps": len(res64["times"]),
                     "rel_linf_vs_oracle": err64, "rel_linf_vs_closed_form_sampled": err_cf,
                     "roofline": r64, "stages_ms": res64["stages"]},
            "precomputed_kernel": {
                "note": "plan option method=1: the quadrature sum as its exact Toeplitz convolution, kernel built "
                        "once per plan by a type-1 NUFFT; each evaluation = two pruned FFTs on the 2n grid",
                "fp64": {"value": len(resk64["times"]) / (sum(resk64["times"]) / 1e3), "unit": "evals/s",
                         "ms_per_step": sum(resk64["times"]) / len(resk64["times"]),
                         "rel_linf_vs_oracle": cf.rel_linf(resk64["phi"], ref), "plan_s": resk64["plan_s"]},
                "fp32": {"value": len(resk32["times"]) / (sum(resk32["times"]) / 1e3), "unit": "evals/s",
                         "ms_per_step": sum(resk32["times"]) / len(resk32["times"]),
                         "rel_linf_vs_oracle": cf.rel_linf(resk32["phi"], ref), "plan_s": resk32["plan_s"]}},
            "improved_split": {
                "note": "plan option method=2, Sec. 2.1 Eq. (3.9): Gaussian partition of unity; I_1 by FFT "
                        "convolution with the analytic multiplier (1-p) U-hat on the 2n grid, I_2 by NUFFT on the "
                        "small ball where p > eps",
                "fp64": {"value": len(ress64["times"]) / (sum(ress64["times"]) / 1e3), "unit": "evals/s",
                         "ms_per_step": sum(ress64["times"]) / len(ress64["times"]),
                         "rel_linf_vs_oracle": cf.rel_linf(ress64["phi"], ref), "plan_s": ress64["plan_s"],
                         "nodes": ress64["info"]["nodes_total"], "radius": ress64["info"]["split_radius"]},
                "fp32": {"value": len(ress32["times"]) / (sum(ress32["times"]) / 1e3), "unit": "evals/s",
                         "ms_per_step": sum(ress32["times"]) / len(ress32["times"]),
                         "rel_linf_vs_oracle": cf.rel_linf(ress32["phi"], ref), "plan_s": ress32["plan_s"],
                         "nodes": ress32["info"]["nodes_total"], "radius": ress32["info"]["split_radius"]}},
            "dipolar_z": {
                "note": "same density, grid, P and quadrature; kernel U-hat = 3 k_z^2/|k|^2 - 1",
                "fp32": {"value": len(resd32["times"]) / (sum(resd32["times"]) / 1e3), "unit": "evals/s",
                         "ms_per_step": sum(resd32["times"]) / len(resd32["times"]),
                         "rel_linf_vs_oracle": cf.rel_linf(resd32["phi"], refd)},
                "fp64": {"value": len(resd64["times"]) / (sum(resd64["times"]) / 1e3), "unit": "evals/s",
                         "ms_per_step": sum(resd64["times"]) / len(resd64["times"]),
                         "rel_linf_vs_oracle": cf.rel_linf(resd64["phi"], refd)}},
            "stages_ms": res32["stages"],
            "roofline": r32,
            "cpu_baseline": {"value": 1.0 / t_or, "unit": "evals/s", "cores": native.max_threads(), "kind": "oracle",
                             "sample": "one full 128^3 evaluation by the FP64 oracle (plain NUFFT, tol 1e-13, "
                                       "full symmetric node set)"},
            "e2e": {"value": ws / e2e, "unit": "evals/s", "h2d_bytes_per_step": res32["bytes_io"],
                    "d2h_bytes_per_step": res32["bytes_io"]},
            "gpu_launches": res32["launches"],
            "clocks": clocks,
            "alu_peaks_tflops": {k: v / 1e12 for k, v in alu.items()},
        }
        print(json.dumps(line))
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def batch_arm(args):
    """Batched workload: 64 densities, grids from {64,96,128,160,192}^3, Coulomb or dipolar-z,
    anisotropic Gaussians (axis ratios in [1,4]), L = 6 a_max, FP32 tol 1e-6, one CUDA graph
    replay per step in the form the batch autotuner keeps (one persistent launch, or the plans'
    own launches on parallel branches), spread tiles from the autotuner."""
    import torch
    import paper_1410_3584_gb300 as nl
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    items = W.batch_spec(args.batch_count)
    cache = os.path.join(ROOT, "_cache", "autotune_cache.txt")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    t0 = time.perf_counter()
    tiles = {}
    for n in sorted(set(it.n for it in items)):
        rep = [it for it in items if it.n == n][0]
        g = W.cube(n, rep.L)
        P, counts = batch_quadrature(g, rep.widths)
        tiles[n], _ = nl.nlp_autotune_tile(g.n, g.L, "coulomb3d", "fp32", cache_path=cache, stream=stream,
                                           kmax=P, counts=counts, tol=1e-6)
    t_tune = time.perf_counter() - t0
    plans, rhos, phis, host = [], [], [], []
    t0 = time.perf_counter()
    nodes = 0
    for it in items:
        g = W.cube(it.n, it.L)
        P, counts = batch_quadrature(g, it.widths)
        pl = nl.Plan(g.n, g.L, it.kernel, "fp32", kmax=P, counts=counts, tol=1e-6, tile=tiles[it.n], stream=stream)
        nodes += pl.info["nodes_total"]
        rho = W.gaussian(g, it.widths)
        with torch.cuda.stream(stream):
            r = torch.from_numpy(rho).to("cuda", torch.float32)
            phis.append(torch.empty_like(r))
        plans.append(pl)
        rhos.append(r)
        host.append((g, rho, it, P, counts))
    stream.synchronize()
    t_plan = time.perf_counter() - t0
    b = nl.nlp_batch_create([p.handle for p in plans], stream=stream)
    grid0 = nl.nlp_batch_get_info(b)["grid"]
    # the batch's own launch knob: persistent CTAs per SM, timed on these inputs
    t0 = time.perf_counter()
    grid_best, tune_ms = nl.nlp_batch_autotune(b, rhos, phis)
    t_btune = time.perf_counter() - t0
    info = nl.nlp_batch_get_info(b)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def time_batch(steps):
        out = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nl.nlp_batch_eval(b, rhos, phis)
            e1.record(stream)
            nl.nlp_batch_sync(b)
            out.append(e0.elapsed_time(e1))
        return sum(out) / len(out)

    # each form on its own (the persistent form at the grid and order the autotuner kept)
    forms = {}
    for mode, br in (("persistent", 1), ("graph", 1), ("graph", 2), ("graph", 4), ("graph", 8)):
        nl.nlp_batch_set_mode(b, mode, br)
        nl.nlp_batch_eval(b, rhos, phis)   # captures the graph form for these pointers
        nl.nlp_batch_sync(b)
        forms[mode if mode == "persistent" else "graph_%d_branches" % br] = time_batch(3)
    nl.nlp_batch_set_mode(b, info["mode"], info["branches"])
    for _ in range(args.warmup):
        nl.nlp_batch_eval(b, rhos, phis)
    nl.nlp_batch_sync(b)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[k][0].record(stream)
        nl.nlp_batch_eval(b, rhos, phis)
        ev[k][1].record(stream)
    nl.nlp_batch_sync(b)
    torch.cuda.synchronize()
    times = [a.elapsed_time(c) for a, c in ev]
    # the same items one plan at a time (every kernel of every plan as its own launch on the
    # same stream), and the same sequence replayed from a captured CUDA graph
    seq = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for pl, r, ph in zip(plans, rhos, phis):
            nl.nlp_eval_potential(pl.handle, r, ph)
        e1.record(stream)
        e1.synchronize()
        seq.append(e0.elapsed_time(e1))
    seq_graph = None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for pl, r, ph in zip(plans, rhos, phis):
                nl.nlp_eval_potential(pl.handle, r, ph)
        sg_t = []
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):   # replay on the stream the events are recorded on
                g.replay()
            e1.record(stream)
            e1.synchronize()
            sg_t.append(e0.elapsed_time(e1))
        seq_graph = sum(sg_t) / len(sg_t)
    except Exception as exc:   # capture not possible here: report it, keep the other numbers
        seq_graph = "not captured: %s" % type(exc).__name__
    # checks: every item against its own single-plan evaluation, a sample against the oracle
    worst_single, worst_oracle = 0.0, 0.0
    from oracle import closed_forms as cf
    from oracle import native, potential
    for i, (pl, r, ph) in enumerate(zip(plans, rhos, phis)):
        ev_out = pl.eval(r)
        pl.sync()
        single = ev_out.double().cpu().numpy()
        out = ph.double().cpu().numpy()
        worst_single = max(worst_single, float(np.max(np.abs(out - single)) / np.max(np.abs(single))))
    # CPU baseline leg: the FP64 oracle on a sample of the items (its results also state the error)
    t_or, n_or = 0.0, 0
    for i in range(0, len(items), max(1, len(items) // 4))[:4]:
        g, rho, it, P, counts = host[i]
        if g.n[0] > 96:
            continue
        t0 = time.perf_counter()
        o = potential.eval_nufft(rho, g, it.kernel, P, counts, tol=1e-12)
        t_or += time.perf_counter() - t0
        n_or += 1
        worst_oracle = max(worst_oracle, cf.rel_linf(phis[i].double().cpu().numpy(), o))
    nl.nlp_batch_destroy(b)
    for p in plans:
        p.close()
    tsum = sum(times) / 1e3
    print(json.dumps({
        "metric": "batched phi=U*rho evals/s (64 mixed 3D densities, one graph launch)",
        "value": len(items) * args.steps / tsum, "unit": "evals/s", "batches_per_s": args.steps / tsum,
        "ms_per_batch": 1e3 * tsum / args.steps, "steps": args.steps, "warmup": args.warmup,
        "items": len(items), "nodes_total": nodes, "tasks": info["tasks"], "grid_ctas": info["grid"],
        "smem_bytes": info["smem"], "tiles": tiles, "plan_s": t_plan, "tune_s": t_tune,
        "batch_autotune": {"form": info["mode"], "branches": info["branches"], "grid_default": grid0,
                           "grid_best": grid_best, "order": info["order"], "ms_best": tune_ms, "tune_s": t_btune},
        "forms_ms": forms,
        "sequential_ms": sum(seq) / len(seq), "sequential_graph_ms": seq_graph,
        "speedup_vs_sequential": (sum(seq) / len(seq)) / (1e3 * tsum / args.steps),
        "max_rel_vs_single_plan": worst_single, "max_rel_vs_oracle_sampled": worst_oracle,
        "cpu_baseline": {"value": n_or / t_or if t_or > 0 else None, "unit": "evals/s", "cores": native.max_threads(),
                         "kind": "oracle", "sample": "%d batch items of at most 96^3 by the FP64 oracle (tol 1e-12)" % n_or},
        "dtype": "f32", "data": "synthetic", "l2": "flushed between timed steps (512 MB write)"}))


def twod_arm(args):
    """2D workload: 1024^2 over [-16,16)^2, rho = three Gaussians (centres in [-4,4]^2, widths
    in [0.5,2], seed 20141014); 2D Coulomb (U-hat = 1/|k|, cancelled by the polar Jacobian) and
    the 2D Laplace kernel (U-hat = 1/|k|^2, Algorithm 1), FP64 tol 1e-12 and FP32 tol 1e-6,
    each against the FP64 oracle on the same nodes and against the closed form."""
    import torch
    import paper_1410_3584_gb300 as nl
    from oracle import closed_forms as cf
    from oracle import native, potential
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    g, rho, P, counts, cs, ws = workload_2d()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    X, Y = g.mesh()
    out = {}
    clk = ClockSampler(0)
    clk.start()
    for kernel in ("coulomb2d", "poisson2d"):
        # CPU baseline leg: the FP64 oracle on the host cores (its result also states the error)
        t0 = time.perf_counter()
        ref = potential.eval_nufft(rho, g, kernel, P, counts, tol=1e-13)
        t_or = time.perf_counter() - t0
        form = cf.coulomb2d_iso if kernel == "coulomb2d" else cf.poisson2d_iso
        exact = np.zeros_like(ref)
        for (cx, cy), s in zip(cs, ws):
            exact += form(np.sqrt((X - cx) ** 2 + (Y - cy) ** 2), s)
        for prec in ("fp32", "fp64"):
            res = run_precision(nl, torch, prec, g, rho, P, counts, args.steps, args.warmup, flush, stream,
                                e2e=False, kernel=kernel)
            t = sum(res["times"]) / 1e3
            out["%s_%s" % (kernel, prec)] = {
                "value": len(res["times"]) / t, "unit": "evals/s", "ms_per_step": 1e3 * t / len(res["times"]),
                "rel_linf_vs_oracle": cf.rel_linf(res["phi"], ref), "rel_linf_vs_closed_form": cf.rel_linf(res["phi"], exact),
                "stages_ms": res["stages"], "nodes": res["info"]["nodes_total"], "width": res["info"]["width"],
                "cpu_baseline": {"value": 1.0 / t_or, "unit": "evals/s", "cores": native.max_threads(), "kind": "oracle",
                                 "sample": "one full 1024^2 %s evaluation by the FP64 oracle (tol 1e-13)" % kernel}}
        # the improved algorithm (method 2) on the same workload
        for prec in ("fp32", "fp64"):
            res = run_precision(nl, torch, prec, g, rho, P, None, args.steps, args.warmup, flush, stream,
                                e2e=False, kernel=kernel, method=2)
            t = sum(res["times"]) / 1e3
            out["%s_%s_method2" % (kernel, prec)] = {
                "value": len(res["times"]) / t, "unit": "evals/s", "ms_per_step": 1e3 * t / len(res["times"]),
                "rel_linf_vs_oracle": cf.rel_linf(res["phi"], ref),
                "rel_linf_vs_closed_form": cf.rel_linf(res["phi"], exact),
                "nodes": res["info"]["nodes_total"], "radius": res["info"]["split_radius"]}
    out["paper_timing_table"] = paper_2d_poisson_table(nl, torch, args, flush, stream)
    clocks = clk.stop()
    print(json.dumps({"metric": "2D phi=U*rho evals/s, 1024^2, three Gaussians", "steps": args.steps,
                      "warmup": args.warmup, "config": {"grid": [1024, 1024], "L": 16.0, "P": P,
                      "quadrature": list(counts), "l2": "flushed between timed steps (512 MB write)"},
                      "results": out, "clocks": clocks, "dtype": "f32/f64", "data": "synthetic"}))


# Table tab:2d:Poisson:time: CPU seconds of the paper's Fortran code (one i7-3520M core, debug
# build) for the 2D Poisson potential of rho = exp(-r^2/1.3) on [-16,16]^2: (h, T_FFT, T_NUFFT, T_total)
PAPER_2D_POISSON_TIME = ((1.0, 0.01, 0.05, 0.06), (0.5, 0.02, 0.08, 0.10), (0.25, 0.12, 0.20, 0.32),
                         (0.125, 0.60, 0.78, 1.38))


def paper_2d_poisson_table(nl, torch, args, flush, stream):
    """The configuration of Table tab:2d:Poisson:time through method 2 (FP64): per h the device
    time of I_2 (small-ball NUFFT with Algorithm 1) and of I_1 (FFT convolution), from the
    stage events of each timed evaluation, beside the printed CPU seconds; the error against the
    E_1 closed form beside the printed e_h of Table tab_NUFFT_2D_Poisson."""
    from oracle import closed_forms as cf
    rows = []
    s = math.sqrt(1.3)
    for h, t_fft, t_nufft, t_tot in PAPER_2D_POISSON_TIME:
        n = int(round(32 / h))
        g = W.Grid((n, n), (16.0, 16.0))
        X, Y = g.mesh()
        rho = np.exp(-(X * X + Y * Y) / (s * s))
        plan = nl.Plan(g.n, g.L, "poisson2d", "fp64", kmax=math.pi / h, method=2, stream=stream)
        with torch.cuda.stream(stream):
            r = torch.from_numpy(rho).to("cuda", torch.float64)
            phi = torch.empty_like(r)
        for _ in range(args.warmup):
            nl.nlp_eval_potential(plan.handle, r, phi)
        nl.nlp_set_stage_timing(plan.handle, True)
        tot, i1, i2 = [], 0.0, 0.0
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            nl.nlp_eval_potential(plan.handle, r, phi)
            b.record(stream)
            st = nl.nlp_get_stage_times(plan.handle)
            names = [nm for nm, _ in st]
            cut = [i for i, nm in enumerate(names) if nm == "fwd_last"][-1]   # I_1 starts at its R2C pass
            i2 += sum(ms for _, ms in st[:cut])
            i1 += sum(ms for _, ms in st[cut:])
            b.synchronize()
            tot.append(a.elapsed_time(b))
        nl.nlp_set_stage_timing(plan.handle, False)
        stream.synchronize()
        err = cf.rel_linf(phi.double().cpu().numpy(), cf.poisson2d_iso(np.sqrt(X * X + Y * Y), s))
        info = plan.info
        plan.close()
        K = args.steps
        rows.append({"h": h, "grid": [n, n], "ms_total": sum(tot) / K, "ms_I1_fft": i1 / K, "ms_I2_nufft": i2 / K,
                     "nodes_I2": info["nodes_total"], "radius_I2": info["split_radius"],
                     "rel_linf_vs_closed_form": err,
                     "paper_cpu_s": {"T_FFT": t_fft, "T_NUFFT": t_nufft, "T_total": t_tot}})
    return {"note": "Table tab:2d:Poisson:time configuration, FP64 method 2; paper: one i7-3520M core, "
                    "Fortran -g, seconds (context, other hardware)", "rows": rows}


def oned_arm(args):
    """1D workload: the 1D Poisson potential (Sec. 2.2, 1D case) on 1024 points of [-16,16),
    rho = three Gaussians (centres in [-4,4], widths in [0.5,2], amplitudes in [0.5,1.5], seed
    20141014), FP64; error against the FP64 oracle and the closed form."""
    import torch
    import paper_1410_3584_gb300 as nl
    from oracle import closed_forms as cf
    from oracle import native
    from oracle import poisson1d as p1
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    n, L = 1024, 16.0
    x = W.cube(n, L, dim=1).axes()[0]
    cs, ws, amps = W.three_gaussians_1d(W.SEED_TRAIN)
    rho = np.zeros(n)
    exact = np.zeros(n)
    for (c,), s, a in zip(cs, ws, amps):
        rho += a * np.exp(-((x - c) / s) ** 2)
        exact += a * cf.poisson1d_gaussian(x, s, c)
    plan = nl.Plan((n,), (L,), "poisson1d", "fp64", stream=stream)
    with torch.cuda.stream(stream):
        r = torch.from_numpy(rho).to("cuda")
        phi = torch.empty_like(r)
    stream.synchronize()
    for _ in range(args.warmup):
        nl.nlp_eval_potential(plan.handle, r, phi)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        ev[k][0].record(stream)
        nl.nlp_eval_potential(plan.handle, r, phi)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    out = phi.cpu().numpy()
    # CPU baseline leg: the FP64 oracle (direct sums) on the host (its result also states the error)
    t0 = time.perf_counter()
    ref = p1.poisson1d(rho, L)
    t_or = time.perf_counter() - t0
    plan.close()
    print(json.dumps({"metric": "1D Poisson phi=U*rho evals/s, 1024 points, three Gaussians", "value": 1e3 / ms,
                      "unit": "evals/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                      "rel_linf_vs_oracle": cf.rel_linf(out, ref), "rel_linf_vs_closed_form": cf.rel_linf(out, exact),
                      "gpu_launches_per_eval": 5, "dtype": "f64", "data": "synthetic",
                      "cpu_baseline": {"value": 1.0 / t_or, "unit": "evals/s", "cores": native.max_threads(),
                                       "kind": "oracle", "sample": "one 1024-point evaluation by the FP64 oracle "
                                       "(direct sums)"},
                      "l2": "inputs resident (16 KB); launch- and latency-bound"}))


def groundstate_arm(args):
    """Ground states with the learned initial guess: training states from the library's own
    gradient flow on 48^3 over [-10,10)^3 (seed 20141014), the network trained by the library's
    kernels, then held-out problems (seed 20141015) solved on 96^3 over [-10,10)^3 from the
    plain Gaussian start and from the network's guess, each to the Sec. 3.2 stopping rule
    max|phi^{n+1} - phi^n|/tau <= 1e-10 (tau = 1e-2, FP64); timing = device-seconds."""
    import torch
    import paper_1410_3584_gb300 as nl
    from paper_1410_3584_gb300 import surrogate as SG
    torch.cuda.set_device(0)
    params = W.gs_problems(args.gs_train, W.SEED_TRAIN)
    t0 = time.perf_counter()
    targets, feats, info = SG.generate(params, workers=12)
    t_gen = time.perf_counter() - t0
    sur = nl.Surrogate(10.0, seed=W.SEED_TRAIN, mode=0)
    resid = SG.residual_targets(sur, targets, params)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = SG.train(sur, feats, resid, steps=args.gs_train_steps, batch=64, lr=3e-3, lr_final=7.5e-5, log_every=500)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    kernels = surrogate_kernel_times(sur, feats, resid, torch)
    del targets, resid
    solver = SG.GroundStateSolver(96, 10.0)
    cases = []
    for beta, gamma, kernel in W.gs_problems(args.gs_heldout, W.SEED_HELDOUT):
        _, n_p, t_p, E_p = solver.solve(beta, gamma, kernel, stop_tol=1e-10)
        phi0 = torch.empty((96, 96, 96), dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sur.initial_guess(beta, gamma, kernel, (96,) * 3, (10.0,) * 3, phi0)
        e1.record()
        e1.synchronize()
        t_g = e0.elapsed_time(e1) * 1e-3
        _, n_s, t_s, E_s = solver.solve(beta, gamma, kernel, phi=phi0, stop_tol=1e-10)
        cases.append({"beta": beta, "gamma": gamma, "kernel": kernel, "plain_steps": n_p, "plain_s": t_p,
                      "surrogate_steps": n_s, "surrogate_s": t_s + t_g, "guess_s": t_g,
                      "E_plain": E_p["E"], "dE": abs(E_s["E"] - E_p["E"]),
                      "converged": bool(E_p["converged"] and E_s["converged"])})
    solver.close()
    sur.close()
    tp = sum(c["plain_s"] for c in cases)
    ts = sum(c["surrogate_s"] for c in cases)
    print(json.dumps({
        "metric": "gradient-flow device-seconds to the stopping rule, 96^3, plain start vs learned start",
        "value": ts / max(1, len(cases)), "unit": "s per ground state (learned start)", "higher_is_better": False,
        "plain_s_per_state": tp / max(1, len(cases)), "speedup": tp / ts if ts > 0 else None,
        "max_dE": max(c["dE"] for c in cases), "cases": cases,
        "training": {"states": len(params), "grid": [48, 48, 48], "generation_wall_s": t_gen,
                     "generation_device_s": sum(i["seconds"] for i in info),
                     "train_steps": args.gs_train_steps, "train_s": t_train, "loss": hist},
        "train_step_kernels": kernels,
        "dtype": "f64 flow / bf16+f32 network", "data": "synthetic"}))


# dense layers of the network (in, out) and its 3^3 convolutions (C_in, C_out, grid edge)
SURROGATE_DENSE = ((64, 512), (512, 512), (512, 512), (512, 512), (512, 1792))
SURROGATE_CONV = ((8, 8, 12), (8, 8, 24), (8, 1, 48))
SURROGATE_GEMM_ROWS = 128   # the padded batch: M of every forward GEMM


def surrogate_kernel_times(sur, feats, resid, torch, steps=20, batch=64):
    """Per-class device time of a training step (the library's CUDA-event timers), measured on
    extra steps after training with the trained parameters restored afterwards, and the
    achieved rate of the tensor-core GEMMs (BF16) and the convolutions (FP32 CUDA cores)."""
    saved = sur.get_params()
    idx = torch.arange(batch, device=feats.device) % feats.shape[0]
    f, t = feats[idx].contiguous(), resid[idx].contiguous()
    sur.set_timing(True)
    for _ in range(steps):
        sur.train_step(f, t, lr=1e-5, want_loss=False)
    torch.cuda.synchronize()
    times = sur.kernel_times()
    sur.set_timing(False)
    sur.set_params(saved)
    M = SURROGATE_GEMM_ROWS
    # forward C = X W^T, backward dW = dP^T X (all layers) and dX = dP W (all but the first)
    gemm_flop = sum(2 * M * a * b for a, b in SURROGATE_DENSE) * 2 + sum(2 * M * a * b for a, b in SURROGATE_DENSE[1:])
    conv_flop = sum(2 * batch * ci * co * 27 * g ** 3 for ci, co, g in SURROGATE_CONV)   # per direction
    out = {}
    for c, (ms, n) in times.items():
        out[c] = {"ms_per_step": ms / steps, "launches_per_step": n / steps}
    g_ms = out["gemm"]["ms_per_step"]
    out["gemm"]["tflops"] = gemm_flop / (g_ms * 1e-3) / 1e12 if g_ms > 0 else None
    out["gemm"]["flop_per_step"] = gemm_flop
    for c in ("conv_fwd", "conv_bwd_in", "conv_bwd_w"):
        ms = out[c]["ms_per_step"]
        out[c]["tflops"] = conv_flop / (ms * 1e-3) / 1e12 if ms > 0 else None
        out[c]["flop_per_step"] = conv_flop
    out["note"] = ("CUDA events after every launch of %d training steps at batch %d (each interval "
                   "includes the launch gap before its kernel); GEMM flop at the padded 128 rows" % (steps, batch))
    return out


def batch_quadrature(g, widths):
    """FP32 batch items: P where rho-hat falls below 1e-8 (never past pi/h), default counts."""
    h = max(g.h)
    P = min(math.pi / h, 2.0 * math.sqrt(math.log(1e8)) / min(widths))
    R = math.sqrt(sum(L * L for L in g.L))
    Rp = math.sqrt(g.L[0] ** 2 + g.L[1] ** 2)
    nr = int(16 * math.ceil((P * R / 2.0 + 16.0) / 16.0))
    nph = int(16 * math.ceil((P * Rp + 32.0) / 16.0))
    return P, (nr, nr, nph)


def reference_arm(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    from oracle import native, potential
    g, rho, P, counts = workload()
    steps, warm = min(args.steps, 2), min(args.warmup, 1)
    for _ in range(warm):
        potential.eval_nufft(rho, g, "coulomb3d", P, counts, tol=1e-13)
    t0 = time.perf_counter()
    for _ in range(steps):
        potential.eval_nufft(rho, g, "coulomb3d", P, counts, tol=1e-13)
    t = time.perf_counter() - t0
    v = steps / t
    sample = ("full 128^3 evaluations by the FP64 oracle (plain NUFFT, tol 1e-13); %d timed, %d warm-up "
              "(capped so the run stays within minutes)" % (steps, warm))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": ws, "steps": steps,
        "warmup": warm, "ms_per_step": 1e3 * t / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [N_GRID] * 3, "L": L_BOX, "kernel": "coulomb3d"},
        "cpu_baseline": {"value": v, "unit": "evals/s", "cores": native.max_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="metric", choices=["metric", "batch", "2d", "1d", "groundstate"])
    ap.add_argument("--gs-train", type=int, default=2000, help="training ground states (groundstate workload)")
    ap.add_argument("--gs-heldout", type=int, default=16, help="held-out problems timed at 96^3")
    ap.add_argument("--gs-train-steps", type=int, default=4000)
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--profile", default=None, choices=["fp32", "fp64"],
                    help="only the timed evaluation loop of one precision (for ncu captures)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu" and not args.profile:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batch":
        batch_arm(args)
    elif args.workload == "2d":
        twod_arm(args)
    elif args.workload == "1d":
        oned_arm(args)
    elif args.workload == "groundstate":
        groundstate_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
