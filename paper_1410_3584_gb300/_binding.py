"""ctypes binding of libnlpot (include/nlpot.h): argument marshalling only.

Every computation runs in the CUDA library.  The functions carry the C-ABI names;
tensors are torch CUDA tensors (device memory and streams only) or numpy arrays for
the *_host entry point.  If the library is missing the import of this module fails
with an error that says how to build it: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libnlpot.so")

NLP_OK, NLP_ERR_INVALID_ARG, NLP_ERR_UNSUPPORTED, NLP_ERR_OOM = 0, 1, 2, 3
NLP_ERR_CUDA, NLP_ERR_TIMEOUT, NLP_ERR_DIVERGED, NLP_ERR_NOT_CONVERGED = 4, 5, 6, 7
KERNELS = {"coulomb3d": 0, "dipole3d": 1, "coulomb2d": 2, "poisson2d": 3, "confined2d": 4, "poisson1d": 5}
PRECISIONS = {"fp64": 0, "fp32": 1}


class nlp_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3)]


class nlp_opts(ctypes.Structure):
    _fields_ = [("kmax", ctypes.c_double), ("n_r", ctypes.c_int), ("n_theta", ctypes.c_int),
                ("n_phi", ctypes.c_int), ("dipole_axis", ctypes.c_double * 3), ("nufft_tol", ctypes.c_double),
                ("tile", ctypes.c_int), ("spread_variant", ctypes.c_int), ("method", ctypes.c_int), ("reserved", ctypes.c_int * 5),
                ("confine_eps", ctypes.c_double)]


class nlp_plan_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("kernel", ctypes.c_int), ("precision", ctypes.c_int),
                ("n", ctypes.c_int * 3), ("nf", ctypes.c_int * 3), ("width", ctypes.c_int),
                ("beta_es", ctypes.c_double), ("kmax", ctypes.c_double), ("n_r", ctypes.c_int),
                ("n_theta", ctypes.c_int), ("n_phi", ctypes.c_int), ("nodes_total", ctypes.c_int64),
                ("nodes_half", ctypes.c_int64), ("tiles", ctypes.c_int64), ("chunks", ctypes.c_int64),
                ("tile", ctypes.c_int), ("workspace_bytes", ctypes.c_size_t), ("sigma_poisson", ctypes.c_double),
                ("sub_tile", ctypes.c_int), ("segments", ctypes.c_int64), ("split_a", ctypes.c_double),
                ("split_radius", ctypes.c_double), ("combine_entries", ctypes.c_int64)]


class NlpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, nlp_status_string(status), status))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libnlpot.so not built (%s); run __graft_entry__.build() or "
                          "python paper_1410_3584_gb300/build.py" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    sig = {
        "nlp_plan_create": ([ctypes.POINTER(nlp_grid), I, I, ctypes.POINTER(nlp_opts), P, ctypes.POINTER(P)], I),
        "nlp_plan_destroy": ([P], None),
        "nlp_plan_get_info": ([P, ctypes.POINTER(nlp_plan_info)], I),
        "nlp_eval_potential": ([P, P, P], I),
        "nlp_eval_potential_host": ([P, P, P], I),
        "nlp_gf_step": ([P, P, P, D, D, D, D, I, ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(D)], I),
        "nlp_energies": ([P, P, P, D, D, ctypes.POINTER(D)], I),
        "nlp_ts_step": ([P, P, P, D, D, D, I], I),
        "nlp_energies_noalloc": ([P, P, P, D, D, ctypes.POINTER(D)], I),
        "nlp_set_stage_timing": ([P, I], I),
        "nlp_get_stage_times": ([P, ctypes.POINTER(I), ctypes.POINTER(D), I, ctypes.POINTER(I)], I),
        "nlp_measure_alu_peak": ([I, P, ctypes.POINTER(D)], I),
        "nlp_batch_create": ([ctypes.POINTER(P), I, P, ctypes.POINTER(P)], I),
        "nlp_batch_eval": ([P, ctypes.POINTER(P), ctypes.POINTER(P)], I),
        "nlp_batch_sync": ([P], I),
        "nlp_batch_get_info": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_size_t)], I),
        "nlp_batch_autotune": ([P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I), ctypes.POINTER(D)], I),
        "nlp_batch_set_wait_limit": ([P, ctypes.c_longlong, I, I], I),
        "nlp_batch_get_order": ([P, ctypes.POINTER(I)], I),
        "nlp_batch_set_mode": ([P, I, I], I),
        "nlp_batch_get_mode": ([P, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "nlp_batch_destroy": ([P], None),
        "nlp_autotune_tile": ([ctypes.POINTER(nlp_grid), I, I, ctypes.POINTER(nlp_opts), P, ctypes.c_char_p,
                               ctypes.POINTER(I), ctypes.POINTER(D)], I),
        "nlp_gf_solve": ([P, P, P, D, D, D, D, I, D, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D)], I),
        "nlp_surrogate_features": ([D, D, I, ctypes.POINTER(ctypes.c_float)], None),
        "nlp_surrogate_create": ([D, ctypes.c_ulonglong, I, P, ctypes.POINTER(P)], I),
        "nlp_surrogate_num_params": ([P], ctypes.c_int64),
        "nlp_surrogate_get_params": ([P, P], I),
        "nlp_surrogate_set_params": ([P, P], I),
        "nlp_surrogate_forward": ([P, P, I, P], I),
        "nlp_surrogate_gradients": ([P, P, P, I, ctypes.POINTER(D), P], I),
        "nlp_surrogate_train_step": ([P, P, P, I, ctypes.c_float, ctypes.c_float, ctypes.POINTER(D)], I),
        "nlp_surrogate_initial_guess": ([P, D, D, I, ctypes.POINTER(nlp_grid), I, P], I),
        "nlp_surrogate_base": ([P, P, I, P], I),
        "nlp_surrogate_destroy": ([P], None),
        "nlp_surrogate_set_timing": ([P, I], I),
        "nlp_surrogate_get_kernel_times": ([P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_int64)], I),
        "nlp_gemm_bf16": ([P, P, P, I, I, I, P], I),
        "nlp_status_string": ([I], ctypes.c_char_p),
        "nlp_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


_lib = _load()


def lib():
    return _lib


def nlp_status_string(status: int) -> str:
    return _lib.nlp_status_string(int(status)).decode()


def nlp_version() -> str:
    return _lib.nlp_version().decode()


def _check(st: int, where: str):
    if st != NLP_OK:
        raise NlpError(st, where)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _grid_opts(n, L, kmax=0.0, counts=None, dipole_axis=(0.0, 0.0, 0.0), tol=0.0, tile=0, spread_variant=0,
               method=0, eps=0.0):
    g = nlp_grid()
    g.dim = len(n)
    for a in range(len(n)):
        g.n[a] = int(n[a])
        g.L[a] = float(L[a])
    o = nlp_opts()
    o.kmax = float(kmax)
    if counts is not None:
        if len(counts) == 3:
            o.n_r, o.n_theta, o.n_phi = (int(c) for c in counts)
        else:
            o.n_r, o.n_phi = (int(c) for c in counts)
    for a in range(3):
        o.dipole_axis[a] = float(dipole_axis[a])
    o.nufft_tol = float(tol)
    o.tile = int(tile)
    o.spread_variant = int(spread_variant)
    o.method = int(method)
    o.confine_eps = float(eps)
    return g, o


def nlp_plan_create(n, L, kernel: str, precision: str = "fp64", kmax: float = 0.0, counts=None,
                    dipole_axis=(0.0, 0.0, 0.0), tol: float = 0.0, tile: int = 0, spread_variant: int = 0,
                    method: int = 0, stream=None, eps: float = 0.0):
    """Create a plan; returns an opaque handle (ctypes.c_void_p).  See nlpot.h."""
    g, o = _grid_opts(n, L, kmax, counts, dipole_axis, tol, tile, spread_variant, method, eps)
    h = ctypes.c_void_p()
    _check(_lib.nlp_plan_create(ctypes.byref(g), KERNELS[kernel], PRECISIONS[precision], ctypes.byref(o),
                                _stream_handle(stream), ctypes.byref(h)), "nlp_plan_create")
    return h


def nlp_plan_destroy(plan):
    _lib.nlp_plan_destroy(plan)


def nlp_plan_get_info(plan) -> dict:
    info = nlp_plan_info()
    _check(_lib.nlp_plan_get_info(plan, ctypes.byref(info)), "nlp_plan_get_info")
    out = {}
    for name, _ in nlp_plan_info._fields_:
        v = getattr(info, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _check_tensor(t, dtype, numel, name):
    if not t.is_cuda or not t.is_contiguous() or t.dtype != dtype or t.numel() != numel:
        raise ValueError("%s: need a contiguous CUDA tensor of %d %s" % (name, numel, dtype))


def nlp_eval_potential(plan, rho, phi):
    """phi <- U * rho (device tensors of the plan precision)."""
    _check(_lib.nlp_eval_potential(plan, _ptr(rho), _ptr(phi)), "nlp_eval_potential")


def nlp_eval_potential_host(plan, rho: np.ndarray, phi: np.ndarray):
    """Host arrays (C-contiguous, plan precision); copies in and out inside the call."""
    assert rho.flags["C_CONTIGUOUS"] and phi.flags["C_CONTIGUOUS"]
    _check(_lib.nlp_eval_potential_host(plan, rho.ctypes.data_as(ctypes.c_void_p),
                                        phi.ctypes.data_as(ctypes.c_void_p)), "nlp_eval_potential_host")


def nlp_gf_step(plan, phi, V, beta: float, g: float = 0.0, tau: float = 1e-2, inner_tol: float = 1e-12,
                max_inner: int = 1000, energies: bool = False, raise_on_nonconv: bool = True):
    """One gradient-flow step in place; returns (max_change, inner_iters, energies or None, status)."""
    ch = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    E = (ctypes.c_double * 5)()
    st = _lib.nlp_gf_step(plan, _ptr(phi), _ptr(V), float(beta), float(g), float(tau), float(inner_tol),
                          int(max_inner), ctypes.byref(ch), ctypes.byref(it), E if energies else None)
    if st != NLP_OK and not (st == NLP_ERR_NOT_CONVERGED and not raise_on_nonconv):
        raise NlpError(st, "nlp_gf_step")
    en = None
    if energies:
        en = dict(zip(("E", "Ekin", "Epot", "Eint", "mu"), list(E)))
    return ch.value, it.value, en, st


def nlp_gf_solve(plan, phi, V, beta: float, g: float = 0.0, tau: float = 1e-2, stop_tol: float = 1e-10,
                 max_steps: int = 100000, inner_tol: float = 1e-12, max_inner: int = 1000,
                 raise_on_nonconv: bool = True):
    """Gradient flow to max|phi^{n+1}-phi^n|/tau <= stop_tol, in place.
    Returns (steps, max_change, energies dict, status)."""
    n = ctypes.c_int(0)
    ch = ctypes.c_double(0.0)
    E = (ctypes.c_double * 5)()
    st = _lib.nlp_gf_solve(plan, _ptr(phi), _ptr(V), float(beta), float(g), float(tau), float(stop_tol),
                           int(max_steps), float(inner_tol), int(max_inner), ctypes.byref(n), ctypes.byref(ch), E)
    if st != NLP_OK and not (st == NLP_ERR_NOT_CONVERGED and not raise_on_nonconv):
        raise NlpError(st, "nlp_gf_solve")
    return n.value, ch.value, dict(zip(("E", "Ekin", "Epot", "Eint", "mu"), list(E))), st


def nlp_energies(plan, phi, V, beta: float, g: float = 0.0) -> dict:
    E = (ctypes.c_double * 5)()
    _check(_lib.nlp_energies(plan, _ptr(phi), _ptr(V), float(beta), float(g), E), "nlp_energies")
    return dict(zip(("E", "Ekin", "Epot", "Eint", "mu"), list(E)))


def nlp_energies_noalloc(plan, phi, V, beta: float, g: float = 0.0) -> dict:
    """As nlp_energies, with no device allocation (static 1 MiB scratch; grids <= 32768 points)."""
    E = (ctypes.c_double * 5)()
    _check(_lib.nlp_energies_noalloc(plan, _ptr(phi), _ptr(V), float(beta), float(g), E), "nlp_energies_noalloc")
    return dict(zip(("E", "Ekin", "Epot", "Eint", "mu"), list(E)))


def nlp_ts_step(plan, psi, V, beta: float, g: float = 0.0, tau: float = 1e-3, order: int = 2):
    """One time-splitting step in place on complex psi (torch complex tensor or interleaved view)."""
    _check(_lib.nlp_ts_step(plan, _ptr(psi), _ptr(V), float(beta), float(g), float(tau), int(order)),
           "nlp_ts_step")


STAGES = {0: "fwd_last", 1: "fwd_mid", 2: "fwd_first", 3: "combine", 4: "interp_spread",
          5: "inv_first", 6: "inv_mid", 7: "inv_last", 8: "poisson_fp64", 9: "window_sum",
          10: "interp"}


def nlp_set_stage_timing(plan, on: bool):
    _check(_lib.nlp_set_stage_timing(plan, 1 if on else 0), "nlp_set_stage_timing")


def nlp_get_stage_times(plan):
    """[(stage name, ms), ...] of the most recent evaluation (timers must be on)."""
    ids = (ctypes.c_int * 32)()
    ms = (ctypes.c_double * 32)()
    cnt = ctypes.c_int(0)
    _check(_lib.nlp_get_stage_times(plan, ids, ms, 32, ctypes.byref(cnt)), "nlp_get_stage_times")
    return [(STAGES.get(ids[i], str(ids[i])), ms[i]) for i in range(cnt.value)]


def nlp_measure_alu_peak(precision: str, stream=None) -> float:
    """Measured FMA throughput (flop/s) of the GPU for 'fp32' or 'fp64'."""
    v = ctypes.c_double(0.0)
    _check(_lib.nlp_measure_alu_peak(PRECISIONS[precision], _stream_handle(stream), ctypes.byref(v)),
           "nlp_measure_alu_peak")
    return v.value


def nlp_autotune_tile(n, L, kernel: str, precision: str = "fp32", cache_path=None, stream=None, **opts):
    """Fastest spread tile edge for this configuration: (tile, ms)."""
    g, o = _grid_opts(n, L, **opts)
    t = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(_lib.nlp_autotune_tile(ctypes.byref(g), KERNELS[kernel], PRECISIONS[precision], ctypes.byref(o),
                                  _stream_handle(stream), cache_path.encode() if cache_path else None,
                                  ctypes.byref(t), ctypes.byref(ms)), "nlp_autotune_tile")
    return t.value, ms.value


def nlp_batch_create(plans, stream=None):
    """Batch of FP32 plan handles -> batch handle (the plans must outlive it)."""
    arr = (ctypes.c_void_p * len(plans))(*[ctypes.cast(p, ctypes.c_void_p) for p in plans])
    h = ctypes.c_void_p()
    _check(_lib.nlp_batch_create(arr, len(plans), _stream_handle(stream), ctypes.byref(h)), "nlp_batch_create")
    return h


def nlp_batch_eval(batch, rhos, phis):
    """One graph-replayed persistent launch over all plans (asynchronous)."""
    r = (ctypes.c_void_p * len(rhos))(*[t.data_ptr() for t in rhos])
    f = (ctypes.c_void_p * len(phis))(*[t.data_ptr() for t in phis])
    _check(_lib.nlp_batch_eval(batch, r, f), "nlp_batch_eval")


def nlp_batch_sync(batch, raise_on_error: bool = True) -> int:
    st = _lib.nlp_batch_sync(batch)
    if raise_on_error:
        _check(st, "nlp_batch_sync")
    return st


def nlp_batch_get_info(batch) -> dict:
    t, g, sm = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_size_t(0)
    _check(_lib.nlp_batch_get_info(batch, ctypes.byref(t), ctypes.byref(g), ctypes.byref(sm)), "nlp_batch_get_info")
    o = ctypes.c_int(0)
    _check(_lib.nlp_batch_get_order(batch, ctypes.byref(o)), "nlp_batch_get_order")
    m, br = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib.nlp_batch_get_mode(batch, ctypes.byref(m), ctypes.byref(br)), "nlp_batch_get_mode")
    return {"tasks": t.value, "grid": g.value, "smem": sm.value, "order": "item-major" if o.value else "stage-major",
            "mode": BATCH_MODES_BY_ID[m.value], "branches": br.value}


BATCH_MODES = {"persistent": 0, "graph": 1}
BATCH_MODES_BY_ID = {v: k for k, v in BATCH_MODES.items()}


def nlp_batch_set_mode(batch, mode: str, branches: int = 1):
    """'persistent': one persistent kernel launch over all plans' stages; 'graph': the plans'
    own stage launches as one graph on `branches` parallel branches."""
    _check(_lib.nlp_batch_set_mode(batch, BATCH_MODES[mode], int(branches)), "nlp_batch_set_mode")


def nlp_batch_autotune(batch, rhos, phis):
    """Pick the batch's form (persistent kernel: task order and grid; graph of the plans' own
    launches: branches) by timing it on these inputs: (grid, ms), grid 0 when the graph form
    won; nlp_batch_get_info(batch) reports the mode, branches and order kept."""
    rp = (ctypes.c_void_p * len(rhos))(*[t.data_ptr() for t in rhos])
    pp = (ctypes.c_void_p * len(phis))(*[t.data_ptr() for t in phis])
    g, ms = ctypes.c_int(0), ctypes.c_double(0.0)
    _check(_lib.nlp_batch_autotune(batch, rp, pp, ctypes.byref(g), ctypes.byref(ms)), "nlp_batch_autotune")
    return g.value, ms.value


def nlp_batch_set_wait_limit(batch, polls: int, block_item: int = -1, block_stage: int = -1):
    _check(_lib.nlp_batch_set_wait_limit(batch, int(polls), int(block_item), int(block_stage)),
           "nlp_batch_set_wait_limit")


def nlp_batch_destroy(batch):
    _lib.nlp_batch_destroy(batch)


class Plan:
    """Owning wrapper: Plan(n, L, kernel, precision, ...) ... .close()."""

    def __init__(self, n, L, kernel, precision="fp64", **kw):
        self.n, self.L, self.kernel, self.precision = tuple(n), tuple(L), kernel, precision
        self.stream = kw.get("stream")
        self.handle = nlp_plan_create(n, L, kernel, precision, **kw)
        self.info = nlp_plan_get_info(self.handle)

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def eval(self, rho, phi=None):
        import torch
        if phi is None:
            phi = torch.empty_like(rho)
        _check_tensor(rho, self.torch_dtype, int(np.prod(self.n)), "rho")
        _check_tensor(phi, self.torch_dtype, int(np.prod(self.n)), "phi")
        nlp_eval_potential(self.handle, rho, phi)
        return phi

    def sync(self):
        """Wait for the work enqueued on the plan's stream (the current stream if none was given)."""
        import torch
        (self.stream or torch.cuda.current_stream()).synchronize()

    def close(self):
        if self.handle:
            nlp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SURROGATE_GRID = 48
SURROGATE_MAX_BATCH = 128


def nlp_surrogate_features(beta: float, gamma: float, kernel: str) -> np.ndarray:
    f = (ctypes.c_float * 4)()
    _lib.nlp_surrogate_features(float(beta), float(gamma), KERNELS[kernel], f)
    return np.array(list(f), dtype=np.float32)


def nlp_gemm_bf16(A, B, C, stream=None):
    """C (fp32 [M,N]) = A (bf16 [M,K]) @ B (bf16 [N,K])^T on the tensor cores (test hook)."""
    M, K = A.shape
    N = B.shape[0]
    _check(_lib.nlp_gemm_bf16(_ptr(A), _ptr(B), _ptr(C), M, N, K, _stream_handle(stream)), "nlp_gemm_bf16")


class Surrogate:
    """Learned gradient-flow initial guess (see nlpot.h): Surrogate(box_L, seed, mode)."""

    def __init__(self, box_L: float = 10.0, seed: int = 0, mode: int = 0, stream=None):
        self.box_L = float(box_L)
        self.stream = stream
        h = ctypes.c_void_p()
        _check(_lib.nlp_surrogate_create(self.box_L, int(seed), int(mode), _stream_handle(stream),
                                         ctypes.byref(h)), "nlp_surrogate_create")
        self.handle = h
        self.num_params = int(_lib.nlp_surrogate_num_params(h))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        _check(_lib.nlp_surrogate_get_params(self.handle, out.ctypes.data_as(ctypes.c_void_p)), "get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.num_params
        _check(_lib.nlp_surrogate_set_params(self.handle, p.ctypes.data_as(ctypes.c_void_p)), "set_params")

    def forward(self, feat, out=None):
        import torch
        B = feat.shape[0]
        _check_tensor(feat, torch.float32, B * 4, "feat")
        if out is None:
            out = torch.empty((B, SURROGATE_GRID, SURROGATE_GRID, SURROGATE_GRID), dtype=torch.float32,
                              device=feat.device)
        _check(_lib.nlp_surrogate_forward(self.handle, _ptr(feat), B, _ptr(out)), "nlp_surrogate_forward")
        return out

    def gradients(self, feat, target):
        B = feat.shape[0]
        loss = ctypes.c_double(0.0)
        g = np.empty(self.num_params, dtype=np.float32)
        _check(_lib.nlp_surrogate_gradients(self.handle, _ptr(feat), _ptr(target), B, ctypes.byref(loss),
                                            g.ctypes.data_as(ctypes.c_void_p)), "nlp_surrogate_gradients")
        return loss.value, g

    def train_step(self, feat, target, lr: float, weight_decay: float = 0.0, want_loss: bool = True):
        B = feat.shape[0]
        loss = ctypes.c_double(0.0)
        _check(_lib.nlp_surrogate_train_step(self.handle, _ptr(feat), _ptr(target), B, float(lr),
                                             float(weight_decay), ctypes.byref(loss) if want_loss else None),
               "nlp_surrogate_train_step")
        return loss.value if want_loss else None

    KERNEL_CLASSES = ("gemm", "conv_fwd", "conv_bwd_in", "conv_bwd_w", "elementwise", "loss", "adamw")

    def set_timing(self, on: bool):
        _check(_lib.nlp_surrogate_set_timing(self.handle, 1 if on else 0), "nlp_surrogate_set_timing")

    def kernel_times(self) -> dict:
        """{class: (milliseconds, launches)} summed over the training steps since set_timing(True)."""
        n = len(self.KERNEL_CLASSES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        _check(_lib.nlp_surrogate_get_kernel_times(self.handle, ms, cnt), "nlp_surrogate_get_kernel_times")
        return {c: (ms[i], int(cnt[i])) for i, c in enumerate(self.KERNEL_CLASSES)}

    def base(self, gamma, out=None):
        """The beta = 0 amplitude on the 48^3 cube for each gamma (device FP32 [B])."""
        import torch
        B = gamma.shape[0]
        _check_tensor(gamma, torch.float32, B, "gamma")
        if out is None:
            out = torch.empty((B, SURROGATE_GRID, SURROGATE_GRID, SURROGATE_GRID), dtype=torch.float32,
                              device=gamma.device)
        _check(_lib.nlp_surrogate_base(self.handle, _ptr(gamma), B, _ptr(out)), "nlp_surrogate_base")
        return out

    def initial_guess(self, beta: float, gamma: float, kernel: str, n, L, phi, precision: str = "fp64"):
        g, _ = _grid_opts(n, L)
        _check(_lib.nlp_surrogate_initial_guess(self.handle, float(beta), float(gamma), KERNELS[kernel],
                                                ctypes.byref(g), PRECISIONS[precision], _ptr(phi)),
               "nlp_surrogate_initial_guess")
        return phi

    def close(self):
        if self.handle:
            _lib.nlp_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
