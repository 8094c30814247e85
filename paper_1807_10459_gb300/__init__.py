"""GB300-native KSG conditional mutual information and greedy mTE parent selection.

Thin Python binding over the C ABI of ``libidtx.so`` (declared in
``include/idtx.h``).  It only marshals arguments: every step of the
estimator runs in the library's CUDA kernels.  Array arguments may be torch
tensors (CUDA or CPU) or numpy arrays; CUDA tensors are passed as device
pointers, everything else as host pointers that the library copies in.

The library is loaded on first use; if it has not been built, or no CUDA
device is present, the call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = ["IdtxError", "Settings", "Context", "load", "cmi_ksg", "cmi_batch", "mte_step",
           "mte_select_target", "mte_prune", "mte_omnibus", "mte_seqmax", "bivariate_te",
           "mte_select_past", "mte_select_sources", "library_path", "Screen", "screen_predict", "screen_loss_grad",
           "screen_train", "screen_set", "StepResult", "probe_issue_rates", "screen_load",
           "screen_features"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libidtx.so")
_lock = threading.Lock()
_lib = None
_default_ctx = {}

IDTX_OK, IDTX_EINVAL, IDTX_ENOMEM, IDTX_ECUDA, IDTX_ETIMEOUT, IDTX_EINTERNAL = range(6)
MODE_BATCHED, MODE_PLAIN, MODE_SCREENED = 0, 1, 2
KERNEL_AUTO, KERNEL_TILE, KERNEL_LIST = 0, 1, 2
SCREEN_F, SCREEN_H = 10, 64
SCREEN_NPARAMS = SCREEN_H * SCREEN_F + SCREEN_H + SCREEN_H * SCREEN_H + SCREEN_H + SCREEN_H + 1
_ERR_NAMES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EINTERNAL"}


class IdtxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"idtx error {_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Settings(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("n_surr", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("alpha", ctypes.c_double), ("timeout_ms", ctypes.c_int32),
                ("mode", ctypes.c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("dx", ctypes.c_int32), ("dy", ctypes.c_int32), ("dz", ctypes.c_int32),
                ("n_surr", ctypes.c_int32), ("n", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("seed", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("fused_launches", ctypes.c_int64),
                ("fused_ms", ctypes.c_double), ("fused_lane_ops", ctypes.c_double),
                ("scanned_a", ctypes.c_double), ("passed_a", ctypes.c_double),
                ("scanned_b", ctypes.c_double), ("passed_b", ctypes.c_double),
                ("exhaustive_pairs", ctypes.c_double), ("wait_cycles", ctypes.c_double),
                ("warp_cycles", ctypes.c_double), ("graph_launches", ctypes.c_int64),
                ("list_launches", ctypes.c_int64), ("list_walk_a", ctypes.c_double),
                ("list_walk_b", ctypes.c_double), ("brute_samples", ctypes.c_double),
                ("fallbacks", ctypes.c_double), ("tune_trials", ctypes.c_int64),
                ("list_cap_a", ctypes.c_int32), ("list_cap_b", ctypes.c_int32),
                ("list_tail_b", ctypes.c_double), ("list_tail_a", ctypes.c_double),
                ("list_sum_nz", ctypes.c_double), ("list_sum_nyz", ctypes.c_double),
                ("useful_lane_ops", ctypes.c_double)]


class IssueRates(ctypes.Structure):
    _fields_ = [("fadd_per_sm_clk", ctypes.c_double), ("fmnmx_per_sm_clk", ctypes.c_double),
                ("fsetp_add_per_sm_clk", ctypes.c_double), ("iadd_per_sm_clk", ctypes.c_double),
                ("count_mix_per_sm_clk", ctypes.c_double), ("fadd_per_s", ctypes.c_double),
                ("fmnmx_per_s", ctypes.c_double), ("fsetp_add_per_s", ctypes.c_double),
                ("iadd_per_s", ctypes.c_double), ("count_mix_per_s", ctypes.c_double),
                ("sm_clock_mhz", ctypes.c_double), ("n_sms", ctypes.c_int32)]


class Step(ctypes.Structure):
    _fields_ = [("cand", ctypes.c_int32), ("significant", ctypes.c_int32),
                ("stat", ctypes.c_double), ("pval", ctypes.c_double),
                ("n_cand", ctypes.c_int32), ("n_full", ctypes.c_int32),
                ("surr_done", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ScreenC(ctypes.Structure):
    _fields_ = [("params", ctypes.c_float * SCREEN_NPARAMS),
                ("feat_mean", ctypes.c_float * SCREEN_F),
                ("feat_scale", ctypes.c_float * SCREEN_F),
                ("delta", ctypes.c_float), ("s0", ctypes.c_int32)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load ``libidtx.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
        lib.idtx_ctx_create.argtypes = [ctypes.POINTER(vp), i32]
        lib.idtx_ctx_destroy.argtypes = [vp]
        lib.idtx_last_error.restype = ctypes.c_char_p
        lib.idtx_cmi_ksg.argtypes = [vp, vp, i32, vp, i32, vp, i32, i64, i64,
                                     ctypes.POINTER(Settings), vp, vp, vp, vp]
        lib.idtx_cmi_batch.argtypes = [vp, ctypes.POINTER(Problem), i32, i32, vp, vp]
        lib.idtx_cmi_ksg_reps.argtypes = [vp, vp, i32, vp, i32, vp, i32, i64, i64, i64,
                                          ctypes.POINTER(Settings), vp, vp, vp, vp]
        lib.idtx_mte_step.argtypes = [vp, vp, i32, i64, i32, i32, i32, i32, vp, i32, i32,
                                      ctypes.POINTER(Settings), ctypes.POINTER(Step), vp, vp]
        lib.idtx_mte_select_target.argtypes = [vp, vp, i32, i64, i32, i32, i32, i32,
                                               ctypes.POINTER(Settings), i32, vp,
                                               ctypes.POINTER(i32), ctypes.POINTER(Step),
                                               ctypes.POINTER(i32), vp]
        lib.idtx_screen_predict.argtypes = [vp, ctypes.POINTER(ScreenC), vp, i32, vp, vp]
        lib.idtx_screen_loss_grad.argtypes = [vp, ctypes.POINTER(ScreenC), vp, vp, i32,
                                              ctypes.c_float, ctypes.POINTER(ctypes.c_double),
                                              vp, vp]
        lib.idtx_screen_train.argtypes = [vp, ctypes.POINTER(ScreenC), vp, vp, i32, i32, i32,
                                          ctypes.c_float, ctypes.c_float, u64,
                                          ctypes.POINTER(ctypes.c_double), vp]
        lib.idtx_screen_set.argtypes = [vp, ctypes.POINTER(ScreenC)]
        lib.idtx_screen_load.argtypes = [vp, ctypes.c_char_p]
        lib.idtx_screen_features.argtypes = [vp, vp, i32, i32, i64, i32, i32, i32, i32, i32,
                                             vp, vp]
        lib.idtx_ctx_set_profiling.argtypes = [vp, i32]
        lib.idtx_ctx_set_graphs.argtypes = [vp, i32]
        lib.idtx_ctx_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        lib.idtx_ctx_reset_stats.argtypes = [vp]
        post = [vp, vp, i32, i64, i32, i32, i32, i32, vp, i32, ctypes.POINTER(Settings)]
        lib.idtx_mte_prune.argtypes = post + [vp, ctypes.POINTER(i32), ctypes.POINTER(Step),
                                              ctypes.POINTER(i32), vp]
        lib.idtx_mte_omnibus.argtypes = post + [ctypes.POINTER(Step), vp]
        lib.idtx_mte_seqmax.argtypes = post + [vp, vp, vp, vp]
        lib.idtx_bivariate_te.argtypes = [vp, vp, i32, i64, i32, i32, i32, i32,
                                          ctypes.POINTER(Settings), vp, vp, vp]
        lib.idtx_mte_select_past.argtypes = [vp, vp, i32, i64, i32, i32, i32,
                                             ctypes.POINTER(Settings), i32, vp,
                                             ctypes.POINTER(i32), ctypes.POINTER(Step),
                                             ctypes.POINTER(i32), vp]
        lib.idtx_mte_select_sources.argtypes = [vp, vp, i32, i64, i32, vp, i32, i32, i32,
                                                ctypes.POINTER(Settings), i32, vp,
                                                ctypes.POINTER(i32), ctypes.POINTER(Step),
                                                ctypes.POINTER(i32), vp]
        lib.idtx_probe_issue_rates.argtypes = [i32, ctypes.POINTER(IssueRates)]
        lib.idtx_ctx_set_kernel.argtypes = [vp, i32]
        lib.idtx_ctx_set_list_caps.argtypes = [vp, i32, i32]
        lib.idtx_ctx_set_wait_limit_ns.argtypes = [vp, i64]
        for name in ("idtx_cmi_ksg_reps", "idtx_mte_prune", "idtx_mte_omnibus", "idtx_mte_seqmax", "idtx_bivariate_te",
                     "idtx_mte_select_past", "idtx_mte_select_sources",
                     "idtx_ctx_set_kernel", "idtx_ctx_set_list_caps","idtx_screen_predict", "idtx_screen_loss_grad", "idtx_screen_train",
                     "idtx_screen_set", "idtx_ctx_set_profiling", "idtx_ctx_set_graphs",
                     "idtx_ctx_get_stats", "idtx_ctx_reset_stats",
                     "idtx_ctx_create", "idtx_ctx_destroy", "idtx_cmi_ksg", "idtx_cmi_batch",
                     "idtx_mte_step", "idtx_mte_select_target", "idtx_version",
                     "idtx_probe_issue_rates", "idtx_ctx_set_wait_limit_ns",
                     "idtx_screen_load", "idtx_screen_features"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def probe_issue_rates(device: int = 0) -> dict:
    """Measured lane-operation rates of the device (idtx_probe_issue_rates)."""
    out = IssueRates()
    rc = load().idtx_probe_issue_rates(device, ctypes.byref(out))
    if rc != IDTX_OK:
        raise IdtxError(rc, "issue-rate probe failed")
    return {name: getattr(out, name) for name, _ in IssueRates._fields_}


def _check(rc):
    if rc != IDTX_OK:
        msg = load().idtx_last_error()
        raise IdtxError(rc, msg.decode() if msg else "")


class Context:
    """A library context bound to one CUDA device (owns the scratch memory)."""

    def __init__(self, device: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.idtx_ctx_create(ctypes.byref(h), int(device)))
        self.handle = h
        self.device = device

    def set_profiling(self, on: bool = True):
        """Time the fused estimator kernel with CUDA events (see stats())."""
        _check(load().idtx_ctx_set_profiling(self.handle, 1 if on else 0))

    def set_graphs(self, on: bool = True):
        """Replay a captured CUDA graph for repeated identical cmi_batch calls."""
        _check(load().idtx_ctx_set_graphs(self.handle, 1 if on else 0))

    def set_kernel(self, kernel: int = KERNEL_AUTO):
        """KERNEL_AUTO (timed choice per shape), KERNEL_TILE or KERNEL_LIST."""
        _check(load().idtx_ctx_set_kernel(self.handle, int(kernel)))

    def set_list_caps(self, cap_a: int = 0, cap_b: int = 0):
        """Capacities of the list kernel's per-query lists (0: defaults)."""
        _check(load().idtx_ctx_set_list_caps(self.handle, int(cap_a), int(cap_b)))

    def set_wait_limit_ns(self, ns: int = 0):
        """Bound of this context's device waits in ns (0: settings' timeout_ms)."""
        _check(load().idtx_ctx_set_wait_limit_ns(self.handle, int(ns)))

    def stats(self) -> dict:
        st = Stats()
        _check(load().idtx_ctx_get_stats(self.handle, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in Stats._fields_}

    def reset_stats(self):
        _check(load().idtx_ctx_reset_stats(self.handle))

    def close(self):
        if self.handle:
            load().idtx_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_context(device: int = 0) -> Context:
    with _lock:
        ctx = _default_ctx.get(device)
    if ctx is None:
        ctx = Context(device)
        with _lock:
            _default_ctx[device] = ctx
    return ctx


class StepResult(tuple):
    """(cand, significant, stat, pval) of one greedy step, with .n_cand, .n_full
    and .surr_done (surrogate indices evaluated)."""

    def __new__(cls, cand, significant, stat, pval, n_cand=0, n_full=0, surr_done=0):
        obj = super().__new__(cls, (cand, significant, stat, pval))
        obj.n_cand = n_cand
        obj.n_full = n_full
        obj.surr_done = surr_done
        return obj


class Screen:
    """Learned screen: network parameters (fp32 master values), feature
    normalisation, margin delta and cheap-surrogate count s0 (idtx_screen)."""

    def __init__(self, params=None, feat_mean=None, feat_scale=None, delta=0.0, s0=8,
                 seed=0):
        if params is None:
            rng = np.random.default_rng(seed)
            params = np.zeros(SCREEN_NPARAMS, np.float32)
            # He-style initial weights, zero biases
            o = 0
            for (fan_in, fan_out) in ((SCREEN_F, SCREEN_H), (SCREEN_H, SCREEN_H), (SCREEN_H, 1)):
                params[o:o + fan_in * fan_out] = rng.standard_normal(fan_in * fan_out) * \
                    np.sqrt(2.0 / fan_in)
                o += fan_in * fan_out + fan_out
        self.params = np.ascontiguousarray(np.asarray(params, np.float32))
        self.feat_mean = np.asarray(feat_mean if feat_mean is not None else np.zeros(SCREEN_F),
                                    np.float32)
        self.feat_scale = np.asarray(feat_scale if feat_scale is not None else np.ones(SCREEN_F),
                                     np.float32)
        self.delta = float(delta)
        self.s0 = int(s0)

    def to_c(self) -> ScreenC:
        c = ScreenC()
        ctypes.memmove(c.params, self.params.ctypes.data, self.params.nbytes)
        ctypes.memmove(c.feat_mean, self.feat_mean.ctypes.data, self.feat_mean.nbytes)
        ctypes.memmove(c.feat_scale, self.feat_scale.ctypes.data, self.feat_scale.nbytes)
        c.delta = self.delta
        c.s0 = self.s0
        return c

    def save(self, path: str, **meta):
        import json
        np.savez(path, params=self.params, feat_mean=self.feat_mean, feat_scale=self.feat_scale,
                 delta=np.float32(self.delta), s0=np.int32(self.s0),
                 meta=np.array(json.dumps(meta)))

    def save_bin(self, path: str):
        """Write the screen in the flat layout idtx_screen_load reads."""
        import struct
        with open(path, "wb") as f:
            f.write(b"IDTXSCR1")
            f.write(struct.pack("<IIIIif", 1, SCREEN_F, SCREEN_H, SCREEN_NPARAMS, self.s0,
                                self.delta))
            for a in (self.params, self.feat_mean, self.feat_scale):
                f.write(np.ascontiguousarray(a, "<f4").tobytes())

    @classmethod
    def load(cls, path: str) -> "Screen":
        import ast
        import json
        d = np.load(path)
        sc = cls(d["params"], d["feat_mean"], d["feat_scale"], float(d["delta"]), int(d["s0"]))
        raw = str(d["meta"]) if "meta" in d else "{}"
        try:
            sc.meta = json.loads(raw)
        except ValueError:
            sc.meta = ast.literal_eval(raw)
        return sc


def screen_load(path: str, ctx: Context | None = None):
    """Install the screen stored at ``path`` (idtx_screen_load's layout)."""
    ctx = ctx or default_context(0)
    _check(load().idtx_screen_load(ctx.handle, os.fsencode(path)))


def screen_features(est, n: int, dz: int, k: int, n_surr: int, s0: int, dx: int = 1,
                    dy: int = 1, ctx: Context | None = None) -> np.ndarray:
    """The screen's features of each row of est [n_cand][>= 1 + s0] (estimate,
    then surrogate estimates), computed as the screened step computes them."""
    e = np.ascontiguousarray(np.asarray(est, np.float64)[:, :1 + s0])
    out = np.empty((e.shape[0], SCREEN_F), np.float32)
    ctx = ctx or default_context(0)
    _check(load().idtx_screen_features(ctx.handle, e.ctypes.data, e.shape[0], s0, n, dx, dy,
                                       dz, k, n_surr, out.ctypes.data, None))
    return out


def screen_predict(screen: Screen, feats, ctx: Context | None = None) -> np.ndarray:
    f = np.ascontiguousarray(np.asarray(feats, np.float32).reshape(-1, SCREEN_F))
    out = np.empty(f.shape[0], np.float32)
    ctx = ctx or default_context(0)
    sc = screen.to_c()
    _check(load().idtx_screen_predict(ctx.handle, ctypes.byref(sc), f.ctypes.data, f.shape[0],
                                      out.ctypes.data, None))
    return out


def screen_loss_grad(screen: Screen, feats, targets, quantile: float = 0.0,
                     ctx: Context | None = None):
    f = np.ascontiguousarray(np.asarray(feats, np.float32).reshape(-1, SCREEN_F))
    t = np.ascontiguousarray(np.asarray(targets, np.float32))
    g = np.empty(SCREEN_NPARAMS, np.float32)
    loss = ctypes.c_double()
    ctx = ctx or default_context(0)
    sc = screen.to_c()
    _check(load().idtx_screen_loss_grad(ctx.handle, ctypes.byref(sc), f.ctypes.data,
                                        t.ctypes.data, f.shape[0], float(quantile),
                                        ctypes.byref(loss), g.ctypes.data, None))
    return loss.value, g


def screen_train(screen: Screen, feats, targets, epochs=100, batch=256, lr=1e-3, seed=0,
                 quantile: float = 0.0, ctx: Context | None = None) -> float:
    """Train screen.params in place on the GPU; returns the final full-data loss."""
    f = np.ascontiguousarray(np.asarray(feats, np.float32).reshape(-1, SCREEN_F))
    t = np.ascontiguousarray(np.asarray(targets, np.float32))
    ctx = ctx or default_context(0)
    sc = screen.to_c()
    loss = ctypes.c_double()
    _check(load().idtx_screen_train(ctx.handle, ctypes.byref(sc), f.ctypes.data, t.ctypes.data,
                                    f.shape[0], int(epochs), int(batch), float(lr),
                                    float(quantile), ctypes.c_uint64(int(seed)).value,
                                    ctypes.byref(loss), None))
    screen.params = np.ctypeslib.as_array(sc.params).astype(np.float32).copy()
    return loss.value


def screen_set(screen: Screen, ctx: Context | None = None) -> None:
    """Install the screen used by MODE_SCREENED greedy calls on the context."""
    ctx = ctx or default_context(0)
    sc = screen.to_c()
    _check(load().idtx_screen_set(ctx.handle, ctypes.byref(sc)))


# ------------------------------------------------------------------ marshalling
def _is_torch(a):
    return type(a).__module__.startswith("torch")


class _Arr:
    """A [d][N] float32 (or other dtype) view with a raw pointer kept alive."""

    def __init__(self, a, dtype=np.float32, name="array"):
        if a is None:
            self.obj, self.ptr, self.d, self.n = None, None, 0, 0
            return
        if _is_torch(a):
            import torch
            t = a
            tdt = {np.float32: torch.float32, np.float64: torch.float64,
                   np.int32: torch.int32}[dtype]
            if t.dtype != tdt:
                raise TypeError(f"{name} must be {tdt}")
            if t.dim() == 1:
                t = t.unsqueeze(0)
            if not t.is_contiguous():
                t = t.contiguous()
            self.obj = t
            self.ptr = t.data_ptr()
            self.d, self.n = int(t.shape[0]), int(t.shape[1])
        else:
            arr = np.asarray(a)
            if arr.dtype != dtype:
                arr = arr.astype(dtype)
            if arr.ndim == 1:
                arr = arr[None, :]
            arr = np.ascontiguousarray(arr)
            self.obj = arr
            self.ptr = arr.ctypes.data
            self.d, self.n = int(arr.shape[0]), int(arr.shape[1])


def _stream_for(*arrays):
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return ctypes.c_void_p(0)


def _out(shape, dtype, like):
    """Output buffer: a CUDA tensor if `like` is a CUDA tensor, else numpy."""
    if like is not None and _is_torch(like) and like.is_cuda:
        import torch
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32}[dtype]
        t = torch.empty(shape, dtype=tdt, device=like.device)
        return t, t.data_ptr()
    a = np.empty(shape, dtype)
    return a, a.ctypes.data


def _settings(k, n_surr, seed, alpha=0.05, timeout_ms=0, mode=MODE_BATCHED):
    return Settings(int(k), int(n_surr), ctypes.c_uint64(int(seed) & (2**64 - 1)).value,
                    float(alpha), int(timeout_ms), int(mode))


def cmi_ksg(x, y, z=None, k: int = 4, n_surr: int = 0, seed: int = 0, want_eps: bool = False,
            want_counts: bool = False, timeout_ms: int = 0, mode: int = MODE_BATCHED,
            n_reps: int = 0, ctx: Context | None = None):
    """One KSG estimate of I(X;Y|Z) plus ``n_surr`` surrogates.

    x, y, z: [d][N] float32 (1-D means d = 1; z may be None).  Returns the
    [1+n_surr] fp64 estimates, and (if asked) eps [1+n_surr][N] and counts
    [1+n_surr][3][N] (n_xz, n_yz, n_z), as CUDA tensors when x is one, else numpy.
    n_reps > 0: surrogates permute n_reps whole replications of X (n_reps divides N).
    """
    ax, ay, az = _Arr(x, name="x"), _Arr(y, name="y"), _Arr(z, name="z")
    n = ax.n
    if ay.n != n or (az.d and az.n != n):
        raise ValueError("x, y, z must have the same number of samples")
    dev = x.device.index if (_is_torch(x) and x.is_cuda) else 0
    ctx = ctx or default_context(dev or 0)
    cmi, p_cmi = _out((1 + n_surr,), np.float64, x)
    eps, p_eps = _out((1 + n_surr, n), np.float32, x) if want_eps else (None, None)
    cnt, p_cnt = _out((1 + n_surr, 3, n), np.int32, x) if want_counts else (None, None)
    s = _settings(k, n_surr, seed, timeout_ms=timeout_ms, mode=mode)
    if n_reps:   # replication-level surrogates
        _check(load().idtx_cmi_ksg_reps(ctx.handle, ax.ptr, ax.d, ay.ptr, ay.d, az.ptr, az.d, n,
                                        n, int(n_reps), ctypes.byref(s), p_cmi, p_eps, p_cnt,
                                        _stream_for(x, y, z)))
    else:
        _check(load().idtx_cmi_ksg(ctx.handle, ax.ptr, ax.d, ay.ptr, ay.d, az.ptr, az.d, n, n,
                                   ctypes.byref(s), p_cmi, p_eps, p_cnt, _stream_for(x, y, z)))
    if want_eps or want_counts:
        out = [cmi]
        if want_eps:
            out.append(eps)
        if want_counts:
            out.append(cnt)
        return tuple(out)
    return cmi


def cmi_batch(problems, k: int = 4, ctx: Context | None = None):
    """Many uneven problems at once.  ``problems``: iterable of objects or dicts
    with x, y, z ([d][N] arrays), n_surr, seed.  Returns a list of [1+n_surr]
    fp64 arrays, one per problem."""
    probs = list(problems)
    keep = []
    arr = (Problem * len(probs))()
    like = None
    counts = []
    for i, p in enumerate(probs):
        get = (lambda key: p[key]) if isinstance(p, dict) else (lambda key: getattr(p, key))
        ax, ay, az = _Arr(get("x"), name="x"), _Arr(get("y"), name="y"), _Arr(get("z"), name="z")
        keep += [ax, ay, az]
        like = like if like is not None else get("x")
        ns = int(get("n_surr"))
        arr[i] = Problem(ax.ptr, ay.ptr, az.ptr if az.d else None, ax.d, ay.d, az.d, ns, ax.n,
                         ax.n, ctypes.c_uint64(int(get("seed")) & (2**64 - 1)).value)
        counts.append(1 + ns)
    dev = like.device.index if (_is_torch(like) and like.is_cuda) else 0
    ctx = ctx or default_context(dev or 0)
    out, p_out = _out((sum(counts),), np.float64, like)
    _check(load().idtx_cmi_batch(ctx.handle, arr, len(probs), int(k), p_out, _stream_for(like)))
    res, o = [], 0
    for c in counts:
        res.append(out[o:o + c])
        o += c
    return res


def mte_step(series, target: int, n_past: int, min_lag: int, max_lag: int, selected=(),
             step_index: int = 0, k: int = 4, n_surr: int = 200, alpha: float = 0.05,
             seed: int = 0, want_estimates: bool = False, timeout_ms: int = 0,
             mode: int = MODE_BATCHED, ctx: Context | None = None):
    """One greedy selection step; returns (cand, significant, stat, pval) and,
    if asked, the [n_proc*n_lags][1+n_surr] estimates (NaN rows: not evaluated)."""
    a = _Arr(series, name="series")
    dev = series.device.index if (_is_torch(series) and series.is_cuda) else 0
    ctx = ctx or default_context(dev or 0)
    sel = np.ascontiguousarray(np.asarray(list(selected), np.int32))
    s = _settings(k, n_surr, seed, alpha, timeout_ms, mode)
    step = Step()
    est, p_est = (None, None)
    if want_estimates:
        est = np.full((a.d * (max_lag - min_lag + 1), 1 + n_surr), np.nan, np.float64)
        p_est = est.ctypes.data
    _check(load().idtx_mte_step(ctx.handle, a.ptr, a.d, a.n, int(target), int(n_past),
                                int(min_lag), int(max_lag),
                                sel.ctypes.data if sel.size else None, int(sel.size),
                                int(step_index), ctypes.byref(s), ctypes.byref(step), p_est,
                                _stream_for(series)))
    res = StepResult(int(step.cand), bool(step.significant), float(step.stat),
                     float(step.pval), int(step.n_cand), int(step.n_full), int(step.surr_done))
    return (res, est) if want_estimates else res


def mte_select_target(series, target: int, n_past: int, min_lag: int, max_lag: int, k: int = 4,
                      n_surr: int = 200, alpha: float = 0.05, seed: int = 0,
                      max_parents: int = 10, timeout_ms: int = 0, mode: int = MODE_BATCHED,
                      ctx: Context | None = None):
    """The greedy loop for one target: dict(parents=[ids], steps=[(cand, sig, stat, p)])."""
    a = _Arr(series, name="series")
    dev = series.device.index if (_is_torch(series) and series.is_cuda) else 0
    ctx = ctx or default_context(dev or 0)
    s = _settings(k, n_surr, seed, alpha, timeout_ms, mode)
    parents = np.zeros(max(1, max_parents), np.int32)
    steps = (Step * (max_parents + 1))()
    n_par, n_steps = ctypes.c_int(), ctypes.c_int()
    _check(load().idtx_mte_select_target(ctx.handle, a.ptr, a.d, a.n, int(target), int(n_past),
                                         int(min_lag), int(max_lag), ctypes.byref(s),
                                         int(max_parents), parents.ctypes.data,
                                         ctypes.byref(n_par), steps, ctypes.byref(n_steps),
                                         _stream_for(series)))
    return dict(parents=[int(p) for p in parents[:n_par.value]],
                steps=[StepResult(int(steps[i].cand), bool(steps[i].significant),
                                  float(steps[i].stat), float(steps[i].pval),
                                  int(steps[i].n_cand), int(steps[i].n_full),
                                  int(steps[i].surr_done))
                       for i in range(n_steps.value)])


def _post_call(name, series, target, n_past, min_lag, max_lag, parents, k, n_surr, alpha, seed,
               timeout_ms, ctx, *outs):
    a = _Arr(series, name="series")
    dev = series.device.index if (_is_torch(series) and series.is_cuda) else 0
    ctx = ctx or default_context(dev or 0)
    s = _settings(k, n_surr, seed, alpha, timeout_ms, MODE_BATCHED)
    par = np.ascontiguousarray(np.asarray(parents, np.int32))
    _check(getattr(load(), name)(ctx.handle, a.ptr, a.d, a.n, int(target), int(n_past),
                                 int(min_lag), int(max_lag), par.ctypes.data, len(par),
                                 ctypes.byref(s), *outs, _stream_for(series)))
    return len(par)


def mte_prune(series, target: int, n_past: int, min_lag: int, max_lag: int, parents, k: int = 4,
              n_surr: int = 200, alpha: float = 0.05, seed: int = 0, timeout_ms: int = 0,
              ctx: Context | None = None):
    """Minimum-statistic pruning of a parent list:
    dict(kept=[ids], rounds=[(cand at the minimum, significant, T_min, p)])."""
    m = len(parents)
    kept = np.zeros(max(1, m), np.int32)
    rounds = (Step * max(1, m))()
    n_kept, n_rounds = ctypes.c_int(), ctypes.c_int()
    _post_call("idtx_mte_prune", series, target, n_past, min_lag, max_lag, parents, k, n_surr,
               alpha, seed, timeout_ms, ctx, kept.ctypes.data, ctypes.byref(n_kept), rounds,
               ctypes.byref(n_rounds))
    return dict(kept=[int(c) for c in kept[:n_kept.value]],
                rounds=[(int(rounds[i].cand), bool(rounds[i].significant), float(rounds[i].stat),
                         float(rounds[i].pval)) for i in range(n_rounds.value)])


def mte_omnibus(series, target: int, n_past: int, min_lag: int, max_lag: int, parents,
                k: int = 4, n_surr: int = 200, alpha: float = 0.05, seed: int = 0,
                timeout_ms: int = 0, ctx: Context | None = None):
    """Omnibus test of a parent set: (stat, p, significant)."""
    r = Step()
    _post_call("idtx_mte_omnibus", series, target, n_past, min_lag, max_lag, parents, k, n_surr,
               alpha, seed, timeout_ms, ctx, ctypes.byref(r))
    return float(r.stat), float(r.pval), bool(r.significant)


def mte_seqmax(series, target: int, n_past: int, min_lag: int, max_lag: int, parents,
               k: int = 4, n_surr: int = 200, alpha: float = 0.05, seed: int = 0,
               timeout_ms: int = 0, ctx: Context | None = None):
    """Sequential maximum statistic: (stats [m], pvals [m], significant [m]) by parent."""
    m = len(parents)
    stats = np.zeros(max(1, m), np.float64)
    pvals = np.zeros(max(1, m), np.float64)
    sig = np.zeros(max(1, m), np.int32)
    _post_call("idtx_mte_seqmax", series, target, n_past, min_lag, max_lag, parents, k, n_surr,
               alpha, seed, timeout_ms, ctx, stats.ctypes.data, pvals.ctypes.data,
               sig.ctypes.data)
    return stats[:m], pvals[:m], sig[:m].astype(bool)


def bivariate_te(series, target: int, n_past: int, min_lag: int, max_lag: int, k: int = 4,
                 n_surr: int = 200, seed: int = 0, timeout_ms: int = 0,
                 ctx: Context | None = None):
    """Bivariate TE of every source variable: (est [n_cand][1+n_surr], pvals [n_cand]),
    NaN at the target's own variables (numpy, host)."""
    a = _Arr(series, name="series")
    dev = series.device.index if (_is_torch(series) and series.is_cuda) else 0
    ctx = ctx or default_context(dev or 0)
    s = _settings(k, n_surr, seed, 0.05, timeout_ms, MODE_BATCHED)
    n_cand = a.d * (max_lag - min_lag + 1)
    est = np.full((n_cand, 1 + n_surr), np.nan, np.float64)
    pvals = np.zeros(n_cand, np.float64)
    _check(load().idtx_bivariate_te(ctx.handle, a.ptr, a.d, a.n, int(target), int(n_past),
                                    int(min_lag), int(max_lag), ctypes.byref(s), est.ctypes.data,
                                    pvals.ctypes.data, _stream_for(series)))
    return est, pvals


def _steps_list(steps, n):
    return [StepResult(int(steps[i].cand), bool(steps[i].significant), float(steps[i].stat),
                       float(steps[i].pval), int(steps[i].n_cand), int(steps[i].n_full),
                       int(steps[i].surr_done)) for i in range(n)]


def mte_select_past(series, target: int, min_lag: int, max_lag: int, k: int = 4,
                    n_surr: int = 200, alpha: float = 0.05, seed: int = 0, max_past: int = 5,
                    timeout_ms: int = 0, mode: int = MODE_BATCHED, ctx: Context | None = None):
    """Greedy selection of the target's own past: dict(past=[ids], steps=[...])."""
    a = _Arr(series, name="series")
    dev = series.device.index if (_is_torch(series) and series.is_cuda) else 0
    ctx = ctx or default_context(dev or 0)
    s = _settings(k, n_surr, seed, alpha, timeout_ms, mode)
    past = np.zeros(max(1, max_past), np.int32)
    steps = (Step * (max_past + 1))()
    n_past, n_steps = ctypes.c_int(), ctypes.c_int()
    _check(load().idtx_mte_select_past(ctx.handle, a.ptr, a.d, a.n, int(target), int(min_lag),
                                       int(max_lag), ctypes.byref(s), int(max_past),
                                       past.ctypes.data, ctypes.byref(n_past), steps,
                                       ctypes.byref(n_steps), _stream_for(series)))
    return dict(past=[int(c) for c in past[:n_past.value]], steps=_steps_list(steps, n_steps.value))


def mte_select_sources(series, target: int, past, min_lag: int, max_lag: int, k: int = 4,
                       n_surr: int = 200, alpha: float = 0.05, seed: int = 0,
                       max_parents: int = 10, timeout_ms: int = 0, mode: int = MODE_BATCHED,
                       ctx: Context | None = None):
    """Greedy source selection given a past (candidate ids): dict(parents=[ids], steps=[...])."""
    a = _Arr(series, name="series")
    dev = series.device.index if (_is_torch(series) and series.is_cuda) else 0
    ctx = ctx or default_context(dev or 0)
    s = _settings(k, n_surr, seed, alpha, timeout_ms, mode)
    pa = np.ascontiguousarray(np.asarray(past, np.int32))
    parents = np.zeros(max(1, max_parents), np.int32)
    steps = (Step * (max_parents + 1))()
    n_par, n_steps = ctypes.c_int(), ctypes.c_int()
    _check(load().idtx_mte_select_sources(ctx.handle, a.ptr, a.d, a.n, int(target),
                                          pa.ctypes.data if len(pa) else None, len(pa),
                                          int(min_lag), int(max_lag), ctypes.byref(s),
                                          int(max_parents), parents.ctypes.data,
                                          ctypes.byref(n_par), steps, ctypes.byref(n_steps),
                                          _stream_for(series)))
    return dict(parents=[int(c) for c in parents[:n_par.value]],
                steps=_steps_list(steps, n_steps.value))
