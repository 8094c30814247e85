"""CPU oracle for the KSG conditional-mutual-information path (TEST INFRASTRUCTURE).

This package is the plain, slow, brute-force statement of what the GPU library
computes (see ``ksg_oracle.c`` for the definitions and the passages of the IDTxl
paper, arXiv 1807.10459, that each function follows).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA library and imports nothing from it.

Parity status: every function is pinned by tests under ``tests/`` (hand-worked
example, closed forms, invariants, published generator outputs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ksg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_F32P = ctypes.POINTER(ctypes.c_float)
_F64P = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)
_U64P = ctypes.POINTER(ctypes.c_uint64)


class OrcStep(ctypes.Structure):
    _fields_ = [("cand", ctypes.c_int32), ("significant", ctypes.c_int32),
                ("stat", ctypes.c_double), ("pval", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile ``ksg_oracle.c`` into ``liboracle.so`` with gcc (no fast-math)."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.orc_psi_table.argtypes = [ctypes.c_int64, _F64P]
        lib.orc_ksg_counts.argtypes = [_F32P, ctypes.c_int, _F32P, ctypes.c_int, _F32P, ctypes.c_int,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _F32P, _I32P,
                                       _I32P, _I32P]
        lib.orc_ksg_counts_at.argtypes = [_F32P, ctypes.c_int, _F32P, ctypes.c_int, _F32P,
                                          ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int, _I64P, ctypes.c_int64, _F32P, _I32P,
                                          _I32P, _I32P]
        lib.orc_cmi_ksg.argtypes = [_F32P, ctypes.c_int, _F32P, ctypes.c_int, _F32P, ctypes.c_int,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _F64P, _F32P,
                                    _I32P]
        lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_int, _U64P]
        lib.orc_perm.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, _I64P]
        lib.orc_cmi_surrogates.argtypes = [_F32P, ctypes.c_int, _F32P, ctypes.c_int, _F32P,
                                           ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _F64P]
        lib.orc_select_target.argtypes = [_F32P, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                          ctypes.c_int, ctypes.POINTER(OrcStep),
                                          ctypes.POINTER(ctypes.c_int), _I32P,
                                          ctypes.POINTER(ctypes.c_int), _F64P]
        lib.orc_bf16_round.argtypes = [ctypes.c_float]
        lib.orc_bf16_round.restype = ctypes.c_float
        lib.orc_mlp_forward.argtypes = [_F32P, ctypes.c_int, ctypes.c_int, _F32P, _F32P, _F32P,
                                        ctypes.c_int64, ctypes.c_int, _F64P]
        lib.orc_mlp_loss_grad.argtypes = [_F32P, ctypes.c_int, ctypes.c_int, _F32P, _F32P, _F32P,
                                          _F32P, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                          _F64P, _F64P]
        post = [_F32P, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                ctypes.c_int, _I32P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                ctypes.c_uint64]
        lib.orc_prune.argtypes = post + [_I32P, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(OrcStep), ctypes.POINTER(ctypes.c_int)]
        lib.orc_omnibus.argtypes = post + [_F64P, _F64P, ctypes.POINTER(ctypes.c_int)]
        lib.orc_seqmax.argtypes = post + [_F64P, _F64P, _I32P]
        lib.orc_bivariate_te.argtypes = [_F32P, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_uint64, _F64P, _F64P]
        lib.orc_select_past.argtypes = [_F32P, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.POINTER(OrcStep), ctypes.POINTER(ctypes.c_int),
                                        _I32P, ctypes.POINTER(ctypes.c_int)]
        lib.orc_select_sources.argtypes = [_F32P, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                           _I32P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(OrcStep),
                                           ctypes.POINTER(ctypes.c_int), _I32P,
                                           ctypes.POINTER(ctypes.c_int)]
        lib.orc_cmi_surrogates_reps.argtypes = [_F32P, ctypes.c_int, _F32P, ctypes.c_int, _F32P,
                                                ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                ctypes.c_int64, _F64P]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _cols(a, n=None):
    """Return (contiguous float32 [d][n] array, d).  ``None`` means d = 0."""
    if a is None:
        return np.zeros((0, n if n is not None else 1), np.float32), 0
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if a.ndim == 1:
        a = a[None, :]
    return a, a.shape[0]


def _fp(a):
    return a.ctypes.data_as(_F32P)


def psi_table(n_max: int) -> np.ndarray:
    """psi(n) for n = 0..n_max (index 0 is NaN), by psi(1) = -gamma and the recurrence."""
    out = np.empty(n_max + 1, np.float64)
    if _load().orc_psi_table(n_max, out.ctypes.data_as(_F64P)) != 0:
        raise ValueError("bad n_max")
    return out


def ksg_counts(x, y, z, k: int):
    """(eps, nxz, nyz, nz) of one estimate; x, y, z are [d][N] (z may be None)."""
    x, dx = _cols(x)
    n = x.shape[1]
    y, dy = _cols(y)
    z, dz = _cols(z, n)
    eps = np.empty(n, np.float32)
    nxz = np.empty(n, np.int32)
    nyz = np.empty(n, np.int32)
    nz = np.empty(n, np.int32)
    rc = _load().orc_ksg_counts(_fp(x), dx, _fp(y), dy, _fp(z), dz, n, n, k, _fp(eps),
                                nxz.ctypes.data_as(_I32P), nyz.ctypes.data_as(_I32P),
                                nz.ctypes.data_as(_I32P))
    if rc != 0:
        raise ValueError("orc_ksg_counts: invalid arguments")
    return eps, nxz, nyz, nz


def ksg_counts_at(x, y, z, k: int, idx):
    """(eps, nxz, nyz, nz) for the listed query indices only (each O(N))."""
    x, dx = _cols(x)
    n = x.shape[1]
    y, dy = _cols(y)
    z, dz = _cols(z, n)
    idx = np.ascontiguousarray(np.asarray(idx, np.int64))
    m = idx.shape[0]
    eps = np.empty(m, np.float32)
    nxz = np.empty(m, np.int32)
    nyz = np.empty(m, np.int32)
    nz = np.empty(m, np.int32)
    rc = _load().orc_ksg_counts_at(_fp(x), dx, _fp(y), dy, _fp(z), dz, n, n, k,
                                   idx.ctypes.data_as(_I64P), m, _fp(eps),
                                   nxz.ctypes.data_as(_I32P), nyz.ctypes.data_as(_I32P),
                                   nz.ctypes.data_as(_I32P))
    if rc != 0:
        raise ValueError("orc_ksg_counts_at: invalid arguments")
    return eps, nxz, nyz, nz


def cmi_ksg(x, y, z, k: int) -> float:
    """One KSG estimate of I(X;Y|Z) in nats."""
    x, dx = _cols(x)
    n = x.shape[1]
    y, dy = _cols(y)
    z, dz = _cols(z, n)
    out = ctypes.c_double()
    rc = _load().orc_cmi_ksg(_fp(x), dx, _fp(y), dy, _fp(z), dz, n, n, k, ctypes.byref(out),
                             None, None)
    if rc != 0:
        raise ValueError("orc_cmi_ksg: invalid arguments")
    return out.value


def splitmix64(state: int, n: int) -> np.ndarray:
    out = np.empty(n, np.uint64)
    _load().orc_splitmix64(ctypes.c_uint64(state), n, out.ctypes.data_as(_U64P))
    return out


def perm(seed: int, stream: int, n: int) -> np.ndarray:
    """The surrogate permutation pi of [0, n) keyed by (seed, stream)."""
    out = np.empty(n, np.int64)
    if _load().orc_perm(ctypes.c_uint64(seed), ctypes.c_uint64(stream), n,
                        out.ctypes.data_as(_I64P)) != 0:
        raise ValueError("bad n")
    return out


def cmi_surrogates(x, y, z, k: int, n_surr: int, seed: int) -> np.ndarray:
    """[1+n_surr] estimates: the original, then X's rows permuted by stream s = 0..n_surr-1."""
    x, dx = _cols(x)
    n = x.shape[1]
    y, dy = _cols(y)
    z, dz = _cols(z, n)
    out = np.empty(1 + n_surr, np.float64)
    rc = _load().orc_cmi_surrogates(_fp(x), dx, _fp(y), dy, _fp(z), dz, n, n, k, n_surr,
                                    ctypes.c_uint64(seed), out.ctypes.data_as(_F64P))
    if rc != 0:
        raise ValueError("orc_cmi_surrogates: invalid arguments")
    return out


def cmi_surrogates_reps(x, y, z, k: int, n_surr: int, seed: int, n_reps: int) -> np.ndarray:
    """[1+n_surr]: the estimate and its replication-level surrogates."""
    x, dx = _cols(x)
    n = x.shape[1]
    y, dy = _cols(y)
    z, dz = _cols(z, n)
    out = np.empty(1 + n_surr, np.float64)
    rc = _load().orc_cmi_surrogates_reps(_fp(x), dx, _fp(y), dy, _fp(z), dz, n, n, k, n_surr,
                                         ctypes.c_uint64(seed), n_reps, out.ctypes.data_as(_F64P))
    if rc != 0:
        raise ValueError("orc_cmi_surrogates_reps: invalid arguments")
    return out


def select_target(series, target: int, n_past: int, min_lag: int, max_lag: int, k: int,
                  n_surr: int, alpha: float, seed: int, max_parents: int,
                  want_first_step: bool = False):
    """Greedy max-statistic parent selection for one target.

    Returns dict(parents=[cand ids], steps=[(cand, significant, stat, pval)],
    first_step=[n_cand_total][1+n_surr] or None).
    """
    s = np.ascontiguousarray(np.asarray(series, np.float32))
    n_proc, T = s.shape
    n_lags = max_lag - min_lag + 1
    steps = (OrcStep * (max_parents + 1))()
    n_steps = ctypes.c_int()
    parents = np.zeros(max(1, max_parents), np.int32)
    n_par = ctypes.c_int()
    est = None
    if want_first_step:
        est = np.full((n_proc * n_lags, 1 + n_surr), np.nan, np.float64)
    rc = _load().orc_select_target(_fp(s), n_proc, T, target, n_past, min_lag, max_lag, k, n_surr,
                                   alpha, ctypes.c_uint64(seed), max_parents, steps,
                                   ctypes.byref(n_steps), parents.ctypes.data_as(_I32P),
                                   ctypes.byref(n_par),
                                   est.ctypes.data_as(_F64P) if est is not None else None)
    if rc != 0:
        raise ValueError("orc_select_target: invalid arguments")
    return dict(parents=[int(p) for p in parents[:n_par.value]],
                steps=[(steps[i].cand, bool(steps[i].significant), steps[i].stat, steps[i].pval)
                       for i in range(n_steps.value)],
                first_step=est)


def _post_args(series, parents):
    s = np.ascontiguousarray(np.asarray(series, np.float32))
    par = np.ascontiguousarray(np.asarray(parents, np.int32))
    return s, par


def prune(series, target: int, n_past: int, min_lag: int, max_lag: int, parents, k: int,
          n_surr: int, alpha: float, seed: int):
    """Minimum-statistic pruning of a selected parent list.

    Returns dict(kept=[cand ids], rounds=[(cand at the minimum, significant, T_min, p)])."""
    s, par = _post_args(series, parents)
    m = len(par)
    kept = np.zeros(max(1, m), np.int32)
    n_kept = ctypes.c_int()
    rounds = (OrcStep * max(1, m))()
    n_rounds = ctypes.c_int()
    rc = _load().orc_prune(_fp(s), s.shape[0], s.shape[1], target, n_past, min_lag, max_lag,
                           par.ctypes.data_as(_I32P), m, k, n_surr, alpha, ctypes.c_uint64(seed),
                           kept.ctypes.data_as(_I32P), ctypes.byref(n_kept), rounds,
                           ctypes.byref(n_rounds))
    if rc != 0:
        raise ValueError("orc_prune: invalid arguments")
    return dict(kept=[int(c) for c in kept[:n_kept.value]],
                rounds=[(rounds[i].cand, bool(rounds[i].significant), rounds[i].stat,
                         rounds[i].pval) for i in range(n_rounds.value)])


def omnibus(series, target: int, n_past: int, min_lag: int, max_lag: int, parents, k: int,
            n_surr: int, alpha: float, seed: int):
    """Omnibus test of a parent set: (stat, p, significant)."""
    s, par = _post_args(series, parents)
    stat, pval, sig = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    rc = _load().orc_omnibus(_fp(s), s.shape[0], s.shape[1], target, n_past, min_lag, max_lag,
                             par.ctypes.data_as(_I32P), len(par), k, n_surr, alpha,
                             ctypes.c_uint64(seed), ctypes.byref(stat), ctypes.byref(pval),
                             ctypes.byref(sig))
    if rc != 0:
        raise ValueError("orc_omnibus: invalid arguments")
    return stat.value, pval.value, bool(sig.value)


def seqmax(series, target: int, n_past: int, min_lag: int, max_lag: int, parents, k: int,
           n_surr: int, alpha: float, seed: int):
    """Sequential maximum statistic: (stats [m], pvals [m], significant [m]) by parent."""
    s, par = _post_args(series, parents)
    m = len(par)
    stats = np.zeros(m, np.float64)
    pvals = np.zeros(m, np.float64)
    sig = np.zeros(m, np.int32)
    rc = _load().orc_seqmax(_fp(s), s.shape[0], s.shape[1], target, n_past, min_lag, max_lag,
                            par.ctypes.data_as(_I32P), m, k, n_surr, alpha, ctypes.c_uint64(seed),
                            stats.ctypes.data_as(_F64P), pvals.ctypes.data_as(_F64P),
                            sig.ctypes.data_as(_I32P))
    if rc != 0:
        raise ValueError("orc_seqmax: invalid arguments")
    return stats, pvals, sig.astype(bool)


def bivariate_te(series, target: int, n_past: int, min_lag: int, max_lag: int, k: int,
                 n_surr: int, seed: int):
    """Bivariate TE of every source variable: (est [n_cand][1+S], pvals [n_cand]);
    rows of the target's own variables are NaN."""
    s = np.ascontiguousarray(np.asarray(series, np.float32))
    n_proc, T = s.shape
    n_cand = n_proc * (max_lag - min_lag + 1)
    est = np.full((n_cand, 1 + n_surr), np.nan, np.float64)
    pvals = np.full(n_cand, np.nan, np.float64)
    rc = _load().orc_bivariate_te(_fp(s), n_proc, T, target, n_past, min_lag, max_lag, k, n_surr,
                                  ctypes.c_uint64(seed), est.ctypes.data_as(_F64P),
                                  pvals.ctypes.data_as(_F64P))
    if rc != 0:
        raise ValueError("orc_bivariate_te: invalid arguments")
    return est, pvals


def select_past(series, target: int, min_lag: int, max_lag: int, k: int, n_surr: int,
                alpha: float, seed: int, max_past: int):
    """Greedy selection of the target's own past: dict(past=[ids], steps=[...])."""
    s = np.ascontiguousarray(np.asarray(series, np.float32))
    steps = (OrcStep * (max_past + 1))()
    n_steps, n_past = ctypes.c_int(), ctypes.c_int()
    past = np.zeros(max(1, max_past), np.int32)
    rc = _load().orc_select_past(_fp(s), s.shape[0], s.shape[1], target, min_lag, max_lag, k,
                                 n_surr, alpha, ctypes.c_uint64(seed), max_past, steps,
                                 ctypes.byref(n_steps), past.ctypes.data_as(_I32P),
                                 ctypes.byref(n_past))
    if rc != 0:
        raise ValueError("orc_select_past: invalid arguments")
    return dict(past=[int(c) for c in past[:n_past.value]],
                steps=[(steps[i].cand, bool(steps[i].significant), steps[i].stat, steps[i].pval)
                       for i in range(n_steps.value)])


def select_sources(series, target: int, past, min_lag: int, max_lag: int, k: int, n_surr: int,
                   alpha: float, seed: int, max_parents: int):
    """Greedy source selection given a past (candidate ids): dict(parents=[ids], steps=[...])."""
    s = np.ascontiguousarray(np.asarray(series, np.float32))
    pa = np.ascontiguousarray(np.asarray(past, np.int32))
    steps = (OrcStep * (max_parents + 1))()
    n_steps, n_par = ctypes.c_int(), ctypes.c_int()
    parents = np.zeros(max(1, max_parents), np.int32)
    rc = _load().orc_select_sources(_fp(s), s.shape[0], s.shape[1], target,
                                    pa.ctypes.data_as(_I32P), len(pa), min_lag, max_lag, k,
                                    n_surr, alpha, ctypes.c_uint64(seed), max_parents, steps,
                                    ctypes.byref(n_steps), parents.ctypes.data_as(_I32P),
                                    ctypes.byref(n_par))
    if rc != 0:
        raise ValueError("orc_select_sources: invalid arguments")
    return dict(parents=[int(c) for c in parents[:n_par.value]],
                steps=[(steps[i].cand, bool(steps[i].significant), steps[i].stat, steps[i].pval)
                       for i in range(n_steps.value)])


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(t: int) -> None:
    _load().orc_set_num_threads(int(t))


# ----------------------------------------------------------------- learned screen
def mlp_nparams(f: int, h: int) -> int:
    return h * f + h + h * h + h + h + 1


def bf16_round(v: float) -> float:
    """Round an fp32 value to bfloat16 (nearest, ties to even), returned as fp32."""
    return float(_load().orc_bf16_round(float(v)))


def mlp_forward(params, f, h, mean, scale, x, bf16: bool = True) -> np.ndarray:
    """Predictions of the screen network (weight matrices rounded to bf16 unless
    bf16=False; fp64 math)."""
    p = np.ascontiguousarray(np.asarray(params, np.float32))
    x = np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1, f))
    mean = np.ascontiguousarray(np.asarray(mean, np.float32))
    scale = np.ascontiguousarray(np.asarray(scale, np.float32))
    y = np.empty(x.shape[0], np.float64)
    if _load().orc_mlp_forward(_fp(p), f, h, _fp(mean), _fp(scale), _fp(x), x.shape[0],
                               1 if bf16 else 0, y.ctypes.data_as(_F64P)) != 0:
        raise ValueError("orc_mlp_forward: invalid arguments")
    return y


def mlp_loss_grad(params, f, h, mean, scale, x, t, bf16: bool = True, quantile: float = 0.0):
    """(loss, gradient [n_params]) in fp64: mean squared error, or the mean pinball
    loss of the given quantile when 0 < quantile < 1."""
    p = np.ascontiguousarray(np.asarray(params, np.float32))
    x = np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1, f))
    t = np.ascontiguousarray(np.asarray(t, np.float32))
    mean = np.ascontiguousarray(np.asarray(mean, np.float32))
    scale = np.ascontiguousarray(np.asarray(scale, np.float32))
    loss = ctypes.c_double()
    g = np.empty(mlp_nparams(f, h), np.float64)
    if _load().orc_mlp_loss_grad(_fp(p), f, h, _fp(mean), _fp(scale), _fp(x), _fp(t),
                                 x.shape[0], 1 if bf16 else 0, float(quantile),
                                 ctypes.byref(loss), g.ctypes.data_as(_F64P)) != 0:
        raise ValueError("orc_mlp_loss_grad: invalid arguments")
    return loss.value, g
