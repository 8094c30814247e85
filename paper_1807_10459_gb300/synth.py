"""Seeded synthetic inputs shared by the GPU path's tests/benchmarks and the oracle.

This module only draws data.  It holds none of the estimator's arithmetic: no
distances, neighbour counts, digamma, permutation or gating.  The IDTxl paper
(arXiv 1807.10459) reports no datasets or experiments, so every workload here
is a synthetic stand-in with the shape of the workloads the build is measured
on (coupled linear VAR networks, coupled logistic maps, correlated Gaussians).
All outputs are standardised (zero mean, unit variance per column, computed in
float64) and returned as float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20181027


def _standardise(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a, np.float64)
    mu = a.mean(axis=-1, keepdims=True)
    sd = a.std(axis=-1, keepdims=True)
    sd[sd == 0] = 1.0
    return ((a - mu) / sd).astype(np.float32)


# --------------------------------------------------------------------------
# Correlated Gaussian CMI problems
# --------------------------------------------------------------------------
@dataclass
class GaussianProblem:
    x: np.ndarray          # [dx][N] float32
    y: np.ndarray          # [dy][N] float32
    z: np.ndarray          # [dz][N] float32 (dz may be 0)
    cov: np.ndarray        # [d][d] float64 covariance the samples were drawn from
    dims: tuple            # (dx, dy, dz)


def random_covariance(d: int, rng: np.random.Generator) -> np.ndarray:
    """Sigma = A A^T + 0.5 I with A ~ N(0,1)^{d x d}."""
    a = rng.standard_normal((d, d))
    return a @ a.T + 0.5 * np.eye(d)


def gaussian_problem(n: int, dx: int = 1, dy: int = 1, dz: int = 2, seed: int = BASE_SEED + 1,
                     cov: np.ndarray | None = None) -> GaussianProblem:
    """Jointly Gaussian samples with a seeded random covariance (float64 Cholesky).

    Columns are NOT standardised, so that ``cov`` stays the exact law of the
    samples (before rounding to float32).
    """
    rng = np.random.default_rng(seed)
    d = dx + dy + dz
    if cov is None:
        cov = random_covariance(d, rng)
    chol = np.linalg.cholesky(cov)
    w = rng.standard_normal((d, n))
    s = (chol @ w).astype(np.float32)
    return GaussianProblem(x=np.ascontiguousarray(s[:dx]), y=np.ascontiguousarray(s[dx:dx + dy]),
                           z=np.ascontiguousarray(s[dx + dy:]), cov=cov, dims=(dx, dy, dz))


# --------------------------------------------------------------------------
# Linear VAR networks
# --------------------------------------------------------------------------
@dataclass
class VarNetwork:
    series: np.ndarray                 # [n_nodes][T] float32, standardised
    coef: np.ndarray                   # [order][n_nodes][n_nodes]: x_t[q] += coef[l-1][q][p] x_{t-l}[p]
    edges: list = field(default_factory=list)  # (source p, target q, lag) for p != q


def _companion_radius(coef: np.ndarray) -> float:
    order, n, _ = coef.shape
    comp = np.zeros((order * n, order * n))
    comp[:n, :] = np.concatenate(list(coef), axis=1)
    comp[n:, :-n] = np.eye((order - 1) * n)
    return float(np.max(np.abs(np.linalg.eigvals(comp))))


def _simulate_var(coef: np.ndarray, T: int, burn: int, rng: np.random.Generator) -> np.ndarray:
    order, n, _ = coef.shape
    total = T + burn
    x = np.zeros((total + order, n))
    e = rng.standard_normal((total, n))
    for t in range(order, total + order):
        acc = e[t - order].copy()
        for lag in range(1, order + 1):
            acc += coef[lag - 1] @ x[t - lag]
        x[t] = acc
    return x[order + burn:].T


def _stabilise(coef: np.ndarray, limit: float = 0.9) -> np.ndarray:
    rho = _companion_radius(coef)
    while rho >= limit:
        coef = coef * (limit / rho) * 0.999
        rho = _companion_radius(coef)
    return coef


def var_network(n_nodes: int = 10, order: int = 5, T: int = 10000, density: float = 0.2,
                weight: float = 0.4, self_range=(0.2, 0.5), burn: int = 1000,
                seed: int = BASE_SEED + 2) -> VarNetwork:
    """Sparse VAR(order): each ordered pair p != q is an edge with probability
    ``density``, at a uniform lag in 1..order with weight U[-weight, weight];
    every node has a lag-1 self-coupling U[self_range].  Weights are scaled
    down until the companion spectral radius is below 0.9.  Unit Gaussian
    innovations."""
    rng = np.random.default_rng(seed)
    coef = np.zeros((order, n_nodes, n_nodes))
    edges = []
    for q in range(n_nodes):
        coef[0, q, q] = rng.uniform(*self_range)
        for p in range(n_nodes):
            if p == q:
                continue
            if rng.random() < density:
                lag = int(rng.integers(1, order + 1))
                coef[lag - 1, q, p] = rng.uniform(-weight, weight)
                edges.append((p, q, lag))
    coef = _stabilise(coef)
    series = _simulate_var(coef, T, burn, rng)
    return VarNetwork(series=_standardise(series), coef=coef, edges=edges)


def var_network_indegree(n_nodes: int = 50, order: int = 3, indegree: int = 3, T: int = 5000,
                         weight: float = 0.4, self_range=(0.2, 0.5), burn: int = 1000,
                         seed: int = BASE_SEED + 5) -> VarNetwork:
    """Sparse VAR(order) where every node has exactly ``indegree`` parents
    (uniform among the other nodes, lag uniform in 1..order)."""
    rng = np.random.default_rng(seed)
    coef = np.zeros((order, n_nodes, n_nodes))
    edges = []
    for q in range(n_nodes):
        coef[0, q, q] = rng.uniform(*self_range)
        others = [p for p in range(n_nodes) if p != q]
        for p in rng.choice(others, size=indegree, replace=False):
            lag = int(rng.integers(1, order + 1))
            w = rng.uniform(-weight, weight)
            coef[lag - 1, q, int(p)] = w
            edges.append((int(p), q, lag))
    coef = _stabilise(coef)
    series = _simulate_var(coef, T, burn, rng)
    return VarNetwork(series=_standardise(series), coef=coef, edges=edges)


# --------------------------------------------------------------------------
# Coupled logistic maps
# --------------------------------------------------------------------------
def logistic_chain(n_maps: int = 4, length: int = 2000, reps: int = 50, r: float = 4.0,
                   coupling: float = 0.1, noise: float = 0.01, burn: int = 500,
                   seed: int = BASE_SEED + 4) -> np.ndarray:
    """Noisy logistic maps coupled along a chain 0 -> 1 -> ... -> n_maps-1:
        x_q(t+1) = (1-c) f(x_q(t)) + c f(x_{q-1}(t)) + eta,  f(u) = r u (1-u),
    eta ~ N(0, noise^2), folded back into [0, 1] by reflection.  Returns
    [reps][n_maps][length] float64 (not standardised)."""
    rng = np.random.default_rng(seed)
    out = np.empty((reps, n_maps, length))
    for rep in range(reps):
        x = rng.uniform(0.05, 0.95, n_maps)
        for t in range(burn + length):
            f = r * x * (1.0 - x)
            nxt = (1.0 - coupling) * f
            nxt[1:] += coupling * f[:-1]
            nxt[0] += coupling * f[0]
            nxt += noise * rng.standard_normal(n_maps)
            nxt = np.abs(nxt)                    # reflect at 0
            nxt = np.where(nxt > 1.0, 2.0 - nxt, nxt)  # reflect at 1
            nxt = np.clip(nxt, 0.0, 1.0)
            x = nxt
            if t >= burn:
                out[rep, :, t - burn] = x
    return out


def logistic_problem(dx: int = 1, dy: int = 1, dz: int = 10, length: int = 2000, reps: int = 50,
                     seed: int = BASE_SEED + 4):
    """A CMI problem embedded from the 4-map logistic chain, replications concatenated.

    Y = map 3 at time t (and map 2 at t if dy = 2); X = map 2 at t-1 (and map 1
    at t-1 if dx = 2); Z = the first dz of: map 3 at t-1, t-2, map 0..3 at
    t-2.., in a fixed list of lags of the four maps.  N = reps * (length - 3).
    Returns (x, y, z) as standardised float32 [d][N]."""
    maps = logistic_chain(n_maps=4, length=length, reps=reps, seed=seed)
    lagmax = 3
    cols_y = [(3, 0), (2, 0)][:dy]
    cols_x = [(2, 1), (1, 1)][:dx]
    z_pool = [(3, 1), (3, 2), (0, 1), (1, 1), (2, 2), (0, 2), (1, 2), (3, 3), (0, 3), (1, 3),
              (2, 3), (0, 0)]
    z_pool = [c for c in z_pool if c not in cols_x and c not in cols_y]
    if dz > len(z_pool):
        raise ValueError("dz too large for the logistic embedding")
    cols_z = z_pool[:dz]

    def take(cols):
        if not cols:
            return np.zeros((0, reps * (length - lagmax)), np.float32)
        parts = []
        for (m, lag) in cols:
            parts.append(np.concatenate([maps[rep, m, lagmax - lag:length - lag]
                                         for rep in range(reps)]))
        return _standardise(np.stack(parts))

    return take(cols_x), take(cols_y), take(cols_z)


# --------------------------------------------------------------------------
# Batched uneven problems
# --------------------------------------------------------------------------
@dataclass
class BatchProblem:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    n_surr: int
    seed: int
    kind: str


def batch_problems(n_probs: int = 64, n_min: int = 2000, n_max: int = 50000, n_surr: int = 500,
                   dz_max: int = 8, seed: int = BASE_SEED + 3) -> list:
    """Uneven CMI problems: N = floor(exp(U[ln n_min, ln n_max])), dx, dy in {1,2},
    dz in 1..dz_max; even indices correlated Gaussian, odd indices coupled
    logistic maps."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n_probs):
        n = int(math.floor(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        dx = int(rng.integers(1, 3))
        dy = int(rng.integers(1, 3))
        dz = int(rng.integers(1, dz_max + 1))
        pseed = int(rng.integers(0, 2**62))
        if p % 2 == 0:
            g = gaussian_problem(n, dx, dy, dz, seed=pseed)
            x, y, z = _standardise(g.x), _standardise(g.y), _standardise(g.z)
            kind = "gaussian"
        else:
            length = 500
            reps = -(-(n + 3 * 0) // (length - 3))
            x, y, z = logistic_problem(dx, dy, dz, length=length, reps=reps, seed=pseed)
            x, y, z = x[:, :n], y[:, :n], z[:, :n]
            kind = "logistic"
        out.append(BatchProblem(x=np.ascontiguousarray(x), y=np.ascontiguousarray(y),
                                z=np.ascontiguousarray(z), n_surr=n_surr,
                                seed=int(rng.integers(0, 2**62)), kind=kind))
    return out
