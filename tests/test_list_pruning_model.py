"""The list builder's tile pruning, modelled on the CPU.

For each query, the list builder forms per tile a lower bound G (the box gap)
and an upper bound F (the far corner) on the fp32 max-norm distances of the
tile's samples, sums tile sizes into a histogram by F to get a radius R within
which more than cap samples lie, histograms only the tiles with G < R, and
collects only the tiles with G below the list's cut.  These tests restate
those steps in numpy fp32 and check the claims the kernel's exactness rests
on: the bounds hold for the computed distances, R really holds more than cap
samples, the pruned histogram gives the same cut as the full one, and the
collected tiles hold every sample below the cut.
"""
import numpy as np
import pytest

TJ = 128          # samples per tile
BIN_SHIFT = 19    # histogram bins on bits 30..19 of a non-negative float
N_BINS = 4096


def bins(v):
    return (np.asarray(v, np.float32).view(np.uint32) >> BIN_SHIFT).astype(np.int64)


def upper_edge(b):
    if b + 1 >= (0x7F800000 >> BIN_SHIFT):
        return np.float32(np.inf)
    return np.uint32((b + 1) << BIN_SHIFT).view(np.float32)


def cut_bin(hist, cap):
    """First bin whose cumulative count exceeds cap (N_BINS if none)."""
    c = np.cumsum(hist)
    over = np.nonzero(c > cap)[0]
    return int(over[0]) if len(over) else N_BINS


def dist(q, rows, cols):
    """fp32 max-norm distance over the given columns."""
    d = np.abs(rows[:, cols] - q[cols]).astype(np.float32)
    return d.max(axis=1)


def box_bounds(q, lo, hi, cols):
    g = np.maximum(np.maximum(lo[:, cols] - q[cols], q[cols] - hi[:, cols]), np.float32(0))
    f = np.maximum(np.abs(q[cols] - lo[:, cols]), np.abs(q[cols] - hi[:, cols]))
    return g.max(axis=1).astype(np.float32), f.max(axis=1).astype(np.float32)


def make_tiles(n, dims, seed):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal((n, dims)).astype(np.float32)
    # a crude spatial order (first coordinate), as the Morton order is
    p = p[np.argsort(p[:, 0], kind="stable")]
    nt = (n + TJ - 1) // TJ
    lo = np.stack([p[t * TJ:(t + 1) * TJ].min(0) for t in range(nt)])
    hi = np.stack([p[t * TJ:(t + 1) * TJ].max(0) for t in range(nt)])
    size = np.array([min(TJ, n - t * TJ) for t in range(nt)])
    return p, lo, hi, size


@pytest.mark.parametrize("n,dims,dz,cap", [(3000, 4, 3, 200), (5000, 11, 10, 300),
                                           (2000, 2, 1, 100)])
def test_pruned_histogram_gives_the_exact_cut(n, dims, dz, cap):
    p, lo, hi, size = make_tiles(n, dims, seed=n + dims)
    tile_of = np.arange(n) // TJ
    rng = np.random.default_rng(1)
    for cols in (list(range(dz)), list(range(dims))):
        for i in rng.choice(n, 12, replace=False):
            q = p[i]
            d = dist(q, p, cols)
            d[i] = np.inf  # the query is not its own neighbour
            g, f = box_bounds(q, lo, hi, cols)
            # the bounds hold for every sample's computed distance
            others = np.arange(n) != i
            assert np.all(g[tile_of][others] <= d[others])
            assert np.all(d[others] <= f[tile_of][others])
            # radius from the far corners: more than cap samples within it
            hf = np.zeros(N_BINS, np.int64)
            np.add.at(hf, bins(f), size)
            fb = cut_bin(hf, cap + 1)
            r_lim = upper_edge(fb) if fb < N_BINS else np.float32(np.inf)
            assert np.count_nonzero(d < r_lim) > cap
            # histogram of the visited tiles only: the same cut as the full one
            full = np.zeros(N_BINS, np.int64)
            np.add.at(full, bins(d[others]), 1)
            visited = g < r_lim
            keep = others & visited[tile_of]
            part = np.zeros(N_BINS, np.int64)
            np.add.at(part, bins(d[keep]), 1)
            cb = cut_bin(full, cap)
            assert cut_bin(part, cap) == cb
            r = np.uint32(cb << BIN_SHIFT).view(np.float32) if cb < N_BINS else np.inf
            # the list: every sample below the cut, at most cap of them,
            # all inside the tiles the collecting pass visits
            members = np.nonzero(d < r)[0]
            assert len(members) <= cap
            assert np.all(g[tile_of[members]] < r)
