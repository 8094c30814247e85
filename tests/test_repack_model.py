"""The list kernel's repacked count phases, modelled on the CPU.

When few of a warp's 32 jobs still need list-B entries, the kernel repacks
them: with c jobs left, M slots (the power of two >= c), slot s on lanes
s, s+M, ..., each lane taking the staged chunk's entries r, r + 32/M, ...
(r = lane / M) two at a time, then sums each slot's lanes by an XOR
butterfly over the lane bits above log2(M) and hands the total to the job's
lane by its rank among the remaining jobs.  These tests restate that index
arithmetic in plain Python and check that every (job, entry) pair of a chunk
is counted exactly once, by one of the job's slot lanes, and that the totals
reach the right jobs, for every set of remaining jobs a warp can have.
"""
import numpy as np
import pytest

PHASE_STEP = 2  # entries a lane takes per step


def slots_for(rem):
    c = bin(rem).count("1")
    lg = 4 if c > 8 else (3 if c > 4 else (2 if c > 2 else (1 if c > 1 else 0)))
    return c, lg, 1 << lg, 32 >> lg


def home_of(rem, s):
    """The lane of the (s+1)-th remaining job."""
    mm = rem
    for _ in range(s):
        mm &= mm - 1
    return (mm & -mm).bit_length() - 1


def phase_counts(rem, co, counts):
    """One chunk of a repacked phase: per lane, the entries it counts for its
    slot's job; counts[job][entry] is the pair's contribution."""
    c, lg, M, per = slots_for(rem)
    lane_sum = np.zeros(32, np.int64)
    seen = {}
    for lane in range(32):
        s, r = lane & (M - 1), lane >> lg
        if s >= c:
            continue
        job = home_of(rem, s)
        for u0 in range(0, M, PHASE_STEP):
            for t in range(PHASE_STEP):
                idx = r + per * (u0 + t)
                if u0 + t < M and idx >= co:
                    assert idx < 32
                    seen[(job, idx)] = seen.get((job, idx), 0) + 1
                    lane_sum[lane] += counts[job][idx]
    # each slot's total over its lanes: XOR butterfly over the bits >= lg
    total = lane_sum.copy()
    off = M
    while off < 32:
        total = total + total[np.arange(32) ^ off]
        off <<= 1
    # slot s's total sits on lane s (r = 0): to the job's lane by rank
    out = np.zeros(32, np.int64)
    for lane in range(32):
        if (rem >> lane) & 1:
            rank = bin(rem & ((1 << lane) - 1)).count("1")
            out[lane] = total[rank]
    return seen, out


@pytest.mark.parametrize("c", [1, 2, 3, 4, 5, 7, 8])
def test_every_pair_counted_once(c):
    rng = np.random.default_rng(c)
    for _ in range(50):
        jobs = rng.choice(32, c, replace=False)
        rem = 0
        for j in jobs:
            rem |= 1 << int(j)
        co = int(rng.integers(0, 32))
        counts = rng.integers(0, 5, size=(32, 32))
        seen, out = phase_counts(rem, co, counts)
        expect = {(int(j), e): 1 for j in jobs for e in range(co, 32)}
        assert seen == expect
        for lane in range(32):
            want = counts[lane][co:].sum() if (rem >> lane) & 1 else 0
            assert out[lane] == want
