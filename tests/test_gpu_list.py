"""The list kernel (per-query sorted neighbour lists) through the C ABI.

Bar: eps and every neighbour count bit-exact against the CPU oracle; every
estimate bit-identical to the tile kernel's (both sum the digamma terms in the
same order) and within 1e-10 nats of the oracle.  Tiny list capacities force
the full-scan fallbacks, so both halves of the kernel are exercised.
"""
import numpy as np
import pytest

import oracle
from paper_1807_10459_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def idtx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_10459_gb300 as m
    from paper_1807_10459_gb300 import build
    build.build()
    return m


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _ctx(idtx, kernel, caps=(0, 0)):
    ctx = idtx.Context(0)
    ctx.set_kernel(kernel)
    ctx.set_list_caps(*caps)
    return ctx


def _run(idtx, ctx, x, y, z, k, S, seed):
    cmi, eps, cnt = idtx.cmi_ksg(_dev(x), _dev(y), _dev(z), k=k, n_surr=S, seed=seed,
                                 want_eps=True, want_counts=True, ctx=ctx)
    torch.cuda.synchronize()
    return cmi.cpu().numpy(), eps.cpu().numpy(), cnt.cpu().numpy()


def _oracle(x, y, z, k, S, seed):
    n = x.shape[1]
    eps, cnt, cmi = [], [], []
    for s in range(S + 1):
        xs = x if s == 0 else x[:, oracle.perm(seed, s - 1, n)]
        e, a, b, c = oracle.ksg_counts(xs, y, z, k)
        eps.append(e)
        cnt.append(np.stack([a, b, c]))
        cmi.append(oracle.cmi_ksg(xs, y, z, k))
    return np.array(eps), np.array(cnt), np.array(cmi)


def _check(idtx, x, y, z, k, S, seed, caps=(0, 0), expect_fallbacks=False):
    lst = _ctx(idtx, idtx.KERNEL_LIST, caps)
    tile = _ctx(idtx, idtx.KERNEL_TILE)
    m_l, e_l, c_l = _run(idtx, lst, x, y, z, k, S, seed)
    m_t, e_t, c_t = _run(idtx, tile, x, y, z, k, S, seed)
    st = lst.stats()
    assert st["list_launches"] == 1 and tile.stats()["list_launches"] == 0
    e_r, c_r, m_r = _oracle(x, y, z, k, S, seed)
    assert np.array_equal(e_l, e_r), "eps differs from the oracle"
    assert np.array_equal(c_l, c_r), "counts differ from the oracle"
    assert np.max(np.abs(m_l - m_r)) < TOL
    assert np.array_equal(m_l, m_t), "list and tile kernels disagree"
    assert np.array_equal(e_l, e_t) and np.array_equal(c_l, c_t)
    if expect_fallbacks:
        assert st["fallbacks"] > 0
    return st


@pytest.mark.parametrize("n", [2, 5, 127, 128, 129, 300, 515, 1000])
def test_ragged_sizes(idtx, n):
    g = synth.gaussian_problem(n, 1, 1, 2, seed=n)
    _check(idtx, g.x, g.y, g.z, min(4, n - 1), 3, 7)


@pytest.mark.parametrize("dims", [(2, 1, 1), (1, 2, 3), (2, 2, 5), (1, 1, 7), (1, 1, 10),
                                  (2, 2, 16), (3, 1, 2), (1, 4, 4), (4, 4, 16)])
def test_dimension_buckets(idtx, dims):
    dx, dy, dz = dims
    g = synth.gaussian_problem(400, dx, dy, dz, seed=sum(dims))
    _check(idtx, g.x, g.y, g.z, 4, 17, 3)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 15])
def test_other_k(idtx, k):
    g = synth.gaussian_problem(333, 1, 1, 2, seed=k)
    _check(idtx, g.x, g.y, g.z, k, 4, 11)


@pytest.mark.parametrize("caps", [(32, 32), (32, 64), (64, 128), (128, 256)])
def test_short_lists_fall_back_exactly(idtx, caps):
    """Lists far shorter than the neighbourhoods: most jobs take the full scan
    in one or both passes; results stay exact."""
    g = synth.gaussian_problem(900, 1, 1, 3, seed=12)
    _check(idtx, g.x, g.y, g.z, 4, 20, 9, caps=caps, expect_fallbacks=True)


def test_lane_op_count_counts_each_fallback_once(idtx):
    """The lane-operation count behind the roofline figure.  Walked list
    entries are counted once per (query, group of 32 jobs) and cost every job
    of the group; a full-scan fallback recomputes ONE job, scanning the N-1
    other samples once.  With lists of 32 entries most jobs fall back, so a
    count that charged each scanned sample to every job of the group would
    exceed the upper bound below by an order of magnitude."""
    n, S, dx, dy, dz = 900, 20, 1, 1, 3
    g = synth.gaussian_problem(n, dx, dy, dz, seed=12)
    ctx = _ctx(idtx, idtx.KERNEL_LIST, (32, 32))
    _, _, cnt = _run(idtx, ctx, g.x, g.y, g.z, 4, S, 9)
    st = ctx.stats()
    assert st["fallbacks"] > 0
    assert st["brute_samples"] == st["fallbacks"] * (n - 1)
    jobs = 1 + S                                      # one group of 32 lanes
    walks = jobs * (st["list_walk_a"] * (2 * dx + 2) + st["list_walk_b"] * (2 * dx + 4))
    tails = st["list_tail_a"] * (2 * dx + 2) + st["list_tail_b"] * (2 * dx + 4)
    dall = 2 * (dx + dy + dz)
    lo = walks + tails + st["brute_samples"] * (dall + 2)
    hi = walks + tails + st["brute_samples"] * (dall + 6)
    assert lo <= st["fused_lane_ops"] <= hi
    # the useful part: exactly the counts the call returned
    assert st["list_sum_nz"] == cnt[:, 2].sum() and st["list_sum_nyz"] == cnt[:, 1].sum()
    assert st["useful_lane_ops"] == (2 * dx + 4) * cnt[:, 2].sum() + (2 * dx + 2) * cnt[:, 1].sum()


def test_useful_work_counters_match_counts(idtx):
    """Default list capacities, a multi-group call: the kernel's sums of n_z
    and n_yz equal the sums of the counts it returns."""
    g = synth.gaussian_problem(2000, 1, 1, 3, seed=41)
    ctx = _ctx(idtx, idtx.KERNEL_LIST)
    _, _, cnt = _run(idtx, ctx, g.x, g.y, g.z, 4, 70, 5)
    st = ctx.stats()
    assert st["list_sum_nz"] == cnt[:, 2].sum() and st["list_sum_nyz"] == cnt[:, 1].sum()


def test_short_lists_other_k_and_dims(idtx):
    g = synth.gaussian_problem(517, 2, 2, 4, seed=3)
    _check(idtx, g.x, g.y, g.z, 7, 9, 2, caps=(32, 32), expect_fallbacks=True)


def test_ties_duplicates_and_zero_distances(idtx):
    """Discrete data: many samples at distance 0, eps = 0 for some queries,
    histogram cuts inside runs of equal distances."""
    rng = np.random.default_rng(5)
    x = rng.integers(0, 4, (1, 260)).astype(np.float32)
    y = rng.integers(0, 4, (1, 260)).astype(np.float32)
    z = rng.integers(0, 3, (2, 260)).astype(np.float32)
    for k in (1, 4, 8):
        for caps in ((0, 0), (32, 32), (64, 96)):
            _check(idtx, x, y, z, k, 3, 1, caps=caps)


def test_all_samples_identical_in_z(idtx):
    """d_Z = 0 for every pair: list B cannot be cut below its capacity."""
    g = synth.gaussian_problem(300, 1, 1, 1, seed=8)
    z = np.zeros_like(g.z)
    _check(idtx, g.x, g.y, z, 4, 5, 3, caps=(32, 32))


def test_dz0_uses_the_tile_kernel(idtx):
    g = synth.gaussian_problem(300, 1, 1, 0, seed=2)
    ctx = _ctx(idtx, idtx.KERNEL_LIST)
    a = idtx.cmi_ksg(_dev(g.x), _dev(g.y), None, k=4, n_surr=3, seed=1, ctx=ctx).cpu().numpy()
    assert ctx.stats()["list_launches"] == 0
    assert np.max(np.abs(a - oracle.cmi_surrogates(g.x, g.y, None, 4, 3, 1))) < TOL


def test_greedy_step_list_equals_tile(idtx):
    net = synth.var_network(n_nodes=5, order=3, T=1500, density=0.4, weight=0.6, seed=21)
    out = []
    for kern in (idtx.KERNEL_LIST, idtx.KERNEL_TILE):
        ctx = _ctx(idtx, kern)
        out.append(idtx.mte_step(_dev(net.series), 0, 2, 1, 3, (), 0, k=4, n_surr=30,
                                 alpha=0.05, seed=17, want_estimates=True, ctx=ctx))
    (a, ea), (b, eb) = out
    ok = ~np.isnan(ea[:, 0])
    assert np.array_equal(ea[ok], eb[ok]) and tuple(a) == tuple(b)


def test_batch_list_equals_tile_and_oracle(idtx):
    probs = synth.batch_problems(n_probs=6, n_min=150, n_max=1500, n_surr=6, dz_max=8, seed=78)
    dev = [dict(x=_dev(p.x), y=_dev(p.y), z=_dev(p.z), n_surr=p.n_surr, seed=p.seed)
           for p in probs]
    lst = _ctx(idtx, idtx.KERNEL_LIST)
    a = [o.cpu().numpy() for o in idtx.cmi_batch(dev, k=4, ctx=lst)]
    b = [o.cpu().numpy() for o in idtx.cmi_batch(dev, k=4, ctx=_ctx(idtx, idtx.KERNEL_TILE))]
    assert lst.stats()["list_launches"] == len(probs)
    for p, u, v in zip(probs, a, b):
        assert np.array_equal(u, v)
        ref = oracle.cmi_surrogates(p.x, p.y, p.z, 4, p.n_surr, p.seed)
        assert np.max(np.abs(u - ref)) < TOL


def test_auto_choice_times_each_shape_once(idtx):
    g = synth.gaussian_problem(1200, 1, 1, 2, seed=30)
    ctx = _ctx(idtx, idtx.KERNEL_AUTO)
    a = idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=4, n_surr=40, seed=2, ctx=ctx)
    b = idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=4, n_surr=40, seed=2, ctx=ctx)
    st = ctx.stats()
    assert st["tune_trials"] == 1
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    ref = oracle.cmi_surrogates(g.x, g.y, g.z, 4, 40, 2)
    assert np.max(np.abs(a.cpu().numpy() - ref)) < TOL
    # another N range is another shape
    g2 = synth.gaussian_problem(5000, 1, 1, 2, seed=31)
    idtx.cmi_ksg(_dev(g2.x), _dev(g2.y), _dev(g2.z), k=4, n_surr=3, seed=2, ctx=ctx)
    assert ctx.stats()["tune_trials"] == 2


def test_bad_list_caps_are_rejected(idtx):
    ctx = idtx.Context(0)
    for caps in ((16, 32), (32, 48), (4096, 32), (32, 8192), (-32, 32)):
        with pytest.raises(idtx.IdtxError):
            ctx.set_list_caps(*caps)
    with pytest.raises(idtx.IdtxError):
        ctx.set_kernel(5)


@pytest.mark.slow
def test_full_size_greedy_step_list_equals_tile(idtx):
    """The benchmarked greedy step (10-node VAR(5), T=10000, history 3, lags
    1..5, k=4, 200 surrogates): every one of the 9447 estimates identical under
    both kernels; sampled estimates against the oracle."""
    net = synth.var_network()
    res = []
    for kern in (idtx.KERNEL_LIST, idtx.KERNEL_TILE):
        ctx = _ctx(idtx, kern)
        res.append(idtx.mte_step(_dev(net.series), 0, 3, 1, 5, (), 0, k=4, n_surr=200,
                                 alpha=0.05, seed=20181029, want_estimates=True, ctx=ctx))
        if kern == idtx.KERNEL_LIST:
            st = ctx.stats()
    (a, ea), (b, eb) = res
    ok = ~np.isnan(ea[:, 0])
    assert ok.sum() == 47
    assert np.array_equal(ea[ok], eb[ok]) and tuple(a) == tuple(b)
    assert st["list_launches"] == 1
    L, T = 5, net.series.shape[1]
    y = net.series[0, L:]
    z = np.stack([net.series[0, L - lag:T - lag] for lag in (1, 2, 3)])
    c = int(np.flatnonzero(ok)[7])
    p, lag = divmod(c, 5)
    xc = net.series[p, L - lag - 1:T - lag - 1][None, :]
    for s in (0, 113):
        xs = xc if s == 0 else xc[:, oracle.perm(20181029, (c << 24) | (s - 1), T - L)]
        assert abs(ea[c, s] - oracle.cmi_ksg(xs, y, z, 4)) < TOL
